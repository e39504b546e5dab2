"""The learned proposal inside the sampler (a network trained in the run
proposes theta_k; the Gaussian L-kernel weights of Eq. 20 correct for it).

Its value is statistical: at equal work it should estimate the posterior
more accurately than the random walk it replaces.  The accuracy of a
configuration is the mean squared error, over independent seeds, of the
recycled posterior mean (Eqs. 23, 29) against a reference pooled from long
random-walk runs with eight times the samples; its efficiency is
1 / (MSE x wall time)."""
import math
import time

import numpy as np
import pytest
import torch

from paper_2311_12973_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2311_12973_gb300 import smc2
    return smc2


def _runs(S, w, seeds, **over):
    ctx = S.SMC2(S.make_config(w, **over), w.y)
    ctx.run(w.K)  # graph capture and first-touch outside the timed runs
    out = []
    for sd in seeds:
        ctx.reset(sd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ctx.run(w.K)
        dt = time.perf_counter() - t0
        mean, logz, _ = ctx.estimate()
        out.append((mean, logz, dt, [s[0] for s in st]))
    ctx.close()
    return out


def test_learned_proposal_trains_and_takes_over(S):
    w = I.workload("seir_t100_n1024_mlp")
    ((mean, logz, _, st),) = _runs(S, w, [5])
    used = [s["mlp_used"] for s in st]
    assert used[0] == 0 and used[1] == 0            # the random walk until a network is published
    assert sum(used) >= w.K // 2, used
    for s in st:
        assert math.isfinite(s["ess"]) and s["ess"] >= 1.0
        assert np.all(np.isfinite(s["est"]))
        if s["mlp_used"]:
            assert 0.0 <= s["mlp_loss"] < 0.5, s    # explains half its target variance
    assert np.all(np.isfinite(mean)) and math.isfinite(logz)


def test_learned_proposal_gain_over_random_walk(S):
    ref_runs = _runs(S, I.workload("seir_t100_n1024", N=8192), list(range(101, 109)), rw_scale=0.2)
    ref = np.mean([r[0] for r in ref_runs], axis=0)
    seeds = list(range(11, 35))
    res = {}
    for name, w in (("rw", I.workload("seir_t100_n1024")), ("learned", I.workload("seir_t100_n1024_mlp"))):
        r = _runs(S, w, seeds)
        means = np.array([x[0] for x in r])
        mse = ((means - ref) ** 2).mean(axis=0)
        t = float(np.mean([x[2] for x in r]))
        used = np.mean([sum(s["mlp_used"] for s in x[3]) for x in r])
        res[name] = (mse, t, means)
        print(f"{name:8s} rmse {np.sqrt(mse)}  {1e3 * t:.2f} ms  iterations proposed by the network {used:.1f}"
              f"  efficiency {1 / (mse.mean() * t):.3g}")
    (mse_rw, t_rw, _), (mse_l, t_l, means_l) = res["rw"], res["learned"]
    gain = (mse_rw.mean() * t_rw) / (mse_l.mean() * t_l)
    print(f"efficiency gain {gain:.2f}")
    # measured on GB300 with 32 seeds: rmse 0.011-0.017 vs 0.026-0.057 per coordinate, gain about 6
    assert np.all(mse_l < mse_rw)
    assert gain > 2.0
    # consistent: the seed average within 4 standard errors of the reference
    se = means_l.std(axis=0, ddof=1) / math.sqrt(len(seeds))
    assert np.all(np.abs(means_l.mean(axis=0) - ref) < 4 * se + 0.005), (means_l.mean(axis=0), ref, se)


def test_learned_proposal_stagewise_against_oracle(S):
    """Each iteration's proposal step recomputed by the oracle from the state the
    device published before it: the decision to use the network and the
    population factor L (choice L4) from the previous iteration's weighted
    covariance and ESS; the score of the published network at the parents
    theta_{k-1} and the preconditioned Langevin proposal with its exact density
    (choice L3), with the proposal stream's Philox normals z.  The score passes
    through the bfloat16 network, so theta_k agrees to the network's
    input-gradient bar; log q depends only on z and L."""
    from oracle import oracle as O
    h = 1.0
    w = I.workload("seir_t100_n1024_mlp", N=256, M=128, T=40, K=14, precision=I.PREC_FP64)
    ctx = S.SMC2(S.make_config(w, mlp_h=h), w.y)
    D, N = w.D, w.N
    checked = 0
    for _ in range(w.K):
        ls = ctx.learned_state()
        k_prev, theta_a, _, _, _ = ctx.get_state()
        hist = ctx.history()
        st = ctx.run(1)[0][0]
        k = st["k"]
        assert k == k_prev + 1
        if k >= 2:
            prev = hist[k - 2]
            L_o, ok_o = O.population_factor(prev["cov"], prev["ess"])
            assert ok_o == ls["pop_ok"], (k, ok_o, ls["pop_ok"])
            if ok_o:
                assert np.allclose(ls["L"], L_o, rtol=1e-12, atol=1e-12 * np.max(np.abs(L_o)))
            assert bool(st["mlp_used"]) == O.learned_decision(k, ls["loss"], ls["var_y"], ok_o), (k, st, ls["loss"])
        if not st["mlp_used"]:
            continue
        theta_b, logq = ctx.proposals()
        g = O.mlp_score(ls["params"].astype(np.float64), ls, theta_a)
        expect_th = np.empty((N, D))
        expect_lq = np.empty(N)
        drift = np.empty((N, D))
        for i in range(N):
            z = np.concatenate([O.normals4(w.seed, gi, 0, i, O.TAG_PROPOSE | (k << 4)) for gi in range(0, D, 4)])[:D]
            expect_th[i], expect_lq[i] = O.langevin_propose(h, ls["L"], theta_a[i], g[i], z)
            drift[i] = O.langevin_propose(h, ls["L"], theta_a[i], g[i], np.zeros(D))[0] - theta_a[i]
        err_th = np.max(np.abs(theta_b - expect_th))
        err_lq = np.max(np.abs(logq - expect_lq))
        print(f"k={k}: theta err {err_th:.3g} (drift scale {np.max(np.abs(drift)):.3g}), log q err {err_lq:.3g}")
        # measured on GB300: theta typically within 2e-7 of a drift of order 1, and within
        # 1e-3 of it when one activation rounds to the neighbouring bfloat16 (one step,
        # 2^-8, as the input-gradient test allows); log q within 4e-15
        assert err_lq < 1e-9
        assert err_th <= 1e-2 * np.max(np.abs(drift)) + 1e-10
        checked += 1
    assert checked >= 3, checked
    ctx.close()


def test_learned_state_needs_the_learned_proposal(S):
    w = I.workload("seir_t100_n1024", N=64, M=64, T=20, K=2)
    ctx = S.SMC2(S.make_config(w), w.y)
    with pytest.raises(S.SMC2Error):
        ctx.learned_state()
    ctx.close()
