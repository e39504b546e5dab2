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


def _weights_bf16(p, D, H=64):
    """W1, W2, w3 rounded to bfloat16 as the kernels use them; biases unchanged."""
    from oracle import oracle as O
    q = np.array(p, dtype=np.float64)
    for a, b in ((0, D * H), (D * H + H, D * H + H + H * H), (D * H + 2 * H + H * H, D * H + 3 * H + H * H)):
        q[a:b] = [O.bf16(v) for v in q[a:b]]
    return q


def test_learned_proposal_stagewise_against_oracle(S):
    """Each learned proposal recomputed by the oracle from the state the device
    published before the iteration: the parents theta_{k-1}, the network and its
    standardisation, the population Cholesky factor L, and the Philox normals z
    of the proposal stream.  theta_k = theta_{k-1} + h L (w + z) with
    w = clip(h/2 L^T grad log pi^, +-3); log q = N(theta_k; theta_{k-1} + h L w,
    h^2 L L^T) exactly.  The score passes through the bf16 network, so theta_k
    agrees to the network's input-gradient bar; log q depends only on z and L."""
    from oracle import oracle as O
    h = 1.0
    w = I.workload("seir_t100_n1024_mlp", N=256, M=128, T=40, K=14, precision=I.PREC_FP64)
    ctx = S.SMC2(S.make_config(w, mlp_h=h), w.y)
    D, N = w.D, w.N
    checked = 0
    for _ in range(w.K):
        ls = ctx.learned_state()
        k_prev, theta_a, _, _, _ = ctx.get_state()
        st = ctx.run(1)[0][0]
        if not st["mlp_used"]:
            continue
        assert ls["pop_ok"] and ls["loss"] < 0.5 * ls["var_y"]
        k = st["k"]
        assert k == k_prev + 1
        theta_b, logq = ctx.proposals()
        pw = _weights_bf16(ls["params"], D)
        x = ((theta_a - ls["mu"]) / ls["sd"]).astype(np.float32).astype(np.float64)
        _, dx = O.mlp_input_grad(pw, x, bf16_points=True)
        g = ls["tau"] * ls["zsd"] * dx / ls["sd"]
        L = ls["L"]
        expect_th = np.empty((N, D))
        expect_lq = np.empty(N)
        drift = np.empty((N, D))
        for i in range(N):
            z = np.concatenate([O.normals4(w.seed, gi, 0, i, O.TAG_PROPOSE | (k << 4)) for gi in range(0, D, 4)])[:D]
            wv = np.clip(0.5 * h * (L.T @ g[i]), -3.0, 3.0)
            drift[i] = h * (L @ wv)
            expect_th[i] = theta_a[i] + h * (L @ (wv + z))
            expect_lq[i] = -0.5 * D * math.log(2 * math.pi) - D * math.log(h) - np.sum(np.log(np.diag(L))) \
                - 0.5 * z @ z
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
