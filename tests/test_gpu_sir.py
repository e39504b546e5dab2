"""The binomial SIR model of Sec. V-A on the device against the oracle.

FP64: the binomial flows are decided by the same correctly rounded operations
on both sides (only exp, log1p, log and lgamma round on their own, a flip
needing a uniform within an ulp of a boundary), so ancestors agree bit for bit
and increments to 1e-12 of T times the magnitude of the Poisson terms.  FP32
particles draw the flows with the float form of the sampler, so they give
independent estimates of the same likelihood: no offset against the oracle,
unbiased for the exact likelihood of a small population, and for the exact
one-day likelihood in every regime of the sampler."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2311_12973_gb300 import inputs as I

from gpu_util import rel_err, soa
from test_oracle_sir import ONE_DAY, one_day_likelihood, sir_exact_loglik

pytestmark = pytest.mark.gpu

PAPER_PF = dict(pf_scheme=O.PF_MULTINOMIAL, pf_ess_frac=0.5)
EVERY_STEP = dict(pf_scheme=O.PF_SYSTEMATIC, pf_ess_frac=0.0)


@pytest.fixture(scope="module")
def S():
    from paper_2311_12973_gb300 import smc2
    return smc2


def _obs_scale(y):
    y = np.maximum(np.asarray(y), 1.0)
    return float(np.max(y * np.log(y) + y + np.array([math.lgamma(v + 1) for v in y])))


def _trace(S, w, thetas, k, pf, ppt=0):
    ctx = S.SMC2(S.make_config(w, ppt=ppt, **pf), w.y)
    ll, delta, anc = ctx.pf_trace(soa(thetas), iteration=k)
    out = ll.cpu().numpy(), delta.cpu().numpy(), anc.cpu().numpy()
    ctx.close()
    cfg = O.config_from(w, **pf)
    ref = [O.pf_loglik(cfg, thetas[i], w.y, k, i, trace=True) for i in range(len(thetas))]
    return out, ref


@pytest.mark.parametrize("pf", ["paper", "every_step"])
@pytest.mark.parametrize("M,n,ppt", [(500, 6, 0), (64, 9, 1), (100, 7, 2), (1000, 3, 0), (2048, 2, 4), (1, 3, 0)])
def test_fp64_traces_bit_exact(S, pf, M, n, ppt):
    w = I.workload("sir_t30_n1024", N=n, M=M, precision=I.PREC_FP64)
    th = I.theta_near_prior(w, n, seed=M + n, spread=0.6)
    th[0] = I.SIR_TRUTH
    (ll, delta, anc), ref = _trace(S, w, th, 2, PAPER_PF if pf == "paper" else EVERY_STEP, ppt)
    sc = _obs_scale(w.y) * w.T
    for i in range(n):
        r_ll, r_delta, r_anc = ref[i]
        assert np.array_equal(anc[i], r_anc), f"filter {i}: ancestors differ"
        fin = np.isfinite(r_delta)
        assert np.array_equal(fin, np.isfinite(delta[i]))
        assert rel_err(delta[i][fin], r_delta[fin], sc) < 1e-12
        if np.isfinite(r_ll):
            assert rel_err(ll[i], r_ll, sc) < 1e-12
        else:
            assert ll[i] == r_ll


def test_fp64_outside_the_prior_support(S):
    # negative rates act as zero probabilities on both sides (the prior gives such theta no weight)
    w = I.workload("sir_t30_n1024", N=4, M=128, precision=I.PREC_FP64)
    th = np.array([[-0.3, 0.2], [0.85, -0.1], [1.7, 0.2], [0.0, 0.0]])
    (ll, delta, anc), ref = _trace(S, w, th, 1, PAPER_PF)
    for i in range(4):
        assert np.array_equal(anc[i], ref[i][2])
        assert ll[i] == ref[i][0] or rel_err(ll[i], ref[i][0], _obs_scale(w.y) * w.T) < 1e-12


@pytest.mark.parametrize("precision", [I.PREC_FP64, I.PREC_MIXED])
@pytest.mark.parametrize("pf", ["paper", "every_step"])
def test_unbiased_for_exact_likelihood(S, precision, pf):
    # a population of 30: the forward algorithm over all (S, I) gives the likelihood exactly
    T, beta, gamma = 10, 0.9, 0.3
    y = I.simulate_sir(T, beta, gamma, 30.0, 3.0, seed=5)
    w = I.workload("sir_t30_n1024", N=4096, M=64, T=T, npop=30.0, i0=3.0, precision=precision)
    w.y = y
    exact = sir_exact_loglik(beta, gamma, 30.0, 3.0, y)
    ctx = S.SMC2(S.make_config(w, **(PAPER_PF if pf == "paper" else EVERY_STEP)), y)
    ll = ctx.pf_loglik(soa(np.tile([beta, gamma], (w.N, 1))), iteration=1).cpu().numpy()
    ctx.close()
    r = np.exp(ll - exact)
    assert abs(r.mean() - 1.0) < 4 * r.std() / math.sqrt(len(r)), (r.mean(), r.std())


@pytest.mark.parametrize("precision", [I.PREC_FP64, I.PREC_MIXED])
@pytest.mark.parametrize("npop,i0,beta,gamma", ONE_DAY)
def test_one_day_filter_unbiased(S, precision, npop, i0, beta, gamma):
    # one day from (npop - i0, i0): E[p^] is the exact convolution of the two binomial
    # laws against Poisson(y_1; I_1); 4096 filters of 1024 particles see the sampler's
    # distribution (rejection, inversion and mirror regimes) to a few 1e-3
    S0, I0 = npop - i0, i0
    mean = I0 + S0 * -math.expm1(-beta * I0 / npop) - I0 * -math.expm1(-gamma)
    for z in (-2.0, 0.0, 1.5):
        y = np.array([max(0.0, round(mean + z * math.sqrt(mean + 1.0) * 1.3))])
        w = I.workload("sir_t30_n1024", N=4096, M=1024, T=1, npop=npop, i0=i0, precision=precision)
        exact = one_day_likelihood(npop, i0, beta, gamma, y[0])
        ctx = S.SMC2(S.make_config(w), y)
        ll = ctx.pf_loglik(soa(np.tile([beta, gamma], (w.N, 1))), iteration=1).cpu().numpy()
        ctx.close()
        r = np.exp(ll - math.log(exact))
        assert abs(r.mean() - 1.0) < 4 * r.std() / math.sqrt(len(r)), (z, r.mean(), r.std())


def test_mixed_precision_no_offset(S):
    w = I.workload("sir_t30_n1024", N=48, M=500)
    th = I.theta_near_prior(w, 48, seed=3, spread=0.3)
    th[:, 0] = 0.85 + 0.05 * (th[:, 0] - 0.5)
    th[:, 1] = 0.20 + 0.05 * (th[:, 1] - 0.5)
    (ll, delta, anc), ref = _trace(S, w, th, 1, PAPER_PF)
    d = ll - np.array([r[0] for r in ref])
    assert np.all(np.isfinite(d))
    assert abs(d.mean()) <= 4.0 * d.std() / np.sqrt(len(d)) + 1e-6, (d.mean(), d.std())


def test_noalloc_entry_point(S):
    w = I.workload("sir_t30_n1024", N=5, M=300, precision=I.PREC_FP64)
    th = I.theta_near_prior(w, 5, seed=2, spread=0.5)
    cfg = S.make_config(w)
    y = torch.tensor(w.y, dtype=torch.float64, device="cuda")
    ll = S.pf_loglik_noalloc(cfg, y, soa(th), iteration=3).cpu().numpy()
    ref = np.array([O.pf_loglik(O.config_from(w), th[i], w.y, 3, i) for i in range(5)])
    assert rel_err(ll, ref, _obs_scale(w.y) * w.T) < 1e-12


@pytest.mark.parametrize("pf", ["paper", "every_step"])
def test_fp64_smc2_run_matches_oracle(S, pf):
    # the paper's experiment at reduced size: uniform prior on [0, 1]^2, Sigma = 0.1 I
    w = I.workload("sir_t30_n1024", N=128, M=100, K=5, precision=I.PREC_FP64)
    v = PAPER_PF if pf == "paper" else EVERY_STEP
    ctx = S.SMC2(S.make_config(w, **v), w.y)
    stats = ctx.run(w.K)
    ref = O.SMC2(O.config_from(w, **v), w.y).run(w.K)
    fin = np.isfinite(ref.logw)
    scale = max(10.0, float(np.max(np.abs(ref.logw[fin]))))
    for k in range(w.K):
        g, o = stats[k][0], ref.stats[k]
        assert g["resampled"] == o["resampled"] and g["lk_fallback"] == o["lk_fallback"]
        for key in ("lse", "lse2", "logz"):
            assert rel_err(g[key], o[key], scale) < 1e-12, (k, key, g[key], o[key])
        assert rel_err(g["ess"], o["ess"]) < 1e-9
        assert rel_err(g["est"], o["est"], 1.0) < 1e-9
    k_, th, lp, ll, lw = ctx.get_state()
    assert rel_err(th, ref.theta, 1.0) < 1e-10
    assert np.array_equal(np.isfinite(lw), fin)
    assert rel_err(lw[fin], ref.logw[fin], scale) < 1e-12
    mean, logz, _ = ctx.estimate()
    assert rel_err(mean, ref.recycled()[0], 1.0) < 1e-9
    ctx.close()


def test_paper_workload_recovers_truth(S):
    # the paper's configuration (N = 1024, M = 500, T = 30, K = 10, FP32 particles):
    # the recycled posterior mean lands near the simulation truth (0.85, 0.20)
    w = I.workload("sir_t30_n1024")
    ctx = S.SMC2(S.make_config(w), w.y)
    stats = ctx.run(w.K)
    mean, logz, ess_sum = ctx.estimate()
    cov = ctx.estimate_cov()
    ctx.close()
    assert np.all(np.isfinite(mean)) and np.isfinite(logz)
    sd = np.sqrt(np.diag(cov))
    assert np.all(np.abs(mean - np.array(I.SIR_TRUTH)) < 0.05 + 4 * sd), (mean, sd)
    assert all(1.0 <= s[0]["ess"] <= w.N for s in stats)


def test_learned_proposal_on_the_papers_experiment(S):
    # At the paper's size the random walk (Sigma = 0.1 I) keeps the ESS near 1, so the
    # learned proposal's guard (ESS >= 2 (D + 1) in the previous population) never
    # passes and the run is the random walk's, bit for bit.  With N = 8192 the guard
    # passes in some iterations and the network's proposals raise the ESS.
    def run(w, proposal):
        ctx = S.SMC2(S.make_config(w, proposal=proposal), w.y)
        st = [s[0] for s in ctx.run(w.K)]
        mean, logz, ess = ctx.estimate()
        ctx.close()
        return st, mean, ess
    w = I.workload("sir_t30_n1024", seed=201)
    st_rw, m_rw, e_rw = run(w, I.PROP_RW)
    st_ml, m_ml, e_ml = run(w, I.PROP_MLP)
    assert all(s["mlp_used"] == 0 for s in st_ml)
    assert np.array_equal(m_rw, m_ml) and e_rw == e_ml
    wb = I.workload("sir_t30_n1024", N=8192, K=20, seed=101)
    st_rw, m_rw, e_rw = run(wb, I.PROP_RW)
    st_ml, m_ml, e_ml = run(wb, I.PROP_MLP)
    used = sum(s["mlp_used"] for s in st_ml)
    print(f"N=8192 K=20: random walk ESS sum {e_rw:.0f}; learned ESS sum {e_ml:.0f} ({used} iterations by the network)")
    assert used >= 1 and e_ml > 2 * e_rw


def test_mixed_smc2_posterior_mean_matches_quadrature(S):
    # mixed precision end to end (the FP32 sampler, the float ESS trigger) against the
    # posterior mean by quadrature of the exact likelihood of a 30-person population
    T = 10
    y = I.simulate_sir(T, 0.9, 0.3, 30.0, 3.0, seed=5)
    G = 24
    g = (np.arange(G) + 0.5) / G
    L = np.array([[sir_exact_loglik(b, c, 30.0, 3.0, y) for c in g] for b in g])
    W = np.exp(L - L.max())
    W /= W.sum()
    quad = np.array([(W.sum(axis=1) * g).sum(), (W.sum(axis=0) * g).sum()])
    w = I.workload("sir_t30_n1024", N=256, M=64, T=T, K=10, npop=30.0, i0=3.0)
    ctx = S.SMC2(S.make_config(w), y)
    est = []
    for s in range(24):
        ctx.reset(300 + s)
        ctx.run(w.K, stats=False)
        est.append(ctx.estimate()[0][:2])
    ctx.close()
    est = np.array(est)
    se = est.std(axis=0, ddof=1) / math.sqrt(len(est))
    assert np.all(np.abs(est.mean(axis=0) - quad) < 4 * se + 2e-3), (est.mean(axis=0), quad, se)
