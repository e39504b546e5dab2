"""Oracle pins for the binomial SIR model of Sec. V-A.

* The binomial sampler against the exact binomial pmf (scipy) in every regime
  (inversion, transformed rejection, the p > 1/2 mirror), its edge cases and
  the number of words it reads.
* The particle filter on the SIR model against the exact likelihood: with a
  population of 30 the state (S, I) has 496 values, so the forward algorithm
  of the hidden Markov chain (scipy pmfs) gives p(y_{1:T} | theta) exactly;
  the filter's estimate must be unbiased for it (Sec. II) and close to it at
  large M, for every resampling scheme; and the whole SMC^2 run's posterior
  mean must agree with quadrature of that likelihood over the prior's box.
* The uniform prior: density, support, and the k = 1 draws."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2311_12973_gb300 import inputs as I


def _draws(n, p, count, seed=11, c3=O.TAG_PF_BINOM | (3 << 4)):
    return np.array([O.binomial(n, p, seed, j % 4096, j // 4096, 5, c3) for j in range(count)])


def _chi2_pvalue(k, n, p):
    """Goodness of fit of the draws k to Bin(n, p), cells with >= 20 expected."""
    R = len(k)
    lo, hi = int(stats.binom.ppf(1e-7, n, p)), int(stats.binom.isf(1e-7, n, p))
    edges = [lo]
    acc = 0.0
    for v in range(lo, hi + 1):
        acc += R * stats.binom.pmf(v, n, p)
        if acc >= 20.0:
            edges.append(v + 1)
            acc = 0.0
    edges[-1] = hi + 1
    obs, exp = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        lo_c = -1 if a == edges[0] else a - 1
        hi_c = n if b == edges[-1] else b - 1
        obs.append(np.sum((k > lo_c) & (k <= hi_c)))
        exp.append(R * (stats.binom.cdf(hi_c, n, p) - stats.binom.cdf(lo_c, n, p)))
    obs, exp = np.array(obs, dtype=float), np.array(exp)
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    return stats.chi2.sf(chi2, len(obs) - 1)


@pytest.mark.parametrize("n,p", [
    (10, 0.3), (1000, 0.002), (19, 0.5), (3, 0.9),        # inversion (n min(p, 1-p) < 10)
    (20, 0.5), (1000, 0.3), (10000, 0.5), (40, 0.26),     # transformed rejection
    (9997, 0.92), (30, 0.8), (4431, 0.181),               # mirror, and an SIR-sized recovery flow
])
def test_binomial_matches_pmf(n, p):
    k = _draws(n, p, 40000)
    assert np.all((k >= 0) & (k <= n)) and np.all(k == np.floor(k))
    assert _chi2_pvalue(k, n, p) > 1e-4
    # the mean within 4 standard errors
    assert abs(k.mean() - n * p) < 4 * math.sqrt(n * p * (1 - p) / len(k))


def test_binomial_edge_cases():
    args = (7, 1, 2, 3, 9)
    assert O.binomial(0, 0.3, *args) == 0
    assert O.binomial(50, 0.0, *args) == 0
    assert O.binomial(50, -0.2, *args) == 0          # a probability below 0 acts as 0
    assert O.binomial(50, float("nan"), *args) == 0
    assert O.binomial(50, 1.0, *args) == 50
    assert O.binomial(50, 1.7, *args) == 50
    assert O.binomial(1, 0.5, *args) in (0, 1)


def test_binomial_mirror_and_word_use():
    # p > 1/2 reads the same words as 1 - p and returns n minus that draw
    for j in range(200):
        a = O.binomial(500, 0.93, 5, j, 2, 1, 9)
        b = O.binomial(500, 1.0 - 0.93, 5, j, 2, 1, 9)
        assert a == 500 - b
    # inversion reads one word; the rejection method two per proposal
    for j in range(200):
        _, w = O.binomial(30, 0.1, 5, j, 1, 1, 9, words=True)
        assert w == 1
        _, w = O.binomial(3000, 0.1, 5, j, 1, 1, 9, words=True)
        assert w >= 2 and w % 2 == 0


def test_binomial_rejection_rate():
    # the squeeze accepts most proposals: about 1.1 proposals per draw for large n p
    used = [O.binomial(10000, 0.3, 5, j, 1, 1, 9, words=True)[1] for j in range(4000)]
    assert 2.0 <= np.mean(used) / 1.0 <= 2.6


# ---------------------------------------------------------------------------
# SIR particle filter against the exact forward algorithm
# ---------------------------------------------------------------------------

def sir_exact_loglik(beta, gamma, npop, i0, y):
    """log p(y_{1:T} | beta, gamma) by the forward algorithm over all (S, I)
    with S + I <= npop: the one-day transition matrix from the two binomial
    laws (scipy pmfs), then alpha_t = (alpha_{t-1} T) * Poisson(y_t; I)."""
    n = int(npop)
    S_idx, I_idx = np.nonzero(np.add.outer(np.arange(n + 1), np.arange(n + 1)) <= n)
    index = -np.ones((n + 1, n + 1), dtype=int)
    index[S_idx, I_idx] = np.arange(len(S_idx))
    k = np.arange(n + 1)
    # pa[I][S, u]: u of S susceptibles infected; pb[I][v]: v of I infected recover
    pa = [stats.binom.pmf(k[None, :], k[:, None], -math.expm1(-beta * Ic / npop)) for Ic in range(n + 1)]
    pb = [stats.binom.pmf(np.arange(Ic + 1), Ic, -math.expm1(-gamma)) for Ic in range(n + 1)]
    trans = np.zeros((len(S_idx), len(S_idx)))
    for s, (S, Ic) in enumerate(zip(S_idx, I_idx)):
        u = np.arange(S + 1)[:, None]
        v = np.arange(Ic + 1)[None, :]
        dest = index[np.broadcast_to(S - u, (S + 1, Ic + 1)), Ic + u - v]  # (S - u, I + u - v)
        np.add.at(trans[s], dest, pa[Ic][S, :S + 1][:, None] * pb[Ic][None, :])
    alpha = np.zeros(len(S_idx))
    alpha[index[n - int(i0), int(i0)]] = 1.0
    ll = 0.0
    for yt in y:
        alpha = alpha @ trans
        lik = stats.poisson.pmf(yt, I_idx.astype(float))
        lik[I_idx == 0] = 1.0 if yt == 0 else 0.0
        alpha = alpha * lik
        tot = alpha.sum()
        ll += math.log(tot)
        alpha /= tot
    return ll


def one_day_likelihood(npop, i0, beta, gamma, y):
    """p(y_1 | theta) after one day from (npop - i0, i0): the S->I and I->R flows
    are independent binomials, so I_1 = i0 + a - b has the convolution of their
    pmfs, and p(y_1) = sum over I_1 of Poisson(y_1; I_1) P(I_1)."""
    S0, I0 = int(npop - i0), int(i0)
    pa = stats.binom.pmf(np.arange(S0 + 1), S0, -math.expm1(-beta * I0 / npop))
    pb = stats.binom.pmf(np.arange(I0 + 1), I0, -math.expm1(-gamma))
    dist = np.convolve(pa, pb[::-1])  # index a + (I0 - b) = I_1
    return float(np.sum(dist * stats.poisson.pmf(y, np.arange(len(dist)))))


# (npop, i0, beta, gamma): both flows by rejection; S->I by rejection and I->R
# by inversion; the I->R flow with p > 1/2 (the mirror)
ONE_DAY = [(1e4, 2000.0, 0.9, 0.2), (1e4, 20.0, 0.9, 0.2), (1e4, 2000.0, 0.9, 1.5)]


@pytest.mark.parametrize("npop,i0,beta,gamma", ONE_DAY)
def test_one_day_filter_unbiased(npop, i0, beta, gamma):
    # E[p^] = p(y_1 | theta) for y_1 in the bulk and the tails of the one-day law
    w = I.workload("sir_t30_n1024", N=1, M=256, T=1, npop=npop, i0=i0, precision=I.PREC_FP64)
    cfg = O.config_from(w)
    S0, I0 = npop - i0, i0
    mean = I0 + S0 * -math.expm1(-beta * I0 / npop) - I0 * -math.expm1(-gamma)
    for z in (-2.0, 0.0, 1.5):
        y = np.array([max(0.0, round(mean + z * math.sqrt(mean + 1.0) * 1.3))])
        exact = one_day_likelihood(npop, i0, beta, gamma, y[0])
        r = np.array([math.exp(O.pf_loglik(cfg, np.array([beta, gamma]), y, k=1, i=s) - math.log(exact))
                      for s in range(200)])
        assert abs(r.mean() - 1.0) < 4 * r.std() / math.sqrt(len(r)), (z, r.mean(), r.std())


def small_sir(T=10, beta=0.9, gamma=0.3, npop=30.0, i0=3.0, seed=5, **over):
    y = I.simulate_sir(T, beta, gamma, npop, i0, seed=seed)
    w = I.workload("sir_t30_n1024", N=1, M=64, T=T, npop=npop, i0=i0, precision=I.PREC_FP64)
    cfg = O.config_from(w, **over)
    return cfg, y, np.array([beta, gamma])


@pytest.mark.parametrize("scheme,frac", [(O.PF_SYSTEMATIC, 0.0), (O.PF_MULTINOMIAL, 0.5),
                                         (O.PF_MULTINOMIAL, 0.0), (O.PF_SYSTEMATIC, 0.5)])
def test_sir_pf_unbiased_for_exact_likelihood(scheme, frac):
    cfg, y, th = small_sir(pf_scheme=scheme, pf_ess_frac=frac)
    exact = sir_exact_loglik(th[0], th[1], cfg.npop, cfg.i0, y)
    R = 400
    r = np.array([math.exp(O.pf_loglik(cfg, th, y, k=1 + s // 100, i=s % 100) - exact) for s in range(R)])
    assert abs(r.mean() - 1.0) < 4 * r.std() / math.sqrt(R), (r.mean(), r.std())


@pytest.mark.parametrize("theta", [(0.9, 0.3), (0.4, 0.6), (1.5, 0.1)])
def test_sir_pf_converges_to_exact(theta):
    # log p^ has variance ~ c / M and bias ~ -var / 2 (it is the log of an
    # unbiased estimate): 12 filters at M = 4096 average within 4 SE plus that
    # bias of the exact value, and the spread shrinks with M like M^-1/2.
    cfg, y, _ = small_sir()
    exact = sir_exact_loglik(theta[0], theta[1], cfg.npop, cfg.i0, y)
    sd = {}
    for M in (1024, 4096):
        cfg.M = M
        e = np.array([O.pf_loglik(cfg, np.array(theta), y, k=2, i=i) for i in range(12)])
        sd[M] = e.std(ddof=1)
    assert abs(e.mean() - exact) < 4 * sd[4096] / math.sqrt(12) + 0.5 * sd[4096] ** 2, (e.mean(), exact)
    assert sd[4096] < 0.75 * sd[1024]


def test_sir_pf_degenerate_data_gives_minus_inf():
    # more infected observed than the population can hold never has weight
    cfg, y, th = small_sir()
    y = y.copy()
    y[:] = 0.0
    y[3] = 1e4
    ll = O.pf_loglik(cfg, th, y, k=1, i=0)
    assert ll < -1e3 or ll == -np.inf


def test_sir_frozen_dynamics_exact():
    # beta = 0 and gamma = 0: nobody moves, I_t = i0, so log p = sum_t log Poisson(y_t; i0)
    cfg, y, _ = small_sir()
    ll = O.pf_loglik(cfg, np.array([0.0, 0.0]), y, k=1, i=0)
    assert ll == pytest.approx(float(np.sum(stats.poisson.logpmf(y, cfg.i0))), rel=1e-13)


def test_sir_smc2_posterior_mean_matches_quadrature():
    # The whole outer sampler on the SIR model with the uniform prior (zero-weight
    # proposals outside [0, 1]^2 included): the recycled posterior mean of 12 runs
    # against the posterior mean by midpoint quadrature of the exact likelihood
    # over a 24 x 24 grid (the posterior sd is 0.13 and 0.06, many cells wide).
    T = 10
    y = I.simulate_sir(T, 0.9, 0.3, 30.0, 3.0, seed=5)
    G = 24
    g = (np.arange(G) + 0.5) / G
    L = np.array([[sir_exact_loglik(b, c, 30.0, 3.0, y) for c in g] for b in g])
    W = np.exp(L - L.max())
    W /= W.sum()
    quad = np.array([(W.sum(axis=1) * g).sum(), (W.sum(axis=0) * g).sum()])
    w = I.workload("sir_t30_n1024", N=256, M=64, T=T, K=10, npop=30.0, i0=3.0, precision=I.PREC_FP64)
    est = np.array([O.SMC2(O.config_from(w, seed=100 + s), y).run(w.K).recycled()[0] for s in range(12)])
    se = est.std(axis=0, ddof=1) / math.sqrt(len(est))
    assert np.all(np.abs(est.mean(axis=0) - quad) < 4 * se + 2e-3), (est.mean(axis=0), quad, se)


# ---------------------------------------------------------------------------
# uniform prior
# ---------------------------------------------------------------------------

def test_uniform_prior_density_and_support():
    w = I.workload("sir_t30_n1024", prior_lo=[0.0, -1.0], prior_hi=[1.0, 3.0])
    cfg = O.config_from(w)
    c = cfg.ctype()
    lp = lambda th: O.lib().oracle_log_prior(c, np.ascontiguousarray(th, dtype=np.float64).ctypes.data_as(
        O.C.POINTER(O.C.c_double)))
    assert lp([0.5, 0.0]) == pytest.approx(-math.log(4.0), rel=1e-15)
    assert lp([0.0, -1.0]) == pytest.approx(-math.log(4.0))        # closed support
    assert lp([1.0000001, 0.0]) == -np.inf
    assert lp([0.5, -1.5]) == -np.inf


def test_uniform_prior_initial_draws():
    # k = 1 draws theta from the prior (Eq. 16); no resampling so the draws survive
    w = I.workload("sir_t30_n1024", N=2048, M=1, T=1, ess_frac=0.0, prior_lo=[0.2, -1.0],
                   prior_hi=[0.7, 3.0], precision=I.PREC_FP64)
    ref = O.SMC2(O.config_from(w), w.y).run(1)
    th = ref.theta
    for d, (lo, hi) in enumerate(zip(w.prior_lo, w.prior_hi)):
        assert np.all((th[:, d] > lo) & (th[:, d] < hi))
        assert stats.kstest((th[:, d] - lo) / (hi - lo), "uniform").pvalue > 1e-3
    # w_1 = pi / q_1 = p^(y | theta): the weights are the likelihood estimates
    assert np.allclose(ref.logw, ref.loglik, rtol=0, atol=1e-12 * np.max(np.abs(ref.loglik)))
