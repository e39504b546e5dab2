"""Pins of the oracle's SMC^2 outer sampler (Sec. IV).

* Eq. (31): with the forward L-kernel and a symmetric random walk, the
  weight update of Eq. (20) reduces to the ratio of targets;
* Eq. (20) with the Gaussian L-kernel, assembled from densities scipy evaluates;
* normalisation, ESS, evidence, resampling and recycling invariants;
* statistical: against a 64^3 quadrature of the exact (Kalman) posterior of
  the linear-Gaussian model, the evidence estimate with a fixed (forward)
  L-kernel is unbiased and the recycled posterior mean is within 4 Monte
  Carlo standard errors for both L-kernels."""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.special import logsumexp

from oracle import oracle as O
from paper_2311_12973_gb300 import inputs as I


def lg(T=10, **kw):
    w = I.workload("lg_t50_n64", T=T)
    return O.config_from(w, **kw), w.y


def start_population(cfg, y, seed=0):
    """A weighted population (no resampling at k=1) to step from."""
    c = O.Config(**{**cfg.__dict__, "ess_frac": 0.0, "seed": seed})
    s = O.SMC2(c, y)
    s.step()
    return s


def test_k1_weights_are_the_likelihood_and_stats_are_consistent():
    cfg, y = lg(N=64, M=32)
    s = O.SMC2(O.Config(**{**cfg.__dict__, "ess_frac": 0.0}), y)
    st = s.step()
    np.testing.assert_allclose(s.logw, s.loglik, rtol=1e-13, atol=1e-12)
    lse = logsumexp(s.logw)
    assert st["lse"] == pytest.approx(lse, rel=1e-13)
    assert st["lse2"] == pytest.approx(logsumexp(2 * s.logw), rel=1e-13)
    assert st["ess"] == pytest.approx(math.exp(2 * lse - logsumexp(2 * s.logw)), rel=1e-11)
    assert st["logz"] == pytest.approx(lse - math.log(64), rel=1e-13)
    assert 1.0 <= st["ess"] <= 64.0
    wn = np.exp(s.logw - lse)
    np.testing.assert_allclose(st["est"], wn @ s.theta, rtol=1e-12)
    # Eq. (21) with f = (theta - f~)(theta - f~)^T: numpy's weighted covariance (no Bessel correction)
    np.testing.assert_allclose(st["cov"], np.cov(s.theta.T, aweights=wn, bias=True), rtol=1e-10, atol=1e-14)
    for d in range(3):
        assert s.theta[:, d].min() <= st["est"][d] <= s.theta[:, d].max()
    for i in range(0, 64, 9):
        assert s.logprior[i] == pytest.approx(stats.norm.logpdf(s.theta[i]).sum(), rel=1e-13)


def test_resampling_resets_to_mean_weight():
    cfg, y = lg(N=128, M=32, ess_frac=1.01)   # always resample
    s = O.SMC2(cfg, y)
    st = s.step()
    assert st["resampled"] == 1
    np.testing.assert_array_equal(s.logw, np.full(128, st["lse"] - math.log(128)))
    # the carried (theta, log prior, log likelihood) are copies of proposals
    for i in range(128):
        j = np.flatnonzero(np.all(s.theta == s.theta[i], axis=1))
        assert np.all(s.loglik[j] == s.loglik[i]) and np.all(s.logprior[j] == s.logprior[i])
    assert logsumexp(s.logw) == pytest.approx(st["lse"], rel=1e-13)   # evidence kept


def test_forward_kernel_reduces_to_target_ratio():
    cfg, y = lg(N=32, M=32, lkernel=O.LK_FORWARD)
    s = start_population(cfg, y)
    old = (s.theta.copy(), s.logprior.copy(), s.loglik.copy(), s.logw.copy())
    st = s.step()
    assert st["resampled"] == 0
    d_target = (s.logprior + s.loglik) - (old[1] + old[2])
    np.testing.assert_allclose(s.logw - old[3], d_target, rtol=1e-12, atol=1e-10)   # Eq. (31)
    step = (s.theta - old[0]) / cfg.rw_scale
    assert np.all(np.abs(step) < 6.0)


def test_gauss_kernel_weight_update():
    cfg, y = lg(N=64, M=32, lkernel=O.LK_GAUSS)
    s = start_population(cfg, y, seed=3)
    th0, lp0, ll0, lw0 = s.theta.copy(), s.logprior.copy(), s.loglik.copy(), s.logw.copy()
    st = s.step()
    assert st["lk_fallback"] == 0
    wn = np.exp(lw0 - logsumexp(lw0))
    fit = O.lkernel_fit(th0, s.theta, wn)
    D = 3
    mu, sig = fit["mu"], fit["sigma"]
    joint = stats.multivariate_normal(mu, sig)
    marg = stats.multivariate_normal(mu[D:], sig[D:, D:])
    for i in range(64):
        logL = joint.logpdf(np.concatenate([th0[i], s.theta[i]])) - marg.logpdf(s.theta[i])
        logq = stats.multivariate_normal(th0[i], cfg.rw_scale**2 * np.eye(D)).logpdf(s.theta[i])
        want = lw0[i] + (s.logprior[i] + s.loglik[i]) - (lp0[i] + ll0[i]) + logL - logq   # Eq. (20)
        assert s.logw[i] == pytest.approx(want, rel=1e-9, abs=1e-8)


def test_recycling_constants():
    cfg, y = lg(N=64, M=32)
    s = O.SMC2(cfg, y).run(5)
    est, ck = s.recycled()
    ess = np.array([st["ess"] for st in s.stats])
    np.testing.assert_allclose(ck, ess / ess.sum(), rtol=1e-14)                   # Eq. (23)
    assert ck.sum() == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose(est, sum(c * st["est"] for c, st in zip(ck, s.stats)), rtol=1e-13)
    for st in s.stats:
        assert st["resampled"] == int(st["ess"] < 0.5 * 64)


# ---------------------------------------------------------------------------
# statistical pins against the exact posterior of the linear-Gaussian model
# ---------------------------------------------------------------------------

def test_recycled_covariance_is_the_recycled_second_moment():
    """Eq. (29) applied to theta theta^T: with c_k from the ESS of each
    iteration, the recycled covariance equals the c-weighted mixture of the
    iterations' weighted populations, which numpy computes from the pooled
    (theta, c_k w~) pairs."""
    cfg, y = lg(N=48, M=16)
    c = O.Config(**{**cfg.__dict__, "ess_frac": 0.0})  # never resample: each state is the weighted population
    s = O.SMC2(c, y)
    pooled_th, pooled_w = [], []
    for _ in range(4):
        st = s.step()
        wn = np.exp(s.logw - logsumexp(s.logw))
        pooled_th.append(s.theta.copy())
        pooled_w.append(st["ess"] * wn)
    th = np.concatenate(pooled_th)
    wt = np.concatenate(pooled_w)
    mean, _ = s.recycled()
    np.testing.assert_allclose(mean, wt @ th / wt.sum(), rtol=1e-12)
    np.testing.assert_allclose(s.recycled_cov(), np.cov(th.T, aweights=wt, bias=True), rtol=1e-10, atol=1e-14)


def _quadrature(y, n, lo, hi):
    g = [np.linspace(lo[d], hi[d], n) for d in range(3)]
    P, LX, LY = np.meshgrid(*g, indexing="ij")
    ll = np.array([O.kalman_loglik(p, math.exp(a), math.exp(b), y)
                   for p, a, b in zip(P.ravel(), LX.ravel(), LY.ravel())]).reshape(P.shape)
    lj = ll + stats.norm.logpdf(P) + stats.norm.logpdf(LX) + stats.norm.logpdf(LY)
    cell = np.prod([(hi[d] - lo[d]) / (n - 1) for d in range(3)])
    w = np.exp(lj - lj.max())
    w /= w.sum()
    mean = np.array([(w * X).sum() for X in (P, LX, LY)])
    sd = np.array([math.sqrt((w * (X - m) ** 2).sum()) for X, m in zip((P, LX, LY), mean)])
    return logsumexp(lj) + math.log(cell), mean, sd


@pytest.mark.slow
def test_recycled_posterior_variance_matches_quadrature(exact_posterior):
    """The recycled covariance's diagonal against the exact posterior variances."""
    y, _, _, sd = exact_posterior
    cfg, _ = lg(N=256, M=64, lkernel=O.LK_GAUSS)
    R = 24
    var = np.array([np.diag(O.SMC2(O.Config(**{**cfg.__dict__, "seed": 3000 + r}), y).run(10).recycled_cov())
                    for r in range(R)])
    se = var.std(axis=0) / math.sqrt(R)
    assert np.all(np.abs(var.mean(axis=0) - sd ** 2) < 4 * se + 0.05 * sd ** 2), (var.mean(axis=0), sd ** 2, se)


@pytest.fixture(scope="module")
def exact_posterior():
    y = I.workload("lg_t50_n64", T=10).y
    _, m, sd = _quadrature(y, 32, [-1.5, -4.0, -3.0], [1.5, 2.0, 1.5])
    return (y,) + _quadrature(y, 64, m - 7 * sd, m + 7 * sd)


@pytest.mark.slow
def test_evidence_unbiased_with_forward_kernel(exact_posterior):
    y, logz, _, _ = exact_posterior
    cfg, _ = lg(N=128, M=64, lkernel=O.LK_FORWARD)
    R, K = 40, 5
    ratio = np.zeros((R, K))
    for r in range(R):
        c = O.Config(**{**cfg.__dict__, "seed": 1000 + r})
        s = O.SMC2(c, y).run(K)
        ratio[r] = [math.exp(st["logz"] - logz) for st in s.stats]
    mean, se = ratio.mean(axis=0), ratio.std(axis=0) / math.sqrt(R)
    assert np.all(np.abs(mean - 1.0) < 4 * se), (mean, se)


@pytest.mark.slow
@pytest.mark.parametrize("lk", [O.LK_FORWARD, O.LK_GAUSS])
def test_recycled_posterior_mean_matches_quadrature(exact_posterior, lk):
    y, _, mean, _ = exact_posterior
    cfg, _ = lg(N=256, M=64, lkernel=lk)
    R = 24
    est = np.array([O.SMC2(O.Config(**{**cfg.__dict__, "seed": 2000 + r}), y).run(10).recycled()[0]
                    for r in range(R)])
    se = est.std(axis=0) / math.sqrt(R)
    assert np.all(np.abs(est.mean(axis=0) - mean) < 4 * se), (est.mean(axis=0), mean, se)
