"""Pins of the oracle's approximately optimal L-kernel (Sec. IV-D, Eqs. 32-35).

The conditional Gaussian density is checked against the identity
log N([a;b]; mu, Sigma) - log N(b; mu_b, Sigma_bb) = log N(a; mu_{a|b}(b), Sigma_{a|b}),
both sides of which scipy evaluates from the fitted joint moments; the
moments against numpy's weighted average and covariance."""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O


def population(rng, N, D, corr=0.8):
    a = rng.standard_normal((N, D)) @ np.diag(rng.uniform(0.3, 2.0, D)) + rng.standard_normal(D)
    b = corr * a + 0.3 * rng.standard_normal((N, D)) + 0.5
    w = rng.random(N) ** 3
    return a, b, w / w.sum()


@pytest.mark.parametrize("D", [1, 3, 4])
def test_moments_match_numpy(D):
    rng = np.random.default_rng(D)
    a, b, w = population(rng, 500, D)
    fit = O.lkernel_fit(a, b, w)
    z = np.concatenate([a, b], axis=1)
    np.testing.assert_allclose(fit["mu"], np.average(z, axis=0, weights=w), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(fit["sigma"], np.cov(z.T, aweights=w, bias=True), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("D", [1, 2, 4])
def test_conditional_density_identity(D):
    rng = np.random.default_rng(10 + D)
    a, b, w = population(rng, 400, D)
    fit = O.lkernel_fit(a, b, w)
    assert fit["fallback"] == 0
    mu, sig = fit["mu"], fit["sigma"]
    joint = stats.multivariate_normal(mu, sig)
    marg_b = stats.multivariate_normal(mu[D:], sig[D:, D:])
    for i in range(10):
        want = joint.logpdf(np.concatenate([a[i], b[i]])) - marg_b.logpdf(b[i])
        assert O.lkernel_logpdf(fit, a[i], b[i]) == pytest.approx(want, rel=1e-9, abs=1e-9)


def test_independent_pairs_reduce_to_marginal():
    # full factorial of 3 parent points x 3 proposal points, uniform weights:
    # the weighted cross-covariance is exactly zero, so L(a|b) = N(a; mu_a, Sigma_aa)
    D = 2
    pa = np.array([[1.0, 2.0], [-1.0, 0.5], [0.5, -2.0]])
    pb = np.array([[0.3, 1.0], [1.0, -0.4], [-0.6, 0.2]])
    a = np.repeat(pa, 3, axis=0)
    b = np.tile(pb, (3, 1))
    w = np.full(9, 1.0 / 9)
    fit = O.lkernel_fit(a, b, w)
    assert fit["fallback"] == 0
    np.testing.assert_allclose(fit["A"], 0.0, atol=1e-14)
    saa = np.cov(pa.T, bias=True)
    for i in range(9):
        want = stats.multivariate_normal(pa.mean(axis=0), saa).logpdf(a[i])
        assert O.lkernel_logpdf(fit, a[i], b[i]) == pytest.approx(want, rel=1e-12)


def test_singular_fit_falls_back():
    D = 3
    a = np.tile(np.array([[0.1, 0.2, 0.3]]), (50, 1))   # every parent identical
    b = a + np.random.default_rng(0).standard_normal((50, D)) * 0.1
    fit = O.lkernel_fit(a, b, np.full(50, 1 / 50))
    assert fit["fallback"] == 1
