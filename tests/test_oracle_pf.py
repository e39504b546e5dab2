"""Pins of the oracle's bootstrap particle filter (Sec. II).

* linear-Gaussian AR(1): the likelihood estimate of Eq. (8) is unbiased for
  the Kalman-filter likelihood, and close to it for many particles;
* special cases where every particle carries the same state, so the estimate
  is exact: LG with phi = 0 and sigma_x = 0, and the SEIR-type model with a
  frozen log beta, checked against scipy's normal and Poisson densities."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2311_12973_gb300 import inputs as I


def lg_cfg(M, T, seed=1):
    w = I.workload("lg_t50_n64")
    return O.config_from(w, M=M, T=T, N=1, seed=seed), w.y[:T]


def test_lg_unbiased_for_kalman_likelihood():
    cfg, y = lg_cfg(M=64, T=20)
    theta = np.array([0.8, math.log(0.5), math.log(1.0)])
    kf = O.kalman_loglik(0.8, 0.5, 1.0, y)
    R = 400
    r = np.array([math.exp(O.pf_loglik(cfg, theta, y, k=1 + s // 64, i=s % 64) - kf) for s in range(R)])
    assert abs(r.mean() - 1.0) < 4 * r.std() / math.sqrt(R)


@pytest.mark.parametrize("theta", [(0.8, math.log(0.5), 0.0), (0.3, math.log(1.2), math.log(0.6))])
def test_lg_many_particles_close_to_kalman(theta):
    cfg, y = lg_cfg(M=8192, T=50)
    kf = O.kalman_loglik(theta[0], math.exp(theta[1]), math.exp(theta[2]), y)
    ll = O.pf_loglik(cfg, np.array(theta), y, k=1, i=0)
    assert abs(ll - kf) < 0.1


def test_lg_degenerate_exact():
    # phi = 0 and sigma_x = 0: x_t = 0 for t >= 1 in every particle
    cfg, y = lg_cfg(M=32, T=30)
    sy = 0.7
    theta = np.array([0.0, -np.inf, math.log(sy)])
    ll, delta, anc = O.pf_loglik(cfg, theta, y, k=3, i=5, trace=True)
    want = stats.norm(0.0, sy).logpdf(y)
    np.testing.assert_allclose(delta, want, rtol=1e-13, atol=1e-13)
    assert ll == pytest.approx(want.sum(), rel=1e-13)


def test_seir_frozen_beta_exact():
    w = I.workload("seir_t100_n1024")
    T = 60
    cfg = O.config_from(w, M=16, T=T, N=1)
    y = w.y[:T]
    beta0, kappa, gamma = 0.55, 0.22, 0.21
    theta = np.array([math.log(beta0), -np.inf, math.log(kappa), math.log(gamma)])
    lam = I.seir_constant_beta_incidence(T, beta0, kappa, gamma, w.npop, w.e0, w.i0, w.n_sub,
                                         w.lambda_floor)
    want = stats.poisson(lam).logpmf(y)
    ll, delta, _ = O.pf_loglik(cfg, theta, y, k=1, i=0, trace=True)
    np.testing.assert_allclose(delta, want, rtol=1e-11, atol=1e-9)
    assert ll == pytest.approx(want.sum(), rel=1e-11)


def test_trace_consistency():
    cfg, y = lg_cfg(M=16, T=12)
    theta = np.array([0.5, -0.5, 0.1])
    ll, delta, anc = O.pf_loglik(cfg, theta, y, k=2, i=7, trace=True)
    assert ll == pytest.approx(delta.sum(), rel=1e-13)
    assert anc.shape == (11, 16)
    assert np.all(np.diff(anc, axis=1) >= 0) and anc.min() >= 0 and anc.max() < 16
    # same key, same result; another filter index, another stream
    assert O.pf_loglik(cfg, theta, y, k=2, i=7) == ll
    assert O.pf_loglik(cfg, theta, y, k=2, i=8) != ll


def test_zero_likelihood_filter():
    cfg, y = lg_cfg(M=8, T=5)
    ll = O.pf_loglik(cfg, np.array([0.5, 0.0, np.nan]), y, k=1, i=0)
    assert ll == -np.inf
