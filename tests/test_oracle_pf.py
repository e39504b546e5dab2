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


# ---------------------------------------------------------------------------
# the paper's own PF resampling: multinomial, when the ESS (Eq. 12) drops below M/2
# ---------------------------------------------------------------------------

def test_multinomial_slots_follow_their_definition():
    """Slot j takes the first i with C_i > floor((2 U_j + 1) S / 2^33): checked in
    Python integers, including zero weights and a dominant weight."""
    rng = np.random.default_rng(11)
    for n in (1, 7, 64, 300):
        q = rng.integers(0, 2 ** 40, size=n, dtype=np.uint64)
        q[rng.random(n) < 0.3] = 0
        q[0] = max(int(q[0]), 1)
        U = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
        anc = O.multinomial_from_q(q, U)
        S = sum(int(v) for v in q)
        C = np.cumsum([int(v) for v in q], dtype=object)
        for j in range(n):
            tau = ((2 * int(U[j]) + 1) * S) >> 33
            assert anc[j] == next(i for i in range(n) if C[i] > tau)
            assert q[anc[j]] > 0                      # a zero weight is never drawn


def test_multinomial_draws_in_proportion_to_the_weights():
    rng = np.random.default_rng(12)
    q = np.array([1, 0, 5, 2, 8, 0, 3, 1], dtype=np.uint64) << np.uint64(40)
    draws = 20000
    U = rng.integers(0, 2 ** 32, size=draws, dtype=np.uint64).astype(np.uint32)
    counts = np.zeros(len(q))
    for c0 in range(0, draws, len(q)):
        a = O.multinomial_from_q(q, U[c0:c0 + len(q)])
        np.add.at(counts, a, 1)
    p = q.astype(float) / q.astype(float).sum()
    se = np.sqrt(draws * p * (1 - p))
    assert np.all(np.abs(counts - draws * p) < 4 * se + 1e-9)


def test_ess_of_integer_weights():
    from fractions import Fraction
    rng = np.random.default_rng(13)
    for n in (1, 5, 512):
        q = rng.integers(1, 2 ** 52, size=n, dtype=np.uint64)
        S = sum(int(v) for v in q)
        exact = Fraction(S * S, sum(int(v) ** 2 for v in q))
        assert O.ess_from_q(q) == pytest.approx(float(exact), rel=4e-16)
    assert O.ess_from_q(np.full(64, 2 ** 45, dtype=np.uint64)) == 64.0   # equal weights
    one = np.zeros(64, dtype=np.uint64)
    one[5] = 2 ** 52
    assert O.ess_from_q(one) == 1.0                                      # one survivor


@pytest.mark.parametrize("scheme,frac", [(O.PF_SYSTEMATIC, 0.5), (O.PF_MULTINOMIAL, 0.5), (O.PF_MULTINOMIAL, 0.0)])
def test_adaptive_and_multinomial_pf_unbiased_for_kalman_likelihood(scheme, frac):
    cfg, y = lg_cfg(M=64, T=20)
    cfg = O.Config(**{**cfg.__dict__, "pf_scheme": scheme, "pf_ess_frac": frac})
    theta = np.array([0.8, math.log(0.5), math.log(1.0)])
    kf = O.kalman_loglik(0.8, 0.5, 1.0, y)
    R = 400
    r = np.array([math.exp(O.pf_loglik(cfg, theta, y, k=1 + s // 64, i=s % 64) - kf) for s in range(R)])
    assert abs(r.mean() - 1.0) < 4 * r.std() / math.sqrt(R)


def test_adaptive_schedule_keeps_weights_between_resampling_events():
    """With the ESS trigger a step either resamples (ancestors of systematic
    resampling, non-decreasing) or keeps every particle (identity), and the
    increments still add up to the estimate.  With uninformative observations
    (a huge sigma_y) the weights stay flat and no step resamples."""
    cfg, y = lg_cfg(M=32, T=15)
    cfg = O.Config(**{**cfg.__dict__, "pf_ess_frac": 0.5})
    theta = np.array([0.5, -0.5, -0.5])
    ll, delta, anc = O.pf_loglik(cfg, theta, y, k=1, i=3, trace=True)
    assert ll == pytest.approx(delta.sum(), rel=1e-13)
    ident = np.arange(32)
    kept = [np.array_equal(a, ident) for a in anc]
    assert any(kept) and not all(kept)
    for a in anc:
        assert np.all(np.diff(a) >= 0)
    flat = np.array([0.5, -0.5, 8.0])
    _, _, anc_flat = O.pf_loglik(cfg, flat, y, k=1, i=3, trace=True)
    assert all(np.array_equal(a, ident) for a in anc_flat)
