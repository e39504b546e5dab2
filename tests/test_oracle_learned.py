"""Pins of the oracle's learned-proposal steps (not in the paper; the
builder's choices L2-L4): the training set's standardisation, the training
call, the surrogate's score, the population factor and the decision rule, and
the preconditioned Langevin proposal with its exact density.

Each is fixed by something other than the oracle: moment invariants, affine
invariance, finite differences, scipy's Gaussian density, Monte Carlo moments
of the proposal, Adam's first-step closed form, and the network learning the
known score of a Gaussian target."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O


def _ring(rng, R=400, D=4, n_low=20, n_inf=5):
    """Rows near a Gaussian target: lp quadratic, some rows far below the clip, some -inf."""
    mu = rng.standard_normal(D)
    th = mu + rng.standard_normal((R, D)) * np.linspace(0.5, 1.5, D)
    lp = -0.5 * np.sum(((th - mu) / np.linspace(0.5, 1.5, D)) ** 2, axis=1) - 40.0
    lp[:n_low] -= 1e3
    lp[n_low:n_low + n_inf] = -np.inf
    return th, lp


def test_standardise_moments_and_clip():
    rng = np.random.default_rng(1)
    th, lp = _ring(rng)
    R, D = th.shape
    x, y, nm = O.mlp_standardise(th, lp)
    tau = max(2.0, D)
    assert nm["tau"] == tau and nm["ymax"] == np.max(lp[np.isfinite(lp)])
    above = np.isfinite(lp) & (lp > nm["ymax"] - 8 * tau)
    assert nm["rows_moments"] == above.sum() == R - 25
    # targets: mean 0, population sd 1 over all rows; clipped and -inf rows share the lowest value
    assert abs(y.mean()) < 1e-12 and abs(y.std() - 1.0) < 1e-12
    assert np.all(y[~above] == y.min()) and np.all(y[above] > y.min())
    # inputs: mean 0 and population sd 1 over the rows above the clip
    assert np.allclose(x[above].mean(axis=0), 0.0, atol=1e-12)
    assert np.allclose(x[above].std(axis=0), 1.0, atol=1e-12)
    assert nm["var_y"] == 1.0


def test_standardise_is_affine_invariant():
    rng = np.random.default_rng(2)
    th, lp = _ring(rng, n_inf=0)
    x, y, nm = O.mlp_standardise(th, lp)
    a, b = np.array([2.0, 0.5, 3.0, 1.5]), np.array([1.0, -2.0, 0.3, 5.0])
    x2, y2, nm2 = O.mlp_standardise(th * a + b, lp + 123.0)  # shifted log target, rescaled theta
    assert np.allclose(x2, x, atol=1e-10) and np.allclose(y2, y, atol=1e-12)
    assert np.allclose(nm2["mu"], a * nm["mu"] + b) and np.allclose(nm2["sd"], a * nm["sd"])
    assert math.isclose(nm2["zmean"], nm["zmean"], abs_tol=1e-12) and math.isclose(nm2["zsd"], nm["zsd"])


def test_standardise_few_rows_above_clip_uses_every_finite_row():
    rng = np.random.default_rng(3)
    D = 3
    th = rng.standard_normal((50, D))
    lp = np.full(50, -1e4)
    lp[:3] = [0.0, -1.0, -2.0]        # three rows above the clip: fewer than 2 D + 2
    lp[40:] = -np.inf
    x, y, nm = O.mlp_standardise(th, lp)
    fin = np.isfinite(lp)
    assert nm["rows_moments"] == fin.sum() == 40
    assert np.allclose(x[fin].mean(axis=0), 0.0, atol=1e-12)
    assert np.allclose(x[fin].std(axis=0), 1.0, atol=1e-12)


def test_standardise_constant_targets():
    th = np.random.default_rng(4).standard_normal((30, 2))
    x, y, nm = O.mlp_standardise(th, np.full(30, -3.5))
    assert nm["var_y"] == 0.0 and nm["zsd"] == 1.0 and np.all(y == 0.0)


def _params(rng, D, H=64):
    return rng.standard_normal(O.mlp_nparams(D, H)) * 0.3


def test_score_is_the_gradient_of_the_fitted_log_target():
    """The fitted log target is ymax + tau (zmean + zsd s((theta - mu)/sd)); its
    central finite differences give the score."""
    rng = np.random.default_rng(5)
    D = 4
    th, lp = _ring(rng, D=D, n_inf=0)
    _, _, nm = O.mlp_standardise(th, lp)
    p = _params(rng, D)
    pts = nm["mu"] + rng.standard_normal((6, D)) * nm["sd"]
    g = O.mlp_score(p, nm, pts, bf16_points=False)

    def f(t):
        x = (np.atleast_2d(t) - nm["mu"]) / nm["sd"]
        return nm["ymax"] + nm["tau"] * (nm["zmean"] + nm["zsd"] * O.mlp_forward(p, x))

    h = 1e-6
    for r in range(len(pts)):
        fd = np.array([(f(pts[r] + h * e)[0] - f(pts[r] - h * e)[0]) / (2 * h) for e in np.eye(D)])
        assert np.allclose(g[r], fd, rtol=1e-6, atol=1e-6 * np.max(np.abs(fd))), (g[r], fd)


def _lower(rng, D):
    A = rng.standard_normal((D, D)) * 0.4 + np.eye(D)
    return np.linalg.cholesky(A @ A.T + 0.1 * np.eye(D))


@pytest.mark.parametrize("D,h", [(2, 1.0), (4, 0.7), (8, 1.3)])
def test_langevin_density_against_scipy(D, h):
    rng = np.random.default_rng(6 + D)
    L = _lower(rng, D)
    a = rng.standard_normal(D)
    g = rng.standard_normal(D)
    mean, _ = O.langevin_propose(h, L, a, g, np.zeros(D))
    for _ in range(5):
        z = rng.standard_normal(D)
        b, lq = O.langevin_propose(h, L, a, g, z)
        ref = stats.multivariate_normal(mean=mean, cov=h * h * L @ L.T).logpdf(b)
        assert math.isclose(lq, ref, rel_tol=1e-12, abs_tol=1e-12), (lq, ref)


def test_langevin_moments_by_monte_carlo():
    rng = np.random.default_rng(8)
    D, h, n = 3, 0.8, 20000
    L = _lower(rng, D)
    a, g = rng.standard_normal(D), 0.5 * rng.standard_normal(D)
    mean, _ = O.langevin_propose(h, L, a, g, np.zeros(D))
    b = np.array([O.langevin_propose(h, L, a, g, rng.standard_normal(D))[0] for _ in range(n)])
    cov = h * h * L @ L.T
    se = np.sqrt(np.diag(cov) / n)
    assert np.all(np.abs(b.mean(axis=0) - mean) < 4 * se)
    assert np.allclose(np.cov(b.T), cov, atol=0.05 * np.max(np.abs(cov)))


def test_langevin_drift_is_half_h2_sigma_score():
    """Unclipped, the mean step is h^2/2 Sigma g with Sigma = L L^T (a transposed L
    or a missing 1/2 would break it)."""
    rng = np.random.default_rng(9)
    D, h = 4, 0.9
    L = _lower(rng, D)
    a, g = rng.standard_normal(D), 0.3 * rng.standard_normal(D)
    mean, _ = O.langevin_propose(h, L, a, g, np.zeros(D))
    assert np.allclose(mean - a, 0.5 * h * h * (L @ L.T) @ g, rtol=1e-12, atol=1e-14)


def test_langevin_drift_is_clipped_at_three_noise_sds():
    rng = np.random.default_rng(10)
    D, h = 3, 1.0
    L = _lower(rng, D)
    a, g = rng.standard_normal(D), 1e6 * rng.standard_normal(D)
    mean, lq = O.langevin_propose(h, L, a, g, np.zeros(D))
    w = 3.0 * np.sign(L.T @ g)
    assert np.allclose(mean - a, h * L @ w, rtol=1e-12)
    # the density at the mean: the Gaussian's peak
    ref = stats.multivariate_normal(mean=mean, cov=h * h * L @ L.T).logpdf(mean)
    assert math.isclose(lq, ref, rel_tol=1e-12)


def test_population_factor():
    rng = np.random.default_rng(11)
    D = 4
    A = rng.standard_normal((D, D))
    cov = A @ A.T + 0.01 * np.eye(D)
    L, ok = O.population_factor(cov, ess=2.0 * (D + 1))
    assert ok and np.allclose(L, np.linalg.cholesky(cov), rtol=1e-12, atol=1e-14)
    assert not O.population_factor(cov, ess=2.0 * (D + 1) - 1e-9)[1]       # too few effective samples
    v = rng.standard_normal(D)
    assert not O.population_factor(np.outer(v, v), ess=100.0)[1]           # rank one: singular
    assert not O.population_factor(cov * np.nan, ess=100.0)[1]


def test_learned_decision():
    assert O.learned_decision(3, 0.1, 1.0, True)
    assert not O.learned_decision(2, 0.1, 1.0, True)        # nothing published before k = 3
    assert not O.learned_decision(5, 0.5, 1.0, True)        # explains no more than half the variance
    assert not O.learned_decision(5, float("nan"), 1.0, True)
    assert not O.learned_decision(5, 0.0, 0.0, True)        # constant targets
    assert not O.learned_decision(5, 0.1, 1.0, False)       # unusable population factor


def test_train_first_step_moves_every_parameter_by_lr():
    """Adam's first step from zero moments moves each parameter by lr g / (|g| + eps),
    i.e. by lr against the sign of its gradient, and lowers the loss at a small lr."""
    rng = np.random.default_rng(12)
    D = 3
    th, lp = _ring(rng, R=120, D=D, n_inf=0, n_low=0)
    p0 = _params(rng, D)
    z = np.zeros_like(p0)
    lr = 1e-4
    p1, m1, v1, t1, loss0, nm, x, y = O.mlp_train(p0, z, z, 0, th, lp, 1, lr, bf16_points=False)
    assert t1 == 1
    d = p1 - p0
    moved = np.abs(m1) > 1e-5          # m1 = (1 - beta1) g
    assert moved.mean() > 0.9
    assert np.allclose(np.abs(d[moved]), lr, rtol=1e-2)
    p2, _, _, _, loss1, _, _, _ = O.mlp_train(p1, m1, v1, t1, th, lp, 1, 0.0, bf16_points=False)
    assert loss1 < loss0


def test_train_continues_its_state_across_calls():
    rng = np.random.default_rng(13)
    D = 2
    th, lp = _ring(rng, R=80, D=D, n_inf=3, n_low=4)
    p0 = _params(rng, D)
    z = np.zeros_like(p0)
    a = O.mlp_train(p0, z, z, 0, th, lp, 7, 5e-3)
    b1 = O.mlp_train(p0, z, z, 0, th, lp, 3, 5e-3)
    b2 = O.mlp_train(b1[0], b1[1], b1[2], b1[3], th, lp, 4, 5e-3)
    assert a[3] == b2[3] == 7
    for u, v in zip(a[:3], b2[:3]):
        assert np.array_equal(u, v)
    assert a[4] == b2[4]


def test_training_learns_the_score_of_a_gaussian_target():
    """Rows drawn from a Gaussian, labelled with its exact log density: after
    training, the surrogate's score near the centre follows -Sigma^-1 (theta - mu)."""
    rng = np.random.default_rng(14)
    D, R = 3, 500
    mu = np.array([0.5, -1.0, 2.0])
    A = rng.standard_normal((D, D)) * 0.3 + np.diag([0.6, 1.0, 0.4])
    Sig = A @ A.T
    th = rng.multivariate_normal(mu, Sig, size=R)
    lp = stats.multivariate_normal(mu, Sig).logpdf(th)
    H = 64
    P = O.mlp_nparams(D, H)
    lim = np.concatenate([np.full(D * H, math.sqrt(6 / (D + H))), np.zeros(H), np.full(H * H, math.sqrt(6 / (2 * H))),
                          np.zeros(H), np.full(H, math.sqrt(6 / (H + 1))), np.zeros(1)])
    p0 = (rng.random(P) * 2 - 1) * lim
    z = np.zeros(P)
    p, m, v, t, loss, nm, _, _ = O.mlp_train(p0, z, z, 0, th, lp, 400, 5e-3, bf16_points=False)
    assert loss < 0.02, loss
    pts = mu + rng.multivariate_normal(np.zeros(D), Sig, size=50) * 0.7
    g = O.mlp_score(p, nm, pts, bf16_points=False)
    ref = -(pts - mu) @ np.linalg.inv(Sig).T
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel < 0.15, rel
