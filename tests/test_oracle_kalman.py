"""Pin of the oracle's Kalman filter: the exact LG-AR(1) likelihood written
as one dense multivariate normal density (scipy), a different computation."""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O


def dense_loglik(phi, sx, sy, y):
    T = len(y)
    # Var(x_t), t = 1..T, with x_0 ~ N(0,1)
    v = np.empty(T)
    prev = 1.0
    for t in range(T):
        prev = phi * phi * prev + sx * sx
        v[t] = prev
    cov = np.empty((T, T))
    for s in range(T):
        for t in range(T):
            a, b = min(s, t), max(s, t)
            cov[s, t] = phi ** (b - a) * v[a]
    cov += sy * sy * np.eye(T)
    return stats.multivariate_normal(np.zeros(T), cov).logpdf(y)


@pytest.mark.parametrize("phi,sx,sy", [(0.8, 0.5, 1.0), (-0.3, 1.2, 0.4), (1.05, 0.2, 0.7), (0.0, 1.0, 1.0)])
def test_kalman_matches_dense_gaussian(phi, sx, sy):
    rng = np.random.default_rng(3)
    y = rng.standard_normal(25) * 1.3
    assert O.kalman_loglik(phi, sx, sy, y) == pytest.approx(dense_loglik(phi, sx, sy, y), rel=1e-10)
