"""Systematic resampling on the device equals the oracle's Eq. (27) counts laid
out by Algorithm 1, bit for bit, on identical quantised weights."""
import numpy as np
import pytest
import torch

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2311_12973_gb300 import smc2
    return smc2


def _gpu(S, q, U):
    qt = torch.tensor(q.view(np.int64), device="cuda")
    anc = torch.full((len(q),), -1, dtype=torch.int32, device="cuda")
    S.resample_systematic(qt, U, anc)
    return anc.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 100, 255, 256, 257, 1000, 1024, 4096, 5000, 8192, 16384])
def test_matches_oracle(S, n):
    rng = np.random.default_rng(n)
    for trial in range(3):
        logw = rng.standard_normal(n) * (1.0 + 4.0 * trial)
        logw[rng.random(n) < 0.25] = -np.inf
        if np.all(np.isinf(logw)):
            logw[n // 2] = 0.0
        q, _ = O.quantise(logw)
        U = int(rng.integers(0, 2**32))
        _, anc = O.systematic_from_q(q, U)
        assert np.array_equal(_gpu(S, q, U), anc)


def test_degenerate_and_extreme_u(S):
    n = 513
    q = np.zeros(n, dtype=np.uint64)
    q[200] = 2**52
    for U in [0, 2**32 - 1]:
        assert np.all(_gpu(S, q, U) == 200)
    q = np.full(n, 2**50, dtype=np.uint64)   # equal weights: identity
    for U in [0, 12345, 2**32 - 1]:
        assert np.array_equal(_gpu(S, q, U), np.arange(n))
