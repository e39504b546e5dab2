"""The device random stream equals the oracle's: Philox words bit for bit,
Box-Muller normals within the rounding of the working precision."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2311_12973_gb300 import smc2
    return smc2


def _counters(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    c[:8] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
             [5, 7, 3 | (2 << 20), 5 | (9 << 4)], [0, 12, 0, 6 | (1 << 4)]]
    return c


def test_known_answer_vectors(S):
    golden = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    for line in open(golden):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        ctr = torch.tensor(np.array([v[0:4]], dtype=np.uint32).view(np.int32), device="cuda")
        words = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
        S.philox_normals(v[4] | (v[5] << 32), ctr, S.PREC_FP64, words=words)
        got = words.cpu().numpy().view(np.uint32)[0]
        assert list(got) == v[6:10]


@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEF12345678])
def test_words_bit_exact(S, seed):
    c = _counters(4096, 7)
    ctr = torch.tensor(c.view(np.int32), device="cuda")
    words = torch.zeros((4096, 4), dtype=torch.int32, device="cuda")
    S.philox_normals(seed, ctr, S.PREC_FP64, words=words)
    got = words.cpu().numpy().view(np.uint32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    want = np.array([O.philox(row, key) for row in c])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 1e-5)])
def test_normals(S, precision, tol):
    # FP64: libm vs CUDA log/sincos, a few ulps.  FP32: hardware lg2, rsqrt,
    # sin and cos: absolute error about 2^-21 on each factor, times r <= 5.8,
    # plus the rounding of 2 pi (u - 1/2): |dz| < 1e-5 (1 + |z|).
    c = _counters(4096, 11)
    ctr = torch.tensor(c.view(np.int32), device="cuda")
    z = torch.zeros((4096, 4), dtype=torch.float64, device="cuda")
    S.philox_normals(99, ctr, precision, z=z)
    got = z.cpu().numpy()
    want = np.array([O.normals4(99, *row) for row in c])
    assert np.max(np.abs(got - want) / (1.0 + np.abs(want))) < tol
