"""Pins of the oracle's random-number stream (no GPU).

Philox4x32-10 is pinned to the published known-answer vectors; the uniform
and Box-Muller conversions to distributional checks."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat_rows())
def test_philox_known_answers(ctr, key, want):
    assert list(O.philox(ctr, key)) == want


def test_uniform23_open_interval_and_exact():
    assert O.uniform23(0) == 0.5 / 2**23
    assert O.uniform23(0xFFFFFFFF) == (2**23 - 0.5) / 2**23
    # every value is an odd multiple of 2^-24: exactly representable in float32 too
    for w in [0, 1, 255, 256, 12345678, 0xDEADBEEF]:
        u = O.uniform23(w)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u


def test_normals_distribution():
    # 20000 draws (5000 Philox calls): mean, variance and a KS test against N(0,1)
    z = np.concatenate([O.normals4(7, j, 0, 3, 5 | (2 << 4)) for j in range(5000)])
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_normals_depend_on_every_counter_word_and_key():
    base = O.normals4(1, 2, 3, 4, 5)
    for args in [(2, 2, 3, 4, 5), (1, 3, 3, 4, 5), (1, 2, 4, 4, 5), (1, 2, 3, 5, 5), (1, 2, 3, 4, 6),
                 (1 << 32 | 1, 2, 3, 4, 5)]:
        assert not np.allclose(O.normals4(*args), base)
