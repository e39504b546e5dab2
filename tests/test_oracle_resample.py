"""Pins of the oracle's systematic resampling (Sec. IV-B, Eqs. 26-28, Algorithm 1).

The oracle evaluates the paper's ncopies formula exactly and lays copies out
with Algorithm 1.  These tests compare it with the textbook definition of
systematic resampling in exact rationals (one stratified position per slot,
each slot takes the first item whose cumulative weight passes its position),
and check the invariants the paper states."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O


def textbook_systematic(q, U):
    """positions p_j = (j + u) S / n with u = (2U+1)/2^33; a_j = first i with C_i > p_j."""
    n = len(q)
    S = sum(int(v) for v in q)
    u = Fraction(2 * U + 1, 2**33)
    C = np.cumsum([int(v) for v in q], dtype=object)
    anc = []
    for j in range(n):
        p = (j + u) * S / n
        anc.append(next(i for i in range(n) if C[i] > p))
    return np.array(anc, dtype=np.int32)


def paper_ncopies(q, U):
    """Eq. (27) with the inclusive cdf of Eq. (26): ceil(cdf^i - u) - ceil(cdf^{i-1} - u)."""
    n = len(q)
    S = sum(int(v) for v in q)
    u = Fraction(2 * U + 1, 2**33)
    out, prev, C = [], 0, 0
    for i in range(n):
        C += int(q[i])
        cur = math.ceil(Fraction(n * C, S) - u)
        out.append(cur - prev)
        prev = cur
    return np.array(out, dtype=np.int32)


def random_q(rng, n, zeros=0.3):
    B = O.fixed_point_bits(n)
    logw = rng.standard_normal(n) * 3.0
    logw[rng.random(n) < zeros] = -np.inf
    if np.all(np.isinf(logw)):
        logw[0] = 0.0
    q, b = O.quantise(logw)
    assert b == B
    return q


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 8, 13, 64])
def test_matches_textbook_and_paper_formula(n):
    rng = np.random.default_rng(n)
    for trial in range(40):
        q = random_q(rng, n)
        U = int(rng.integers(0, 2**32))
        nc, anc = O.systematic_from_q(q, U)
        assert np.array_equal(anc, textbook_systematic(q, U))
        assert np.array_equal(nc, paper_ncopies(q, U))


def test_extreme_u_values():
    rng = np.random.default_rng(11)
    for U in [0, 1, 2**31, 2**32 - 1]:
        for n in [4, 7, 16]:
            q = random_q(rng, n)
            nc, anc = O.systematic_from_q(q, U)
            assert np.array_equal(anc, textbook_systematic(q, U))


@pytest.mark.parametrize("n", [4, 100, 1024, 8192])
def test_invariants(n):
    rng = np.random.default_rng(n + 1)
    for trial in range(5):
        q = random_q(rng, n)
        U = int(rng.integers(0, 2**32))
        nc, anc = O.systematic_from_q(q, U)
        S = sum(int(v) for v in q)
        assert nc.sum() == n                                  # Eq. (28b)
        assert nc.min() >= 0 and nc.max() <= n                # Eq. (28a)
        assert np.all(np.diff(anc) >= 0)                      # Algorithm 1 order
        assert np.all(nc[q == 0] == 0)                        # zero weight, no copy
        for i in range(n):                                    # floor / ceil of n w~
            lo = (n * int(q[i])) // S
            assert nc[i] in (lo, lo + (1 if (n * int(q[i])) % S else 0))


def test_expected_copies_equal_n_times_weight():
    rng = np.random.default_rng(5)
    n = 6
    q = random_q(rng, n, zeros=0.0)
    S = sum(int(v) for v in q)
    Us = rng.integers(0, 2**32, size=20000)
    counts = np.array([O.systematic_from_q(q, int(U))[0] for U in Us])
    mean = counts.mean(axis=0)
    want = n * q.astype(np.float64) / S
    se = counts.std(axis=0) / np.sqrt(len(Us)) + 1e-12
    assert np.all(np.abs(mean - want) < 5 * se + 1e-9)


def test_quantise_properties():
    B = O.fixed_point_bits
    assert [B(1), B(2), B(1024), B(2048), B(4096), B(8192), B(2**20)] == [52, 52, 52, 52, 51, 50, 43]
    logw = np.array([-1.0, 0.5, -np.inf, np.nan, 0.5 - 40.0, 0.5])
    q, b = O.quantise(logw)
    assert b == 52
    assert q[1] == 2**52 and q[5] == 2**52
    assert q[2] == 0 and q[3] == 0
    assert q[0] == math.floor(math.exp(-1.5) * 2**52)
    assert q[4] == math.floor(math.exp(-40.0) * 2**52)
    # all weights equal at the largest n: the total still fits in 64 bits
    n = 8192
    q, b = O.quantise(np.zeros(n))
    assert int(q.sum(dtype=np.uint64)) == n * 2**b < 2**64
    q, b = O.quantise(np.full(3, -np.inf))
    assert b == -1
