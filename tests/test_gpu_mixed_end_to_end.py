"""Mixed precision (FP32 particles, FP64 outer) against the FP64 form end to end.

For each seed the two forms draw the same random streams, and the FP64 form
equals the oracle (test_gpu_smc2.py), so the paired difference of their
recycled posterior means (Eq. 29) and log-evidence estimates isolates what
FP32 particles change.  A filter whose FP32 weights move one resampling
decision follows another trajectory afterwards, so the differences are Monte
Carlo noise, not rounding: the bar is that they have no offset (3 standard
errors of the paired differences over 32 seeds)."""
import math

import numpy as np
import pytest

from paper_2311_12973_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2311_12973_gb300 import smc2
    return smc2


def _paired(S, name, seeds, **kw):
    res = {}
    for prec in (I.PREC_FP64, I.PREC_MIXED):
        w = I.workload(name, precision=prec, **kw)
        ctx = S.SMC2(S.make_config(w), w.y)
        out = []
        for sd in seeds:
            ctx.reset(sd)
            ctx.run(w.K, stats=False)
            m, lz, _ = ctx.estimate()
            out.append((m, lz))
        res[prec] = out
        ctx.close()
    dm = np.array([a[0] - b[0] for a, b in zip(res[I.PREC_MIXED], res[I.PREC_FP64])])
    dz = np.array([a[1] - b[1] for a, b in zip(res[I.PREC_MIXED], res[I.PREC_FP64])])
    return dm, dz


@pytest.mark.parametrize("name,kw", [("lg_t50_n64", {}),
                                     ("seir_t100_n1024", dict(N=256, M=256, T=60, K=10))])
def test_mixed_precision_matches_fp64_without_offset(S, name, kw):
    n = 32
    dm, dz = _paired(S, name, list(range(1, n + 1)), **kw)
    se_m = dm.std(axis=0, ddof=1) / math.sqrt(n)
    se_z = dz.std(ddof=1) / math.sqrt(n)
    print(f"{name}: mean diff {dm.mean(axis=0)} +- {se_m}; log Z diff {dz.mean():.3f} +- {se_z:.3f}, "
          f"median |diff| {np.median(np.abs(dz)):.3f}")
    # measured on GB300: means within 2.1 SE; log Z -0.07 +- 0.18 (LG), -0.46 +- 0.62 (SEIR)
    assert np.all(np.abs(dm.mean(axis=0)) < 3 * se_m + 1e-12)
    assert abs(dz.mean()) < 3 * se_z
    if name.startswith("lg"):
        assert np.median(np.abs(dz)) < 0.1  # measured 0.049 nats


def test_equal_accuracy_at_the_headline_size(S):
    """The SEIR workload at full size (N = 1024, M = 512, T = 100, K = 20): over
    192 paired seeds the mixed form's recycled posterior mean is as accurate as
    the FP64 form's, against a reference pooled from four FP64 runs with 8192
    samples (the FP64 form equals the oracle run for run).  The errors are
    heavy-tailed: a few runs dominate a mean of squares (blocks of 24 seeds gave
    MSE ratios from 1.2 to 2.9, 192 seeds 0.96), and a block of 96 seeds put the
    FP64 form's own mean 3 SE from its long-run value.  So equal accuracy is a
    sign test -- in each coordinate the mixed form is the worse of the pair in
    50 % +- 3 SD of the seeds -- and neither the means nor the log-evidence have
    an offset beyond 3.5 SE of the paired differences (four coordinates: a
    family-wise level near 0.2 %)."""
    n = 192
    seeds = list(range(501, 501 + n))
    ref_w = I.workload("seir_t100_n1024", N=8192, precision=I.PREC_FP64)
    ctx = S.SMC2(S.make_config(ref_w, rw_scale=0.2), ref_w.y)
    ref = []
    for sd in range(9001, 9005):
        ctx.reset(sd)
        ctx.run(ref_w.K, stats=False)
        ref.append(ctx.estimate()[0])
    ctx.close()
    ref = np.mean(ref, axis=0)
    res = {}
    for prec in (I.PREC_FP64, I.PREC_MIXED):
        w = I.workload("seir_t100_n1024", precision=prec)
        ctx = S.SMC2(S.make_config(w), w.y)
        out = []
        for sd in seeds:
            ctx.reset(sd)
            ctx.run(w.K, stats=False)
            m, lz, _ = ctx.estimate()
            out.append((m, lz))
        res[prec] = out
        ctx.close()
    m64 = np.array([a[0] for a in res[I.PREC_FP64]])
    m32 = np.array([a[0] for a in res[I.PREC_MIXED]])
    z64 = np.array([a[1] for a in res[I.PREC_FP64]])
    z32 = np.array([a[1] for a in res[I.PREC_MIXED]])
    e64, e32 = (m64 - ref) ** 2, (m32 - ref) ** 2
    worse = (e32 > e64).mean(axis=0)
    dm, dz = m32 - m64, z32 - z64
    se_m = dm.std(axis=0, ddof=1) / math.sqrt(n)
    se_z = dz.std(ddof=1) / math.sqrt(n)
    print(f"rmse fp64 {np.sqrt(e64.mean(axis=0))} mixed {np.sqrt(e32.mean(axis=0))}; median squared error "
          f"fp64 {np.median(e64, axis=0)} mixed {np.median(e32, axis=0)}; mixed worse in {worse}; "
          f"log Z mixed - fp64 {dz.mean():.3f} +- {se_z:.3f} (median |diff| {np.median(np.abs(dz)):.3f})")
    print(f"paired mean differences {dm.mean(axis=0)} +- {se_m}")
    assert np.all(np.abs(worse - 0.5) <= 3 * 0.5 / math.sqrt(n))
    assert np.all(np.abs(dm.mean(axis=0)) < 3.5 * se_m + 1e-12)
    assert abs(dz.mean()) < 3.5 * se_z
