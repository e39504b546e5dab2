"""Whole SMC^2 iterations on the device against the oracle (Sec. IV).

FP64 runs follow the oracle's random stream, so the resampling decisions and
indices agree exactly and every statistic agrees to rounding: relative 1e-12
on log-weight-like quantities (scaled by their magnitude, 1e-12 |log w| being
the rounding floor of sums of logs), and the ESS and estimates within the
error that this absolute log-weight error induces."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2311_12973_gb300 import inputs as I

from gpu_util import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2311_12973_gb300 import smc2
    return smc2


def _compare_stats(g, o, scale):
    assert g["k"] == o["k"] and g["resampled"] == o["resampled"], (g, o)
    assert g["lk_fallback"] == o["lk_fallback"], (g, o)
    for key in ("lse", "lse2", "logz"):
        assert rel_err(g[key], o[key], scale) < 1e-12, (key, g[key], o[key])
    assert rel_err(g["ess"], o["ess"]) < 1e-9, (g["ess"], o["ess"])
    assert rel_err(g["est"], o["est"], 1.0) < 1e-9, (g["est"], o["est"])
    # covariance: one pass about the first proposal on the device, two passes in the oracle;
    # the one-pass form's rounding floor is about 1e-16 of the squared scale of theta, which
    # dominates when the population collapses onto one point (ESS near 1)
    floor = 1e-15 * max(1.0, float(np.max(np.abs(o["est"]))) ** 2)
    assert np.max(np.abs(g["cov"] - o["cov"])) <= 1e-8 * float(np.max(np.abs(o["cov"]))) + floor, (g["cov"], o["cov"])


def _compare_state(S_ctx, ref, scale):
    k, th, lp, ll, lw = S_ctx.get_state()
    assert k == ref.k
    assert rel_err(th, ref.theta, 1.0) < 1e-10
    assert rel_err(lp, ref.logprior, 10.0) < 1e-12
    assert rel_err(ll, ref.loglik, scale) < 1e-12
    assert rel_err(lw, ref.logw, scale) < 1e-12


CASES = {
    "lg_cfg1": dict(name="lg_t50_n64"),
    "lg_max_n": dict(name="lg_t50_n64", N=16384, M=8, T=5, K=3),      # the largest N: 128 KB of q per block
    "seir_max_m": dict(name="seir_t100_n1024", N=40, M=2048, T=6, K=3, precision=I.PREC_FP64),  # FP64 SEIR limit
    "lg_max_m": dict(name="lg_t50_n64", N=20, M=4096, T=6, K=3),
    "lg_n_odd": dict(name="lg_t50_n64", N=1000, M=33, T=7, K=4),
    "lg_forward": dict(name="lg_t50_n64", lkernel=I.LK_FORWARD, N=96, K=6),
    "lg_ragged": dict(name="lg_t50_n64", N=300, M=100, T=20, K=4),
    "seir_fp64": dict(name="seir_t100_n1024", N=64, M=128, T=40, K=5, precision=I.PREC_FP64),
    "lg_tiny": dict(name="lg_t50_n64", N=1, M=1, T=1, K=3),
}


@pytest.mark.parametrize("case", list(CASES))
def test_fp64_run_matches_oracle(S, case):
    kw = dict(CASES[case])
    w = I.workload(kw.pop("name"), **kw)
    ctx = S.SMC2(S.make_config(w), w.y)
    stats = ctx.run(w.K)
    ref = O.SMC2(O.config_from(w), w.y).run(w.K)
    scale = max(10.0, float(np.max(np.abs(ref.logw[np.isfinite(ref.logw)]))))
    for k in range(w.K):
        _compare_stats(stats[k][0], ref.stats[k], scale)
    _compare_state(ctx, ref, scale)
    mean, logz, ess_sum = ctx.estimate()
    ref_mean, _ = ref.recycled()
    assert rel_err(mean, ref_mean, 1.0) < 1e-9
    ref_cov = ref.recycled_cov()
    assert rel_err(ctx.estimate_cov(), ref_cov, max(float(np.max(np.abs(ref_cov))), 1e-300)) < 1e-8
    assert rel_err(logz, ref.stats[-1]["logz"], scale) < 1e-12
    assert rel_err(ess_sum, sum(s["ess"] for s in ref.stats)) < 1e-9
    ctx.close()


@pytest.mark.parametrize("lk", [I.LK_GAUSS, I.LK_FORWARD])
@pytest.mark.parametrize("name", ["lg_t50_n64", "seir_t100_n1024"])
def test_stagewise_iteration_from_oracle_state(S, name, lk):
    """The oracle's population after iteration k is loaded into the context;
    one device iteration must equal the oracle's iteration k+1."""
    kw = dict(N=128, M=64, T=30, K=4, lkernel=lk, precision=I.PREC_FP64)
    w = I.workload(name, **kw)
    ref = O.SMC2(O.config_from(w, ess_frac=0.3), w.y).run(2)
    ctx = S.SMC2(S.make_config(w, ess_frac=0.3), w.y)
    ctx.set_state(ref.k, ref.theta, ref.logprior, ref.loglik, ref.logw)
    g = ctx.run(1)[0][0]
    o = ref.step()
    scale = max(10.0, float(np.max(np.abs(ref.logw[np.isfinite(ref.logw)]))))
    _compare_stats(g, o, scale)
    _compare_state(ctx, ref, scale)
    ctx.close()


def test_checkpoint_resume_is_bit_identical(S):
    w = I.workload("lg_t50_n64", N=128, K=8)
    a = S.SMC2(S.make_config(w), w.y)
    full = a.run(w.K)
    mean_a, logz_a, ess_a = a.estimate()
    b = S.SMC2(S.make_config(w), w.y)
    b.run(5)
    k, th, lp, ll, lw = b.get_state()
    hist, kh = b.raw_history()
    b.close()
    c = S.SMC2(S.make_config(w), w.y)
    c.set_state(k, th, lp, ll, lw)
    c.set_history(hist, kh)
    rest = c.run(w.K - 5)
    for i in range(w.K - 5):
        assert rest[i][0]["lse"] == full[5 + i][0]["lse"]
        assert np.array_equal(rest[i][0]["est"], full[5 + i][0]["est"])
    mean_c, logz_c, ess_c = c.estimate()
    assert np.array_equal(mean_a, mean_c) and logz_a == logz_c and ess_a == ess_c
    sa, sc = a.get_state(), c.get_state()
    for x, y in zip(sa[1:], sc[1:]):
        assert np.array_equal(x, y)


def test_run_state_errors(S):
    w = I.workload("lg_t50_n64", N=16, M=16, T=5, K=2)
    ctx = S.SMC2(S.make_config(w), w.y)
    ctx.run(2)
    with pytest.raises(S.SMC2Error) as e:
        ctx.run(1)
    assert e.value.status == S.ESTATE
    ctx.reset(w.seed)
    again = ctx.run(2)
    ctx.reset(w.seed + 1)
    other = ctx.run(2)
    assert again[1][0]["lse"] != other[1][0]["lse"]


def test_nonfinite_outer_weights_reported(S):
    # every observation impossible under every theta: y = nan makes all PF weights vanish
    w = I.workload("lg_t50_n64", N=16, M=16, T=5, K=1)
    y = np.full(5, np.nan)
    ctx = S.SMC2(S.make_config(w), y)
    with pytest.raises(S.SMC2Error) as e:
        ctx.run(1)
    assert e.value.status == S.ENONFINITE


BATCHED = {
    "lg": ("lg_t50_n64", [(64, 128, 50), (100, 64, 30), (33, 200, 45)], {}),
    "lg_paper_pf": ("lg_t50_n64", [(64, 128, 50), (100, 64, 30), (33, 200, 45)],
                    dict(pf_scheme=I.PF_MULTINOMIAL, pf_ess_frac=0.5)),
    "sir": ("sir_t30_n1024", [(64, 100, 30), (96, 64, 20), (40, 150, 25)], dict(precision=I.PREC_FP64)),
}


@pytest.mark.parametrize("case", list(BATCHED))
def test_batched_datasets_match_oracle(S, case):
    """Datasets of different N, M and T in one context: each follows its own
    random stream (dataset index in the counter) and must equal the oracle's
    single-dataset run of that dataset; with the paper's particle filter, and
    for the SIR model with its uniform prior."""
    name, shapes, over = BATCHED[case]
    ws = [I.workload(name, N=n, M=m, T=t, K=4, dataset=d, data_seed=10 + d, **over)
          for d, (n, m, t) in enumerate(shapes)]
    y = np.concatenate([w.y for w in ws])
    ctx = S.SMC2(S.make_config(ws[0]), y, datasets=shapes)
    stats = ctx.run(4)
    for d, w in enumerate(ws):
        ref = O.SMC2(O.config_from(w), w.y).run(w.K)
        fin = np.isfinite(ref.logw)
        scale = max(10.0, float(np.max(np.abs(ref.logw[fin]))))
        for k in range(w.K):
            assert stats[k][d]["dataset"] == d
            _compare_stats(stats[k][d], ref.stats[k], scale)
        k, th, lp, ll, lw = ctx.get_state(d)
        assert k == ref.k
        assert rel_err(th, ref.theta, 1.0) < 1e-10
        assert np.array_equal(np.isfinite(lw), fin)  # zero-weight samples (outside a uniform prior) alike
        assert rel_err(ll[fin], ref.loglik[fin], scale) < 1e-12
        assert rel_err(lw[fin], ref.logw[fin], scale) < 1e-12
        mean, logz, ess_sum = ctx.estimate(d)
        ref_mean, _ = ref.recycled()
        assert rel_err(mean, ref_mean, 1.0) < 1e-9
    ctx.close()


@pytest.mark.parametrize("family", ["groups", "fp32"])
def test_batched_seir_mixed_runs(S, family):
    """Sixty-four SEIR-type datasets of uneven T, N and M in one mixed-precision
    context: every dataset's statistics are finite, and dataset 0 (whose random
    stream is that of a single-dataset context) equals a context holding it
    alone, bit for bit, with the same filter kernel: pf_kernel at the same
    launch shape, or the FP32 filter (grouped in the batched context, one
    filter per CTA alone)."""
    ws = I.batched_workloads(64, K=3)
    shapes = [(w.N, w.M, w.T) for w in ws]
    shape = dict(ppt=4, cta_threads=256, pf_family=S.PF_GROUPS) if family == "groups" else \
        dict(ppt=4, pf_family=S.PF_FP32)
    ctx = S.SMC2(S.make_config(ws[0], **shape), np.concatenate([w.y for w in ws]), datasets=shapes)
    assert ctx.launch_shape()["fp32_filter"] == (0 if family == "groups" else 2)
    stats = ctx.run(3)
    for k in range(3):
        for d in range(64):
            s = stats[k][d]
            assert s["dataset"] == d and s["k"] == k + 1
            assert math.isfinite(s["lse"]) and s["ess"] >= 1.0 and np.all(np.isfinite(s["est"]))
    w = ws[0]
    single = S.SMC2(S.make_config(w, **shape), w.y)
    alone = single.run(3)
    for k in range(3):
        for key in ("ess", "lse", "lse2", "logz", "resampled"):
            assert alone[k][0][key] == stats[k][0][key], (k, key)
        assert np.array_equal(alone[k][0]["est"], stats[k][0]["est"])
    single.close()
    ctx.close()
