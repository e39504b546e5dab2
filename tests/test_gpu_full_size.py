"""Parity at the full sizes of the benchmark configurations, in the launch
configuration the benchmark times (shapes picked by the built-in tuner).

The oracle cannot run a whole mixed-precision job at these sizes, so:
* FP64 form: sampled filters of a full-size launch, and a full first SMC^2
  iteration of the N=1024 workload, against the oracle (bit-exact ancestors,
  1e-12 relative increments, as at small sizes);
* mixed form: against the FP64 form of the same full-size launch (same random
  streams), through properties that hold at any size: most filters agree to
  FP32 rounding (a filter whose FP32 weights move one resampling decision
  follows another trajectory afterwards), and the differences have no
  systematic offset."""
import math
import time

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


def _soa(theta_rows):
    return torch.tensor(np.ascontiguousarray(np.asarray(theta_rows).T), dtype=torch.float64, device="cuda")


def _full_pf(S, w, theta, precision):
    ctx = S.SMC2(S.make_config(w, precision=precision), w.y)
    ll = ctx.pf_loglik(_soa(theta), iteration=1).cpu().numpy()
    shape = ctx.launch_shape()
    ctx.close()
    return ll, shape


def _mixed_vs_fp64(ll32, ll64, tag):
    d = ll32 - ll64
    rel = np.abs(d) / np.abs(ll64)
    se = d.std(ddof=1) / math.sqrt(len(d))
    print(f"{tag}: median rel {np.median(rel):.3g}, 90% {np.quantile(rel, 0.9):.3g}, max {rel.max():.3g}, "
          f"mean diff {d.mean():.3g} +- {se:.3g}, sd {d.std():.3g}")
    return rel, d, se


@pytest.mark.parametrize("name", ["seir_t100_n1024", "seir_t200_n8192"])
def test_full_size_pf_fp64_sampled_and_mixed(S, name):
    w = I.workload(name)
    theta = I.theta_near_prior(w, w.N, seed=11, spread=0.3)
    t0 = time.perf_counter()
    ll64, shape64 = _full_pf(S, w, theta, I.PREC_FP64)
    ll32, shape32 = _full_pf(S, w, theta, I.PREC_MIXED)
    print(f"{name}: shapes fp64 {shape64} mixed {shape32}, {time.perf_counter() - t0:.1f} s")
    cfg = O.config_from(w)
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(w.N, size=8, replace=False))
    ref = np.array([O.pf_loglik(cfg, theta[i], w.y, 1, i) for i in idx])
    scale = np.maximum(np.abs(ref), 10.0)
    err = np.abs(ll64[idx] - ref) / scale
    print(f"{name}: FP64 sampled max rel err {err.max():.3g}")
    assert err.max() < 1e-12
    rel, d, se = _mixed_vs_fp64(ll32, ll64, name)
    # measured on GB300: median 1.4e-3 / 1.0e-3, mean difference within 1.8 SE of zero
    assert np.median(rel) < 5e-3
    assert abs(d.mean()) < 4 * se


def test_full_size_sir_fp64_sampled_and_mixed(S):
    """The paper's SIR experiment at full size (N = 1024, M = 500, T = 30, the
    paper's filter): sampled filters of the FP64 launch bit-exact against the
    oracle; the mixed launch, whose FP32 sampler reads its words differently,
    without offset against the FP64 one over all 1024 filters."""
    w = I.workload("sir_t30_n1024")
    u = np.random.default_rng(12).random((w.N, 2))
    theta = np.column_stack([0.85 + 0.1 * (u[:, 0] - 0.5), 0.20 + 0.05 * (u[:, 1] - 0.5)])
    ll64, shape64 = _full_pf(S, w, theta, I.PREC_FP64)
    ll32, shape32 = _full_pf(S, w, theta, I.PREC_MIXED)
    cfg = O.config_from(w)
    idx = np.sort(np.random.default_rng(4).choice(w.N, size=8, replace=False))
    for i in idx:
        r_ll, r_delta, r_anc = O.pf_loglik(cfg, theta[i], w.y, 1, i, trace=True)
        if np.isfinite(r_ll):
            assert abs(ll64[i] - r_ll) / max(abs(r_ll), 10.0) < 1e-12, (i, ll64[i], r_ll)
        else:
            assert ll64[i] == r_ll
    fin = np.isfinite(ll64) & np.isfinite(ll32)
    assert fin.mean() > 0.9
    d = ll32[fin] - ll64[fin]
    se = d.std(ddof=1) / math.sqrt(len(d))
    print(f"sir: shapes fp64 {shape64} mixed {shape32}; mixed - fp64 mean {d.mean():.3g} +- {se:.3g}")
    # E[p^] is the same in both forms; log p^ of independent filters differs in mean by
    # at most the difference of their log-variance biases, small against the spread here
    assert abs(d.mean()) < 4 * se + 0.1 * d.std()


def _compare_stats(g, o, scale):
    assert g["k"] == o["k"] and g["resampled"] == o["resampled"], (g, o)
    assert g["lk_fallback"] == o["lk_fallback"]
    for key in ("lse", "lse2", "logz"):
        assert rel_err(g[key], o[key], scale) < 1e-12, (key, g[key], o[key])
    assert rel_err(g["ess"], o["ess"]) < 1e-9
    assert rel_err(g["est"], o["est"], 1.0) < 1e-9
    # covariance: one pass about the first proposal on the device, two passes in the oracle
    assert rel_err(g["cov"], o["cov"], max(float(np.max(np.abs(o["cov"]))), 1e-300)) < 1e-8, (g["cov"], o["cov"])


def test_full_size_iterations_fp64_match_oracle(S):
    """The whole first SMC^2 iteration of the N=1024, M=512, T=100 workload in
    FP64, then a second iteration stage-wise from the oracle's state."""
    w = I.workload("seir_t100_n1024", precision=I.PREC_FP64)
    ref = O.SMC2(O.config_from(w), w.y)
    o1 = ref.step()
    ctx = S.SMC2(S.make_config(w), w.y)
    g1 = ctx.run(1)[0][0]
    scale = max(10.0, float(np.max(np.abs(ref.logw[np.isfinite(ref.logw)]))))
    _compare_stats(g1, o1, scale)
    k, th, lp, ll, lw = ctx.get_state()
    assert k == 1 and rel_err(th, ref.theta, 1.0) < 1e-10
    assert rel_err(ll, ref.loglik, scale) < 1e-12 and rel_err(lw, ref.logw, scale) < 1e-12
    ctx.set_state(ref.k, ref.theta, ref.logprior, ref.loglik, ref.logw)
    g2 = ctx.run(1)[0][0]
    o2 = ref.step()
    scale = max(10.0, float(np.max(np.abs(ref.logw[np.isfinite(ref.logw)]))))
    _compare_stats(g2, o2, scale)
    k, th, lp, ll, lw = ctx.get_state()
    assert rel_err(th, ref.theta, 1.0) < 1e-10 and rel_err(lw, ref.logw, scale) < 1e-12
    ctx.close()


def test_full_size_mixed_iterations_are_consistent(S):
    """Two mixed-precision iterations of the N=8192, M=1024, T=200 workload in
    the tuner's launch shape: statistics finite and within their ranges, the
    recycled estimate inside the prior's bulk."""
    w = I.workload("seir_t200_n8192")
    ctx = S.SMC2(S.make_config(w), w.y)
    st = [s[0] for s in ctx.run(2)]
    for s in st:
        assert 1.0 <= s["ess"] <= w.N and math.isfinite(s["lse"]) and s["lse2"] <= 2 * s["lse"] + 1e-9
        assert np.all(np.abs(s["est"][:w.D] - np.array(w.prior_mean)) < 4 * np.array(w.prior_sd))
    mean, logz, ess = ctx.estimate()
    assert np.all(np.isfinite(mean)) and math.isfinite(logz) and ess == pytest.approx(sum(s["ess"] for s in st))
    ctx.close()


def test_full_size_batched_sampled_filters(S):
    """The 64-dataset workload (T in 50..400, N in {256, 1024, 4096}, M in
    {128, 512, 1024}) in one context: sampled filters of three datasets in FP64
    against the oracle with that dataset's random stream; the mixed context
    against the FP64 one over every filter of those datasets."""
    ws = I.batched_workloads(64)
    shapes = [(w.N, w.M, w.T) for w in ws]
    y = np.concatenate([w.y for w in ws])
    ctx64 = S.SMC2(S.make_config(ws[0], precision=I.PREC_FP64), y, datasets=shapes)
    ctx32 = S.SMC2(S.make_config(ws[0]), y, datasets=shapes)
    rng = np.random.default_rng(5)
    diffs, rels = [], []
    for d in (0, 31, 63):
        w = ws[d]
        theta = I.theta_near_prior(w, w.N, seed=20 + d, spread=0.3)
        ll64 = ctx64.pf_loglik(_soa(theta), iteration=1, dataset=d).cpu().numpy()
        ll32 = ctx32.pf_loglik(_soa(theta), iteration=1, dataset=d).cpu().numpy()
        cfg = O.config_from(w)
        idx = np.sort(rng.choice(w.N, size=4, replace=False))
        ref = np.array([O.pf_loglik(cfg, theta[i], w.y, 1, i) for i in idx])
        err = np.abs(ll64[idx] - ref) / np.maximum(np.abs(ref), 10.0)
        print(f"dataset {d} (N={w.N}, M={w.M}, T={w.T}): FP64 sampled max rel err {err.max():.3g}")
        assert err.max() < 1e-12
        diffs.append(ll32 - ll64)
        rels.append(np.abs(ll32 - ll64) / np.abs(ll64))
    dd = np.concatenate(diffs)
    rr = np.concatenate(rels)
    se = dd.std(ddof=1) / math.sqrt(len(dd))
    print(f"batched mixed vs FP64: median rel {np.median(rr):.3g}, mean diff {dd.mean():.3g} +- {se:.3g}")
    assert np.median(rr) < 5e-3
    assert abs(dd.mean()) < 4 * se
    ctx64.close()
    ctx32.close()


def test_full_size_batched_fp64_iterations_against_oracle(S):
    """The 64-dataset workload at full size in one FP64 context (every dataset
    runs; 1.7e10 particle-steps per iteration): two whole SMC^2 iterations of
    its three cheapest datasets (N = 256, M = 128, T = 218, 228, 259) against
    the oracle's single-dataset runs with their dataset indices -- the
    statistics of each iteration (Sec. IV: Eqs. 17, 20-22, 24-25, the
    resampling decision) and the population after the second."""
    ws = [w.with_(precision=I.PREC_FP64, K=2) for w in I.batched_workloads(64, K=2)]
    shapes = [(w.N, w.M, w.T) for w in ws]
    ctx = S.SMC2(S.make_config(ws[0]), np.concatenate([w.y for w in ws]), datasets=shapes)
    t0 = time.perf_counter()
    stats = ctx.run(2)
    print(f"two FP64 iterations of the 64 datasets: {time.perf_counter() - t0:.1f} s")
    for d in (24, 57, 1):
        w = ws[d]
        ref = O.SMC2(O.config_from(w), w.y).run(2)
        fin = np.isfinite(ref.logw)
        scale = max(10.0, float(np.max(np.abs(ref.logw[fin]))))
        for k in range(2):
            g, o = stats[k][d], ref.stats[k]
            assert g["dataset"] == d and g["k"] == o["k"] and g["resampled"] == o["resampled"], (d, k, g, o)
            for key in ("lse", "lse2", "logz"):
                assert abs(g[key] - o[key]) <= 1e-12 * max(scale, abs(o[key])), (d, k, key, g[key], o[key])
            assert abs(g["ess"] - o["ess"]) <= 1e-9 * o["ess"], (d, k, g["ess"], o["ess"])
            assert np.max(np.abs(g["est"] - o["est"])) <= 1e-9 * max(1.0, float(np.max(np.abs(o["est"]))))
        kk, th, lp, ll, lw = ctx.get_state(d)
        assert kk == ref.k
        assert np.max(np.abs(th - ref.theta)) <= 1e-10 * max(1.0, float(np.max(np.abs(ref.theta))))
        assert np.array_equal(np.isfinite(lw), fin)
        assert np.max(np.abs(ll[fin] - ref.loglik[fin])) <= 1e-12 * scale
        assert np.max(np.abs(lw[fin] - ref.logw[fin])) <= 1e-12 * scale
        print(f"dataset {d} (N={w.N}, M={w.M}, T={w.T}): two iterations equal the oracle's")
    ctx.close()
