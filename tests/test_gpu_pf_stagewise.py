"""Stage-wise parity of the FP32 particle filter (Sec. II) on identical inputs.

The device writes, for every step t, each particle's state after propagation,
its log-weight, its quantised weight and the ancestors of the resampling after
the step (smc2_pf_trace_states).  For every step the oracle recomputes, from
the device's own numbers:
  * the propagation (Eq. 1) of the device's resampled states of step t - 1 with
    the step's normals: relative 2e-5;
  * the log-weights (Eq. 2) of the device's propagated states: 2e-5 of
    max(1, |l|);
  * the quantised weights floor(exp(l - max l) 2^B) of the device's log-weights:
    the FP32 argument a = (l - max l) log2(e) carries an absolute error of about
    |a| 2^-23 and the hardware 2^a one of 2^-22 relative, so each weight is held
    to (|a| 2^-22 ln 2 + 2^-20) relative, twice that bound, plus one unit;
  * the ancestors, systematic resampling (Eqs. 26-27, Algorithm 1) of the
    device's quantised weights with the step's word U: bit for bit;
  * the increment log((1/M) sum w) (Eq. 8) from the device's log-weights:
    2e-5 of max(1, |increment|).
It covers the filter shapes the tuner picks for the headline workloads."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2311_12973_gb300 import inputs as I

from gpu_util import soa

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def S():
    from paper_2311_12973_gb300 import smc2
    return smc2


CASES = [
    # (workload, M, T, filters, ppt, kernel family)
    ("seir_t100_n1024", 512, 100, 4, 8, 2),
    ("seir_t100_n1024", 512, 100, 4, 4, 2),
    ("seir_t100_n1024", 512, 100, 3, 2, 2),
    ("seir_t100_n1024", 512, 60, 3, 2, 1),      # the groups kernel at its headline shape
    ("seir_t200_n8192", 1024, 120, 3, 4, 2),
    ("seir_t100_n1024", 300, 50, 3, 4, 2),      # ragged: padding particles in the last thread
    ("lg_t50_n64", 512, 50, 4, 8, 2),
    ("lg_t50_n64", 128, 50, 4, 4, 2),
]


def _check_stagewise(w, th, k, ll, delta, anc, xs, lw, q):
    """Every step of every traced filter against the oracle (the bars of the
    module docstring); returns the worst relative errors."""
    M, T, n = w.M, w.T, th.shape[0]
    q = q.view(np.uint64)
    cfg = O.config_from(w)
    ns = 1 if w.model == I.LG else 4
    B = O.fixed_point_bits(M)
    worst = {"x": 0.0, "l": 0.0, "q": 0.0, "delta": 0.0}
    for i in range(n):
        x_pre = O.pf_initial(cfg, th[i], k, i)
        for t in range(1, T + 1):
            x_dev = xs[i, t - 1].astype(np.float64)          # [M][5]
            l_dev = lw[i, t - 1].astype(np.float64)
            # propagation from the device's resampled states of the previous step
            x_or, _ = O.pf_propagate(cfg, th[i], k, i, t, w.y[t - 1], x_pre)
            cols = list(range(ns)) + ([4] if w.model == I.SEIR else [])
            ex = np.max(np.abs(x_dev[:, cols] - x_or[:, cols]) / np.maximum(np.abs(x_or[:, cols]), 1.0))
            worst["x"] = max(worst["x"], ex)
            assert ex <= TOL, (i, t, ex)
            # log-weights of the device's propagated states
            l_or = O.pf_log_weights(cfg, th[i], x_dev, w.y[t - 1])
            fin = np.isfinite(l_or)
            assert np.array_equal(fin, np.isfinite(l_dev)), (i, t)
            el = np.max(np.abs(l_dev[fin] - l_or[fin]) / np.maximum(np.abs(l_or[fin]), 1.0)) if fin.any() else 0.0
            worst["l"] = max(worst["l"], el)
            assert el <= TOL, (i, t, el)
            # quantised weights of the device's log-weights
            m = np.max(l_dev)
            q_ref = np.floor(np.exp(l_dev - m) * 2.0 ** B)
            qd = q[i, t - 1].astype(np.float64)
            a = np.where(np.isfinite(l_dev), (l_dev - m) * np.log2(np.e), 0.0)
            bound = q_ref * (np.abs(a) * 2.0 ** -22 * np.log(2.0) + 2.0 ** -20) + 1.0
            eq = np.max(np.abs(qd - q_ref) / bound)
            worst["q"] = max(worst["q"], eq)
            assert eq <= 1.0, (i, t, eq)
            # increment from the device's log-weights
            lse = m + np.log(np.sum(np.exp(l_dev - m))) - np.log(M)
            ed = abs(delta[i, t - 1] - lse) / max(1.0, abs(lse))
            worst["delta"] = max(worst["delta"], ed)
            assert ed <= TOL, (i, t, delta[i, t - 1], lse)
            if t < T:
                # ancestors: systematic resampling of the device's integer weights, bit for bit
                _, a_or = O.systematic_from_q(q[i, t - 1], O.pf_resample_word(cfg, k, i, t))
                assert np.array_equal(anc[i, t - 1], a_or), (i, t, np.nonzero(anc[i, t - 1] != a_or)[0][:8])
                x_pre = x_dev[anc[i, t - 1]]
        assert abs(ll[i] - np.sum(delta[i])) <= 1e-9 * max(1.0, abs(ll[i]))
    return worst


@pytest.mark.parametrize("name,M,T,n,ppt,fam", CASES)
def test_fp32_filter_stagewise_against_oracle(S, name, M, T, n, ppt, fam):
    w = I.workload(name, precision=I.PREC_MIXED).with_(M=M, T=T)
    th = I.theta_near_prior(w, n, seed=23, spread=0.3)
    if w.model == I.LG:
        th[:, 0] = np.clip(th[:, 0], -0.95, 0.95)
    ctx = S.SMC2(S.make_config(w, ppt=ppt, pf_family=fam), w.y)
    shape = ctx.launch_shape()
    if fam == 2:
        assert shape["fp32_filter"] == 1 and shape["ppt"] == ppt, shape
    k = 3
    trace = [a.cpu().numpy() for a in ctx.pf_trace_states(soa(th), iteration=k)]
    ctx.close()
    worst = _check_stagewise(w, th, k, *trace)
    print(f"{name} M={M} ppt={ppt} family={fam}: worst relative errors {worst}")


GROUPED = [
    # (ppt, [(M, T)] of the datasets of one context): groups of one warp, of
    # several warps on named barriers, and as wide as the CTA, with ragged M
    (4, [(128, 40), (512, 60), (1024, 50), (250, 45)]),
    (8, [(128, 40), (512, 60), (1024, 50), (250, 45)]),
]


@pytest.mark.parametrize("ppt,shapes", GROUPED)
def test_grouped_fp32_filter_equals_one_group_per_cta(S, ppt, shapes):
    """Datasets of unequal M in one context run the grouped instantiation of the
    FP32 filter (filter groups of unequal width sharing a CTA).  The filter's
    arithmetic does not depend on the group's width, so every dataset's
    log-likelihoods, increments and ancestors equal bit for bit those of the
    one-group-per-CTA instantiation on the same dataset (the traced run), and
    the traced run of the ragged dataset is checked step by step against the
    oracle."""
    n = 5  # fewer filters than a unit of the narrowest groups holds
    ws = [I.workload("seir_t100_n1024", precision=I.PREC_MIXED, N=n, M=m, T=t, dataset=d, data_seed=30 + d)
          for d, (m, t) in enumerate(shapes)]
    ctx = S.SMC2(S.make_config(ws[0], ppt=ppt, pf_family=S.PF_FP32), np.concatenate([w.y for w in ws]),
                 datasets=[(n, m, t) for m, t in shapes])
    shape = ctx.launch_shape()
    assert shape["fp32_filter"] == 2 and shape["ppt"] == ppt, shape
    k = 2
    for d, w in enumerate(ws):
        th = I.theta_near_prior(w, n, seed=40 + d, spread=0.3)
        ll_g = ctx.pf_loglik(soa(th), iteration=k, dataset=d).cpu().numpy()
        _, delta_g, anc_g = (a.cpu().numpy() for a in ctx.pf_trace(soa(th), iteration=k, dataset=d))
        trace = [a.cpu().numpy() for a in ctx.pf_trace_states(soa(th), iteration=k, dataset=d)]
        assert np.array_equal(ll_g, trace[0]), (d, ll_g, trace[0])
        assert np.array_equal(delta_g, trace[1]), d
        assert np.array_equal(anc_g, trace[2]), d
        if w.M % ppt or (w.M // ppt) % 32:
            worst = _check_stagewise(w, th[:2], k, *(a[:2] for a in trace))
            print(f"dataset {d} (M={w.M}, T={w.T}) ppt={ppt}: worst relative errors {worst}")
    ctx.close()


@pytest.mark.parametrize("name,M,T", [("seir_t100_n1024", 512, 80), ("seir_t100_n1024", 300, 40), ("lg_t50_n64", 256, 50)])
def test_fp32_filter_results_do_not_depend_on_the_launch_shape(S, name, M, T):
    """The tuner may pick any particles-per-thread shape, and the sampler's
    results must not change with it: per particle the arithmetic is the same,
    the slot counts are exact whatever the thread's float running sum, and S
    and the increment come from exact integer totals.  Log-likelihoods and
    increments at ppt 2, 4 and 8 agree bit for bit."""
    w = I.workload(name, precision=I.PREC_MIXED).with_(M=M, T=T)
    th = I.theta_near_prior(w, 40, seed=29, spread=0.5)
    if w.model == I.LG:
        th[:, 0] = np.clip(th[:, 0], -0.95, 0.95)
    out = {}
    for ppt in (2, 4, 8):
        ctx = S.SMC2(S.make_config(w, ppt=ppt, pf_family=S.PF_FP32), w.y)
        assert ctx.launch_shape()["fp32_filter"] == 1
        ll = ctx.pf_loglik(soa(th), iteration=5).cpu().numpy()
        _, delta, anc = (a.cpu().numpy() for a in ctx.pf_trace(soa(th), iteration=5))
        ctx.close()
        out[ppt] = (ll, delta, anc)
    for ppt in (4, 8):
        assert np.array_equal(out[ppt][0], out[2][0]), (ppt, out[ppt][0][:4], out[2][0][:4])
        assert np.array_equal(out[ppt][1], out[2][1]), ppt
        assert np.array_equal(out[ppt][2], out[2][2]), ppt
