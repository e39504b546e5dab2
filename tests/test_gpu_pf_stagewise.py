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


@pytest.mark.parametrize("name,M,T,n,ppt,fam", CASES)
def test_fp32_filter_stagewise_against_oracle(S, name, M, T, n, ppt, fam):
    w = I.workload(name, precision=I.PREC_MIXED).with_(M=M, T=T)
    th = I.theta_near_prior(w, n, seed=23, spread=0.3)
    if w.model == I.LG:
        th[:, 0] = np.clip(th[:, 0], -0.95, 0.95)
    ctx = S.SMC2(S.make_config(w, ppt=ppt, pf_family=fam), w.y)
    shape = ctx.launch_shape()
    if fam == 2:
        assert shape["one_group_per_cta"] and shape["ppt"] == ppt, shape
    k = 3
    ll, delta, anc, xs, lw, q = (a.cpu().numpy() for a in ctx.pf_trace_states(soa(th), iteration=k))
    ctx.close()
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
    print(f"{name} M={M} ppt={ppt} family={fam}: worst relative errors {worst}")
