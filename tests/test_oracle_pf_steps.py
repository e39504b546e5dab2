"""The oracle's exposed step body composes to its particle filter: initial
states, propagation, log-weights, quantisation and systematic resampling with
the step's word, run step by step, give oracle_pf_loglik's increments and
ancestors bit for bit (so the stage-wise GPU checks exercise the filter the
other pins fix)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_12973_gb300 import inputs as I


@pytest.mark.parametrize("name,M,T", [("lg_t50_n64", 64, 20), ("seir_t100_n1024", 100, 25)])
def test_step_body_composes_to_the_filter(name, M, T):
    w = I.workload(name, M=M, T=T)
    cfg = O.config_from(w)
    th = I.theta_near_prior(w, 3, seed=4, spread=0.3)
    for i in range(3):
        ll, delta, anc = O.pf_loglik(cfg, th[i], w.y, 2, i, trace=True)
        x = O.pf_initial(cfg, th[i], 2, i)
        total = 0.0
        for t in range(1, T + 1):
            x, ell = O.pf_propagate(cfg, th[i], 2, i, t, w.y[t - 1], x)
            assert np.array_equal(ell, O.pf_log_weights(cfg, th[i], x, w.y[t - 1]))
            m = ell.max()
            step = m + np.log(np.sum(np.exp(ell - m))) - np.log(M)
            assert abs(step - delta[t - 1]) <= 1e-12 * max(1.0, abs(step))
            total += delta[t - 1]
            if t < T:
                qq, _ = O.quantise(ell)
                _, a = O.systematic_from_q(qq, O.pf_resample_word(cfg, 2, i, t))
                assert np.array_equal(a, anc[t - 1])
                x = x[a]
        assert abs(total - ll) <= 1e-12 * max(1.0, abs(ll))
