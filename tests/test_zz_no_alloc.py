"""smc2_pf_loglik_noalloc, the entry point for callers that cannot allocate
device memory once running (a fixed budget, a framework-owned memory pool, or
a loop that cannot pay for cudaMalloc's synchronisation): through the C ABI,
two calls in a row must give what smc2_pf_loglik gives on the same inputs.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import numpy as np
import pytest
import torch

from paper_2311_12973_gb300 import inputs as I

from gpu_util import rel_err, soa

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2311_12973_gb300 import smc2
    return smc2


@pytest.mark.parametrize("precision,tol", [(I.PREC_FP64, 1e-12), (I.PREC_MIXED, 2e-5)])
@pytest.mark.parametrize("name,M,n,T", [("seir_t100_n1024", 512, 300, 60), ("lg_t50_n64", 128, 37, 50)])
def test_matches_context_entry_point_twice(S, precision, tol, name, M, n, T):
    w = I.workload(name, M=M, N=n, T=T, precision=precision)
    th = I.theta_near_prior(w, n, seed=41, spread=0.3)
    if w.model == I.LG:
        th[:, 0] = np.clip(th[:, 0], -0.95, 0.95)
    theta = soa(th)
    cfg = S.make_config(w)
    ctx = S.SMC2(cfg, w.y)
    ref = ctx.pf_loglik(theta, iteration=3).cpu().numpy()
    ctx.close()
    y_dev = torch.tensor(w.y, dtype=torch.float64, device="cuda")
    for call in range(2):
        got = S.pf_loglik_noalloc(S.make_config(w), y_dev, theta, iteration=3).cpu().numpy()
        torch.cuda.synchronize()
        assert rel_err(got, ref, 10.0) <= tol, (call, got[:4], ref[:4])


def test_rejects_series_longer_than_the_scratch(S):
    w = I.workload("lg_t50_n64", M=64, N=4)
    cfg = S.make_config(w)
    cfg.T = 32001
    y_dev = torch.zeros(32001, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SMC2Error) as e:
        S.pf_loglik_noalloc(cfg, y_dev, soa(I.theta_near_prior(w, 4, seed=1)), iteration=1)
    assert e.value.status == S.EINVAL
