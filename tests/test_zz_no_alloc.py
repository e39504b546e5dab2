"""smc2_pf_loglik_noalloc, the entry point for callers that cannot allocate
device memory once running (a fixed budget, a framework-owned memory pool, or
a loop that cannot pay for cudaMalloc's synchronisation): through the C ABI,
two calls in a row must give what smc2_pf_loglik gives on the same inputs and
launch shape (a context pinned to pf_kernel, the kernel the allocation-free
entry point runs), and repeated calls must leave the device's free memory as
it was.

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


def _theta(w, n):
    th = I.theta_near_prior(w, n, seed=41, spread=0.3)
    if w.model == I.LG:
        th[:, 0] = np.clip(th[:, 0], -0.95, 0.95)
    return soa(th)


@pytest.mark.parametrize("precision", [I.PREC_FP64, I.PREC_MIXED])
@pytest.mark.parametrize("ppt", [2, 4])
@pytest.mark.parametrize("name,M,n,T", [("seir_t100_n1024", 512, 300, 60), ("lg_t50_n64", 128, 37, 50)])
def test_matches_context_entry_point_twice(S, precision, ppt, name, M, n, T):
    """Both entry points run the same kernel at the same particles per thread,
    with the same random streams and observation terms: FP64 results agree bit
    for bit; the mixed form within the FP32 stage bar (2e-5)."""
    w = I.workload(name, M=M, N=n, T=T, precision=precision)
    theta = _theta(w, n)
    # the context pinned to the kernel the allocation-free entry point runs (pf_kernel)
    ctx = S.SMC2(S.make_config(w, ppt=ppt, pf_family=S.PF_GROUPS), w.y)
    ref = ctx.pf_loglik(theta, iteration=3).cpu().numpy()
    ctx.close()
    y_dev = torch.tensor(w.y, dtype=torch.float64, device="cuda")
    for call in range(2):
        got = S.pf_loglik_noalloc(S.make_config(w, ppt=ppt), y_dev, theta, iteration=3).cpu().numpy()
        torch.cuda.synchronize()
        if precision == I.PREC_FP64:
            assert np.array_equal(got, ref), (call, got[:4], ref[:4])
        else:
            assert rel_err(got, ref, 10.0) <= 2e-5, (call, got[:4], ref[:4])


def test_repeated_calls_leave_free_memory_unchanged(S):
    """After the first call (which may load the kernel and the scratch array),
    further calls change the device's free memory by nothing: the scratch is
    the library's static array and the outputs are the caller's."""
    w = I.workload("seir_t100_n1024", M=256, N=200, T=40, precision=I.PREC_MIXED)
    theta = _theta(w, 200)
    y_dev = torch.tensor(w.y, dtype=torch.float64, device="cuda")
    out = torch.empty(200, dtype=torch.float64, device="cuda")
    cfg = S.make_config(w, ppt=2)
    S.pf_loglik_noalloc(cfg, y_dev, theta, iteration=1, out=out)
    torch.cuda.synchronize()
    first = out.cpu().numpy().copy()
    free0 = torch.cuda.mem_get_info()[0]
    for it in range(3):
        S.pf_loglik_noalloc(cfg, y_dev, theta, iteration=1, out=out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, it
    assert np.array_equal(out.cpu().numpy(), first)


def test_a_smaller_call_does_not_shrink_a_context_launch(S):
    """A context whose filter needs much shared memory (M = 2048 at four
    particles per thread, one 512-thread group per CTA) still launches after an
    allocation-free call of the same kernel with a far smaller M."""
    w = I.workload("seir_t100_n1024", M=2048, N=40, T=30, precision=I.PREC_MIXED)
    theta = _theta(w, 40)
    ctx = S.SMC2(S.make_config(w, ppt=4, cta_threads=512, pf_family=S.PF_GROUPS), w.y)
    before = ctx.pf_loglik(theta, iteration=2).cpu().numpy()
    ws = I.workload("seir_t100_n1024", M=32, N=40, T=30, precision=I.PREC_MIXED)
    y_dev = torch.tensor(ws.y, dtype=torch.float64, device="cuda")
    S.pf_loglik_noalloc(S.make_config(ws, ppt=4), y_dev, theta, iteration=2)
    torch.cuda.synchronize()
    after = ctx.pf_loglik(theta, iteration=2).cpu().numpy()
    ctx.sync()
    ctx.close()
    assert np.array_equal(before, after)


def test_rejects_series_longer_than_the_scratch(S):
    w = I.workload("lg_t50_n64", M=64, N=4)
    cfg = S.make_config(w)
    cfg.T = 32001
    y_dev = torch.zeros(32001, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SMC2Error) as e:
        S.pf_loglik_noalloc(cfg, y_dev, soa(I.theta_near_prior(w, 4, seed=1)), iteration=1)
    assert e.value.status == S.EINVAL


def test_binding_rejects_short_or_mistyped_buffers(S):
    w = I.workload("lg_t50_n64", M=64, N=4)
    cfg = S.make_config(w)
    theta = soa(I.theta_near_prior(w, 4, seed=1))
    for y_bad in (torch.zeros(w.T - 1, dtype=torch.float64, device="cuda"),
                  torch.zeros(w.T, dtype=torch.float32, device="cuda")):
        with pytest.raises(S.SMC2Error) as e:
            S.pf_loglik_noalloc(cfg, y_bad, theta, iteration=1)
        assert e.value.status == S.EINVAL
    with pytest.raises(S.SMC2Error):
        S.pf_loglik_noalloc(cfg, torch.zeros(w.T, dtype=torch.float64, device="cuda"), theta[:2], iteration=1)
