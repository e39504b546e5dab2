"""The C-ABI library loads without a GPU, exports every entry point that
include/smc2.h declares, and rejects invalid arguments before touching the GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(smc2_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def S():
    from paper_2311_12973_gb300 import build
    build.build()
    from paper_2311_12973_gb300 import smc2
    return smc2


def test_every_declared_symbol_is_exported(S):
    names = declared_symbols()
    assert len(names) >= 19
    for n in names:
        assert hasattr(S.lib, n), n


def test_status_strings(S):
    for code in range(9):
        assert S.status_string(code) not in ("", "unknown status")
    assert S.status_string(99) == "unknown status"


def _cfg(S, **over):
    from paper_2311_12973_gb300 import inputs as I
    cfg = S.make_config(I.workload("lg_t50_n64"))
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


@pytest.mark.parametrize("over", [
    {"model": 7}, {"precision": 3}, {"proposal": 5}, {"lkernel": 9}, {"D": 4}, {"N": 0},
    {"N": 16385}, {"M": 0}, {"M": 4097}, {"T": 0}, {"K": 0}, {"rw_scale": 0.0},
    {"rw_scale": float("nan")}, {"ess_frac": -1.0}, {"ppt": 3}, {"cta_threads": 48},
    {"cta_threads": 1024}, {"ppt": 1, "M": 4096}, {"ppt": 4, "cta_threads": 64, "M": 1024},
    # learned proposal: needs the Gaussian L-kernel; bounded training settings
    {"proposal": 1, "lkernel": 0}, {"proposal": 1, "mlp_steps": 257}, {"proposal": 1, "mlp_window": 17},
    {"proposal": 1, "mlp_h": -1.0}, {"mlp_lr": 1.5}, {"mlp_h": float("nan")}, {"mlp_steps": -1},
    # particle-filter variants: known scheme, ESS fraction in [0, 1], register-resident shapes only
    {"pf_scheme": 2}, {"pf_scheme": -1}, {"pf_ess_frac": 1.5}, {"pf_ess_frac": -0.1},
    {"pf_ess_frac": float("nan")}, {"pf_scheme": 1, "ppt": 8},
    {"pf_ess_frac": 0.5, "ppt": 16}, {"pf_scheme": 1, "M": 4096},
    # priors and the SIR model: D = 2, integer population and infected, ppt <= 4
    {"prior_kind": 2}, {"model": 2}, {"model": 2, "D": 2, "npop": 10.5, "i0": 3.0},
    {"model": 2, "D": 2, "npop": 1e4, "i0": 2e4}, {"model": 2, "D": 2, "npop": 1e4, "i0": 2.5},
    {"model": 2, "D": 2, "npop": 1e8, "i0": 3.0}, {"model": 2, "D": 2, "npop": 1e4, "i0": 3.0, "ppt": 8},
])
def test_invalid_configs_rejected_before_gpu_work(S, over):
    import numpy as np
    cfg = _cfg(S, **over)
    y = np.zeros(64)
    ctx = C.c_void_p()
    assert S.lib.smc2_init(C.byref(cfg), y.ctypes.data, None, C.byref(ctx)) == S.EINVAL
    assert not ctx.value


def test_uniform_prior_needs_an_interval(S):
    import numpy as np
    from paper_2311_12973_gb300 import inputs as I
    y = np.zeros(64)
    ctx = C.c_void_p()
    for lo, hi in [(0.5, 0.5), (1.0, 0.0), (float("nan"), 1.0), (0.0, float("inf"))]:
        cfg = S.make_config(I.workload("sir_t30_n1024"))
        cfg.prior_lo[1], cfg.prior_hi[1] = lo, hi
        assert S.lib.smc2_init(C.byref(cfg), y.ctypes.data, None, C.byref(ctx)) == S.EINVAL
        assert not ctx.value


def test_invalid_prior_and_seir_constants(S):
    import numpy as np
    from paper_2311_12973_gb300 import inputs as I
    y = np.zeros(200)
    ctx = C.c_void_p()
    cfg = _cfg(S)
    cfg.prior_sd[1] = 0.0
    assert S.lib.smc2_init(C.byref(cfg), y.ctypes.data, None, C.byref(ctx)) == S.EINVAL
    w = I.workload("seir_t100_n1024")
    for over in ({"npop": 0.0}, {"n_sub": 0}, {"lambda_floor": 0.0}, {"i0": 2e6}):
        cfg = S.make_config(w, **over)
        assert S.lib.smc2_init(C.byref(cfg), y.ctypes.data, None, C.byref(ctx)) == S.EINVAL
    assert S.lib.smc2_init(None, y.ctypes.data, None, C.byref(ctx)) == S.EINVAL
    assert S.lib.smc2_init(C.byref(cfg), None, None, C.byref(ctx)) == S.EINVAL


def test_filters_that_do_not_fit_shared_memory_are_rejected(S):
    import numpy as np
    from paper_2311_12973_gb300 import inputs as I
    ctx = C.c_void_p()
    y = np.zeros(10)
    cfg = S.make_config(I.workload("seir_t100_n1024", T=10), precision=S.PREC_FP64, M=4096)
    assert S.lib.smc2_init(C.byref(cfg), y.ctypes.data, None, C.byref(ctx)) == S.EINVAL
    assert not ctx.value


def test_learned_proposal_needs_one_dataset(S):
    import numpy as np
    cfg = _cfg(S, proposal=1)
    arrs = [np.array([64, 64], dtype=np.int32), np.array([32, 32], dtype=np.int32),
            np.array([20, 20], dtype=np.int32)]
    cfg.n_datasets = 2
    cfg.ds_N, cfg.ds_M, cfg.ds_T = (a.ctypes.data_as(C.POINTER(C.c_int)) for a in arrs)
    y = np.zeros(40)
    ctx = C.c_void_p()
    assert S.lib.smc2_init(C.byref(cfg), y.ctypes.data, None, C.byref(ctx)) == S.EINVAL
    assert not ctx.value


def test_surrogate_entry_points_reject_bad_arguments(S):
    """Rejected on the host, before any device work: no buffer is touched."""
    a16, a20 = 4096, 4100  # never dereferenced
    assert S.lib.smc2_mlp_loss_grad(0, a16, a16, a16, 8, a16, a16, None) == S.EINVAL
    assert S.lib.smc2_mlp_loss_grad(4, a16, a16, a16, 0, a16, a16, None) == S.EINVAL
    assert S.lib.smc2_mlp_loss_grad(4, a20, a16, a16, 8, a16, a16, None) == S.EINVAL
    assert S.lib.smc2_mlp_input_grad(9, a16, a16, 8, None, a16, None) == S.EINVAL
    assert S.lib.smc2_mlp_input_grad(4, a20, a16, 8, None, a16, None) == S.EINVAL
    assert S.lib.smc2_mlp_adam_step(4, a16, a16, a16, None, a16, a16, 8, 1e-3, a16, None) == S.EINVAL
    assert S.lib.smc2_mlp_adam_step(4, a20, a16, a16, a16, a16, a16, 8, 1e-3, a16, None) == S.EINVAL
    assert S.lib.smc2_mlp_adam_step(4, a16, a16, a16, a16, a16, a16, 8, 2.0, a16, None) == S.EINVAL


def test_null_context_calls_rejected(S):
    assert S.lib.smc2_run(None, 1, None) == S.EINVAL
    assert S.lib.smc2_sync(None) == S.EINVAL
    assert S.lib.smc2_pf_loglik(None, None, 1, 1, 0, None) == S.EINVAL
    assert S.lib.smc2_resample_systematic(None, 4, 0, None, None) == S.EINVAL
    assert S.lib.smc2_philox_normals(1, None, 4, 0, None, None, None) == S.EINVAL
    S.lib.smc2_destroy(None)
