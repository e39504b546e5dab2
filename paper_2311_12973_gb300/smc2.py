"""Python binding of libsmc2.so: the C ABI of include/smc2.h, argument marshalling only.

Device buffers are torch CUDA tensors (passed as raw pointers); streams are
torch CUDA streams.  Every computation happens in the library's CUDA kernels;
importing this module fails loudly when the library has not been built, and no
call falls back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MAX_D = 8
OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ECHOL, ETIMEOUT, EBOUNDS, ESTATE = range(9)
MODEL_LG_AR1, MODEL_SEIR = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
PROP_RW, PROP_MLP = 0, 1
PF_SYSTEMATIC, PF_MULTINOMIAL = 0, 1
PRIOR_GAUSS, PRIOR_UNIFORM = 0, 1
PF_ANY, PF_GROUPS, PF_FP32 = 0, 1, 2
LK_FORWARD, LK_GAUSS_OPT = 0, 1


class Config(C.Structure):
    _fields_ = [
        ("model", C.c_int), ("precision", C.c_int), ("proposal", C.c_int), ("lkernel", C.c_int),
        ("D", C.c_int), ("N", C.c_int), ("M", C.c_int), ("T", C.c_int), ("K", C.c_int),
        ("rw_scale", C.c_double), ("ess_frac", C.c_double), ("seed", C.c_uint64),
        ("prior_mean", C.c_double * MAX_D), ("prior_sd", C.c_double * MAX_D),
        ("npop", C.c_double), ("e0", C.c_double), ("i0", C.c_double), ("lambda_floor", C.c_double),
        ("n_sub", C.c_int), ("ppt", C.c_int), ("cta_threads", C.c_int), ("n_datasets", C.c_int),
        ("ds_N", C.POINTER(C.c_int)), ("ds_M", C.POINTER(C.c_int)), ("ds_T", C.POINTER(C.c_int)),
        ("mlp_h", C.c_double), ("mlp_lr", C.c_double), ("mlp_steps", C.c_int), ("mlp_window", C.c_int),
        ("pf_ess_frac", C.c_double), ("pf_scheme", C.c_int), ("prior_kind", C.c_int),
        ("prior_lo", C.c_double * MAX_D), ("prior_hi", C.c_double * MAX_D), ("pf_family", C.c_int),
    ]


class IterStats(C.Structure):
    _fields_ = [
        ("k", C.c_int), ("resampled", C.c_int), ("lk_fallback", C.c_int), ("dataset", C.c_int),
        ("ess", C.c_double), ("lse", C.c_double), ("lse2", C.c_double), ("logz", C.c_double),
        ("est", C.c_double * MAX_D), ("mlp_used", C.c_int), ("pad", C.c_int), ("mlp_loss", C.c_double),
        ("cov", C.c_double * (MAX_D * MAX_D)),
    ]

    def as_dict(self, D: int) -> dict:
        return {"k": self.k, "resampled": self.resampled, "lk_fallback": self.lk_fallback,
                "dataset": self.dataset, "ess": self.ess, "lse": self.lse, "lse2": self.lse2,
                "logz": self.logz, "est": np.array(self.est[:D]), "mlp_used": self.mlp_used,
                "mlp_loss": self.mlp_loss,
                "cov": np.array(self.cov[:]).reshape(MAX_D, MAX_D)[:D, :D].copy()}


class SMC2Error(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        detail = ""
        if status in (ECUDA, ENOMEM):
            detail = " [" + lib.smc2_last_error_string().decode() + "]"
        super().__init__(f"{what}: {status_string(status)} ({status}){detail}")


def _load() -> C.CDLL:
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libsmc2.so is not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, dp, i32p, u32p, u64p = C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p
    st = C.c_int
    ctx = C.c_void_p
    sig = {
        "smc2_init": ([C.POINTER(Config), dp, vp, C.POINTER(ctx)], st),
        "smc2_set_observations": ([ctx, dp], st),
        "smc2_reset": ([ctx, C.c_uint64], st),
        "smc2_pf_loglik": ([ctx, dp, C.c_int, C.c_int, C.c_int, dp], st),
        "smc2_pf_trace": ([ctx, dp, C.c_int, C.c_int, C.c_int, dp, dp, i32p], st),
        "smc2_iterate": ([ctx, C.POINTER(IterStats)], st),
        "smc2_run": ([ctx, C.c_int, C.POINTER(IterStats)], st),
        "smc2_estimate": ([ctx, C.c_int, dp, dp, dp, dp], st),
        "smc2_get_history": ([ctx, C.c_int, C.POINTER(IterStats), C.c_int, C.POINTER(C.c_int)], st),
        "smc2_get_state": ([ctx, C.c_int, C.POINTER(C.c_int), dp, dp, dp, dp], st),
        "smc2_set_state": ([ctx, C.c_int, C.c_int, dp, dp, dp, dp], st),
        "smc2_set_history": ([ctx, C.c_int, C.POINTER(IterStats), C.c_int], st),
        "smc2_resample_systematic": ([u64p, C.c_int, C.c_uint32, i32p, vp], st),
        "smc2_philox_normals": ([C.c_uint64, u32p, C.c_int, C.c_int, u32p, dp, vp], st),
        "smc2_sync": ([ctx], st),
        "smc2_set_timing": ([ctx, C.c_int], st),
        "smc2_get_timing": ([ctx, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                             C.POINTER(C.c_int64), C.c_int], st),
        "smc2_get_launch_shape": ([ctx, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int)], st),
        "smc2_pf_trace_states": ([ctx, dp, C.c_int, C.c_int, C.c_int, dp, dp, i32p, dp, dp, dp], st),
        "smc2_pf_loglik_noalloc": ([C.POINTER(Config), dp, dp, C.c_int, C.c_int, dp, vp], st),
        "smc2_mlp_loss_grad": ([C.c_int, dp, dp, dp, C.c_int, dp, dp, vp], st),
        "smc2_mlp_input_grad": ([C.c_int, dp, dp, C.c_int, dp, dp, vp], st),
        "smc2_mlp_adam_step": ([C.c_int, dp, dp, dp, dp, dp, dp, C.c_int, C.c_float, dp, vp], st),
        "smc2_get_proposals": ([ctx, C.c_int, dp, dp], st),
        "smc2_fma_rates": ([dp, dp, vp], st),
        "smc2_get_learned_state": ([ctx, dp, dp, dp, C.POINTER(C.c_int)], st),
        "smc2_get_learned_training": ([ctx, dp, dp, dp, C.POINTER(C.c_int), dp, dp, dp, C.POINTER(C.c_int)], st),
        "smc2_mlp_train_ring": ([C.c_int, dp, dp, dp, dp, dp, dp, C.c_int, C.c_int, C.c_float, dp, dp, dp, vp],
                                st),
        "smc2_destroy": ([ctx], None),
        "smc2_status_string": ([st], C.c_char_p),
        "smc2_last_error_string": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def status_string(s: int) -> str:
    return lib.smc2_status_string(int(s)).decode()


def _check(status: int, what: str):
    if status != OK:
        raise SMC2Error(status, what)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def make_config(w, **over) -> Config:
    """smc2_config from a workload description (attributes named as in the config)."""
    c = Config()
    get = lambda k, d=None: over.get(k, getattr(w, k, d))
    c.model, c.precision = get("model"), get("precision", PREC_FP64)
    c.proposal, c.lkernel = get("proposal", PROP_RW), get("lkernel", LK_GAUSS_OPT)
    c.D, c.N, c.M, c.T, c.K = get("D"), get("N"), get("M"), get("T"), get("K")
    c.rw_scale, c.ess_frac, c.seed = get("rw_scale"), get("ess_frac"), get("seed")
    for d in range(c.D):
        c.prior_mean[d] = get("prior_mean")[d]
        c.prior_sd[d] = get("prior_sd")[d]
    c.npop, c.e0, c.i0 = get("npop", 0.0), get("e0", 0.0), get("i0", 0.0)
    c.lambda_floor, c.n_sub = get("lambda_floor", 1e-3), get("n_sub", 1)
    c.ppt = get("ppt", 0)
    c.cta_threads = get("cta_threads", 0)
    c.n_datasets = 0
    c.mlp_h, c.mlp_lr = get("mlp_h", 0.0), get("mlp_lr", 0.0)
    c.mlp_steps, c.mlp_window = get("mlp_steps", 0), get("mlp_window", 0)
    c.pf_ess_frac, c.pf_scheme = get("pf_ess_frac", 0.0), get("pf_scheme", PF_SYSTEMATIC)
    c.prior_kind = get("prior_kind", PRIOR_GAUSS)
    c.pf_family = get("pf_family", PF_ANY)
    if c.prior_kind == PRIOR_UNIFORM:
        for d in range(c.D):
            c.prior_lo[d] = get("prior_lo")[d]
            c.prior_hi[d] = get("prior_hi")[d]
    return c


class SMC2:
    """One sampler context (smc2_ctx) on the current CUDA device and stream."""

    def __init__(self, cfg: Config, y, stream=None, datasets=None):
        self.cfg = cfg
        self.D = cfg.D
        self._keep = []
        if datasets is not None:   # list of (N, M, T)
            n = len(datasets)
            arrs = [np.ascontiguousarray([d[a] for d in datasets], dtype=np.int32) for a in range(3)]
            self._keep += arrs
            cfg.n_datasets = n
            cfg.ds_N, cfg.ds_M, cfg.ds_T = (a.ctypes.data_as(C.POINTER(C.c_int)) for a in arrs)
        self.n_ds = max(1, cfg.n_datasets)
        self.Ns = [d[0] for d in datasets] if datasets is not None else [cfg.N]
        self.Ms = [d[1] for d in datasets] if datasets is not None else [cfg.M]
        self.Ts = [d[2] for d in datasets] if datasets is not None else [cfg.T]
        self.stream = _stream_handle(stream)
        y = self._host_or_device(y)
        self._ctx = C.c_void_p()
        _check(lib.smc2_init(C.byref(cfg), _ptr(y), self.stream, C.byref(self._ctx)), "smc2_init")

    @staticmethod
    def _host_or_device(y):
        if hasattr(y, "data_ptr"):
            return y.contiguous()
        return np.ascontiguousarray(y, dtype=np.float64)

    def close(self):
        if self._ctx:
            lib.smc2_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- sampler ----------------------------------------------------------
    def run(self, n_iter: int, stats: bool = True):
        if not stats:
            _check(lib.smc2_run(self._ctx, int(n_iter), None), "smc2_run")
            return None
        arr = (IterStats * (n_iter * self.n_ds))()
        _check(lib.smc2_run(self._ctx, int(n_iter), arr), "smc2_run")
        return [[arr[i * self.n_ds + d].as_dict(self.D) for d in range(self.n_ds)] for i in range(n_iter)]

    def iterate(self):
        return self.run(1)[0]

    def estimate(self, dataset: int = 0):
        mean = np.zeros(self.D)
        logz, ess = C.c_double(), C.c_double()
        _check(lib.smc2_estimate(self._ctx, dataset, mean.ctypes.data, C.byref(logz), C.byref(ess), None),
               "smc2_estimate")
        return mean, logz.value, ess.value

    def estimate_cov(self, dataset: int = 0):
        """Recycled posterior covariance [D][D] (Eq. 29 applied to theta theta^T)."""
        cov = np.zeros((self.D, self.D))
        _check(lib.smc2_estimate(self._ctx, dataset, None, None, None, cov.ctypes.data), "smc2_estimate")
        return cov

    def history(self, dataset: int = 0, cap: int | None = None):
        cap = cap or self.cfg.K
        arr = (IterStats * cap)()
        k = C.c_int()
        _check(lib.smc2_get_history(self._ctx, dataset, arr, cap, C.byref(k)), "smc2_get_history")
        return [arr[i].as_dict(self.D) for i in range(min(k.value, cap))]

    def raw_history(self, dataset: int = 0):
        cap = self.cfg.K
        arr = (IterStats * cap)()
        k = C.c_int()
        _check(lib.smc2_get_history(self._ctx, dataset, arr, cap, C.byref(k)), "smc2_get_history")
        return arr, k.value

    def set_history(self, arr, k: int, dataset: int = 0):
        _check(lib.smc2_set_history(self._ctx, dataset, arr, int(k)), "smc2_set_history")

    def get_state(self, dataset: int = 0):
        N = self.Ns[dataset]
        th, lp, ll, lw = np.zeros((N, self.D)), np.zeros(N), np.zeros(N), np.zeros(N)
        k = C.c_int()
        _check(lib.smc2_get_state(self._ctx, dataset, C.byref(k), th.ctypes.data, lp.ctypes.data,
                                  ll.ctypes.data, lw.ctypes.data), "smc2_get_state")
        return k.value, th, lp, ll, lw

    def set_state(self, k, theta, logprior, loglik, logw, dataset: int = 0):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (theta, logprior, loglik, logw)]
        _check(lib.smc2_set_state(self._ctx, dataset, int(k), *(a.ctypes.data for a in arrs)),
               "smc2_set_state")

    def proposals(self, dataset: int = 0):
        """theta_k of the latest iteration [N][D] and log q(theta_k | theta_{k-1}) [N]."""
        N = self.Ns[dataset]
        th, lq = np.zeros((N, self.D)), np.zeros(N)
        _check(lib.smc2_get_proposals(self._ctx, dataset, th.ctypes.data, lq.ctypes.data), "smc2_get_proposals")
        return th, lq

    def learned_state(self):
        """The learned proposal's published network and standardisation, and the
        population Cholesky factor the next iteration proposes with."""
        D = self.D
        params = np.zeros(64 * D + 4289, dtype=np.float32)
        stdz = np.zeros(2 * D + 6)
        L = np.zeros((D, D))
        ok = C.c_int()
        _check(lib.smc2_get_learned_state(self._ctx, params.ctypes.data, stdz.ctypes.data, L.ctypes.data,
                                          C.byref(ok)), "smc2_get_learned_state")
        return {"params": params, **_stdz_dict(stdz, D), "L": L, "pop_ok": bool(ok.value)}

    def learned_training(self):
        """The learned proposal's training state after the latest training call
        (not yet published): parameters, Adam moments and step, the call's
        standardisation and loss, and the ring of training pairs."""
        D = self.D
        P = 64 * D + 4289
        rows = 16 * self.Ns[0]   # room for the largest ring (mlp_window <= 16 iterations of N rows)
        params, m, v = (np.zeros(P, dtype=np.float32) for _ in range(3))
        stdz = np.zeros(2 * D + 6)
        th = np.zeros((rows, D), dtype=np.float32)
        lp = np.zeros(rows, dtype=np.float32)
        step, filled = C.c_int(), C.c_int()
        _check(lib.smc2_get_learned_training(self._ctx, params.ctypes.data, m.ctypes.data, v.ctypes.data,
                                             C.byref(step), stdz.ctypes.data, th.ctypes.data, lp.ctypes.data,
                                             C.byref(filled)), "smc2_get_learned_training")
        return {"params": params, "m": m, "v": v, "step": step.value, **_stdz_dict(stdz, D),
                "ring_th": th[:filled.value].copy(), "ring_lp": lp[:filled.value].copy(),
                "ring_rows": filled.value}

    def reset(self, seed: int):
        _check(lib.smc2_reset(self._ctx, int(seed)), "smc2_reset")

    def set_observations(self, y):
        y = self._host_or_device(y)
        self._keep_y = y
        _check(lib.smc2_set_observations(self._ctx, _ptr(y)), "smc2_set_observations")

    def sync(self):
        _check(lib.smc2_sync(self._ctx), "smc2_sync")

    # -- particle filter ---------------------------------------------------
    def pf_loglik(self, theta_soa, iteration: int, dataset: int = 0, out=None):
        """theta_soa: CUDA float64 tensor [D][n]; returns CUDA float64 [n]."""
        import torch
        n = self._theta_n(theta_soa, "smc2_pf_loglik")
        self._dataset_dims(dataset)
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=theta_soa.device)
        elif not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() >= n):
            raise SMC2Error(EINVAL, "smc2_pf_loglik: out must be a contiguous CUDA float64 tensor of n values")
        _check(lib.smc2_pf_loglik(self._ctx, _ptr(theta_soa), n, int(iteration), dataset, _ptr(out)),
               "smc2_pf_loglik")
        return out

    def pf_trace(self, theta_soa, iteration: int, dataset: int = 0):
        """Log-likelihoods [n], increments [n][T] and ancestors [n][T-1][M] of the
        dataset's filters (T, M of that dataset)."""
        import torch
        n = self._theta_n(theta_soa, "smc2_pf_trace")
        M, T = self._dataset_dims(dataset)
        dev = theta_soa.device
        ll = torch.empty(n, dtype=torch.float64, device=dev)
        delta = torch.empty((n, T), dtype=torch.float64, device=dev)
        anc = torch.empty((n, max(T - 1, 0), M), dtype=torch.int32, device=dev)
        _check(lib.smc2_pf_trace(self._ctx, _ptr(theta_soa), n, int(iteration), dataset, _ptr(ll),
                                 _ptr(delta), _ptr(anc)), "smc2_pf_trace")
        return ll, delta, anc

    def _theta_n(self, theta_soa, what: str) -> int:
        """n of a [D][n] CUDA float64 parameter array, checked."""
        import torch
        if not (hasattr(theta_soa, "is_cuda") and theta_soa.is_cuda and theta_soa.dtype == torch.float64
                and theta_soa.is_contiguous() and theta_soa.dim() == 2 and theta_soa.shape[0] == self.D):
            raise SMC2Error(EINVAL, f"{what}: theta must be a contiguous CUDA float64 tensor [D][n]")
        return theta_soa.shape[1]

    def _dataset_dims(self, dataset: int):
        if not 0 <= dataset < len(self.Ms):
            raise SMC2Error(EINVAL, f"dataset {dataset} of {len(self.Ms)}")
        return self.Ms[dataset], self.Ts[dataset]

    def launch_shape(self):
        a, b, c, f = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(lib.smc2_get_launch_shape(self._ctx, C.byref(a), C.byref(b), C.byref(c), C.byref(f)),
               "smc2_get_launch_shape")
        return {"ppt": a.value, "cta_threads": b.value, "grid": c.value, "fp32_filter": f.value}

    def pf_trace_states(self, theta_soa, iteration: int, dataset: int = 0):
        """The FP32 filter's per-step trace: log-likelihoods [n], increments [n][T],
        ancestors [n][T-1][M], post-propagation states [n][T][M][5], log-weights
        [n][T][M] and quantised weights [n][T][M] (int64 storage of uint64)."""
        import torch
        n = self._theta_n(theta_soa, "smc2_pf_trace")
        M, T = self._dataset_dims(dataset)
        dev = theta_soa.device
        ll = torch.empty(n, dtype=torch.float64, device=dev)
        delta = torch.empty((n, T), dtype=torch.float64, device=dev)
        anc = torch.empty((n, max(T - 1, 0), M), dtype=torch.int32, device=dev)
        x = torch.empty((n, T, M, 5), dtype=torch.float32, device=dev)
        lw = torch.empty((n, T, M), dtype=torch.float32, device=dev)
        q = torch.empty((n, T, M), dtype=torch.int64, device=dev)
        _check(lib.smc2_pf_trace_states(self._ctx, _ptr(theta_soa), n, int(iteration), dataset, _ptr(ll),
                                        _ptr(delta), _ptr(anc), _ptr(x), _ptr(lw), _ptr(q)),
               "smc2_pf_trace_states")
        return ll, delta, anc, x, lw, q

    # -- timing -------------------------------------------------------------
    def set_timing(self, on: bool):
        _check(lib.smc2_set_timing(self._ctx, int(bool(on))), "smc2_set_timing")

    def timing(self, reset: bool = False):
        ms, n, kl = C.c_double(), C.c_int64(), C.c_int64()
        _check(lib.smc2_get_timing(self._ctx, C.byref(ms), C.byref(n), C.byref(kl), int(reset)),
               "smc2_get_timing")
        return ms.value, n.value, kl.value


def _stdz_dict(stdz, D: int) -> dict:
    """The 2 D + 6 standardisation values of the learned proposal, by name."""
    return {"mu": stdz[:D].copy(), "sd": stdz[D:2 * D].copy(), "tau": stdz[2 * D], "zmean": stdz[2 * D + 1],
            "zsd": stdz[2 * D + 2], "var_y": stdz[2 * D + 3], "loss": stdz[2 * D + 4], "ymax": stdz[2 * D + 5]}


def mlp_train_ring(params, m, v, step, ring_th, ring_lp, steps: int, lr: float, stream=None):
    """The sampler's training call on CUDA float32 tensors (in place on params,
    m, v and the int32 step counter); returns (x, y, stdz dict) of the training set."""
    import torch
    R, D = ring_th.shape
    x = torch.empty((R, D), dtype=torch.float32, device=params.device)
    y = torch.empty(R, dtype=torch.float32, device=params.device)
    stdz = torch.empty(2 * D + 6, dtype=torch.float64, device=params.device)
    _check(lib.smc2_mlp_train_ring(D, _ptr(params), _ptr(m), _ptr(v), _ptr(step), _ptr(ring_th), _ptr(ring_lp),
                                   R, int(steps), float(lr), _ptr(x), _ptr(y), _ptr(stdz),
                                   _stream_handle(stream)), "smc2_mlp_train_ring")
    return x, y, _stdz_dict(stdz.cpu().numpy(), D)


def pf_loglik_noalloc(cfg: Config, y_dev, theta_soa, iteration: int, out=None, stream=None):
    """smc2_pf_loglik_noalloc: no context and no device allocation by the library.
    y_dev: CUDA float64 [T]; theta_soa: CUDA float64 [D][n]; returns CUDA float64 [n]."""
    import torch

    def device_f64(t, what):
        if not (hasattr(t, "is_cuda") and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise SMC2Error(EINVAL, f"smc2_pf_loglik_noalloc: {what} must be a contiguous CUDA float64 tensor")

    # the C entry point reads T doubles of y and D rows of theta through raw pointers
    device_f64(y_dev, "y_dev")
    device_f64(theta_soa, "theta_soa")
    if y_dev.numel() < cfg.T:
        raise SMC2Error(EINVAL, f"smc2_pf_loglik_noalloc: y_dev holds {y_dev.numel()} < T = {cfg.T} values")
    if theta_soa.dim() != 2 or theta_soa.shape[0] != cfg.D:
        raise SMC2Error(EINVAL, f"smc2_pf_loglik_noalloc: theta_soa must be [D = {cfg.D}][n]")
    n = theta_soa.shape[1]
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=theta_soa.device)
    else:
        device_f64(out, "out")
        if out.numel() < n:
            raise SMC2Error(EINVAL, "smc2_pf_loglik_noalloc: out holds fewer than n values")
    _check(lib.smc2_pf_loglik_noalloc(C.byref(cfg), _ptr(y_dev), _ptr(theta_soa), n, int(iteration),
                                      _ptr(out), _stream_handle(stream)), "smc2_pf_loglik_noalloc")
    return out


def mlp_loss_grad(params, x, y, stream=None):
    """params, x [R][D], y: CUDA float32 tensors; returns (loss, grad) as CUDA tensors."""
    import torch
    R, D = x.shape
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _check(lib.smc2_mlp_loss_grad(D, _ptr(params), _ptr(x), _ptr(y), R, _ptr(grad), _ptr(loss),
                                  _stream_handle(stream)), "smc2_mlp_loss_grad")
    return loss, grad


def mlp_input_grad(params, x, stream=None):
    import torch
    R, D = x.shape
    s = torch.empty(R, dtype=torch.float32, device=params.device)
    dx = torch.empty((R, D), dtype=torch.float32, device=params.device)
    _check(lib.smc2_mlp_input_grad(D, _ptr(params), _ptr(x), R, _ptr(s), _ptr(dx),
                                   _stream_handle(stream)), "smc2_mlp_input_grad")
    return s, dx


def mlp_adam_step(params, m, v, step, x, y, lr: float, stream=None):
    """One gradient + Adam step in place on CUDA float32 tensors params, m, v and
    the CUDA int32 step counter; returns the loss before the step (CUDA tensor)."""
    import torch
    R, D = x.shape
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _check(lib.smc2_mlp_adam_step(D, _ptr(params), _ptr(m), _ptr(v), _ptr(step), _ptr(x), _ptr(y), R,
                                  float(lr), _ptr(loss), _stream_handle(stream)), "smc2_mlp_adam_step")
    return loss


def fma_rates(stream=None):
    """Measured FP32 and FP64 FMA throughput of the device, FLOP/s."""
    f32, f64 = C.c_double(), C.c_double()
    _check(lib.smc2_fma_rates(C.byref(f32), C.byref(f64), _stream_handle(stream)), "smc2_fma_rates")
    return f32.value, f64.value


def resample_systematic(q, U: int, anc, stream=None):
    """q: CUDA uint64 (int64 storage) [n]; anc: CUDA int32 [n]."""
    _check(lib.smc2_resample_systematic(_ptr(q), q.numel(), int(U) & 0xFFFFFFFF, _ptr(anc),
                                        _stream_handle(stream)), "smc2_resample_systematic")
    return anc


def philox_normals(seed: int, ctr, precision: int, words=None, z=None, stream=None):
    """ctr: CUDA int32 [n][4] holding uint32 counters."""
    n = ctr.shape[0]
    _check(lib.smc2_philox_normals(int(seed), _ptr(ctr), n, int(precision), _ptr(words), _ptr(z),
                                   _stream_handle(stream)), "smc2_philox_normals")
