"""ctypes wrapper of the FP64 CPU oracle (smc2_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` load it.  The CUDA library never imports,
links or calls anything here, and nothing here imports the CUDA package.

Every function is a thin marshalling layer over the C oracle; the arithmetic
is all in ``smc2_oracle.c``, which follows the paper section by section.
Arrays cross the boundary as numpy arrays; the population layout on this side
is row-major ``theta[N][D]``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smc2_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

LG, SEIR, SIR = 0, 1, 2
PRIOR_GAUSS, PRIOR_UNIFORM = 0, 1
LK_FORWARD, LK_GAUSS = 0, 1
MAX_D = 8
TAG_THETA_INIT, TAG_PROPOSE, TAG_OUTER_RES = 1, 2, 3
TAG_PF_INIT, TAG_PF_PROP, TAG_PF_RES = 4, 5, 6
TAG_PF_MULTI, TAG_PF_BINOM = 8, 9
PF_SYSTEMATIC, PF_MULTINOMIAL = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    hdr = os.path.join(_HERE, "smc2_oracle.h")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class OracleCfg(C.Structure):
    _fields_ = [
        ("model", C.c_int), ("D", C.c_int), ("N", C.c_int), ("M", C.c_int), ("T", C.c_int),
        ("lkernel", C.c_int), ("dataset", C.c_int),
        ("rw_scale", C.c_double), ("ess_frac", C.c_double), ("seed", C.c_uint64),
        ("prior_mean", C.c_double * MAX_D), ("prior_sd", C.c_double * MAX_D),
        ("npop", C.c_double), ("e0", C.c_double), ("i0", C.c_double),
        ("lambda_floor", C.c_double), ("n_sub", C.c_int),
        ("pf_scheme", C.c_int), ("pf_ess_frac", C.c_double),
        ("prior_kind", C.c_int), ("prior_lo", C.c_double * MAX_D), ("prior_hi", C.c_double * MAX_D),
    ]


class OracleStats(C.Structure):
    _fields_ = [
        ("k", C.c_int), ("resampled", C.c_int), ("lk_fallback", C.c_int), ("pad", C.c_int),
        ("lse", C.c_double), ("lse2", C.c_double), ("ess", C.c_double), ("logz", C.c_double),
        ("est", C.c_double * MAX_D), ("cov", C.c_double * (MAX_D * MAX_D)),
    ]


class MlpNorm(C.Structure):
    _fields_ = [
        ("mu", C.c_double * MAX_D), ("sd", C.c_double * MAX_D), ("ymax", C.c_double), ("tau", C.c_double),
        ("zmean", C.c_double), ("zsd", C.c_double), ("var_y", C.c_double), ("rows", C.c_int),
        ("rows_moments", C.c_int),
    ]

    def as_dict(self, D: int) -> dict:
        return {"mu": np.array(self.mu[:D]), "sd": np.array(self.sd[:D]), "ymax": self.ymax, "tau": self.tau,
                "zmean": self.zmean, "zsd": self.zsd, "var_y": self.var_y, "rows": self.rows,
                "rows_moments": self.rows_moments}

    @classmethod
    def from_dict(cls, d: dict) -> "MlpNorm":
        n = cls()
        D = len(d["mu"])
        for i in range(D):
            n.mu[i] = float(d["mu"][i])
            n.sd[i] = float(d["sd"][i])
        for k in ("ymax", "tau", "zmean", "zsd", "var_y"):
            setattr(n, k, float(d.get(k, 0.0)))
        n.rows = int(d.get("rows", 0))
        n.rows_moments = int(d.get("rows_moments", 0))
        return n


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _declare(L):
    dp, ip, up = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_uint32)
    u64p = C.POINTER(C.c_uint64)
    L.oracle_philox4x32_10.argtypes = [up, up, up]
    L.oracle_uniform23.argtypes = [C.c_uint32]
    L.oracle_uniform23.restype = C.c_double
    L.oracle_normals4.argtypes = [C.c_uint64] + [C.c_uint32] * 4 + [dp]
    L.oracle_kalman_loglik.argtypes = [C.c_double, C.c_double, C.c_double, dp, C.c_int]
    L.oracle_kalman_loglik.restype = C.c_double
    L.oracle_fixed_point_bits.argtypes = [C.c_int]
    L.oracle_fixed_point_bits.restype = C.c_int
    L.oracle_quantise.argtypes = [dp, C.c_int, u64p]
    L.oracle_quantise.restype = C.c_int
    L.oracle_systematic_from_q.argtypes = [u64p, C.c_int, C.c_uint32, ip, ip]
    L.oracle_systematic_from_q.restype = C.c_int
    L.oracle_log_obs.argtypes = [C.POINTER(OracleCfg), dp, dp, C.c_double]
    L.oracle_log_obs.restype = C.c_double
    L.oracle_pf_loglik.argtypes = [C.POINTER(OracleCfg), dp, dp, C.c_uint32, C.c_uint32, dp, ip]
    L.oracle_pf_initial.argtypes = [C.POINTER(OracleCfg), dp, C.c_uint32, C.c_uint32, dp]
    L.oracle_pf_propagate.argtypes = [C.POINTER(OracleCfg), dp, C.c_uint32, C.c_uint32, C.c_int, C.c_double, dp, dp]
    L.oracle_pf_resample_word.argtypes = [C.POINTER(OracleCfg), C.c_uint32, C.c_uint32, C.c_int]
    L.oracle_pf_resample_word.restype = C.c_uint32
    L.oracle_pf_log_weights.argtypes = [C.POINTER(OracleCfg), dp, dp, C.c_double, dp]
    L.oracle_pf_loglik.restype = C.c_double
    L.oracle_log_prior.argtypes = [C.POINTER(OracleCfg), dp]
    L.oracle_log_prior.restype = C.c_double
    L.oracle_lkernel_fit.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp, dp, dp, dp]
    L.oracle_lkernel_fit.restype = C.c_int
    L.oracle_gauss_lkernel_logpdf.argtypes = [C.c_int, dp, dp, dp, C.c_double, dp, dp]
    L.oracle_gauss_lkernel_logpdf.restype = C.c_double
    L.oracle_smc2_step.argtypes = [C.POINTER(OracleCfg), dp, C.c_int, dp, dp, dp, dp,
                                   C.POINTER(OracleStats)]
    L.oracle_smc2_step.restype = C.c_int
    L.oracle_recycle.argtypes = [C.c_int, C.c_int, C.POINTER(OracleStats), dp, dp]
    L.oracle_multinomial_from_q.argtypes = [C.POINTER(C.c_uint64), C.c_int, C.POINTER(C.c_uint32),
                                            C.POINTER(C.c_int32)]
    L.oracle_multinomial_from_q.restype = C.c_int
    L.oracle_ess_from_q.argtypes = [C.POINTER(C.c_uint64), C.c_int]
    L.oracle_ess_from_q.restype = C.c_double
    L.oracle_recycle_cov.argtypes = [C.c_int, C.c_int, C.POINTER(OracleStats), dp]
    L.oracle_binomial.argtypes = [C.c_double, C.c_double, C.c_uint64] + [C.c_uint32] * 4 + [ip]
    L.oracle_binomial.restype = C.c_double
    L.oracle_bf16.argtypes = [C.c_double]
    L.oracle_bf16.restype = C.c_double
    L.oracle_mlp_nparams.argtypes = [C.c_int, C.c_int]
    L.oracle_mlp_nparams.restype = C.c_int
    L.oracle_mlp_forward.argtypes = [C.c_int, C.c_int, dp, dp, C.c_int, C.c_int, dp]
    L.oracle_mlp_loss_grad.argtypes = [C.c_int, C.c_int, dp, dp, dp, C.c_int, C.c_int, dp]
    L.oracle_mlp_loss_grad.restype = C.c_double
    L.oracle_mlp_input_grad.argtypes = [C.c_int, C.c_int, dp, dp, C.c_int, C.c_int, dp, dp]
    L.oracle_adam_step.argtypes = [C.c_int, dp, dp, dp, dp, C.c_int, C.c_double, C.c_double,
                                   C.c_double, C.c_double]
    L.oracle_mlp_weights_bf16.argtypes = [C.c_int, C.c_int, dp, dp]
    L.oracle_mlp_standardise.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, C.POINTER(MlpNorm)]
    L.oracle_mlp_standardise.restype = C.c_int
    L.oracle_mlp_train.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, C.c_double, C.c_int,
                                   dp, dp, dp, C.POINTER(C.c_int), C.POINTER(MlpNorm), dp, dp]
    L.oracle_mlp_train.restype = C.c_double
    L.oracle_mlp_score.argtypes = [C.c_int, C.c_int, dp, C.POINTER(MlpNorm), dp, C.c_int, C.c_int, dp]
    L.oracle_population_factor.argtypes = [C.c_int, dp, C.c_double, dp]
    L.oracle_population_factor.restype = C.c_int
    L.oracle_learned_decision.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int]
    L.oracle_learned_decision.restype = C.c_int
    L.oracle_langevin_propose.argtypes = [C.c_int, C.c_double, dp, dp, dp, dp, dp, dp]


# --------------------------------------------------------------------------
# configuration
# --------------------------------------------------------------------------

@dataclass
class Config:
    """Plain description of one SMC^2 problem, as the oracle sees it."""
    model: int
    D: int
    N: int
    M: int
    T: int
    K: int = 1
    lkernel: int = LK_GAUSS
    dataset: int = 0
    rw_scale: float = 0.1
    ess_frac: float = 0.5
    seed: int = 1
    prior_mean: list = field(default_factory=list)
    prior_sd: list = field(default_factory=list)
    npop: float = 0.0
    e0: float = 0.0
    i0: float = 0.0
    lambda_floor: float = 1e-3
    n_sub: int = 2
    pf_scheme: int = 0          # 0 systematic, 1 multinomial
    pf_ess_frac: float = 0.0    # <= 0: resample every step; else when ESS < pf_ess_frac * M
    prior_kind: int = PRIOR_GAUSS
    prior_lo: list = field(default_factory=list)   # uniform prior support (PRIOR_UNIFORM)
    prior_hi: list = field(default_factory=list)

    def ctype(self) -> OracleCfg:
        c = OracleCfg()
        c.model, c.D, c.N, c.M, c.T = self.model, self.D, self.N, self.M, self.T
        c.lkernel, c.dataset = self.lkernel, self.dataset
        c.rw_scale, c.ess_frac, c.seed = self.rw_scale, self.ess_frac, self.seed
        for d in range(self.D):
            c.prior_mean[d] = self.prior_mean[d]
            c.prior_sd[d] = self.prior_sd[d]
        c.npop, c.e0, c.i0 = self.npop, self.e0, self.i0
        c.lambda_floor, c.n_sub = self.lambda_floor, self.n_sub
        c.pf_scheme, c.pf_ess_frac = self.pf_scheme, self.pf_ess_frac
        c.prior_kind = self.prior_kind
        if self.prior_kind == PRIOR_UNIFORM:
            for d in range(self.D):
                c.prior_lo[d] = self.prior_lo[d]
                c.prior_hi[d] = self.prior_hi[d]
        return c


def config_from(w, **over) -> Config:
    """Build a Config from any object with the workload's attribute names."""
    keys = Config.__dataclass_fields__.keys()
    kw = {k: getattr(w, k) for k in keys if hasattr(w, k)}
    kw.update(over)
    return Config(**kw)


# --------------------------------------------------------------------------
# primitives
# --------------------------------------------------------------------------

def philox(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def uniform23(w: int) -> float:
    return lib().oracle_uniform23(int(w))


def normals4(seed, c0, c1, c2, c3) -> np.ndarray:
    z = np.zeros(4)
    lib().oracle_normals4(int(seed), int(c0), int(c1), int(c2), int(c3), _p(z, C.c_double))
    return z


def kalman_loglik(phi, sx, sy, y) -> float:
    y = np.ascontiguousarray(y, dtype=np.float64)
    return lib().oracle_kalman_loglik(float(phi), float(sx), float(sy), _p(y, C.c_double), len(y))


def fixed_point_bits(n: int) -> int:
    return lib().oracle_fixed_point_bits(int(n))


def quantise(logw):
    logw = np.ascontiguousarray(logw, dtype=np.float64)
    q = np.zeros(len(logw), dtype=np.uint64)
    B = lib().oracle_quantise(_p(logw, C.c_double), len(logw), _p(q, C.c_uint64))
    return q, B


def multinomial_from_q(q, U):
    """Multinomial slots on integer weights: a_j = min{i : C_i > floor((2 U_j + 1) S / 2^33)}."""
    qq = np.ascontiguousarray(q, dtype=np.uint64)
    UU = np.ascontiguousarray(U, dtype=np.uint32)
    anc = np.zeros(len(qq), dtype=np.int32)
    rc = lib().oracle_multinomial_from_q(_p(qq, C.c_uint64), len(qq), _p(UU, C.c_uint32), _p(anc, C.c_int32))
    if rc != 0:
        raise ValueError("all weights zero")
    return anc


def binomial(n, p, seed, c0, c1, c2, c3, words: bool = False):
    """Bin(n, p) from a fresh word stream (counters c0 + 4096 m, c1, c2, c3)."""
    used = np.zeros(1, dtype=np.int32)
    k = lib().oracle_binomial(float(n), float(p), int(seed), int(c0), int(c1), int(c2), int(c3),
                              _p(used, C.c_int32))
    return (k, int(used[0])) if words else k


def ess_from_q(q) -> float:
    qq = np.ascontiguousarray(q, dtype=np.uint64)
    return lib().oracle_ess_from_q(_p(qq, C.c_uint64), len(qq))


def systematic_from_q(q, U):
    q = np.ascontiguousarray(q, dtype=np.uint64)
    n = len(q)
    nc = np.zeros(n, dtype=np.int32)
    anc = np.zeros(n, dtype=np.int32)
    rc = lib().oracle_systematic_from_q(_p(q, C.c_uint64), n, int(U), _p(nc, C.c_int32),
                                        _p(anc, C.c_int32))
    if rc != 0:
        raise ValueError("systematic resampling: no positive weight")
    return nc, anc


def log_obs(cfg: Config, theta, x, y) -> float:
    c = cfg.ctype()
    th = np.ascontiguousarray(theta, dtype=np.float64)
    xs = np.zeros(5)
    xs[:len(x)] = x
    return lib().oracle_log_obs(C.byref(c), _p(th, C.c_double), _p(xs, C.c_double), float(y))


def pf_loglik(cfg: Config, theta, y, k: int, i: int, trace: bool = False):
    """log p^(y_{1:T} | theta) of filter i at iteration k (with the trace if asked)."""
    c = cfg.ctype()
    th = np.ascontiguousarray(theta, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    delta = np.zeros(cfg.T) if trace else None
    anc = np.zeros((max(cfg.T - 1, 0), cfg.M), dtype=np.int32) if trace else None
    ll = lib().oracle_pf_loglik(C.byref(c), _p(th, C.c_double), _p(yy, C.c_double), int(k), int(i),
                                _p(delta, C.c_double), _p(anc, C.c_int32))
    return (ll, delta, anc) if trace else ll


def pf_initial(cfg: Config, theta, k: int, i: int) -> np.ndarray:
    """Initial particle states of filter i at iteration k, [M][5]."""
    c = cfg.ctype()
    th = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.zeros((cfg.M, 5))
    lib().oracle_pf_initial(C.byref(c), _p(th, C.c_double), int(k), int(i), _p(x, C.c_double))
    return x


def pf_propagate(cfg: Config, theta, k: int, i: int, t: int, y_t: float, x):
    """One step t of the filter from states x [M][5] (copied): (propagated states, log-weights)."""
    c = cfg.ctype()
    th = np.ascontiguousarray(theta, dtype=np.float64)
    xx = np.array(x, dtype=np.float64, order="C")
    ell = np.zeros(cfg.M)
    lib().oracle_pf_propagate(C.byref(c), _p(th, C.c_double), int(k), int(i), int(t), float(y_t),
                              _p(xx, C.c_double), _p(ell, C.c_double))
    return xx, ell


def pf_log_weights(cfg: Config, theta, x, y_t: float) -> np.ndarray:
    """log g(y_t | x_j) for the M states x [M][5]."""
    c = cfg.ctype()
    th = np.ascontiguousarray(theta, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    ell = np.zeros(cfg.M)
    lib().oracle_pf_log_weights(C.byref(c), _p(th, C.c_double), _p(xx, C.c_double), float(y_t), _p(ell, C.c_double))
    return ell


def pf_resample_word(cfg: Config, k: int, i: int, t: int) -> int:
    return int(lib().oracle_pf_resample_word(C.byref(cfg.ctype()), int(k), int(i), int(t)))


def pf_loglik_many(cfg: Config, thetas, y, k: int, i0: int = 0, threads: int = 1) -> np.ndarray:
    """PF log-likelihoods of theta rows i0, i0+1, ... (embarrassingly parallel over theta).

    The C calls release the GIL, so a thread pool uses several host cores."""
    thetas = np.ascontiguousarray(thetas, dtype=np.float64)
    n = thetas.shape[0]
    out = np.zeros(n)

    def run(lo, hi):
        for r in range(lo, hi):
            out[r] = pf_loglik(cfg, thetas[r], y, k, i0 + r)

    if threads <= 1:
        run(0, n)
    else:
        chunks = np.linspace(0, n, threads + 1).astype(int)
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda a: run(*a), zip(chunks[:-1], chunks[1:])))
    return out


def log_prior(cfg: Config, theta) -> float:
    c = cfg.ctype()
    th = np.ascontiguousarray(theta, dtype=np.float64)
    return lib().oracle_log_prior(C.byref(c), _p(th, C.c_double))


def lkernel_fit(theta_prev, theta_new, wn_prev):
    a = np.ascontiguousarray(theta_prev, dtype=np.float64)
    b = np.ascontiguousarray(theta_new, dtype=np.float64)
    w = np.ascontiguousarray(wn_prev, dtype=np.float64)
    N, D = a.shape
    mu = np.zeros(2 * D)
    sigma = np.zeros((2 * D, 2 * D))
    A = np.zeros((D, D))
    Lc = np.zeros((D, D))
    ld = C.c_double(0.0)
    rc = lib().oracle_lkernel_fit(D, N, _p(a, C.c_double), _p(b, C.c_double), _p(w, C.c_double),
                                  _p(mu, C.c_double), _p(sigma, C.c_double), _p(A, C.c_double),
                                  _p(Lc, C.c_double), C.byref(ld))
    return {"fallback": rc, "mu": mu, "sigma": sigma, "A": A, "Lc": Lc, "logdet": ld.value}


def lkernel_logpdf(fit, a, b) -> float:
    D = fit["A"].shape[0]
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return lib().oracle_gauss_lkernel_logpdf(D, _p(fit["mu"], C.c_double), _p(fit["A"], C.c_double),
                                             _p(fit["Lc"], C.c_double), fit["logdet"],
                                             _p(a, C.c_double), _p(b, C.c_double))


# --------------------------------------------------------------------------
# the SMC^2 sampler
# --------------------------------------------------------------------------

def _stats_dict(s: OracleStats, D: int) -> dict:
    return {"k": s.k, "resampled": s.resampled, "lk_fallback": s.lk_fallback, "lse": s.lse,
            "lse2": s.lse2, "ess": s.ess, "logz": s.logz, "est": np.array(s.est[:D]),
            "cov": np.array(s.cov[:D * D]).reshape(D, D)}


class SMC2:
    """The oracle sampler: state held in numpy arrays, one C call per iteration."""

    def __init__(self, cfg: Config, y):
        self.cfg = cfg
        self.y = np.ascontiguousarray(y, dtype=np.float64)
        N, D = cfg.N, cfg.D
        self.theta = np.zeros((N, D))
        self.logprior = np.zeros(N)
        self.loglik = np.zeros(N)
        self.logw = np.zeros(N)
        self.k = 0
        self.stats: list[dict] = []
        self._raw: list[OracleStats] = []
        self._c = cfg.ctype()

    def set_state(self, k, theta, logprior, loglik, logw):
        self.k = int(k)
        self.theta[:] = theta
        self.logprior[:] = logprior
        self.loglik[:] = loglik
        self.logw[:] = logw

    def step(self) -> dict:
        st = OracleStats()
        k = self.k + 1
        rc = lib().oracle_smc2_step(C.byref(self._c), _p(self.y, C.c_double), k,
                                    _p(self.theta, C.c_double), _p(self.logprior, C.c_double),
                                    _p(self.loglik, C.c_double), _p(self.logw, C.c_double),
                                    C.byref(st))
        if rc != 0:
            raise FloatingPointError(f"oracle SMC2 iteration {k}: status {rc}")
        self.k = k
        self._raw.append(st)
        d = _stats_dict(st, self.cfg.D)
        self.stats.append(d)
        return d

    def run(self, K=None) -> "SMC2":
        for _ in range((K or self.cfg.K) - self.k):
            self.step()
        return self

    def recycled(self):
        K = len(self._raw)
        arr = (OracleStats * K)(*self._raw)
        est = np.zeros(self.cfg.D)
        ck = np.zeros(K)
        lib().oracle_recycle(K, self.cfg.D, arr, _p(est, C.c_double), _p(ck, C.c_double))
        return est, ck

    def recycled_cov(self):
        K = len(self._raw)
        arr = (OracleStats * K)(*self._raw)
        cov = np.zeros((self.cfg.D, self.cfg.D))
        lib().oracle_recycle_cov(K, self.cfg.D, arr, _p(cov, C.c_double))
        return cov


# --------------------------------------------------------------------------
# surrogate network of the learned proposal
# --------------------------------------------------------------------------

def bf16(v: float) -> float:
    return lib().oracle_bf16(float(v))


def mlp_nparams(D: int, H: int = 64) -> int:
    return lib().oracle_mlp_nparams(D, H)


def mlp_forward(params, x, H: int = 64, bf16_points: bool = False) -> np.ndarray:
    p = np.ascontiguousarray(params, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    R, D = xx.shape
    out = np.zeros(R)
    lib().oracle_mlp_forward(D, H, _p(p, C.c_double), _p(xx, C.c_double), R, int(bf16_points),
                             _p(out, C.c_double))
    return out


def mlp_loss_grad(params, x, y, H: int = 64, bf16_points: bool = False):
    p = np.ascontiguousarray(params, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    R, D = xx.shape
    g = np.zeros_like(p)
    loss = lib().oracle_mlp_loss_grad(D, H, _p(p, C.c_double), _p(xx, C.c_double), _p(yy, C.c_double),
                                      R, int(bf16_points), _p(g, C.c_double))
    return loss, g


def mlp_input_grad(params, x, H: int = 64, bf16_points: bool = False):
    p = np.ascontiguousarray(params, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    R, D = xx.shape
    s = np.zeros(R)
    dx = np.zeros((R, D))
    lib().oracle_mlp_input_grad(D, H, _p(p, C.c_double), _p(xx, C.c_double), R, int(bf16_points),
                                _p(s, C.c_double), _p(dx, C.c_double))
    return s, dx


def adam_step(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on params, m, v (float64 numpy arrays)."""
    lib().oracle_adam_step(len(params), _p(params, C.c_double), _p(np.ascontiguousarray(grad), C.c_double),
                           _p(m, C.c_double), _p(v, C.c_double), int(t), lr, beta1, beta2, eps)


# --------------------------------------------------------------------------
# the learned proposal's sampler-side steps (choices L2-L4)
# --------------------------------------------------------------------------

def mlp_weights_bf16(params, D: int, H: int = 64) -> np.ndarray:
    """W1, W2, w3 rounded to bfloat16 as the kernels use them; biases unchanged."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    out = np.zeros_like(p)
    lib().oracle_mlp_weights_bf16(D, H, _p(p, C.c_double), _p(out, C.c_double))
    return out


def mlp_standardise(theta, lp):
    """Training set of the surrogate from rows (theta [R][D], log pi^ [R]): (x, y, norm dict)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    l = np.ascontiguousarray(lp, dtype=np.float64)
    R, D = th.shape
    x = np.zeros((R, D))
    y = np.zeros(R)
    nm = MlpNorm()
    lib().oracle_mlp_standardise(D, R, _p(th, C.c_double), _p(l, C.c_double), _p(x, C.c_double),
                                 _p(y, C.c_double), C.byref(nm))
    return x, y, nm.as_dict(D)


def mlp_train(params, m, v, t: int, theta, lp, steps: int, lr: float, H: int = 64, bf16_points: bool = True):
    """One training call: standardise the rows, then `steps` Adam steps from the
    state (params, m, v, step counter t).  Returns (params, m, v, t, loss of the
    last step before its update, norm dict, x, y); the inputs are not modified."""
    p = np.array(params, dtype=np.float64)
    mm = np.array(m, dtype=np.float64)
    vv = np.array(v, dtype=np.float64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    l = np.ascontiguousarray(lp, dtype=np.float64)
    R, D = th.shape
    tt = C.c_int(int(t))
    nm = MlpNorm()
    x = np.zeros((R, D))
    y = np.zeros(R)
    loss = lib().oracle_mlp_train(D, H, R, _p(th, C.c_double), _p(l, C.c_double), int(steps), float(lr),
                                  int(bf16_points), _p(p, C.c_double), _p(mm, C.c_double), _p(vv, C.c_double),
                                  C.byref(tt), C.byref(nm), _p(x, C.c_double), _p(y, C.c_double))
    return p, mm, vv, tt.value, loss, nm.as_dict(D), x, y


def mlp_score(params, norm: dict, theta, H: int = 64, bf16_points: bool = True) -> np.ndarray:
    """d log pi^ / d theta of the surrogate at rows theta [R][D]."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    R, D = th.shape
    nm = MlpNorm.from_dict(norm)
    out = np.zeros((R, D))
    lib().oracle_mlp_score(D, H, _p(p, C.c_double), C.byref(nm), _p(th, C.c_double), R, int(bf16_points),
                           _p(out, C.c_double))
    return out


def population_factor(cov, ess: float):
    """(L, usable) for the population covariance [D][D] and its ESS."""
    c = np.ascontiguousarray(cov, dtype=np.float64)
    D = c.shape[0]
    L = np.zeros((D, D))
    ok = lib().oracle_population_factor(D, _p(c, C.c_double), float(ess), _p(L, C.c_double))
    return L, bool(ok)


def learned_decision(k: int, loss: float, var_y: float, pop_ok: bool) -> bool:
    return bool(lib().oracle_learned_decision(int(k), float(loss), float(var_y), int(bool(pop_ok))))


def langevin_propose(h: float, L, theta_prev, score, z):
    """theta_k = theta_{k-1} + h L (w + z), w = clip(h/2 L^T g, +-3); returns (theta_k, log q)."""
    LL = np.ascontiguousarray(L, dtype=np.float64)
    a = np.ascontiguousarray(theta_prev, dtype=np.float64)
    g = np.ascontiguousarray(score, dtype=np.float64)
    zz = np.ascontiguousarray(z, dtype=np.float64)
    D = len(a)
    out = np.zeros(D)
    lq = np.zeros(1)
    lib().oracle_langevin_propose(D, float(h), _p(LL, C.c_double), _p(a, C.c_double), _p(g, C.c_double),
                                  _p(zz, C.c_double), _p(out, C.c_double), _p(lq, C.c_double))
    return out, float(lq[0])
