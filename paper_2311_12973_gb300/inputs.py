"""Seeded synthetic inputs for the SMC^2 hot path.

This module holds no step of the sampler.  It simulates observation series
from the two state-space models with numpy's own generator (not the
sampler's counter-based stream) and describes the workloads: sizes, priors and
model constants.  The CUDA path and the oracle both take their inputs from
here, so it imports neither of them.

Workloads (sizes follow the benchmark configurations of the method):

* ``lg_t50_n64``       linear-Gaussian AR(1), T=50, N=64, M=128, K=10, FP64
* ``seir_t100_n1024``  SEIR-type, population 1e6, T=100, N=1024, M=512, K=20, FP32 particles
* ``seir_t200_n8192``  SEIR-type, T=200, N=8192, M=1024, K=30, FP32 particles
* ``seir_t100_n1024_mlp``  as ``seir_t100_n1024`` with the learned proposal
* ``seir_batched_64``  64 SEIR-type datasets, T ~ U{50..400}, N in {256,1024,4096},
  M in {128,512,1024}, K=10
* ``sir_t30_n1024``    the paper's binomial SIR experiment (Sec. V-A): population 1e4,
  3 infected, T=30, theta = (beta, gamma) ~ U[0,1]^2, random walk Sigma = 0.1 I,
  N=1024 (256 and 512 by override), M=500, K=10, the paper's particle filter
  (multinomial resampling when the ESS falls below M/2), FP32 particles
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

LG, SEIR, SIR = 0, 1, 2
PREC_FP64, PREC_MIXED = 0, 1
PRIOR_GAUSS, PRIOR_UNIFORM = 0, 1
PF_SYSTEMATIC, PF_MULTINOMIAL = 0, 1
PROP_RW, PROP_MLP = 0, 1
LK_FORWARD, LK_GAUSS = 0, 1

LG_TRUTH = (0.8, 0.5, 1.0)                # phi, sigma_x, sigma_y
SEIR_TRUTH = (0.6, 0.05, 0.25, 0.2)       # beta0, sigma_rw, kappa, gamma
SEIR_PRIOR_MEDIAN = (0.5, 0.1, 0.2, 0.2)  # log-normal prior medians, log-sd 0.5
SIR_TRUTH = (0.85, 0.20)                  # beta, gamma (Sec. V-A)


@dataclass
class Workload:
    name: str
    model: int
    D: int
    N: int
    M: int
    T: int
    K: int
    precision: int = PREC_FP64
    proposal: int = PROP_RW
    lkernel: int = LK_GAUSS
    rw_scale: float = 0.1
    ess_frac: float = 0.5
    seed: int = 1
    data_seed: int = 1
    dataset: int = 0
    prior_mean: list = field(default_factory=list)
    prior_sd: list = field(default_factory=list)
    npop: float = 0.0
    e0: float = 0.0
    i0: float = 0.0
    lambda_floor: float = 1e-3
    n_sub: int = 2
    prior_kind: int = PRIOR_GAUSS
    prior_lo: list = field(default_factory=list)
    prior_hi: list = field(default_factory=list)
    pf_scheme: int = PF_SYSTEMATIC
    pf_ess_frac: float = 0.0
    ppt: int = 0            # particle-filter launch shape (0: the library's tuner)
    cta_threads: int = 0
    pf_family: int = 0      # particle-filter kernel family the tuner may pick (0: either)
    y: np.ndarray | None = None

    @property
    def particle_steps_per_iter(self) -> int:
        return self.N * self.M * self.T

    def with_(self, **kw) -> "Workload":
        w = replace(self, **kw)
        if "T" in kw or "data_seed" in kw:
            w.y = simulate(w)
        return w


def simulate_lg(T: int, phi: float, sx: float, sy: float, seed: int) -> np.ndarray:
    """y_t = x_t + sy n_t, x_t = phi x_{t-1} + sx e_t, x_0 ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal()
    y = np.empty(T)
    for t in range(T):
        x = phi * x + sx * rng.standard_normal()
        y[t] = x + sy * rng.standard_normal()
    return y


def seir_day(S: float, E: float, I: float, beta: float, kappa: float, gamma: float,
             npop: float, n_sub: int) -> tuple[float, float, float, float]:
    """One day of the SEIR-type dynamics: n_sub explicit Euler substeps of the
    S -> E -> I -> R flows, clamped at zero.  Returns (S, E, I, incidence)."""
    dt = 1.0 / n_sub
    lam = 0.0
    for _ in range(n_sub):
        inf, onset, rec = beta * S * I / npop, kappa * E, gamma * I
        lam += dt * onset
        S = max(S - dt * inf, 0.0)
        E = max(E + dt * (inf - onset), 0.0)
        I = max(I + dt * (onset - rec), 0.0)
    return S, E, I, lam


def simulate_seir(T: int, beta0: float, sigma_rw: float, kappa: float, gamma: float,
                  npop: float, e0: float, i0: float, n_sub: int, lambda_floor: float,
                  seed: int) -> np.ndarray:
    """Daily Poisson counts of new infectious cases from the SEIR-type model,
    with log beta following a Gaussian random walk."""
    rng = np.random.default_rng(seed)
    S, E, I, lb = npop - e0 - i0, e0, i0, math.log(beta0)
    y = np.empty(T)
    for t in range(T):
        lb = lb + sigma_rw * rng.standard_normal()
        S, E, I, lam = seir_day(S, E, I, math.exp(lb), kappa, gamma, npop, n_sub)
        y[t] = rng.poisson(max(lam, lambda_floor))
    return y.astype(np.float64)


def seir_constant_beta_incidence(T: int, beta0: float, kappa: float, gamma: float,
                                 npop: float, e0: float, i0: float, n_sub: int,
                                 lambda_floor: float) -> np.ndarray:
    """Daily incidence of the SEIR-type model when log beta does not move."""
    S, E, I = npop - e0 - i0, e0, i0
    lam = np.empty(T)
    for t in range(T):
        S, E, I, l = seir_day(S, E, I, beta0, kappa, gamma, npop, n_sub)
        lam[t] = max(l, lambda_floor)
    return lam


def simulate_sir(T: int, beta: float, gamma: float, npop: float, i0: float, seed: int) -> np.ndarray:
    """Daily Poisson counts of the infected from the binomial SIR model: each day
    Bin(S, 1 - exp(-beta I / npop)) susceptibles are infected and Bin(I, 1 - exp(-gamma))
    infected recover, both from the previous day's compartments; y_t ~ Poisson(I_t)."""
    rng = np.random.default_rng(seed)
    S, I = int(npop - i0), int(i0)
    y = np.empty(T)
    for t in range(T):
        n_si = rng.binomial(S, -math.expm1(-beta * I / npop))
        n_ir = rng.binomial(I, -math.expm1(-gamma))
        S, I = S - n_si, I + n_si - n_ir
        y[t] = rng.poisson(I)
    return y.astype(np.float64)


def simulate(w: Workload) -> np.ndarray:
    if w.model == SIR:
        return simulate_sir(w.T, *SIR_TRUTH, w.npop, w.i0, seed=w.data_seed)
    if w.model == LG:
        return simulate_lg(w.T, *LG_TRUTH, seed=w.data_seed)
    return simulate_seir(w.T, *SEIR_TRUTH, w.npop, w.e0, w.i0, w.n_sub, w.lambda_floor,
                         seed=w.data_seed)


def _lg(**kw) -> Workload:
    w = Workload(name="lg", model=LG, D=3, N=64, M=128, T=50, K=10, precision=PREC_FP64,
                 prior_mean=[0.0, 0.0, 0.0], prior_sd=[1.0, 1.0, 1.0], seed=1, data_seed=1)
    w = replace(w, **kw)
    w.y = simulate(w)
    return w


def _seir(**kw) -> Workload:
    w = Workload(name="seir", model=SEIR, D=4, N=1024, M=512, T=100, K=20,
                 precision=PREC_MIXED,
                 prior_mean=[math.log(v) for v in SEIR_PRIOR_MEDIAN], prior_sd=[0.5] * 4,
                 npop=1e6, e0=0.0, i0=100.0, n_sub=2, seed=2, data_seed=2)
    w = replace(w, **kw)
    w.y = simulate(w)
    return w


def _sir(**kw) -> Workload:
    w = Workload(name="sir", model=SIR, D=2, N=1024, M=500, T=30, K=10, precision=PREC_MIXED,
                 rw_scale=math.sqrt(0.1), prior_kind=PRIOR_UNIFORM, prior_lo=[0.0, 0.0],
                 prior_hi=[1.0, 1.0], prior_mean=[0.5, 0.5], prior_sd=[1.0, 1.0],
                 npop=1e4, i0=3.0, pf_scheme=PF_MULTINOMIAL, pf_ess_frac=0.5, seed=4, data_seed=4)
    w = replace(w, **kw)
    w.y = simulate(w)
    return w


def workload(name: str, **kw) -> Workload:
    if name == "sir_t30_n1024":
        return _sir(name=name, **kw)
    if name == "lg_t50_n64":
        return _lg(name=name, **kw)
    if name == "seir_t100_n1024":
        return _seir(name=name, **kw)
    if name == "seir_t200_n8192":
        return _seir(name=name, T=200, N=8192, M=1024, K=30, seed=3, data_seed=3, **kw)
    if name == "seir_t100_n1024_mlp":
        return _seir(name=name, proposal=PROP_MLP, **kw)
    raise KeyError(name)


def batched_workloads(n: int = 64, K: int = 10, seed: int = 100) -> list[Workload]:
    """n independent SEIR-type datasets of uneven length and size."""
    rng = np.random.default_rng(seed)
    out = []
    for d in range(n):
        T = int(rng.integers(50, 401))
        N = int(rng.choice([256, 1024, 4096]))
        M = int(rng.choice([128, 512, 1024]))
        out.append(_seir(name=f"seir_batched_{d}", T=T, N=N, M=M, K=K, seed=seed,
                         data_seed=seed + d, dataset=d))
    return out


def theta_near_prior(w: Workload, n: int, seed: int, spread: float = 1.0) -> np.ndarray:
    """n parameter vectors drawn around the prior (row-major [n][D])."""
    rng = np.random.default_rng(seed)
    if w.prior_kind == PRIOR_UNIFORM:  # uniform on the support shrunk about its centre
        lo, hi = np.asarray(w.prior_lo, dtype=np.float64), np.asarray(w.prior_hi, dtype=np.float64)
        return 0.5 * (lo + hi) + (rng.random((n, w.D)) - 0.5) * (hi - lo) * min(spread, 1.0)
    mu = np.asarray(w.prior_mean, dtype=np.float64)
    sd = np.asarray(w.prior_sd, dtype=np.float64) * spread
    return mu + sd * rng.standard_normal((n, w.D))
