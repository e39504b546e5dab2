"""Benchmark of the SMC^2 hot path on one GB300 (or N replicas under torchrun).

One step = one complete SMC^2 run of the workload: K iterations, each scoring
N parameter samples with an M-particle filter over T observations, plus the
L-kernel weights, ESS, outer resampling and recycling.  Inputs (observations)
are resident on the device for `value`; `e2e` repeats the step through the C
ABI with host buffers (observations copied in, recycled estimate copied out).

Default workload: the largest single-GPU configuration, SEIR-type model,
population 1e6, T=200, N=8192, M=1024, K=30, FP32 particles with FP64 outer
arithmetic.  The accuracy comparison of the forms (mixed precision, the plain
FP64 GPU form, the learned proposal) runs on the N=1024, M=512, T=100, K=20
workload and is printed as extra keys.  `--impl reference` times the CPU
oracle on a bounded sample of the workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PF particle-steps/s and SMC² ESS/s vs plain FP64 GPU form; % of roofline"
UNIT = "particle-steps/s"

# Algorithmic lane operations per particle-step of the particle-filter kernel,
# counted from the kernel source by category: Philox share 20.5, Box-Muller
# share 10.5, propagation 32 (LG 1), log-weight 15 (LG 5), checks and max 4,
# quantisation 5, prefix sum and store 6, resampling 15.  Binomial SIR with
# the paper's filter: 1.28 Philox calls of 82 for the two flows' shared word
# stream (105), the two binomial draws 80 (about 40 each: BTRS setup 15, 1.2
# proposals of 13 and 2.4 word conversions of 3; inversion's setup and short
# search cost about the same), the hazard and flows 12, log-weight 15, checks,
# max, quantisation and prefix sum 15, the ESS's sum of q^2 5, and multinomial
# slots on the 86 % of steps that resample (a quarter Philox call, a 9-step
# binary search, the state read: 51.5) 44.
ALG_OPS_PER_PARTICLE_STEP = {
    0: 67.0,    # linear-Gaussian AR(1)
    1: 108.0,   # SEIR-type
    2: 276.0,   # binomial SIR (Sec. V-A), the paper's filter
}
# The same counts for the other particle filter: the every-step systematic
# resampling (15) replaced by the paper's ESS test (5) and multinomial slots
# (51.5) on the fraction of steps that resample, measured on the oracle (SEIR
# 58 % at theta near the prior; SIR 86 %), or the other way round.
ALG_OPS_OTHER_PF = {
    (1, "paper"): 108.0 - 15.0 + 5.0 + 0.584 * 51.5,     # 128
    (2, "systematic"): 276.0 - 5.0 - 0.86 * 51.5 + 15.0,  # 242
}


def alg_ops(w) -> float:
    """Algorithmic lane operations per particle-step of the filter w runs."""
    paper = bool(w.pf_scheme) or w.pf_ess_frac > 0
    default_paper = w.model == 2
    if paper == default_paper:
        return ALG_OPS_PER_PARTICLE_STEP[w.model]
    return ALG_OPS_OTHER_PF.get((w.model, "paper" if paper else "systematic"),
                                ALG_OPS_PER_PARTICLE_STEP[w.model])
MODEL_NAMES = {0: "LG-AR(1)", 1: "SEIR-type", 2: "binomial SIR"}
# DRAM bytes per particle-filter launch (dram__bytes_read.sum + dram__bytes_write.sum)
# from one ncu capture of a full-size launch of the workload, valid only for that
# workload and the kernel source it was taken on (sha-256 prefixes of the sources).
PF_TRAFFIC = {
    "seir_t200_n8192": {"bytes": 748800.0, "sources": {"pf_fast.cuh": "bde90cf5170865a6", "pf_impl.cuh": "ed94a1cf40e60688",
                                                       "common.cuh": "e78c60dc197c7ed7"}},
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="seir_t200_n8192")
    p.add_argument("--forms-workload", default="seir_t100_n1024",
                   help="workload of the accuracy comparison of the forms (extra keys of the line)")
    p.add_argument("--no-fp64-form", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batched", action="store_true",
                   help="skip the 64-dataset workload (extra keys of the line)")
    p.add_argument("--batched-datasets", type=int, default=64,
                   help="datasets of the batched workload (smaller cases for profiler captures)")
    p.add_argument("--no-forms", action="store_true",
                   help="skip the accuracy comparison of the random-walk, FP64 and learned forms")
    p.add_argument("--pf", default="workload", choices=["workload", "systematic", "paper"],
                   help="particle-filter resampling: the workload's own, systematic after every step, "
                        "or the paper's (multinomial when the ESS falls below M/2)")
    p.add_argument("--ppt", type=int, default=0, help="pin particles per thread (0: tuner)")
    p.add_argument("--cta", type=int, default=0, help="pin threads per PF CTA (0: tuner)")
    p.add_argument("--pf-family", default="any", choices=["any", "groups", "fp32"],
                   help="particle-filter kernel family: the tuner's pick, pf_kernel, or the FP32 filter")
    p.add_argument("--filters", type=int, default=0,
                   help="run N parameter samples instead of the workload's (smaller cases for profiler captures)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_workload(w, rank: int, ppt: int = 0, cta: int = 0, pf_family: int = 0):
    """Rank `rank`'s independent replica of the workload: same data, own seed."""
    return w.with_(seed=w.seed + 1000 * rank, ppt=ppt, cta_threads=cta, pf_family=pf_family)


def reduce_max(x: float, dist=None, device: str = "cpu") -> float:
    """The largest value over the ranks of the default process group (x itself
    without one): the job's step time is that of its slowest replica."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_replica_step: float, world: int, step_ms_max: float) -> float:
    """Whole-job units per second: every replica's units over the slowest step."""
    return units_per_replica_step * world / (step_ms_max * 1e-3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def pf_traffic_if_current(workload: str):
    import hashlib
    rec = PF_TRAFFIC.get(workload)
    if rec is None:
        return None
    d = os.path.join(ROOT, "paper_2311_12973_gb300", "csrc")
    for f, h in rec["sources"].items():
        if hashlib.sha256(open(os.path.join(d, f), "rb").read()).hexdigest()[:16] != h:
            return None
    return rec["bytes"]


def measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def alu_peak_ops(sm_count: int, sm_mhz: float) -> float:
    """Lane-operation issue peak: 4 schedulers x 32 lanes per SM per clock."""
    return sm_count * 4 * 32 * sm_mhz * 1e6


def cpu_baseline(w, seconds: float = 12.0) -> dict:
    """The oracle particle filter (>= 99.9% of the method's work) on a bounded
    sample of the workload's filters, all host cores, as it stands."""
    import numpy as np
    from oracle import oracle as O
    from paper_2311_12973_gb300 import inputs as I
    cores = os.cpu_count() or 1
    cfg = O.config_from(w)
    per_chunk = cores * 2
    th = I.theta_near_prior(w, per_chunk * 64, seed=17, spread=0.3)
    done, t0, chunk = 0, time.perf_counter(), 0
    while True:
        rows = th[(chunk * per_chunk) % len(th):][:per_chunk]
        O.pf_loglik_many(cfg, rows, w.y, k=1, i0=chunk * per_chunk, threads=cores)
        done += len(rows)
        chunk += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": done * w.M * w.T / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} particle filters of the workload (M={w.M}, T={w.T}), FP64 oracle, "
                      f"{cores} threads, {el:.1f} s"}


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2311_12973_gb300 import inputs as I
    cores = os.cpu_count() or 1
    cfg = O.config_from(w)
    per_step = cores * 4
    th = I.theta_near_prior(w, per_step, seed=17, spread=0.3)
    for _ in range(args.warmup):
        O.pf_loglik_many(cfg, th[:cores], w.y, k=1, threads=cores)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        O.pf_loglik_many(cfg, th, w.y, k=1 + s, threads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * w.M * w.T * args.steps / total
    sample = f"{per_step} particle filters per step (M={w.M}, T={w.T}), FP64 oracle, {cores} threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, "fp64 oracle"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def workload_config(w, precision: str) -> dict:
    c = {"workload": w.name, "model": MODEL_NAMES[w.model], "N": w.N,
         "M": w.M, "T": w.T, "K": w.K, "precision": precision, "proposal": "random walk",
         "lkernel": "approx. optimal Gaussian",
         "l2": "flushed between timed steps (256 MiB write outside the step events)"}
    if w.pf_scheme or w.pf_ess_frac:
        c["pf_resampling"] = (("multinomial" if w.pf_scheme else "systematic") +
                              (f" when ESS < {w.pf_ess_frac:g} M" if w.pf_ess_frac else " every step"))
    if w.prior_kind:
        c["prior"] = f"uniform on {list(zip(w.prior_lo, w.prior_hi))}"
    return c


def time_runs(S, torch, ctx, w, steps, warmup, flush, rank_sync):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ctx.reset(w.seed)
        ctx.run(w.K, stats=False)
    torch.cuda.synchronize()
    ctx.timing(reset=True)
    ctx.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    ess_sums = []
    rank_sync()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for s in range(steps):
        flush.zero_()
        ev[s][0].record(stream)
        ctx.reset(w.seed)
        ctx.run(w.K, stats=False)
        ev[s][1].record(stream)
        _, _, ess = ctx.estimate()
        ess_sums.append(ess)
    torch.cuda.synchronize()
    rank_sync()
    wall = time.perf_counter() - t_wall
    ctx.set_timing(False)
    ms = [a.elapsed_time(b) for a, b in ev]
    pf_ms, pf_n, launches = ctx.timing(reset=True)
    return ms, ess_sums, pf_ms, pf_n, launches, wall


def batched_datasets(S, torch, I, flush, rank_sync, peak, steps=2, n_datasets=64):
    """The 64-dataset SEIR-type workload (T in 50..400, N in {256, 1024, 4096},
    M in {128, 512, 1024}, K = 10) in one mixed-precision context: particle-steps
    per second of whole runs, and of its particle-filter launches against the
    ALU issue peak."""
    import numpy as np
    ws = I.batched_workloads(n_datasets)
    ctx = S.SMC2(S.make_config(ws[0]), np.concatenate([w.y for w in ws]),
                 datasets=[(w.N, w.M, w.T) for w in ws])
    shape = ctx.launch_shape()
    ms, _, pf_ms, pf_n, launches, _ = time_runs(S, torch, ctx, ws[0], steps, 1, flush, rank_sync)
    ctx.close()
    per_iter = float(sum(w.N * w.M * w.T for w in ws))
    run_ms = sum(ms) / len(ms)
    pf_avg = pf_ms / max(pf_n, 1)
    ops = alg_ops(ws[0]) * per_iter
    return {"workload": f"seir_batched_{n_datasets}", "datasets": n_datasets, "K": ws[0].K, "particle_steps_per_iteration": per_iter,
            "ms_per_run": run_ms, "value": per_iter * ws[0].K / (run_ms * 1e-3), "unit": UNIT,
            "pf_ms_per_launch": pf_avg, "pf_particle_steps_per_s": per_iter / (pf_avg * 1e-3),
            "pf_roofline_frac": ops / (pf_avg * 1e-3) / peak, "launch_shape": shape,
            "gpu_launches_per_run": launches / max(len(ms), 1)}


def accuracy_forms(S, torch, I, wr, world, seeds=384):
    """Posterior accuracy per unit time of three forms of the SMC^2 step on the
    same data: mixed precision with the random walk, the plain FP64 GPU form,
    and mixed precision with the learned proposal.  Accuracy is the mean
    squared error over `seeds` runs of the recycled posterior mean against a
    reference pooled from four FP64 random-walk runs with 8x the samples (the
    FP64 form matches the oracle run for run); mse x time is inversely
    proportional to accuracy per second.  The FP64 and mixed random-walk forms
    run the same seeds, so their log-evidence estimates and squared errors are
    compared pairwise.  The errors are heavy-tailed (blocks of 96 seeds gave
    worse-of-the-pair fractions from 0.40 to 0.68), so the line also carries
    the median squared error, per coordinate the fraction of seeds in which
    the mixed form is the worse of the pair, and the paired differences of the
    posterior means with their standard errors."""
    import numpy as np

    def runs(w, seed_list, **over):
        ctx = S.SMC2(S.make_config(w, **over), w.y)
        ctx.run(w.K, stats=False)
        stream = torch.cuda.current_stream()
        out = []
        for sd in seed_list:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ctx.reset(sd)
            a.record(stream)
            ctx.run(w.K, stats=False)
            b.record(stream)
            mean, logz, ess = ctx.estimate()
            out.append((mean, ess, a.elapsed_time(b), logz))
        ctx.close()
        return out

    base = 10_000 * (1 + wr.seed)
    ref_w = wr.with_(N=8 * wr.N, precision=I.PREC_FP64, ppt=0, cta_threads=0)
    ref = runs(ref_w, [base + i for i in range(4)], rw_scale=0.2)
    ref_mean = np.mean([r[0] for r in ref], axis=0)
    forms = {"mixed_rw": wr.with_(ppt=0, cta_threads=0),
             "fp64_rw": wr.with_(precision=I.PREC_FP64, ppt=0, cta_threads=0),
             "mixed_learned": wr.with_(proposal=I.PROP_MLP, ppt=0, cta_threads=0)}
    res, logz, sqerr, post = {}, {}, {}, {}
    for name, wf in forms.items():
        r = runs(wf, [base + 100 + i for i in range(seeds)])
        means = np.array([x[0] for x in r])
        sq = (means - ref_mean) ** 2
        mse = sq.mean(axis=0)
        ms = float(np.mean([x[2] for x in r]))
        logz[name] = np.array([x[3] for x in r])
        sqerr[name] = sq
        post[name] = means
        res[name] = {"ms_per_run": ms, "ess_per_s": float(np.mean([x[1] for x in r])) * world / (ms * 1e-3),
                     "rmse": [float(v) for v in np.sqrt(mse)], "mse_x_s": float(mse.mean() * ms * 1e-3),
                     "mse": float(mse.mean()), "median_sq_err": float(np.median(sq))}
    for name in ("fp64_rw", "mixed_learned"):
        res[name]["accuracy_per_s_vs_mixed_rw"] = res["mixed_rw"]["mse_x_s"] / res[name]["mse_x_s"]
    res["mixed_learned"]["accuracy_per_s_vs_fp64_rw"] = res["fp64_rw"]["mse_x_s"] / res["mixed_learned"]["mse_x_s"]
    res["mixed_learned"]["ess_per_s_vs_fp64_rw"] = res["mixed_learned"]["ess_per_s"] / res["fp64_rw"]["ess_per_s"]
    d = logz["mixed_rw"] - logz["fp64_rw"]   # same seeds: paired
    res["mixed_minus_fp64_logz"] = {"mean": float(d.mean()), "se": float(d.std(ddof=1) / np.sqrt(len(d))),
                                    "median_abs": float(np.median(np.abs(d))), "pairs": len(d),
                                    "target_nats": 0.05}
    res["mixed_over_fp64_mse"] = res["mixed_rw"]["mse"] / res["fp64_rw"]["mse"]
    res["mixed_over_fp64_median_sq_err"] = res["mixed_rw"]["median_sq_err"] / res["fp64_rw"]["median_sq_err"]
    res["mixed_worse_fraction"] = [float(v) for v in (sqerr["mixed_rw"] > sqerr["fp64_rw"]).mean(axis=0)]
    dm = post["mixed_rw"] - post["fp64_rw"]
    res["mixed_minus_fp64_posterior_mean"] = {"mean": [float(v) for v in dm.mean(axis=0)],
                                              "se": [float(v) for v in dm.std(axis=0, ddof=1) / np.sqrt(len(dm))]}
    res["reference"] = {"runs": 4, "N": ref_w.N, "precision": "fp64", "rw_scale": 0.2, "seeds_per_form": seeds,
                        "workload": wr.name}
    return res


def sir_paper_table(S, torch, I, wr, runs=10):
    """The paper's SIR results table (Sec. V) on this GPU: `runs` Monte Carlo
    runs of the workload with their own seeds; the mean of the recycled
    estimates of (beta, gamma), their mean squared error against the
    simulation truth, and the device time of one run."""
    import numpy as np
    ctx = S.SMC2(S.make_config(wr), wr.y)
    ctx.run(wr.K, stats=False)
    stream = torch.cuda.current_stream()
    est, ms = [], []
    for r in range(runs):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx.reset(wr.seed + 7919 * (r + 1))
        a.record(stream)
        ctx.run(wr.K, stats=False)
        b.record(stream)
        mean, _, _ = ctx.estimate()
        est.append(mean[:2])
        ms.append(a.elapsed_time(b))
    ctx.close()
    est = np.array(est)
    truth = np.array(I.SIR_TRUTH)
    return {"runs": runs, "E_beta": float(est[:, 0].mean()), "E_gamma": float(est[:, 1].mean()),
            "mse": float(((est - truth) ** 2).mean()), "ms_per_run": float(np.mean(ms)),
            "truth": list(I.SIR_TRUTH), "K_x_N": wr.K * wr.N, "M": wr.M}


def main():
    args = parse()
    rank, world, local = dist_env()
    from paper_2311_12973_gb300 import inputs as I
    w = I.workload(args.workload)
    if args.filters:
        w = w.with_(N=args.filters)
    if args.pf == "systematic":
        w = w.with_(pf_scheme=I.PF_SYSTEMATIC, pf_ess_frac=0.0)
    elif args.pf == "paper":
        w = w.with_(pf_scheme=I.PF_MULTINOMIAL, pf_ess_frac=0.5)
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def rank_sync():
        if dist is not None:
            dist.barrier()

    def reduce_max_gpu(x: float) -> float:
        return reduce_max(x, dist, "cuda")

    from paper_2311_12973_gb300 import build as B
    B.build()
    from paper_2311_12973_gb300 import smc2 as S

    # each rank runs an independent replica (its own seed): weak scaling
    wr = replica_workload(w, rank, args.ppt, args.cta, {"any": 0, "groups": 1, "fp32": 2}[args.pf_family])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ctx = S.SMC2(S.make_config(wr), wr.y)
    shape = ctx.launch_shape()
    props = torch.cuda.get_device_properties(local)

    with ClockSampler(local) as clk:
        ms, ess_sums, pf_ms, pf_n, launches, wall = time_runs(S, torch, ctx, wr, args.steps, args.warmup,
                                                              flush, rank_sync)
    clocks = clk.summary()
    step_ms = reduce_max_gpu(sum(ms) / len(ms))
    units_per_step = wr.N * wr.M * wr.T * wr.K
    value = job_throughput(units_per_step, world, step_ms)
    ess_per_s = statistics.mean(ess_sums) * world / (step_ms * 1e-3)

    # end to end through the C ABI with host buffers, on the host clock: each step
    # copies the observations in from pinned host memory, runs, and reads the
    # recycled estimate back (which synchronises); L2 is flushed before each step,
    # outside the timed region, as for `value`
    import numpy as np
    y_host = torch.tensor(wr.y, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for s in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_observations(y_host)
        ctx.reset(wr.seed)
        ctx.run(wr.K, stats=False)
        mean, logz, ess = ctx.estimate()
        if s >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_step = reduce_max(sum(e2e_ms) / len(e2e_ms), dist, "cuda")
    d2h = 8 * wr.D + 112 + 8 + 4

    # plain FP64 GPU form of the same workload
    fp64 = None
    if not args.no_fp64_form:
        w64 = wr.with_(precision=I.PREC_FP64, ppt=0, cta_threads=0, pf_family=0)
        ctx64 = S.SMC2(S.make_config(w64), w64.y)
        ms64, ess64, _, _, _, _ = time_runs(S, torch, ctx64, w64, max(2, args.steps // 5), 1, flush,
                                            rank_sync)
        st64 = reduce_max_gpu(sum(ms64) / len(ms64))
        fp64 = {"value": units_per_step * world / (st64 * 1e-3), "unit": UNIT,
                "ess_per_s": statistics.mean(ess64) * world / (st64 * 1e-3), "ms_per_step": st64}
        ctx64.close()

    forms = None
    if not args.no_forms and wr.model == I.SEIR and wr.D <= 8:
        forms = accuracy_forms(S, torch, I, replica_workload(I.workload(args.forms_workload), rank), world)
    paper_table = None
    if not args.no_forms and wr.model == I.SIR:
        paper_table = sir_paper_table(S, torch, I, wr)
    peak = alu_peak_ops(props.multi_processor_count, measured_peaks().get("sm_max_mhz", 2070.0))
    batched = None
    if not args.no_batched and wr.model == I.SEIR:
        batched = batched_datasets(S, torch, I, flush, rank_sync, peak, n_datasets=args.batched_datasets)

    if rank != 0:
        return
    peaks = measured_peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    fma32, fma64 = S.fma_rates()
    pf_avg_ms = pf_ms / max(pf_n, 1)
    ops_pps = alg_ops(wr)
    ops = ops_pps * wr.N * wr.M * wr.T
    achieved = ops / (pf_avg_ms * 1e-3)
    peak = alu_peak_ops(props.multi_processor_count, sm_mhz)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 particles, f64 outer", "data": "synthetic",
        "config": workload_config(wr, "mixed"),
        "ess_per_s": ess_per_s,
        "fp64_form": fp64,
        "speedup_vs_fp64_form": (value / fp64["value"]) if fp64 else None,
        "ess_speedup_vs_fp64_form": (ess_per_s / fp64["ess_per_s"]) if fp64 else None,
        "forms": forms,
        "paper_table": paper_table,
        "batched": batched,
        "roofline": {"kernel": (f"pf_fast_kernel<{MODEL_NAMES[wr.model]}, {shape['ppt']}>"
                                if shape["fp32_filter"] else f"pf_kernel<float, {MODEL_NAMES[wr.model]}, "
                                f"{shape['ppt']}>"), "bound": "alu", "achieved": achieved / 1e9,
                     "peak": peak / 1e9, "unit": "Gop/s", "frac": achieved / peak,
                     "traffic": pf_traffic_if_current(wr.name) if wr.N == I.workload(wr.name).N else None,
                     "ops_per_particle_step": ops_pps,
                     "pf_ms_per_launch": pf_avg_ms, "pf_launches": pf_n,
                     "pf_share_of_step": pf_ms / max(sum(ms), 1e-9),
                     "launch_shape": shape,
                     "peak_basis": f"{props.multi_processor_count} SMs x 128 lanes x {sm_mhz:.0f} MHz "
                                   "(max SM clock of MEASURED_PEAKS.json)",
                     "measured_fma_tflops": {"fp32": fma32 / 1e12, "fp64": fma64 / 1e12}},
        # the whole step against the time its particle filter work needs at the issue peak
        "ess_roofline": {"bound": "alu", "t_roof_ms": 1e3 * units_per_step * ops_pps / peak,
                         "ms_per_step": step_ms,
                         "frac": 1e3 * units_per_step * ops_pps / peak / step_ms},
        "e2e": {"value": units_per_step * world / (e2e_step * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": 8 * wr.T, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step,
                "clock": "host (perf_counter), L2 flushed before each step"},
        "gpu_launches": launches,
        "clocks": clocks,
        "wall_s": wall,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(wr)
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
