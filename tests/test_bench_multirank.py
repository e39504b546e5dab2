"""The multi-process path of bench.py on the CPU (gloo, world size 2).

The sampler shards by replicas: every rank runs the whole workload with its
own seed and no data-path collective; the only exchange is the maximum step
time over the ranks, from which the job throughput is formed.  These tests
run that exchange and the reference arm's torchrun launch without a GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    from paper_2311_12973_gb300 import inputs as I
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    step_ms = 10.0 + 5.0 * rank                       # the second replica is slower
    slowest = bench.reduce_max(step_ms, dist, "cpu")
    w = bench.replica_workload(I.workload("lg_t50_n64"), rank)
    out.put((rank, slowest, w.seed, bench.job_throughput(100.0, world, slowest)))
    dist.destroy_process_group()


def test_replicas_exchange_only_the_slowest_step_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]            # every rank sees the max
    assert res[0][2] != res[1][2]                         # independent replicas
    assert res[0][3] == pytest.approx(100.0 * 2 / 15e-3)  # all units over the slowest step


def test_reference_arm_under_torchrun_prints_one_line():
    """Rank 0 alone times the oracle and prints; the other rank exits 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--workload", "lg_t50_n64"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300,
                       env={**os.environ, "OMP_NUM_THREADS": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle"


@pytest.mark.parametrize("pf", ["workload", "systematic"])
def test_reference_arm_on_the_papers_sir_experiment(pf):
    """The reference arm on the SIR workload, with its own filter and with the default one."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "0", "--workload", "sir_t30_n1024", "--pf", pf]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["config"]["model"] == "binomial SIR"
    assert line["config"]["prior"].startswith("uniform")
    assert ("pf_resampling" in line["config"]) == (pf == "workload")
