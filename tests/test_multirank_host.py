"""The multi-rank path of bench.py on the host (gloo, world size 2): the
reductions behind its max-over-ranks timing and whole-job sums, the barrier,
disjoint per-rank workloads, and the reference arm under torchrun (rank 0
prints one line, rank 1 exits without work)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    bench.barrier(2)
    res = (bench.max_over_ranks(2, 1.5 + rank), bench.sum_over_ranks(2, 10.0 * (rank + 1)))
    bench.barrier(2)
    dist.destroy_process_group()
    out.put((rank, res))


def test_reductions_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == (2.5, 30.0)


def test_rank_workloads_are_disjoint():
    """each rank draws its particles from its own seed and id range (weak
    scaling: no rank shares a particle with another)"""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2110_00256_gb300 import workloads
    seeds = [bench.SEED + 7919 * r + 1 for r in range(2)]
    a = workloads.paper_benchmark(1000, seeds[0], 0 + 0 * 10 ** 10)
    b = workloads.paper_benchmark(1000, seeds[1], 0 + 1 * 10 ** 10)
    assert not set(a["id"].tolist()) & set(b["id"].tolist())
    assert not np.array_equal(a["px"], b["px"])


def test_reference_arm_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
