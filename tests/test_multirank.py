"""The N > 1 host path on CPU: gloo process groups, world size 2.

bench.py runs one independent lattice per rank (replicas: no data-path
collective) and reports the whole-job rate timed by the slowest rank.  These
tests run that logic in two gloo ranks, and the reference arm of bench.py
(the CPU oracle) under torch.distributed.run with two processes.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_1810_04201_gb300 import gen
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    # each rank draws its own lattice (different seeds, no exchange)
    U, b = bench.make_inputs(bench.WORKLOADS["c1"], rank)
    step_ms = 10.0 + 5.0 * rank
    slowest = bench.max_over_ranks(step_ms, dist, "cpu")
    value = bench.job_throughput(1e9, slowest, world)
    q.put((rank, float(abs(b).sum()), slowest, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_and_max_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, v0), (r1, s1, t1, v1) = out
    assert s0 != s1  # different lattices per rank
    assert t0 == t1 == 15.0  # both ranks report the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 1e9 / 15e-3 / 1e9)


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus",
           "2", "--workload", "c1", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
