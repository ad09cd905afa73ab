"""bench.py with several ranks, on the CPU (gloo, world size 2).

Every rank runs a full replica of the step; the reported time is the
slowest rank's and the rate counts every rank's bytes.  The reference arm
runs on rank 0 alone and the other ranks exit without work."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(torch, times[rank], torch.device("cpu"))
        q.put((rank, ms))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    times = [3.25, 7.5]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 7.5, 1: 7.5}


def test_job_rate_counts_every_rank():
    # 2 ranks x 1e9 bytes x 10 steps in 20 ms of the slowest rank -> 1000 GB/s
    assert bench.job_rate(2, 1e9, 10, 20.0) == pytest.approx(1000.0)
    assert bench.job_rate(1, 1e9, 10, 20.0) == pytest.approx(500.0)


def test_reference_arm_under_torchrun_world2(tmp_path):
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3", "--ops", "reduce"]
    env = dict(os.environ, TMPDIR=str(tmp_path))        # torchrun's log directory goes under pytest's
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1                          # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
