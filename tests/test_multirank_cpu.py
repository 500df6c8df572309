"""The bench's multi-rank host logic on CPU: two gloo ranks, no GPU.

Each rank applies its own instance (no data-path collective); the job's time
is the slowest rank's (one MAX all-reduce), and the whole-job rate counts the
units of every rank.  The reference arm runs on rank 0 only.
"""
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(times[rank], dist, "cpu")
        out.put((rank, slowest, bench.rank_seed(7, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    times = [0.125, 0.5]
    port = 29500 + os.getpid() % 1000
    mp.start_processes(_rank_main, args=(2, port, times, out), nprocs=2, join=True, start_method="spawn")
    got = sorted(out.get(timeout=60) for _ in range(2))
    assert [g[1] for g in got] == [0.5, 0.5]          # both ranks see the max
    assert got[0][2] != got[1][2]                     # independent instances


def test_job_throughput_counts_every_rank():
    assert bench.job_throughput(1, 10, 100, 2.0) == 500.0
    assert bench.job_throughput(4, 10, 100, 2.0) == 2000.0
    assert bench.max_over_ranks(3.5) == 3.5           # one process: no reduction


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--gpus", "2"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
