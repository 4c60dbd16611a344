"""bench.py's multi-rank logic on the CPU: world-size-2 gloo ranks (each rank times its own
replica; the step time is the slowest rank's, the value adds up over ranks) and the reference
arm under a launcher (rank 0 alone runs and prints)."""
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


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], world, dist, "cpu")
        out[rank] = (ms, bench.whole_job_percent(1e9, world, ms, 1000.0))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_with_two_gloo_ranks():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    times = [1.25, 2.5]
    mp.start_processes(_rank, args=(world, port, times, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 2.5                                     # the slowest rank's step
    assert value == pytest.approx(100.0 * 2 * 1e9 / 2.5e-3 / 1e9 / 1000.0)   # both ranks' bytes


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.0, 1, None, "cpu") == 3.0
    assert bench.whole_job_percent(2e9, 1, 1.0, 2000.0) == pytest.approx(100.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
