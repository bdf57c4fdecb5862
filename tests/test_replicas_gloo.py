"""The N > 1 bench path on CPU (two gloo ranks): the solve does not shard, so
every rank runs an independent replica and the bench reduces only the
timing.  Checks that every rank receives the slowest rank's time, that the
whole-job throughput counts all ranks' iterations over that time, and that
the reference arm prints nothing on a rank other than 0."""
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


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_max = bench.max_over_ranks(torch, dist, times[rank], "cpu")
        out[rank] = t_max
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    world, port = 2, _free_port()
    times = [10.0, 14.5]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 14.5
    # 2 replicas x 3 solves x 200 iterations in 14.5 ms
    assert bench.replica_throughput(world, 3, 200, out[0]) == pytest.approx(2 * 3 * 200 / 14.5e-3)


def test_single_process_keeps_its_time():
    assert bench.max_over_ranks(torch, None, 7.25, "cpu") == 7.25


def test_reference_arm_other_ranks_print_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
