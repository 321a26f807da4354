"""The bench's multi-rank path on CPU: two gloo ranks, each with its own
timing, agree on the job's wall time (max over ranks) and on the whole-job
throughput of the replicas."""

import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.5, 2.25][rank]             # per-rank timed region
        wall = bench.max_over_ranks(local, dist, "cpu")
        solves, tflops = bench.replica_throughput(3.0e12, 4, world, wall)
        out[rank] = (wall, solves, tflops)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_wall_time_and_throughput():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    wall, solves, tflops = out[0]
    assert wall == 2.25                        # the slowest rank sets the job's time
    assert solves == 8                         # 4 steps on each of 2 replicas
    assert tflops == pytest.approx(3.0e12 * 8 / 2.25 / 1e12)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.replica_throughput(2.0e12, 3, 1, 2.0) == (3, 3.0)
