"""bench.py's multi-rank aggregation (N replicas, one per GPU) with world_size 2 gloo
ranks on the CPU: barrier, max over ranks, whole-job value."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_seconds = 1.0 + rank  # rank 1 is the slow one
    dist.barrier()
    m = bench.max_over_ranks(local_seconds, dist, "cpu")
    v = bench.weak_value(world, 1000.0, m)
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == pytest.approx(2.0)          # the slowest rank's time
        assert v == pytest.approx(2 * 1000 / 2.0)  # all ranks' units / that time


def test_single_process_defaults():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.weak_value(1, 10.0, 2.0) == 5.0
