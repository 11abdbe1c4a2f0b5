"""The benchmark's multi-rank timing on CPU: two gloo ranks (one process
each, rendezvous on 127.0.0.1), each with its own timed total; every rank
must see the slowest rank's time, and the whole-job throughput counts the
iterations of all ranks over that time.  The data path has no collective
(replicas: independent identical solves), so this reduction is the only
exchange between ranks."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [120.0, 310.5][rank]
        total = bench.max_over_ranks(local_ms, dist, "cpu")
        dist.barrier()
        q.put((rank, total, bench.job_value(total, world, 10, 1000)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [310.5, 310.5]
    assert all(g[2] == pytest.approx(world * 10 * 1000 / 0.3105) for g in got)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0
    assert bench.job_value(500.0, 1, 10, 1000) == pytest.approx(20000.0)
