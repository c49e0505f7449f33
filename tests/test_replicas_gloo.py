"""The N > 1 path of bench.py (replicas only: no collective in the data path)
with two gloo ranks on the CPU: the barrier + max-over-ranks timing, the
whole-job value, and the reference arm's rank-0-only rule."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
        value = bench.replica_value(world, 1000, 4, ms)
        ref = bench.run_reference(None, world, rank) if rank != 0 else None
        q.put((rank, ms, value, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    assert all(p.exitcode == 0 for p in ps)
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, value, ref in got:
        assert ms == 20.0                      # max over ranks, seen by every rank
        assert value == 2 * 1000 * 4 / 0.020   # both replicas' pairs / slowest time
    assert got[1][3] == 0                      # rank 1 of the reference arm exits 0 without work


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.replica_value(1, 10, 2, 1000.0) == 20.0
