"""LPT graph shards of the batched form (host logic, no GPU)."""
import itertools
import os

import numpy as np
import pytest

from paper_1607_06156_gb300.sharding import graph_cost, lpt_shards, shard_loads


def _opt_makespan(cost, world):
    best = None
    for assign in itertools.product(range(world), repeat=len(cost)):
        loads = [0] * world
        for c, r in zip(cost, assign):
            loads[r] += c
        best = max(loads) if best is None else min(best, max(loads))
    return best


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_every_graph_in_exactly_one_shard(world):
    rng = np.random.default_rng(world)
    cost = rng.integers(1, 10**6, size=200)
    shards = lpt_shards(cost, world)
    assert len(shards) == world
    allg = np.concatenate(shards)
    assert np.array_equal(np.sort(allg), np.arange(200))
    for s in shards:
        assert np.all(np.diff(s) > 0)
    assert sum(shard_loads(cost, shards)) == int(cost.sum())


@pytest.mark.parametrize("seed", range(25))
def test_graham_bound_against_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    world = int(rng.integers(2, 4))
    cost = rng.integers(1, 50, size=int(rng.integers(1, 9))).tolist()
    mk = max(shard_loads(cost, lpt_shards(cost, world)))
    opt = _opt_makespan(cost, world)
    assert mk <= (4 / 3 - 1 / (3 * world)) * opt + 1e-9


def test_lpt_known_case_and_ties():
    # the classic tight case for N = 2: 3,3,2,2,2 -> LPT 7, optimum 6
    assert max(shard_loads([3, 3, 2, 2, 2], lpt_shards([3, 3, 2, 2, 2], 2))) == 7
    # equal costs: round robin in graph order, ranks in order
    sh = lpt_shards([5] * 6, 3)
    assert [s.tolist() for s in sh] == [[0, 3], [1, 4], [2, 5]]
    assert [s.tolist() for s in lpt_shards([], 2)] == [[], []]


def test_batch_shards_cover_the_batch_sizes():
    import graphgen as gg

    ng, mg = gg.batch_sizes(seed=2, G=60, nmin=1000, nmax=20000)
    cost = graph_cost(ng, mg)
    shards = lpt_shards(cost, 4)
    loads = shard_loads(cost, shards)
    assert max(loads) <= int(cost.sum()) / 4 + int(cost.max())
    sub = gg.batch(seed=2, G=60, nmin=1000, nmax=20000, graphs=shards[1])
    whole = gg.batch(seed=2, G=60, nmin=1000, nmax=20000)
    for i, g in enumerate(shards[1]):
        assert np.array_equal(sub.graph(i).edges, whole.graph(int(g)).edges)


def _ranks_agree(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(7)
    cost = rng.integers(1, 1000, size=101)
    mine = lpt_shards(cost, world)[rank]
    sizes = [None] * world
    dist.all_gather_object(sizes, mine.tolist())
    dist.destroy_process_group()
    out.put((rank, sizes))


def test_two_gloo_ranks_take_disjoint_shards():
    import multiprocessing as mp
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_ranks_agree, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, sizes in res:
        allg = sorted(sizes[0] + sizes[1])
        assert allg == list(range(101))
        assert not set(sizes[0]) & set(sizes[1])
