"""Full-size parity: the benchmark workloads, every label compared with the oracle.

R-MAT scale 24 (268M int32 pairs) in the benchmark's launch configuration
(default options, heuristic route) plus the forced BFS route, and the
grid + chains graph (8192^2 percolated grid at p = 0.55 unioned with 10M
branched chains, ~267M int64 vertices). The oracle's union-find runs once
per graph on the host (tens of seconds each).
"""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _labels(torch, edges_d, n, route, id_bytes):
    import paper_1607_06156_gb300 as cc

    eng = cc.Engine(id_bytes=id_bytes, route=route)
    out = eng.labels(edges_d, n)
    torch.cuda.synchronize()
    st = eng.stats()
    eng.close()
    return out, st


def test_rmat24_full_size():
    torch = torch_cuda()
    g = gg.rmat(seed=1, scale=24, edge_factor=16)
    want = oracle.labels_uf(g.edges, g.n)
    e = torch.from_numpy(g.edges).cuda()
    for route in ("auto", "bfs"):
        got, st = _labels(torch, e, g.n, route, 4)
        got = got.cpu().numpy()
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (route, bad[:10], st)
        if route == "bfs":
            assert st["route"] == 1 and st["bfs_visited"] > g.n // 3
    # component structure: one giant component plus isolated/tiny ones
    comp_sizes = np.bincount(want)
    assert comp_sizes.max() > g.n // 3


def test_grid_chains_full_size():
    torch = torch_cuda()
    g = gg.grid_chains(seed=1, W=8192, p=0.55, nchains=10_000_000, mean_len=20.0, branch_p=0.02, id_bytes=8)
    assert 250_000_000 < g.n < 290_000_000 and 250_000_000 < g.m < 290_000_000
    want = oracle.labels_uf(g.edges, g.n)
    e = torch.from_numpy(g.edges).cuda()
    got, st = _labels(torch, e, g.n, "auto", 8)
    assert st["route"] == 0  # mesh + chains: no power-law tail, SV only
    got = got.cpu().numpy()
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (bad[:10], st)
    # every chain is its own component
    assert np.unique(want).size >= 10_000_000


def test_batch4096_full_size():
    """The 4,096-graph batch: every graph's labels against the oracle's
    union-find (the graphs are spread over host threads; the oracle releases
    the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    b = gg.batch(seed=1, G=4096, nmin=1000, nmax=1_000_000)
    eng = cc.Engine(id_bytes=4)
    out = eng.labels_batched(torch.from_numpy(b.edges).cuda(), torch.from_numpy(b.edge_offsets),
                             torch.from_numpy(b.vertex_offsets))
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.int64)
    eng.close()
    eo, vo = b.edge_offsets, b.vertex_offsets

    def mismatch(g):
        want = oracle.labels_uf(b.edges[eo[g]:eo[g + 1]], int(vo[g + 1] - vo[g]))
        return not np.array_equal(want, got[vo[g]:vo[g + 1]])

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        bad = [g for g, x in enumerate(ex.map(mismatch, range(b.G))) if x]
    assert not bad, bad[:10]
