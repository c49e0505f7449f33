"""Multi-start BFS (the BFS step of Section 3.2 run as several traversals at
once, options.bfs_starts) against the oracle.

Unique results are compared exactly: the labels, the number of trees
started (the ranges whose max-degree vertex has degree > 0), and the number
of vertices the traversal reached (with a cutoff of L levels, those within
distance L of a start; with none, the starts' components). Which tree claims
a vertex that two trees reach in the same level is not unique and is not
compared; the labels show that every tree was merged correctly.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import multi_bfs
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _power_law_union(seed=1, parts=24, id_bytes=4):
    """Mid-size power-law components of several sizes plus a sprinkle of
    isolated pairs, ids and pairs shuffled."""
    rng = np.random.default_rng(seed)
    gs = [gg.chung_lu(seed=seed * 100 + i, n=int(rng.integers(2000, 40000)), avg_degree=8, alpha=2.3)
          for i in range(parts)]
    gs.append(gg.Graph(np.array([(2 * i, 2 * i + 1) for i in range(500)], np.int32), 1200, "pairs"))
    return gg.union(gs, seed=seed, id_bytes=id_bytes)


def _graphs():
    return {
        "power_law_union": lambda: _power_law_union(1),
        "power_law_union_int64": lambda: _power_law_union(2, id_bytes=8),
        "planted": lambda: gg.planted(seed=3, n=60000, ncomp=300),
        "rmat": lambda: gg.rmat(seed=4, scale=15, edge_factor=8),
        "grid_chains": lambda: gg.grid_chains(seed=5, W=120, nchains=2000),
    }


def _run(torch, g, **opts):
    import paper_1607_06156_gb300 as cc

    eng = cc.Engine(id_bytes=g.id_bytes, **opts)
    lab = eng.labels(torch.from_numpy(g.edges).cuda(), g.n)
    torch.cuda.synchronize()
    st = eng.stats()
    eng.close()
    return lab.cpu().numpy().astype(np.int64), st


@pytest.mark.parametrize("name", list(_graphs()))
@pytest.mark.parametrize("k", [2, 64, 4096])
@pytest.mark.parametrize("profile", [0, 1])
def test_forced_bfs_route_multi_start(name, k, profile):
    torch = torch_cuda()
    g = _graphs()[name]()
    want = oracle.cc_labels(g.edges, g.n)
    for cutoff in (0, 1, 3):
        got, st = _run(torch, g, route="bfs", bfs_starts=k, bfs_cutoff_levels=cutoff, profile=profile)
        assert np.array_equal(got, want), (name, k, cutoff)
        starts, reached = multi_bfs.multi_bfs_reached(g.edges, g.n, k, cutoff)
        assert st["route"] == 1 and st["bfs_starts"] == len(starts), (st["bfs_starts"], len(starts))
        assert st["bfs_visited"] == int(reached.sum()), (name, k, cutoff, st["bfs_visited"], int(reached.sum()))
        if cutoff:
            assert st["bfs_levels"] <= cutoff


def test_one_start_is_the_single_tree_route():
    """bfs_starts = 1 is Algorithm 2's single BFS from the max-degree vertex."""
    torch = torch_cuda()
    g = _power_law_union(3)
    want = oracle.cc_labels(g.edges, g.n)
    got, st = _run(torch, g, route="bfs", bfs_starts=1)
    assert np.array_equal(got, want) and st["bfs_starts"] == 1
    starts, reached = multi_bfs.multi_bfs_reached(g.edges, g.n, 1)
    assert starts.tolist() == [int(np.argmax(oracle.degrees(g.edges, g.n)))]
    assert st["bfs_visited"] == int(reached.sum())


def test_heuristic_route_with_many_starts_reaches_more_components():
    """On power-law components the K-S heuristic takes the BFS step; with
    many starts the trees cover far more of the graph than one tree, and
    the labels stay exact."""
    torch = torch_cuda()
    g = _power_law_union(4, parts=40)
    want = oracle.cc_labels(g.edges, g.n)
    got1, st1 = _run(torch, g)
    got, st = _run(torch, g, bfs_starts=1024)
    assert np.array_equal(got1, want) and np.array_equal(got, want)
    assert st1["route"] == 1 and st["route"] == 1
    assert st["bfs_visited"] > 2 * st1["bfs_visited"], (st["bfs_visited"], st1["bfs_visited"])
    assert st["m_active"][0] < st1["m_active"][0]


def test_captured_and_replayed_on_new_inputs():
    """The multi-start route inside the caller's CUDA graph: starts, trees
    and merge all decided on the device for each replay's input."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    a, b = _power_law_union(5, parts=12), _power_law_union(6, parts=12)
    m = min(a.m, b.m)
    n = max(a.n, b.n)
    ea, eb = a.edges[:m].copy(), b.edges[:m].copy()
    eng = cc.Engine(route="bfs", bfs_starts=256)
    edges = torch.from_numpy(ea).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    eng.labels(edges, n, out=out)
    eng.check()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr):
        eng.labels(edges, n, out=out)
    for src in (ea, eb, ea):
        edges.copy_(torch.from_numpy(src))
        out.fill_(-1)
        gr.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.int64), oracle.cc_labels(src, n))
        st = eng.stats()
        starts, reached = multi_bfs.multi_bfs_reached(src, n, 256)
        assert st["status"] == 0 and st["bfs_starts"] == len(starts) and st["bfs_visited"] == int(reached.sum())
    del gr
    eng.close()


def test_starts_option_is_checked():
    torch_cuda()
    import paper_1607_06156_gb300 as cc

    with pytest.raises(cc.CCError) as ei:
        cc.Engine(bfs_starts=4097)
    assert ei.value.status == 1
