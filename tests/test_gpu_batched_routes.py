"""Per-graph route prediction of the batched form (Algorithm 2 lines 1-3 per
graph): the device fit of every graph against the fp64 oracle's fit of that
graph alone, and the labels of batches whose graphs take different routes."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _concat(graphs):
    eo = np.zeros(len(graphs) + 1, dtype=np.int64)
    vo = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, (e, n) in enumerate(graphs):
        eo[i + 1] = eo[i] + e.shape[0]
        vo[i + 1] = vo[i] + n
    edges = np.concatenate([e.astype(np.int32).reshape(-1, 2) for e, _ in graphs]) if eo[-1] else \
        np.zeros((0, 2), np.int32)
    return np.ascontiguousarray(edges), eo, vo


def _mixed_graphs(with_overflow=False):
    gs = []
    for k in range(4):
        g = gg.chung_lu(seed=40 + k, n=20000 + 5000 * k, avg_degree=10, alpha=2.3)  # power law: BFS
        gs.append((g.edges, g.n))
    for k in range(3):
        g = gg.rmat(seed=50 + k, scale=12 + k, edge_factor=8)
        gs.append((g.edges, g.n))
    g = gg.planted(seed=6, n=8000, ncomp=40)
    gs.append((g.edges, g.n))
    g = gg.grid_chains(seed=7, W=60, nchains=400)
    gs.append((g.edges, g.n))
    gs.append((np.zeros((0, 2), np.int32), 17))                       # edgeless
    gs.append((np.array([(0, 1), (1, 2)], np.int32), 3))             # tiny
    star = np.stack([np.zeros(5000, np.int64), np.arange(1, 5001)], axis=1)
    gs.append((star, 5001))                                          # one vertex of degree >= 4096
    if with_overflow:
        # more than 4096 vertices of degree >= 4096: the single-graph fit takes this graph
        n = 10000
        h = np.repeat(np.arange(4200), 4096)
        o = (h * 7 + np.tile(np.arange(4096), 4200) + 4200) % n
        gs.append((np.stack([h, o], axis=1), n))
    return gs


@pytest.mark.parametrize("with_overflow", [False, True])
def test_per_graph_fit_matches_oracle(with_overflow):
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    gs = _mixed_graphs(with_overflow)
    edges, eo, vo = _concat(gs)
    eng = cc.Engine()
    r = eng.ks_statistic_batched(torch.from_numpy(edges).cuda(), eo, vo)
    eng.close()
    for i, (e, n) in enumerate(gs):
        deg = oracle.degrees(e, n)
        want = oracle.ks_fit(oracle.histogram(deg))
        assert r["ncand"][i] == want["ncand"], (i, r["ncand"][i], want)
        assert abs(r["D"][i] - want["D"]) < 1e-9, (i, r["D"][i], want)
        assert r["xmin"][i] == want["xmin"], (i, r["xmin"][i], want)
        if want["ncand"]:
            assert abs(r["alpha"][i] - want["alpha"]) < 1e-9 * max(1.0, want["alpha"])
        assert r["route"][i] == int(oracle.route_is_bfs(want["D"]))
        assert r["seed"][i] == int(np.argmax(deg))
    assert r["route"][:4].all()  # the power-law graphs go to BFS


@pytest.mark.parametrize("route,profile", [("auto", 0), ("auto", 1), ("bfs", 0), ("sv", 0), ("learned", 0)])
def test_batched_labels_whatever_each_graph_routes(route, profile):
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    gs = _mixed_graphs()
    edges, eo, vo = _concat(gs)
    eng = cc.Engine(route=route, profile=profile)
    out = eng.labels_batched(torch.from_numpy(edges).cuda(), torch.from_numpy(eo), torch.from_numpy(vo))
    st = eng.stats()
    eng.close()
    got = out.cpu().numpy().astype(np.int64)
    for i, (e, n) in enumerate(gs):
        assert np.array_equal(got[vo[i]:vo[i + 1]], oracle.cc_labels(e, n)), i
    if route == "auto":
        assert st["route"] >= 4  # the power-law graphs took the BFS step
    if route == "sv":
        assert st["route"] == 0
    if route == "bfs":
        assert st["route"] == sum(1 for e, n in gs if n > 0 and e.shape[0] > 0)


def test_batch_with_bfs_cutoff():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    gs = _mixed_graphs()[:5]
    edges, eo, vo = _concat(gs)
    for cutoff in (1, 2):
        eng = cc.Engine(bfs_cutoff_levels=cutoff)
        out = eng.labels_batched(torch.from_numpy(edges).cuda(), torch.from_numpy(eo), torch.from_numpy(vo))
        eng.close()
        got = out.cpu().numpy().astype(np.int64)
        for i, (e, n) in enumerate(gs):
            assert np.array_equal(got[vo[i]:vo[i + 1]], oracle.cc_labels(e, n)), (cutoff, i)
