"""Batched form: G independent graphs in one cc_labels_batched call.

Each graph's labels are local (the minimum local id of each component) and
must equal the oracle's labels of that graph alone, and the labels a loop of
per-graph cc_labels calls gives.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _run_batched(torch, edges, eoff, voff, **opts):
    import paper_1607_06156_gb300 as cc

    eng = cc.Engine(id_bytes=4, **opts)
    out = eng.labels_batched(torch.from_numpy(np.ascontiguousarray(edges)).cuda(), torch.from_numpy(eoff),
                             torch.from_numpy(voff))
    torch.cuda.synchronize()
    st = eng.stats()
    eng.close()
    return out.cpu().numpy().astype(np.int64), st


def _check_each(b, got, graphs=None):
    for g in (range(b.G) if graphs is None else graphs):
        gr = b.graph(g)
        want = oracle.cc_labels(gr.edges, gr.n)
        have = got[b.vertex_offsets[g]:b.vertex_offsets[g + 1]]
        bad = np.nonzero(have != want)[0]
        assert bad.size == 0, (g, gr.n, gr.m, bad[:5])


def test_mixed_batch_matches_oracle_per_graph():
    torch = torch_cuda()
    b = gg.batch(seed=3, G=90, nmin=1000, nmax=60000)
    got, st = _run_batched(torch, b.edges, b.edge_offsets, b.vertex_offsets)
    _check_each(b, got)
    assert st["sv_iters"] >= 2
    # the schedule the call used (the default below the tuner's size); the
    # degree pass of a batch of 2^20 pairs or more counts in shared-memory
    # windows, which have no regions (0)
    assert b.edge_offsets[-1] >= 1 << 20
    assert (st["batch_unroll"], st["batch_grid_mult"], st["batch_deg_regions"]) == (2, 1, 0)


@pytest.mark.parametrize("stride,route,profile", [(8, "auto", 0), (0, "auto", 0), (8, "sv", 0), (8, "auto", 1),
                                                   (8, "sv", 1)])
def test_front_end_per_graph(stride, route, profile):
    """The SV front end of the batched form (requested by a stride > 1): each
    graph with 2 m_g / n_g >= 4 (the R-MAT graphs here) is sampled at its own
    stride, the sparse ones (grids, chains) are hooked in full, and tiles
    cross graph boundaries. Labels equal the oracle's with the front end on
    and off (the default), on the captured and the profiled paths; with it
    on, the first gather pass leaves fewer pairs crossing trees."""
    torch = torch_cuda()
    b = gg.batch(seed=5, G=60, nmin=500, nmax=120000)
    got, st = _run_batched(torch, b.edges, b.edge_offsets, b.vertex_offsets, sv_sample_stride=stride, route=route,
                           profile=profile)
    _check_each(b, got)
    assert st["sv_sample_stride"] == (-1 if stride > 1 else 1)
    if stride > 1 and route == "auto" and not profile:
        _, off = _run_batched(torch, b.edges, b.edge_offsets, b.vertex_offsets)
        assert st["m_active"][2] < off["m_active"][2] // 2, (st["m_active"], off["m_active"])


@pytest.mark.parametrize("regions,profile", [(-1, 0), (1, 0), (8, 0), (32, 0), (8, 1), (1000, 0)])
def test_hook_passes_in_region_order(regions, profile):
    """The batched hook passes with their tiles taken from a counter over
    contiguous regions of the pairs (the tuner's other tile order): every
    tile exactly once, the odd last pair included, whatever the number of
    regions (more regions than tiles leave fetches with nothing to do)."""
    torch = torch_cuda()
    b = gg.batch(seed=6, G=40, nmin=500, nmax=80000)
    edges, eo, vo = b.edges, b.edge_offsets, b.vertex_offsets
    if eo[-1] % 2 == 0:  # an odd number of pairs: drop the last pair of the last graph
        edges, eo = edges[:-1], eo.copy()
        eo[-1] -= 1
    got, st = _run_batched(torch, edges, eo, vo, batch_hook_regions=regions, profile=profile)
    for g in range(b.G):
        want = oracle.cc_labels(np.ascontiguousarray(edges[eo[g]:eo[g + 1]]), int(vo[g + 1] - vo[g]))
        assert np.array_equal(got[vo[g]:vo[g + 1]], want), g
    assert st["batch_sv_regions"] == max(regions, 0)


def test_batched_equals_per_graph_loop():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    b = gg.batch(seed=4, G=24, nmin=2000, nmax=200000)
    got, _ = _run_batched(torch, b.edges, b.edge_offsets, b.vertex_offsets)
    eng = cc.Engine(id_bytes=4)
    for g in range(b.G):
        gr = b.graph(g)
        one = eng.labels(torch.from_numpy(np.ascontiguousarray(gr.edges)).cuda(), gr.n).cpu().numpy()
        assert np.array_equal(one, got[b.vertex_offsets[g]:b.vertex_offsets[g + 1]])
    eng.close()


def test_empty_tiny_and_ragged_graphs():
    torch = torch_cuda()
    rng = np.random.default_rng(5)
    sizes = [1, 5, 1000, 1, 3, 777, 2, 40000, 1]
    pairs = [0, 2, 3001, 0, 3, 1555, 1, 80001, 0]  # odd total; some graphs without pairs
    parts = [rng.integers(0, n, size=(k, 2)) for n, k in zip(sizes, pairs)]
    edges = np.concatenate(parts).astype(np.int32)
    eoff = np.concatenate([[0], np.cumsum(pairs)]).astype(np.int64)
    voff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    got, _ = _run_batched(torch, edges, eoff, voff)
    for g, (n, p) in enumerate(zip(sizes, parts)):
        want = oracle.cc_labels(p.astype(np.int32), n)
        assert np.array_equal(got[voff[g]:voff[g + 1]], want), g


def test_local_id_out_of_its_graph_is_rejected():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    edges = np.array([[0, 1], [1, 2], [0, 3]], dtype=np.int32)  # graph 1 has 3 vertices: id 3 is invalid there
    eoff = np.array([0, 1, 3], dtype=np.int64)
    voff = np.array([0, 10, 13], dtype=np.int64)
    with pytest.raises(cc.CCError) as ei:
        _run_batched(torch, edges, eoff, voff, debug_checks=1)
    assert ei.value.status == 2


def test_single_graph_batch_equals_cc_labels():
    torch = torch_cuda()
    g = gg.rmat(seed=6, scale=16, edge_factor=8)
    got, _ = _run_batched(torch, g.edges, np.array([0, g.m], np.int64), np.array([0, g.n], np.int64))
    assert np.array_equal(got, oracle.cc_labels(g.edges, g.n))


def test_batched_over_2_25_vertices():
    """A batch of more than 2^25 vertices in all (a parent array larger than L2)."""
    torch = torch_cuda()
    b = gg.batch(seed=12, G=40, nmin=800_000, nmax=1_000_000, edge_factor=2)
    assert b.vertex_offsets[-1] >= 1 << 25
    got, _ = _run_batched(torch, b.edges, b.edge_offsets, b.vertex_offsets)
    _check_each(b, got)


@pytest.mark.parametrize("bad", [-2, 1025])
def test_hook_regions_option_is_checked(bad):
    torch_cuda()
    import paper_1607_06156_gb300 as cc

    with pytest.raises(cc.CCError) as ei:
        cc.Engine(batch_hook_regions=bad)
    assert ei.value.status == 1


def _window_edge_case_batch():
    """A batch for the windowed degree pass (windows of 4,096 vertices per
    graph, 2^20 pairs or more in all) with each of its exact fallbacks:
    a graph of more than 2^20 vertices (counted and hooked with global
    atomics), 1,500 graphs of three pairs and two windows each (their chunks
    span more than 512 windows), a star whose window runs far past its
    capacity, an R-MAT graph with hubs and a long path."""
    rng = np.random.default_rng(77)
    gs = []
    n_big = (1 << 20) + 3
    gs.append((rng.integers(0, n_big, size=(400_000, 2)), n_big))
    for k in range(700):
        n = 4097 + k % 3
        gs.append((rng.integers(0, n, size=(3, 2)), n))
    n = 50_000
    star = np.stack([np.full(300_000, 7), rng.integers(0, n, size=300_000)], axis=1)
    star[::5] = star[::5, ::-1]
    gs.append((star, n))
    r = gg.rmat(seed=78, scale=17, edge_factor=8)
    gs.append((r.edges.astype(np.int64), r.n))
    for k in range(800):
        n = 4097 + k % 5
        gs.append((rng.integers(0, n, size=(3, 2)), n))
    n = 200_000
    perm = rng.permutation(n)
    gs.append((np.stack([perm[:-1], perm[1:]], axis=1), n))
    gs.append((np.array([[0, 0], [1, 1], [2, 1]]), 3))  # self-loops
    eo = np.zeros(len(gs) + 1, np.int64)
    vo = np.zeros(len(gs) + 1, np.int64)
    for i, (e, n) in enumerate(gs):
        eo[i + 1] = eo[i] + len(e)
        vo[i + 1] = vo[i] + n
    edges = np.ascontiguousarray(np.concatenate([e for e, _ in gs]).astype(np.int32))
    assert eo[-1] >= 1 << 20
    return gs, edges, eo, vo


def test_windowed_degree_pass_fallbacks_per_graph_fit():
    """The batched degree pass in shared-memory windows against the oracle:
    every graph's fit (which depends on every degree) and max-degree seed."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    gs, edges, eo, vo = _window_edge_case_batch()
    eng = cc.Engine()
    r = eng.ks_statistic_batched(torch.from_numpy(edges).cuda(), eo, vo)
    eng.close()
    for i, (e, n) in enumerate(gs):
        deg = oracle.degrees(e, n)
        want = oracle.ks_fit(oracle.histogram(deg))
        assert r["ncand"][i] == want["ncand"] and r["xmin"][i] == want["xmin"], (i, want)
        assert abs(r["D"][i] - want["D"]) < 1e-9, (i, r["D"][i], want)
        assert r["seed"][i] == int(np.argmax(deg)), i


@pytest.mark.parametrize("profile,stride", [(0, 0), (1, 0), (0, 8)])
def test_windowed_degree_pass_fallbacks_labels(profile, stride):
    """Labels per graph with the first hook pass inside the windowed degree
    pass (profile 0 and 1), and with the front end, whose degree pass hooks
    nothing (stride 8)."""
    torch = torch_cuda()
    gs, edges, eo, vo = _window_edge_case_batch()
    got, st = _run_batched(torch, edges, eo, vo, profile=profile, sv_sample_stride=stride)
    assert st["batch_deg_regions"] == 0
    for i, (e, n) in enumerate(gs):
        assert np.array_equal(got[vo[i]:vo[i + 1]], oracle.cc_labels(e.astype(np.int32), n)), i
