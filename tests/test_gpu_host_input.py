"""cc_labels_host: pairs and labels in host memory. Above 2^24 pairs the copy
is chunked and the degree count and the first SV pass consume each chunk as
it lands; the labels must equal the oracle's whatever the route, id width,
ragged tail or kind of host memory."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _host_labels(edges, n, pin=True, **opts):
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    eng = cc.Engine(id_bytes=edges.dtype.itemsize, **opts)
    try:
        e = torch.from_numpy(np.ascontiguousarray(edges))
        if pin:
            e = e.pin_memory()
        out = eng.labels_host(e, n)
        return out.numpy().astype(np.int64), eng.stats()
    finally:
        eng.close()


@pytest.mark.parametrize("route", ["auto", "sv", "bfs", "learned"])
def test_small_graphs_take_one_copy(route):
    g = gg.planted(seed=3, n=20000, ncomp=90)
    got, _ = _host_labels(g.edges, g.n, route=route)
    assert np.array_equal(got, oracle.cc_labels(g.edges, g.n))


@pytest.mark.parametrize("id_bytes,extra,route", [(4, 3, "auto"), (8, 1, "auto"), (4, 0, "sv"), (4, 5, "bfs")])
def test_chunked_copy_matches_oracle(id_bytes, extra, route):
    g = gg.rmat(seed=17, scale=20, edge_factor=16, m=(1 << 24) + extra, id_bytes=id_bytes)
    want = oracle.cc_labels(g.edges, g.n, cross_check=False)
    got, st = _host_labels(g.edges, g.n, route=route)
    assert np.array_equal(got, want)
    if route == "auto":
        # the degrees counted chunk by chunk give the same statistics as the device call
        deg = oracle.degrees(g.edges, g.n)
        assert st["max_degree"] == int(deg.max())
        assert st["seed_vertex"] == int(np.argmax(deg))


def test_chunked_copy_then_bfs_route():
    """A power-law graph above 2^24 pairs: the SV iterations streamed during
    the copy are discarded when the K-S fit picks BFS first."""
    g = gg.chung_lu(seed=5, n=1 << 21, avg_degree=17, alpha=2.3)
    assert g.m >= 1 << 24
    want = oracle.cc_labels(g.edges, g.n, cross_check=False)
    got, st = _host_labels(g.edges, g.n, route="auto")
    assert st["route"] == 1
    assert np.array_equal(got, want)
    got, st = _host_labels(g.edges, g.n, route="auto", bfs_mode=1)
    assert st["route"] == 1
    assert np.array_equal(got, want)


def test_chunked_copy_from_pageable_memory_and_repeat():
    g = gg.grid_chains(seed=9, W=2000, nchains=800000, id_bytes=4)
    assert g.m >= 1 << 24
    want = oracle.cc_labels(g.edges, g.n, cross_check=False)
    for pin in (False, True, True):
        got, _ = _host_labels(g.edges, g.n, pin=pin)
        assert np.array_equal(got, want)
    # the host-driven loop (per-kernel profiling on) continues the streamed iterations too
    got, st = _host_labels(g.edges, g.n, profile=1)
    assert np.array_equal(got, want)


def test_invalid_id_in_host_pairs():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    e = np.array([(0, 1), (2, 9)], dtype=np.int32)
    eng = cc.Engine()
    with pytest.raises(cc.CCError) as ei:
        eng.labels_host(torch.from_numpy(e), 5)
    assert ei.value.status == 2
    ok = eng.labels_host(torch.from_numpy(np.array([(0, 1)], dtype=np.int32)), 3)
    assert ok.tolist() == [0, 0, 2]
    eng.close()
