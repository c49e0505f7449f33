"""The paper's sort-based SV (Algorithm 1) on the device: cc_labels_tuple_sv.

Algorithm 1 is deterministic (every step is a minimum over a group), so
the device run must match the oracle's sequential tuple-array Algorithm 1
in both the labels and the number of iterations on small graphs, and the
union-find labels on larger ones.
"""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.tuple_sv import tuple_sv
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1b_example.txt")


def _run(edges: np.ndarray, n: int, id_bytes: int = 4, **opts):
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    eng = cc.Engine(id_bytes=id_bytes, **opts)
    try:
        dt = np.int32 if id_bytes == 4 else np.int64
        e = torch.from_numpy(np.ascontiguousarray(edges, dtype=dt).reshape(-1, 2)).cuda()
        lab = eng.labels_tuple_sv(e, n)
        torch.cuda.synchronize()
        return lab.cpu().numpy().astype(np.int64), eng.stats()
    finally:
        eng.close()


@pytest.mark.parametrize("seed", range(6))
def test_matches_algorithm1_labels_iterations_and_working_set(seed):
    """Labels, iterations, and the tuples left in the working set entering
    every iteration after completed partitions leave (Section 3.1.4)."""
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 300))
    m = int(rng.integers(0, 2 * n + 1))
    e = rng.integers(0, n, size=(m, 2))
    trace = []
    want_lab, want_it = tuple_sv(n, e.tolist(), trace=trace)
    got, st = _run(e, n)
    assert got.tolist() == want_lab
    assert st["sv_iters"] == want_it
    assert st["m_active"][:want_it] == [t["active"] for t in trace]


def test_many_small_components_leave_early():
    """The planted graph's 512 components finish at different iterations:
    the working set shrinks each iteration exactly as in the oracle."""
    g = gg.planted(seed=6, n=4096, ncomp=128)
    trace = []
    want_lab, want_it = tuple_sv(g.n, g.edges.tolist(), trace=trace)
    got, st = _run(g.edges, g.n)
    assert got.tolist() == want_lab
    active = [t["active"] for t in trace]
    assert st["m_active"][:want_it] == active
    assert active[-1] < active[0]


def test_long_path_iterations():
    """A path with ids in random order: many iterations, each one checked
    against the sequential Algorithm 1 by its count."""
    rng = np.random.default_rng(9)
    n = 400
    order = rng.permutation(n)
    e = np.stack([order[:-1], order[1:]], axis=1)
    want_lab, want_it = tuple_sv(n, e.tolist())
    got, st = _run(e, n)
    assert got.tolist() == want_lab
    assert st["sv_iters"] == want_it
    assert want_it > 3


def test_figure_1b_example():
    d = {}
    edges = []
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        k, *rest = line.split()
        if k == "edge":
            edges.append([int(x) for x in rest])
        elif k in ("n", "label"):
            d[k] = [int(x) for x in rest]
    got, _ = _run(np.array(edges), d["n"][0])
    assert got.tolist() == d["label"]


@pytest.mark.parametrize("maker,id_bytes", [
    (lambda: gg.rmat(seed=5, scale=16, edge_factor=16), 4),
    (lambda: gg.planted(seed=6), 4),
    (lambda: gg.grid_chains(seed=7, W=300, nchains=20000, id_bytes=8), 8),
    (lambda: gg.chung_lu(seed=8, n=1 << 17, avg_degree=6, alpha=2.3), 4),
])
def test_larger_graphs_match_union_find(maker, id_bytes):
    g = maker()
    got, st = _run(g.edges, g.n, id_bytes=id_bytes)
    assert np.array_equal(got, oracle.cc_labels(g.edges, g.n))
    assert st["sv_iters"] >= 1


def test_edgeless_and_self_loops():
    got, st = _run(np.zeros((0, 2)), 37)
    assert got.tolist() == list(range(37))
    assert st["sv_iters"] == 1
    e = np.array([[3, 3], [5, 5], [5, 2], [2, 2]])
    got, _ = _run(e, 8)
    assert got.tolist() == [0, 1, 2, 3, 4, 2, 6, 7]


def test_invalid_id_and_size_limits():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    with pytest.raises(cc.CCError) as ei:
        _run(np.array([[0, 1], [2, 9]]), 5)
    assert ei.value.status == 2  # CC_ERR_INVALID_EDGE
    eng = cc.Engine()
    e = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    small = torch.empty(1, dtype=torch.int32, device="cuda")
    # the C boundary refuses n >= 2^31 before it touches the output
    assert cc.lib().cc_labels_tuple_sv(eng._h, e.data_ptr(), 1 << 31, 1, small.data_ptr(), 0) == 7  # UNSUPPORTED
    # the binding refuses an output shorter than n before the call
    with pytest.raises(ValueError):
        eng.labels_tuple_sv(e, 1 << 31, out=small)
    eng.close()


def test_sort_time_reported_when_profiling():
    """options.profile = 1 times every radix sort: four per iteration."""
    g = gg.rmat(seed=11, scale=15, edge_factor=8)
    got, st = _run(g.edges, g.n, profile=1)
    assert np.array_equal(got, oracle.cc_labels(g.edges, g.n))
    assert st["kernel_launches"]["tuple_sort"] == 4 * st["sv_iters"]
    assert 0.0 < st["kernel_ms"]["tuple_sort"] <= st["ms_total"]
