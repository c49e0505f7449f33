"""Pins for the oracle's component labels (CPU only).

The oracle computes label[v] = min{u : u reachable from v} (Section 1;
Section 3.1.1 and the Figure 1(b) caption). These tests tie it to things
other than itself: exhaustive brute force over all small graphs, a
pure-Python reachability search, scipy's connected components, planted
component structure, the paper's worked example and the paper's own
tuple-array algorithm.
"""
import itertools
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.tuple_sv import tuple_sv


def _py_reach_labels(n, edges):
    """Pure-Python DFS reachability: the definition with no shared code."""
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[int(u)].append(int(v))
        adj[int(v)].append(int(u))
    out = []
    for v in range(n):
        seen = {v}
        stack = [v]
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if y not in seen:
                    seen.add(y)
                    stack.append(y)
        out.append(min(seen))
    return out


def _arr(edges, dtype=np.int32):
    return np.array(edges, dtype=dtype).reshape(-1, 2)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_exhaustive_all_edge_subsets(n):
    """Every simple graph on n <= 5 labelled vertices: three oracles + the definition agree."""
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        e = _arr(edges)
        want = _py_reach_labels(n, edges)
        assert oracle.labels_closure(e, n).tolist() == want
        assert oracle.labels_uf(e, n).tolist() == want
        assert oracle.labels_bfs(e, n).tolist() == want


def test_random_small_with_loops_and_duplicates():
    rng = np.random.default_rng(7)
    for trial in range(300):
        n = int(rng.integers(1, 65))
        m = int(rng.integers(0, 3 * n))
        e = rng.integers(0, n, size=(m, 2)).astype(np.int64)
        want = _py_reach_labels(n, e.tolist())
        assert oracle.labels_closure(e, n).tolist() == want
        assert oracle.labels_uf(e, n).tolist() == want
        assert oracle.labels_bfs(e, n).tolist() == want


def test_special_cases():
    n = 50
    path = _arr([(i, i + 1) for i in range(n - 1)])
    assert (oracle.cc_labels(path, n) == 0).all()
    rpath = _arr([(i + 1, i) for i in reversed(range(n - 1))])
    assert (oracle.cc_labels(rpath, n) == 0).all()
    empty = np.zeros((0, 2), dtype=np.int32)
    assert oracle.cc_labels(empty, n).tolist() == list(range(n))
    complete = _arr(list(itertools.combinations(range(n), 2)))
    assert (oracle.cc_labels(complete, n) == 0).all()
    star = _arr([(n - 1, i) for i in range(n - 1)])
    assert (oracle.cc_labels(star, n) == 0).all()
    loops = _arr([(i, i) for i in range(n)])
    assert oracle.cc_labels(loops, n).tolist() == list(range(n))
    dup = _arr([(3, 9)] * 10 + [(9, 4)] * 3)
    lab = oracle.cc_labels(dup, 12)
    assert lab[3] == lab[9] == lab[4] == 3 and lab[0] == 0 and lab[11] == 11
    assert oracle.cc_labels(np.zeros((0, 2), np.int32), 0).size == 0
    assert oracle.cc_labels(np.zeros((0, 2), np.int32), 1).tolist() == [0]


def test_out_of_range_ids_rejected():
    with pytest.raises(ValueError):
        oracle.labels_uf(_arr([(0, 5)]), 5)
    with pytest.raises(ValueError):
        oracle.labels_bfs(_arr([(-1, 2)]), 5)


def _golden(path):
    d = {}
    edges = []
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        k, *rest = line.split()
        if k == "edge":
            edges.append(tuple(int(x) for x in rest))
        elif k == "ids":
            d[k] = dict(x.split("=") for x in rest)
        else:
            d[k] = [int(x) for x in rest]
    return d, edges


def test_fig1b_worked_example(golden_dir):
    """Section 3.1.1 / Figure 1(b): u, v1, v2 end in component v1 = min."""
    d, edges = _golden(os.path.join(golden_dir, "fig1b_example.txt"))
    n = d["n"][0]
    ids = {k: int(v) for k, v in d["ids"].items()}
    e = _arr(edges)
    assert oracle.cc_labels(e, n).tolist() == d["label"]
    assert oracle.labels_closure(e, n).tolist() == d["label"]
    lab, _ = tuple_sv(n, edges)
    assert lab == d["label"]
    # the initial tuple array of Algorithm 1: <x,_,x> per vertex, <x,_,y>, <y,_,x> per pair
    A0 = [(x, x) for x in range(n)] + [t for x, y in edges for t in ((x, y), (y, x))]
    u, v1 = ids["u"], ids["v1"]
    M0 = lambda r: sorted({p for p, rr in A0 if rr == r})
    V0 = lambda p: sorted({r for pp, r in A0 if pp == p})
    assert M0(u) == d["M0_u"]
    assert V0(u) == d["V0_u"]
    assert sorted({q for r in V0(v1) for q in M0(r)}) == d["N0_v1"]


def test_planted_components_match_planted_sets():
    g = gg.planted(seed=3)
    lab = oracle.cc_labels(g.edges, g.n)
    comp = g.meta["comp"]
    assert np.unique(lab).size == g.meta["ncomp"] == 512
    mins = np.full(g.meta["ncomp"], g.n, dtype=np.int64)
    np.minimum.at(mins, comp, np.arange(g.n))
    assert np.array_equal(lab, mins[comp])


def test_chain_forest_matches_planted_chains():
    g = gg.grid_chains(seed=5, W=1, nchains=2000, mean_len=20.0, branch_p=0.02, id_bytes=8)
    lab = oracle.cc_labels(g.edges, g.n)
    off = g.meta["chain_off"]
    pre = np.arange(g.n - 1, dtype=np.uint64) + 1  # pre-permutation ids of chain vertices (W*W = 1)
    post = gg.permute(g.n, 5, 24, pre).astype(np.int64)
    chain_of = np.repeat(np.arange(off.size - 1), np.diff(off))
    mins = np.full(off.size - 1, g.n, dtype=np.int64)
    np.minimum.at(mins, chain_of, post)
    assert np.array_equal(lab[post], mins[chain_of])
    assert np.unique(lab).size == 2000 + 1  # chains plus the single grid vertex


def _scipy_min_labels(edges, n):
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    e = np.asarray(edges, dtype=np.int64)
    A = sp.coo_matrix((np.ones(e.shape[0]), (e[:, 0], e[:, 1])), shape=(n, n))
    k, comp = csg.connected_components(A, directed=False)
    mins = np.full(k, n, dtype=np.int64)
    np.minimum.at(mins, comp, np.arange(n))
    return mins[comp]


@pytest.mark.parametrize("maker", [
    lambda: gg.rmat(seed=2, scale=14, edge_factor=4),
    lambda: gg.grid_chains(seed=9, W=128, p=0.55, nchains=3000, id_bytes=8),
    lambda: gg.planted(seed=11, n=20000, ncomp=300),
])
def test_against_scipy_connected_components(maker):
    g = maker()
    assert np.array_equal(oracle.cc_labels(g.edges, g.n), _scipy_min_labels(g.edges, g.n))


def test_label_invariants_rmat():
    g = gg.rmat(seed=4, scale=16, edge_factor=16)
    lab = oracle.cc_labels(g.edges, g.n)
    e = g.edges.astype(np.int64)
    assert (lab[e[:, 0]] == lab[e[:, 1]]).all()
    v = np.arange(g.n)
    assert (lab <= v).all()
    assert (lab[lab] == lab).all()


def test_tuple_sv_algorithm1_agrees():
    """The paper's Algorithm 1 reaches the same min labels, in few iterations."""
    rng = np.random.default_rng(3)
    for trial in range(60):
        n = int(rng.integers(1, 40))
        m = int(rng.integers(0, 2 * n + 1))
        e = rng.integers(0, n, size=(m, 2))
        lab, it = tuple_sv(n, e.tolist())
        assert lab == oracle.labels_uf(e.astype(np.int64), n).tolist()
    # a path with shuffled ids: pointer doubling keeps iterations logarithmic
    n = 256
    perm = rng.permutation(n)
    edges = [(int(perm[i]), int(perm[i + 1])) for i in range(n - 1)]
    lab, it = tuple_sv(n, edges)
    assert lab == [0] * n
    assert it <= 2 * int(np.ceil(np.log2(n))) + 2
