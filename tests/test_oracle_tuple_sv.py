"""Pins for the tuple-array SV oracle and its exclusion of completed
partitions (Section 3.1.4), against fixed points that do not come from the
oracle: scipy's connected components, a hand-traced example, and the tuple
counts a component contributes (k vertices and e pairs give k + 2e tuples,
Section 3.1.1)."""
import numpy as np
import pytest

from oracle.tuple_sv import tuple_sv


def _components(n, edges):
    """{component id: sorted vertex list} from scipy (a library routine)."""
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    A = sp.coo_matrix((np.ones(e.shape[0]), (e[:, 0], e[:, 1])), shape=(n, n))
    _, comp = csg.connected_components(A, directed=False)
    out = {}
    for v, c in enumerate(comp.tolist()):
        out.setdefault(c, []).append(v)
    return out


def _random_graphs(count, seed):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(1, 48))
        m = int(rng.integers(0, 2 * n + 1))
        yield n, rng.integers(0, n, size=(m, 2)).tolist()


def test_hand_traced_exclusion():
    """Vertex 0 isolated, pair (2, 1), path 5-4-3.
    Iteration 1: only vertex 0 has M(0) = {0}, so only partition 0 is
    completed; the joins move 2 -> 1 and 4, 5 -> 3. Iteration 2: partitions 1
    and 3 each cover their component, nothing moves, the run stops."""
    trace = []
    lab, it = tuple_sv(6, [(2, 1), (5, 4), (4, 3)], trace=trace)
    assert lab == [0, 1, 1, 3, 3, 3]
    assert it == 2
    assert [t["excluded"] for t in trace] == [{0}, {1, 3}]
    assert [t["active"] for t in trace] == [6 + 2 * 3, 6 + 2 * 3 - 1]


def test_exclusion_keeps_labels_and_iterations():
    for n, e in _random_graphs(150, 11):
        assert tuple_sv(n, e) == tuple_sv(n, e, exclude_completed=False)


def test_excluded_partitions_are_the_components_completed_one_iteration_earlier():
    """A partition is excluded in iteration i exactly when one partition
    held every tuple of its component at the end of iteration i - 1 (the
    start of the run for i = 1) and it was not excluded before; it is the
    component's smallest vertex, and the working set shrinks by the
    component's k + 2e tuples."""
    for n, e in _random_graphs(120, 12):
        comps = _components(n, e)
        pairs_in = {c: 0 for c in comps}
        comp_of = {v: c for c, vs in comps.items() for v in vs}
        for x, _y in e:
            pairs_in[comp_of[x]] += 1
        trace = []
        tuple_sv(n, e, trace=trace)
        # tuples at each vertex before iteration 1: partition x for the self
        # tuple and for every pair (x, y) or (y, x) seen from vertex x
        parts_at = {v: {v} for v in range(n)}
        for x, y in e:
            parts_at[y].add(x)
            parts_at[x].add(y)
        excluded_before = set()
        active = n + 2 * len(e)
        for rec in trace:
            whole = set()
            for c, vs in comps.items():
                if c in excluded_before:
                    continue
                ps = set().union(*(parts_at[v] for v in vs))
                if len(ps) == 1:
                    whole.add(c)
            assert {comp_of[p] for p in rec["excluded"]} == whole
            assert all(p == min(comps[comp_of[p]]) for p in rec["excluded"])
            assert rec["active"] == active
            active -= sum(len(comps[c]) + 2 * pairs_in[c] for c in whole)
            excluded_before |= whole
            parts_at = {v: set(s) for v, s in rec["parts_at"].items()}
        assert excluded_before == set(comps)


def test_no_exclusion_keeps_every_tuple():
    trace = []
    tuple_sv(7, [(0, 1), (3, 4), (4, 6)], exclude_completed=False, trace=trace)
    assert all(t["active"] == 7 + 2 * 3 and not t["excluded"] for t in trace)


def test_pointer_doubling_on_ordered_paths():
    """Path 0-1-2-3, traced by hand: the join moves 1, 2 -> 0 and 3 -> 1;
    the extra tuple (1, 1) then pulls partition 1 to min M(1) = 0, so one
    iteration joins everything and the second finds nothing to move (a join
    alone would need three). On longer ordered paths the doubling keeps the
    iteration count within log2 of the length (a join alone covers about
    two hops per iteration)."""
    assert tuple_sv(4, [(0, 1), (1, 2), (2, 3)])[1] == 2
    for k in (16, 64, 256):
        lab, it = tuple_sv(k, [(i, i + 1) for i in range(k - 1)])
        assert lab == [0] * k
        assert it <= int(np.log2(k)), (k, it)
