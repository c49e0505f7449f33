"""Pins of the multi-start BFS oracle (Section 3.2, one traversal per start):
the starts on a hand-built graph, the distances against scipy's shortest
paths, and the reached set without a cutoff against scipy's components."""
import numpy as np
import pytest

from oracle import multi_bfs

scipy_sparse = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


def _hand_graph():
    # n = 10, ranges for k = 3: [0, 3), [3, 6), [6, 10)
    # degrees: 0:1 1:3 2:3 | 3:0 4:0 5:0 | 6:1 7:1 8:4 9:1 (a self-loop adds 2)
    e = np.array([(1, 2), (1, 2), (1, 0), (2, 6), (8, 8), (8, 9), (8, 7)], dtype=np.int64)
    return e, 10


def test_starts_by_hand():
    e, n = _hand_graph()
    # range 0: vertices 1 and 2 tie at degree 3 -> 1; range 1: all degree 0 -> no start;
    # range 2: vertex 8 (degree 4: a self-loop and two pairs)
    assert multi_bfs.bfs_starts(e, n, 3).tolist() == [1, 8]
    # one range: the max-degree vertex, ties to the smallest id (8 has degree 4)
    assert multi_bfs.bfs_starts(e, n, 1).tolist() == [8]
    # ten ranges of one vertex: every vertex of degree > 0
    assert multi_bfs.bfs_starts(e, n, 10).tolist() == [0, 1, 2, 6, 7, 8, 9]
    # more ranges than vertices: empty ranges start nothing
    assert multi_bfs.bfs_starts(e, n, 16).tolist() == [0, 1, 2, 6, 7, 8, 9]


def test_distances_by_hand_with_cutoffs():
    e, n = _hand_graph()
    starts = np.array([1, 8])
    d = multi_bfs.multi_bfs_distances(e, n, starts)
    assert d.tolist() == [1, 0, 1, -1, -1, -1, 2, 1, 0, 1]
    d1 = multi_bfs.multi_bfs_distances(e, n, starts, cutoff=1)
    assert d1.tolist() == [1, 0, 1, -1, -1, -1, -1, 1, 0, 1]


def _random_graph(rng, n, m):
    e = rng.integers(0, n, size=(m, 2))
    return e


@pytest.mark.parametrize("seed", range(6))
def test_distances_match_scipy_shortest_paths(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(50, 400))
    e = _random_graph(rng, n, int(rng.integers(n // 2, 2 * n)))
    k = int(rng.integers(1, 12))
    starts = multi_bfs.bfs_starts(e, n, k)
    a = scipy_sparse.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n)).tocsr()
    sp = csgraph.shortest_path(a, method="D", directed=False, unweighted=True, indices=starts)
    want = np.min(np.atleast_2d(sp), axis=0)
    got = multi_bfs.multi_bfs_distances(e, n, starts)
    reach = np.isfinite(want)
    assert np.array_equal(got >= 0, reach)
    assert np.array_equal(got[reach], want[reach].astype(np.int64))
    for L in (1, 2, 3):
        gl = multi_bfs.multi_bfs_distances(e, n, starts, cutoff=L)
        assert np.array_equal(gl >= 0, reach & (want <= L)), L


@pytest.mark.parametrize("seed", range(4))
def test_full_traversal_reaches_the_starts_components(seed):
    rng = np.random.default_rng(100 + seed)
    n = 600
    e = _random_graph(rng, n, 380)  # below the giant-component threshold: many components
    k = 20
    starts, reached = multi_bfs.multi_bfs_reached(e, n, k)
    a = scipy_sparse.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n)).tocsr()
    _, comp = csgraph.connected_components(a, directed=False)
    assert np.array_equal(reached, np.isin(comp, comp[starts]))


def test_starts_are_the_range_maxima():
    """Every start has the largest degree of its range and the smallest id
    among the range's vertices of that degree (checked by a plain scan)."""
    rng = np.random.default_rng(7)
    n = 1000
    e = rng.integers(0, n, size=(1500, 2))
    deg = np.zeros(n, dtype=np.int64)
    for u, v in e:
        deg[u] += 1
        deg[v] += 1
    k = 37
    starts = list(multi_bfs.bfs_starts(e, n, k))
    want = []
    for j in range(k):
        lo, hi = j * n // k, (j + 1) * n // k
        best = None
        for v in range(lo, hi):
            if best is None or deg[v] > deg[best]:
                best = v
        if best is not None and deg[best] > 0:
            want.append(best)
    assert starts == want
