"""Multi-start BFS, the oracle's form of the BFS step run from several
vertices at once (Section 3.2).

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle``, only the tests,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` use it.

Section 3.2 computes components with BFS, one traversal per component, each
from a vertex that no earlier traversal reached; Algorithm 2 runs one such
traversal (from one seed) before SV. The multi-start form runs several
traversals at once, one tree per start. Its starts are a reading (the paper
names one seed, picked at random in Section 5): the id range [0, n) is cut
into k ranges [j n / k, (j + 1) n / k), and each range's vertex of largest
degree starts a tree, ties going to the smallest id. A range whose largest
degree is 0 starts none. With k = 1 this is the single start, the
max-degree vertex.

What the traversal reaches does not depend on the order in which the trees
grow. With a cutoff of L levels it is the set of vertices at distance <= L
from some start; with no cutoff it is the union of the starts' components.
Which tree claims a vertex that two trees reach at the same level is not
unique, so the oracle gives the starts and the distances only.
"""
from __future__ import annotations

import numpy as np

from . import degrees
from . import multi_bfs_distances as _distances


def bfs_starts(edges: np.ndarray, n: int, k: int) -> np.ndarray:
    """The starts of a k-start BFS: per id range, the first vertex of
    largest degree (numpy's argmax returns the first maximum), if that
    degree is above 0."""
    deg = degrees(edges, n)
    starts = []
    for j in range(k):
        lo, hi = j * n // k, (j + 1) * n // k
        if hi <= lo:
            continue
        v = lo + int(np.argmax(deg[lo:hi]))
        if deg[v] > 0:
            starts.append(v)
    return np.asarray(starts, dtype=np.int64)


def multi_bfs_distances(edges: np.ndarray, n: int, starts: np.ndarray, cutoff: int = 0) -> np.ndarray:
    """Level-synchronous BFS from all starts at once: dist[v] = the smallest
    number of pairs on a path from a start to v, -1 if v is not reached.
    With cutoff L > 0 the traversal stops after L levels, so only distances
    <= L are found (cutoff 0: run to completion). The queue BFS of the
    oracle's C library."""
    return _distances(edges, n, starts, cutoff)


def multi_bfs_reached(edges: np.ndarray, n: int, k: int, cutoff: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(starts, reached mask) of a k-start BFS with the given cutoff."""
    starts = bfs_starts(edges, n, k)
    return starts, multi_bfs_distances(edges, n, starts, cutoff) >= 0
