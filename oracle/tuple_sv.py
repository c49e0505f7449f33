"""The paper's tuple-array Shiloach-Vishkin (Algorithm 1), sequential semantics.

TEST INFRASTRUCTURE ONLY (see the package docstring). Pure Python, for tiny
graphs: it exists to pin the final-label rule and the iteration behaviour to
the paper's own algorithm rather than to a union-find.

Section 3.1.1 / Algorithm 1: the array A_0 holds <x,_,x> for each vertex and
<x,_,y>, <y,_,x> for each undirected pair. Every iteration
  1. groups A by the third entry r (the vertex bucket VB(u)) and writes
     u_min = min of the partitions in VB(u) into the second entry q;
  2. groups A by the first entry p (the partition bucket PB(p)); each
     partition takes p_min = min of its candidates q; if p != p_min for any
     partition the run has not converged; every tuple of PB(p) moves to
     p_min, and a temporary tuple <p_min,_,p_min> is added per partition;
  3. repeats steps 1 and 2 once more with the temporary tuples present,
     which makes p_min join min M(p_min) (pointer doubling, Fig. 3);
  4. erases the temporary tuples.
At convergence the label of u is the partition of any tuple <c,_,u>
(Section 3.1.1, last paragraph), the minimum id of u's component.
"""
from __future__ import annotations

from collections import defaultdict


def _vertex_pass(A):
    """Step 1: q <- min of the partitions in the tuple's vertex bucket."""
    umin = {}
    for p, _q, r, _t in A:
        if r not in umin or p < umin[r]:
            umin[r] = p
    return [(p, umin[r], r, t) for p, _q, r, t in A]


def _partition_pass(A):
    """Step 2: every partition bucket moves to its minimum candidate."""
    pmin = {}
    for p, q, _r, _t in A:
        if p not in pmin or q < pmin[p]:
            pmin[p] = q
    changed = any(p != pm for p, pm in pmin.items())
    return [(pmin[p], q, r, t) for p, q, r, t in A], pmin, changed


def tuple_sv(n: int, edges) -> tuple[list[int], int]:
    """Run Algorithm 1 on vertices 0..n-1; returns (labels, iterations)."""
    A = [(x, None, x, False) for x in range(n)]
    for x, y in edges:
        A.append((int(x), None, int(y), False))
        A.append((int(y), None, int(x), False))
    iterations = 0
    converged = False
    while not converged:
        iterations += 1
        A = _vertex_pass(A)
        A, pmin, changed = _partition_pass(A)
        converged = not changed
        # one temporary tuple <p_min,_,p_min> per partition of this iteration
        A.extend((pm, None, pm, True) for pm in pmin.values())
        A = _vertex_pass(A)
        A, _pmin2, changed2 = _partition_pass(A)
        if changed2:
            converged = False
        A = [tup for tup in A if not tup[3]]
        if iterations > 4 * max(n, 1) + 8:
            raise RuntimeError("tuple SV failed to converge")
    label = defaultdict(lambda: None)
    for p, _q, r, _t in A:
        label[r] = p
    return [label[v] for v in range(n)], iterations
