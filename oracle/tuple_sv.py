"""The paper's tuple-array Shiloach-Vishkin (Section 3.1), sequential semantics.

TEST INFRASTRUCTURE ONLY (see the package docstring). Pure Python, for tiny
graphs: it pins the final-label rule, the iteration count and the shrinking
working set to the paper's own formulation rather than to a union-find.

The formulation (Section 3.1.1). A graph is a bag of tuples (p, r): one
(x, x) per vertex and (x, y), (y, x) per undirected pair. r is a vertex and
never changes; p is the tuple's partition. From the bag:
  M(u)  = the partitions of the tuples whose vertex is u,
  V(p)  = the vertices of the tuples in partition p,
  C(p)  = { min M(u) : u in V(p) }, the candidates of p,
and N(p), the union of M(u) over V(p), is p's neighbourhood.

One iteration (Sections 3.1.2-3.1.3; Fig. 3):
  * join:     every partition p moves all its tuples to min C(p), the
              smallest neighbouring partition; if any partition moved, the
              run has not converged;
  * doubling: the partition p_min that p joined is pulled one step further.
              For every partition of the join, one extra tuple
              (p_min, p_min) ties partition p_min to vertex p_min, and the
              join runs again on the bag with these extras, which moves
              p_min to min M(p_min); the extras are then dropped.
The run stops after the first iteration in which neither join moved a
partition. The label of u is then the partition of any tuple with vertex u,
the smallest id of u's component (Section 3.1.1, last paragraph).

Exclusion of completed partitions (Section 3.1.4). A partition p is
completed when N(p) = {p}. While grouping by vertex at the start of an
iteration, every tuple of u is "potentially completed" if M(u) holds one
partition; while grouping by partition, p is "completed" if all of its
tuples are potentially completed. Completed partitions are whole
components; their labels are final and their tuples leave the working set
after the iteration that found them, one iteration after they became
complete.
"""
from __future__ import annotations


def _group_min(keys, vals):
    """{key: min of the values with that key} (a sort-and-scan in the paper)."""
    out = {}
    for k, v in zip(keys, vals):
        if k not in out or v < out[k]:
            out[k] = v
    return out


def _join(P, R):
    """Every partition moves to its smallest candidate, min C(p).

    Returns the moved partitions of the tuples and {p: min C(p)}."""
    u_min = _group_min(R, P)                         # min M(u), per vertex u
    p_min = _group_min(P, [u_min[r] for r in R])     # min C(p), per partition p
    return [p_min[p] for p in P], p_min


def _completed(P, R):
    """Partitions whose every tuple sits at a vertex u with |M(u)| = 1."""
    parts_at = {}
    for p, r in zip(P, R):
        parts_at.setdefault(r, set()).add(p)
    potentially = [len(parts_at[r]) == 1 for r in R]
    all_pot = {}
    for p, ok in zip(P, potentially):
        all_pot[p] = all_pot.get(p, True) and ok
    return {p for p, ok in all_pot.items() if ok}


def tuple_sv(n: int, edges, exclude_completed: bool = True, trace: list | None = None
             ) -> tuple[list[int], int]:
    """Labels of vertices 0..n-1 and the number of iterations.

    With `trace` (a list), one record per iteration is appended:
    {"active": tuples in the working set at the start of the iteration,
     "excluded": set of partitions found completed in it (they leave after
     it), "parts_at": {vertex: frozenset of the partitions of its tuples} for
     the vertices still active after it}.
    Exclusion never changes the labels or the iteration count: completed
    partitions have no neighbour to join.
    """
    P = list(range(n))
    R = list(range(n))
    for x, y in edges:
        x, y = int(x), int(y)
        P += [x, y]
        R += [y, x]
    label = [None] * n
    iterations = 0
    while True:
        iterations += 1
        if iterations > 4 * max(n, 1) + 8:
            raise RuntimeError("tuple SV failed to converge")
        active = len(P)
        done = _completed(P, R) if exclude_completed else set()
        P, first = _join(P, R)
        moved = any(p != q for p, q in first.items())
        # one extra tuple (p_min, p_min) per partition of the first join
        extra = list(first.values())
        P2, second = _join(P + extra, R + extra)
        moved = moved or any(p != q for p, q in second.items())
        P = P2[:len(P)]
        if done:
            keep = [i for i, p in enumerate(P) if p not in done]
            for p, r in zip(P, R):
                if p in done:
                    label[r] = p
            P = [P[i] for i in keep]
            R = [R[i] for i in keep]
        if trace is not None:
            parts_at = {}
            for p, r in zip(P, R):
                parts_at.setdefault(r, set()).add(p)
            trace.append({"active": active, "excluded": set(done),
                          "parts_at": {r: frozenset(s) for r, s in parts_at.items()}})
        if not moved:
            break
    for p, r in zip(P, R):
        label[r] = p
    return label, iterations
