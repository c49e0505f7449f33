"""Graph shards of the batched form across GPUs, one process per GPU.

The graphs of a batch are independent units: no pair joins two graphs, so
N GPUs label a batch with no exchange at all, each its own graphs through
cc_labels_batched. The shards balance the work with the longest-processing-
time-first rule (Graham, "Bounds on multiprocessing timing anomalies", 1969):
graphs in decreasing order of cost, each to the rank with the least cost so
far, which keeps the largest shard within 4/3 - 1/(3N) of the best possible.
A graph costs its pairs plus its vertices: the hook passes stream the pairs,
the shortcuts and the labels touch the vertices.

Host-side logic only; every rank computes the same shards from the sizes.
"""
from __future__ import annotations

import heapq

import numpy as np


def graph_cost(n_g: np.ndarray, m_g: np.ndarray) -> np.ndarray:
    """Per-graph work estimate: pairs + vertices."""
    return np.asarray(m_g, dtype=np.int64) + np.asarray(n_g, dtype=np.int64)


def lpt_shards(cost, world: int) -> list[np.ndarray]:
    """Graph numbers of each rank (ascending), longest processing time first.

    Ties in cost keep the graph order; ties in load go to the lower rank, so
    every rank computes the same shards."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = np.asarray(cost, dtype=np.int64)
    order = np.argsort(-cost, kind="stable")
    heap = [(0, r) for r in range(world)]
    shards: list[list[int]] = [[] for _ in range(world)]
    for g in order:
        load, r = heapq.heappop(heap)
        shards[r].append(int(g))
        heapq.heappush(heap, (load + int(cost[g]), r))
    return [np.sort(np.asarray(s, dtype=np.int64)) for s in shards]


def shard_loads(cost, shards: list[np.ndarray]) -> list[int]:
    cost = np.asarray(cost, dtype=np.int64)
    return [int(cost[s].sum()) for s in shards]
