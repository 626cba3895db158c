"""Sharding of independent realizations across ranks (one process per GPU).

Realizations never exchange data, so a batch shards with no collective on
the data path: rank r advances its own subset and the host gathers results.
Subsets are balanced by cell count with the longest-processing-time rule
(largest realization first, each to the currently lightest rank), which is
within 4/3 of the optimal makespan (Graham, 1969).
"""
from __future__ import annotations

import heapq


def lpt_partition(sizes, nranks):
    """Indices of `sizes` per rank; deterministic (ties by index, then rank)."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    heap = [(0, r) for r in range(nranks)]
    parts = [[] for _ in range(nranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + sizes[i], r))
    return [sorted(p) for p in parts]


def shard_loads(sizes, parts):
    return [sum(sizes[i] for i in p) for p in parts]
