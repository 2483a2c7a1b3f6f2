"""Sharding a batch of independent systems over ranks (one GPU per rank).

Independent instances need no exchange: each rank factors and solves its own
share as one block-diagonal batch (wd_analyze_batch), and only timings and
statuses are combined at the end.  Shares are balanced by the factorization
cost of each instance (sum_j c_j^2 from a host-only symbolic analysis) with
the greedy longest-processing-time rule: instances in decreasing cost (ties:
lower index first) each go to the rank with the smallest load so far (ties:
lower rank).  The rule is deterministic, so every rank computes the same
partition without communicating.
"""
from __future__ import annotations

import heapq

import numpy as np

from . import Solver


def lpt_partition(costs, nranks: int) -> list:
    """Indices of the instances of each rank (each list in increasing order)."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(costs.size), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(nranks)]
    heapq.heapify(heap)
    shares = [[] for _ in range(nranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(x) for x in shares]


def instance_costs(patterns, bases=None) -> np.ndarray:
    """Factorization flops (sum_j c_j^2) of every instance from a host-only
    analysis; instances given with the same arrays are analyzed once."""
    cache = {}
    out = np.empty(len(patterns))
    for i, (cp, ri) in enumerate(patterns):
        b = None if bases is None else bases[i]
        key = (id(cp), id(ri), id(b))
        if key not in cache:
            s = Solver(symbolic_only=True).analyze(cp, ri, b)
            cache[key] = s.info()["flops_factor"]
            s.close()
        out[i] = cache[key]
    return out


def local_share(patterns, bases, rank: int, nranks: int, costs=None):
    """(indices, patterns, bases) of this rank's instances."""
    costs = instance_costs(patterns, bases) if costs is None else costs
    idx = lpt_partition(costs, nranks)[rank]
    return idx, [patterns[i] for i in idx], (None if bases is None else [bases[i] for i in idx])
