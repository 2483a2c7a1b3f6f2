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


def subtree_partition(sym: dict, nranks: int, per_rank: int = 2) -> dict:
    """Mapping of one matrix's nested-dissection subtrees to ranks.

    Below the top separators the subtrees of the supernodal elimination tree
    are independent (Section 4: no entry couples V1 and V2), so each rank can
    factor its own; one exchange follows, in which the update matrix of every
    subtree root (its front rows below the pivots) goes to rank 0, which owns
    the separator supernodes above the cut.  `sym` is Solver.symbolic().

    The cut is top-down and deterministic: starting from the roots, the most
    expensive subtree (sum_j c_j^2, ties: the lower supernode) is replaced by
    its children and its own supernode joins the top, until there are
    per_rank * nranks subtrees or none can be split; the subtrees go to ranks
    by lpt_partition.  Returns owner[ns] (the rank of every supernode),
    subtrees [(root, first column, end column, rank, cost)] in increasing root
    order, boundary {root: the rows of its update matrix (permuted indices)}
    and send_entries {root: lower entries of its update matrix}."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    sf = np.asarray(sym["super_first"], dtype=np.int64)
    srp = np.asarray(sym["super_rowptr"], dtype=np.int64)
    srows = np.asarray(sym["super_rows"], dtype=np.int64)
    parent = np.asarray(sym["parent"], dtype=np.int64)
    cc = np.asarray(sym["colcount"], dtype=np.float64)
    ns = sf.size - 1
    n = int(sf[-1])
    snode = np.repeat(np.arange(ns), np.diff(sf))
    spar = np.full(ns, -1, dtype=np.int64)
    for s in range(ns):
        p = parent[sf[s + 1] - 1]
        if p >= 0:
            spar[s] = snode[p]
    children = [[] for _ in range(ns)]
    for s in range(ns):
        if spar[s] >= 0:
            children[spar[s]].append(s)
    own = np.add.reduceat(cc ** 2, sf[:-1]) if n > 0 else np.zeros(0)
    cost = own.copy()
    lo = sf[:-1].copy()
    for s in range(ns):                       # children precede parents
        if spar[s] >= 0:
            cost[spar[s]] += cost[s]
            lo[spar[s]] = min(lo[spar[s]], lo[s])
    heap = [(-cost[s], s) for s in range(ns) if spar[s] < 0]
    heapq.heapify(heap)
    final = []
    while heap and len(heap) + len(final) < per_rank * nranks:
        c, s = heapq.heappop(heap)
        if not children[s]:
            final.append(s)
            continue
        for ch in children[s]:
            heapq.heappush(heap, (-cost[ch], ch))
    roots = sorted(final + [s for _, s in heap])
    shares = lpt_partition([cost[r] for r in roots], nranks)
    rank_of = {}
    for r, idx in enumerate(shares):
        for i in idx:
            rank_of[roots[i]] = r
    owner = np.zeros(ns, dtype=np.int32)
    subtrees, boundary, send = [], {}, {}
    for root in roots:
        c0, c1 = int(lo[root]), int(sf[root + 1])
        owner[snode[c0:c1]] = rank_of[root]
        k = int(sf[root + 1] - sf[root])
        rows = srows[srp[root] + k: srp[root + 1]]
        boundary[root] = rows
        send[root] = rows.size * (rows.size + 1) // 2
        subtrees.append((root, c0, c1, rank_of[root], float(cost[root])))
    return {"owner": owner, "subtrees": subtrees, "boundary": boundary, "send_entries": send}
