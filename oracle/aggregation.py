"""Deterministic greedy aggregation of a cell graph (oracle; test only).

The paper partitions the cell graph G_T into connected, non-overlapping aggregates with METIS and applies this
recursively (Sec. 3.1, App. A.1); a coarse edge joins two aggregates when some fine edge joins their cells. METIS is
replaced by the following rule, which is reproducible bit for bit (the CUDA library implements it separately):

  1. Visit vertices in increasing index. Each vertex not yet aggregated seeds a new aggregate (ids 0, 1, ...).
  2. Grow it breadth first: pop vertices from a FIFO queue (starting with the seed) and take their unaggregated
     neighbours in increasing index, one at a time, until the aggregate holds `target` vertices or the queue is
     empty.
  3. Visit aggregate ids in increasing order. An aggregate whose current size s satisfies 2 s < target is merged
     into the adjacent aggregate that shares the most edges with it (ties: the smallest id); an aggregate without
     neighbours is kept.
  4. Renumber the surviving aggregates 0, 1, ... in increasing order of their id.
Aggregates stay connected: step 2 grows connected sets and step 3 only joins sets that share an edge.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def adjacency(n, edges):
    """Sorted, duplicate-free neighbour lists from an (E, 2) edge array."""
    nb = [set() for _ in range(n)]
    for u, v in np.asarray(edges).reshape(-1, 2):
        u, v = int(u), int(v)
        if u != v:
            nb[u].add(v)
            nb[v].add(u)
    return [sorted(s) for s in nb]


def aggregate(n, nbrs, target):
    """Return agg_of[n] (int64) following the four rules above."""
    agg = np.full(n, -1, dtype=np.int64)
    nagg = 0
    for s in range(n):
        if agg[s] != -1:
            continue
        aid = nagg
        nagg += 1
        agg[s] = aid
        count = 1
        q = deque([s])
        while q and count < target:
            v = q.popleft()
            for u in nbrs[v]:
                if count >= target:
                    break
                if agg[u] == -1:
                    agg[u] = aid
                    count += 1
                    q.append(u)
    # edge multiplicities between aggregates are recomputed on the current labels at each merge
    for aid in range(nagg):
        members = np.where(agg == aid)[0]
        if members.size == 0 or 2 * members.size >= target:
            continue
        shared = {}
        for v in members:
            for u in nbrs[v]:
                b = int(agg[u])
                if b != aid:
                    shared[b] = shared.get(b, 0) + 1
        if not shared:
            continue
        best = min(shared.items(), key=lambda kv: (-kv[1], kv[0]))[0]
        agg[members] = best
    ids = np.unique(agg)
    remap = np.full(nagg, -1, dtype=np.int64)
    remap[ids] = np.arange(ids.size)
    return remap[agg]


def coarse_edges(agg_of, nbrs):
    """Sorted list of (a, b), a < b, for every pair of aggregates joined by at least one fine edge."""
    out = set()
    for v, nb in enumerate(nbrs):
        a = int(agg_of[v])
        for u in nb:
            b = int(agg_of[u])
            if a != b:
                out.add((min(a, b), max(a, b)))
    return sorted(out)
