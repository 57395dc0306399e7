"""Shortest-path-tree invariants -- TEST INFRASTRUCTURE ONLY.

Several parent arrays are correct for one graph (ties), so parents are checked
by the properties every correct answer has rather than by equality.  For
distances from ``src`` in a digraph with weights w >= 1 (the dynamic SSSP
listings of the paper's Appendix "SSSP" store dist and parent per vertex, and
unreachable vertices keep INT_MAX/2 and parent -1):

1. dist[src] == 0 and parent[src] == -1;
2. every edge u->v with dist[u] finite satisfies dist[v] <= dist[u] + w
   (no edge can still be relaxed -- the fixedPoint of the Incremental listing);
3. every finite dist[v], v != src, is realised by its parent edge:
   p = parent[v] names an existing edge p->v with dist[p] + w(p,v) == dist[v];
4. an unreachable vertex (dist == INT_MAX/2) has parent -1.

With w >= 1, property 3 makes dist strictly increase along parent edges, so
parent pointers form a tree rooted at src (no cycles) and 1-3 together imply
dist is exactly the shortest-path distance.
"""
from __future__ import annotations

import numpy as np

INF = 2147483647 // 2


class InvariantError(AssertionError):
    pass


def _edge_arrays(n, row_off, col, w):
    deg = np.diff(np.asarray(row_off, dtype=np.int64))
    u = np.repeat(np.arange(n, dtype=np.int64), deg)
    return u, np.asarray(col, dtype=np.int64), np.asarray(w, dtype=np.int64)


def check_sssp(n, row_off, col, w, src, dist, parent=None):
    """Raise InvariantError naming the first violated property."""
    dist = np.asarray(dist, dtype=np.int64)
    if dist.shape != (n,):
        raise InvariantError("dist has the wrong shape")
    if dist[src] != 0:
        raise InvariantError(f"dist[src]={dist[src]} != 0")
    if np.any(dist < 0) or np.any(dist > INF):
        raise InvariantError("dist outside [0, INF]")
    u, v, wt = _edge_arrays(n, row_off, col, w)
    fin = dist[u] < INF
    bad = fin & (dist[v] > dist[u] + wt)
    if np.any(bad):
        i = int(np.nonzero(bad)[0][0])
        raise InvariantError(
            f"edge {u[i]}->{v[i]} (w={wt[i]}) relaxable: "
            f"dist {dist[u[i]]} + {wt[i]} < {dist[v[i]]}")
    if parent is None:
        return
    parent = np.asarray(parent, dtype=np.int64)
    if parent[src] != -1:
        raise InvariantError(f"parent[src]={parent[src]} != -1")
    unreach = dist >= INF
    if np.any(parent[unreach] != -1):
        raise InvariantError("unreachable vertex with a parent")
    reach = np.nonzero(~unreach)[0]
    reach = reach[reach != src]
    p = parent[reach]
    if np.any((p < 0) | (p >= n)):
        i = int(np.nonzero((p < 0) | (p >= n))[0][0])
        raise InvariantError(f"vertex {reach[i]} has parent {p[i]} out of range")
    # look up each parent edge p->v in the sorted edge keys
    keys = u * n + v
    order = np.argsort(keys, kind="stable")
    skeys, sw = keys[order], wt[order]
    q = p * n + reach
    pos = np.searchsorted(skeys, q)
    pos_c = np.minimum(pos, max(skeys.size - 1, 0))
    exists = (skeys.size > 0) & (skeys[pos_c] == q)
    if not np.all(exists):
        i = int(np.nonzero(~exists)[0][0])
        raise InvariantError(f"parent edge {p[i]}->{reach[i]} does not exist")
    tight = dist[p] + sw[pos_c] == dist[reach]
    if not np.all(tight):
        i = int(np.nonzero(~tight)[0][0])
        raise InvariantError(
            f"parent edge {p[i]}->{reach[i]} not tight: "
            f"{dist[p[i]]} + {sw[pos_c[i]]} != {dist[reach[i]]}")
