"""Seeded synthetic inputs for dynamic SSSP: graphs and update batches.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds input generation only -- graph shapes, weights and
the choice of which edges a batch deletes or inserts -- and none of the
shortest-path arithmetic: no relaxation, no distance computation, no CSR
merge.  Everything is numpy with explicit seeds (PCG64), so x86 and Arm hosts
produce identical inputs.

Workload shapes follow the paper's evaluation (Section 6, Table "Input
graphs"): an R-MAT graph with a=0.57, b=0.19, c=0.19, d=0.05 stands in for
the skewed social graphs and RM; a 2-D 4-neighbour grid stands in for the
high-diameter road graphs US and GR; an Erdos-Renyi digraph stands in for UR.
Updates are random edge deletions and insertions applied as one batch whose
size is a percentage of |E| (Section 6, experimental setup).  Edge weights
are integers (``propEdge<int>`` in the dynamic SSSP listing of Section 3).

Graphs are returned as CSR with each row sorted by destination:
``row_off`` int64[n+1], ``col`` int32[m], ``w`` int32[m].
"""
from __future__ import annotations

import dataclasses

import numpy as np

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------

def _csr_from_keys(n: int, keys: np.ndarray, w: np.ndarray):
    """Build a row-sorted CSR from unique edge keys ``u*n+v`` (sorted)."""
    keys = np.asarray(keys, dtype=np.int64)
    u = keys // n
    v = (keys % n).astype(np.int32)
    counts = np.bincount(u, minlength=n).astype(np.int64)
    row_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_off[1:])
    return row_off, v, np.asarray(w, dtype=np.int32)


def csr_keys(n: int, row_off: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Edge keys ``u*n+v`` (int64) of a CSR, in CSR order."""
    deg = np.diff(row_off)
    u = np.repeat(np.arange(n, dtype=np.int64), deg)
    return u * n + col.astype(np.int64)


def _first_unique_in_order(keys: np.ndarray) -> np.ndarray:
    """Keys with duplicates removed, keeping first occurrences in input order."""
    _, idx = np.unique(keys, return_index=True)
    idx.sort()
    return keys[idx]


def max_out_degree_source(row_off: np.ndarray) -> int:
    """Vertex with the largest out-degree, smallest id on ties."""
    return int(np.argmax(np.diff(row_off)))


# --------------------------------------------------------------------------
# graph generators
# --------------------------------------------------------------------------

def er_digraph(n: int, m: int, wlo: int, whi: int, seed: int):
    """Erdos-Renyi digraph with exactly m edges: uniform (u, v), u != v, no
    duplicates; weights uniform in [wlo, whi]."""
    if m > n * (n - 1):
        raise ValueError("too many edges for a simple digraph")
    rng = np.random.default_rng(seed)
    keys = np.empty(0, dtype=np.int64)
    while keys.size < m:
        need = m - keys.size
        k = int(need * 1.2) + 16
        u = rng.integers(0, n, size=k, dtype=np.int64)
        v = rng.integers(0, n, size=k, dtype=np.int64)
        cand = u * n + v
        cand = cand[u != v]
        keys = _first_unique_in_order(np.concatenate([keys, cand]))
    keys = np.sort(keys[:m])
    w = rng.integers(wlo, whi + 1, size=m, dtype=np.int64).astype(np.int32)
    return _csr_from_keys(n, keys, w)


def _rmat_pairs(rng, scale: int, count: int, abcd=RMAT_ABCD):
    """Draw ``count`` R-MAT (u, v) pairs on 2**scale vertices (no noise)."""
    a, b, c, _ = abcd
    u = np.zeros(count, dtype=np.int64)
    v = np.zeros(count, dtype=np.int64)
    for _level in range(scale):
        r = rng.random(count)
        ubit = r >= (a + b)                        # quadrants c, d: lower half
        vbit = ((r >= a) & (r < a + b)) | (r >= a + b + c)   # quadrants b, d
        u = (u << 1) | ubit
        v = (v << 1) | vbit
    return u, v


@dataclasses.dataclass
class RmatSampler:
    """R-MAT edge sampler with a fixed random vertex relabelling."""
    scale: int
    perm: np.ndarray
    abcd: tuple = RMAT_ABCD

    def draw(self, rng, count: int):
        u, v = _rmat_pairs(rng, self.scale, count, self.abcd)
        return self.perm[u], self.perm[v]


def rmat_digraph(scale: int, m: int, wlo: int, whi: int, seed: int,
                 abcd=RMAT_ABCD):
    """R-MAT digraph on n = 2**scale vertices with exactly m unique edges.

    Self-loops and duplicates are dropped and pairs are redrawn until m unique
    edges exist (first occurrences in draw order are kept).  A seeded random
    relabelling of the vertices is applied, as Graph500 does.  Returns
    ``(row_off, col, w, sampler)``; the sampler draws further edges from the
    same distribution and labelling (used for insertions).
    """
    n = 1 << scale
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n).astype(np.int64)
    sampler = RmatSampler(scale, perm, abcd)
    keys = np.empty(0, dtype=np.int64)
    while keys.size < m:
        need = m - keys.size
        k = int(need * 1.3) + 1024
        u, v = sampler.draw(rng, k)
        cand = u * n + v
        cand = cand[u != v]
        keys = _first_unique_in_order(np.concatenate([keys, cand]))
    keys = np.sort(keys[:m])
    w = rng.integers(wlo, whi + 1, size=m, dtype=np.int64).astype(np.int32)
    row_off, col, w = _csr_from_keys(n, keys, w)
    return row_off, col, w, sampler


def grid_digraph(rows: int, cols: int, wlo: int, whi: int, seed: int):
    """4-neighbour grid, both directions as two directed edges with
    independent weights uniform in [wlo, whi].  Vertex (i, j) is i*cols+j."""
    n = rows * cols
    i, j = np.divmod(np.arange(n, dtype=np.int64), cols)
    us, vs = [], []
    for di, dj in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        ok = (i + di >= 0) & (i + di < rows) & (j + dj >= 0) & (j + dj < cols)
        us.append(np.nonzero(ok)[0])
        vs.append((i[ok] + di) * cols + (j[ok] + dj))
    keys = np.sort(np.concatenate(us) * n + np.concatenate(vs))
    rng = np.random.default_rng(seed)
    w = rng.integers(wlo, whi + 1, size=keys.size, dtype=np.int64).astype(np.int32)
    return _csr_from_keys(n, keys, w)


# --------------------------------------------------------------------------
# update batches
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Batch:
    """One update batch: deletions (del_src, del_dst) and insertions
    (add_src, add_dst, add_w), all int32 arrays."""
    del_src: np.ndarray
    del_dst: np.ndarray
    add_src: np.ndarray
    add_dst: np.ndarray
    add_w: np.ndarray

    @property
    def size(self) -> int:
        return int(self.del_src.size + self.add_src.size)

    @staticmethod
    def empty() -> "Batch":
        z = np.zeros(0, dtype=np.int32)
        return Batch(z, z.copy(), z.copy(), z.copy(), z.copy())


class BatchStream:
    """Draws update batches against the evolving edge set of one graph.

    The stream keeps the current edge keys (sorted) and weights so that every
    deletion names an existing edge and every insertion a non-edge; a batch
    never deletes and inserts the same edge and never repeats an edge.  This
    bookkeeping is input generation: it decides which updates to issue, and
    shares no code with the method under test or with the oracle.

    ``insert_kind``:
      * ``"uniform"``  -- uniform pairs u != v;
      * ``"rmat"``     -- pairs from ``sampler`` (R-MAT, same labelling);
      * ``"local5"``   -- a uniform vertex of a ``rows x cols`` grid joined to
        a uniform vertex of its 5x5 neighbourhood (local shortcuts that keep
        the diameter high).
    """

    def __init__(self, n, row_off, col, w, wlo, whi, insert_kind="uniform",
                 sampler=None, grid_shape=None):
        self.n = int(n)
        self.keys = csr_keys(self.n, row_off, col)
        order = np.argsort(self.keys, kind="stable")
        self.keys = self.keys[order]
        self.wts = np.asarray(w, dtype=np.int32)[order]
        self.wlo, self.whi = int(wlo), int(whi)
        self.insert_kind = insert_kind
        self.sampler = sampler
        self.grid_shape = grid_shape

    @property
    def m(self) -> int:
        return int(self.keys.size)

    def _draw_pairs(self, rng, k):
        n = self.n
        if self.insert_kind == "uniform":
            u = rng.integers(0, n, size=k, dtype=np.int64)
            v = rng.integers(0, n, size=k, dtype=np.int64)
        elif self.insert_kind == "rmat":
            u, v = self.sampler.draw(rng, k)
        elif self.insert_kind == "local5":
            rows, cols = self.grid_shape
            u = rng.integers(0, n, size=k, dtype=np.int64)
            ui, uj = np.divmod(u, cols)
            di = rng.integers(-2, 3, size=k, dtype=np.int64)
            dj = rng.integers(-2, 3, size=k, dtype=np.int64)
            vi = np.clip(ui + di, 0, rows - 1)
            vj = np.clip(uj + dj, 0, cols - 1)
            v = vi * cols + vj
        else:
            raise ValueError(self.insert_kind)
        return u, v

    def _pick_deletions(self, rng, n_del, dist=None, tree_fraction=0.0):
        m = self.m
        if n_del > m:
            raise ValueError("more deletions than edges")
        if dist is None or tree_fraction <= 0.0:
            return rng.choice(m, size=n_del, replace=False)
        # Deletions biased toward shortest-path-tree edges: an edge u->v is
        # taken as a tree edge when it is tight for the given distances.
        n = self.n
        u = self.keys // n
        v = self.keys % n
        du = dist[u].astype(np.int64)
        dv = dist[v].astype(np.int64)
        tight = (du + self.wts == dv)
        tidx = np.nonzero(tight)[0]
        oidx = np.nonzero(~tight)[0]
        n_tree = min(int(round(n_del * tree_fraction)), tidx.size)
        n_other = n_del - n_tree
        a = rng.choice(tidx, size=n_tree, replace=False) if n_tree else tidx[:0]
        b = rng.choice(oidx, size=n_other, replace=False) if n_other else oidx[:0]
        return np.concatenate([a, b])

    def next(self, n_del: int, n_add: int, seed: int, dist=None,
             tree_fraction=0.0) -> Batch:
        """Draw the next batch and advance the edge set past it."""
        rng = np.random.default_rng(seed)
        n = self.n
        di = self._pick_deletions(rng, n_del, dist, tree_fraction)
        dkeys = self.keys[di]
        # insertions: fresh non-edges, distinct, not deleted in this batch
        chosen = np.empty(0, dtype=np.int64)
        tries = 0
        while chosen.size < n_add:
            tries += 1
            if tries > 64:
                raise RuntimeError("could not draw enough new edges")
            k = int((n_add - chosen.size) * 1.5) + 64
            u, v = self._draw_pairs(rng, k)
            cand = u * n + v
            cand = cand[u != v]
            pos = np.searchsorted(self.keys, cand)
            pos = np.minimum(pos, max(self.keys.size - 1, 0))
            present = (self.keys.size > 0) & (self.keys[pos] == cand)
            cand = cand[~present]
            cand = cand[~np.isin(cand, dkeys)]
            chosen = _first_unique_in_order(np.concatenate([chosen, cand]))
        akeys = chosen[:n_add]
        aw = rng.integers(self.wlo, self.whi + 1, size=n_add,
                          dtype=np.int64).astype(np.int32)
        batch = Batch(
            del_src=(dkeys // n).astype(np.int32),
            del_dst=(dkeys % n).astype(np.int32),
            add_src=(akeys // n).astype(np.int32),
            add_dst=(akeys % n).astype(np.int32),
            add_w=aw,
        )
        # advance the edge set
        keep = np.ones(self.keys.size, dtype=bool)
        keep[di] = False
        keys = self.keys[keep]
        wts = self.wts[keep]
        order = np.argsort(akeys, kind="stable")
        ak, aww = akeys[order], aw[order]
        pos = np.searchsorted(keys, ak)
        self.keys = np.insert(keys, pos, ak)
        self.wts = np.insert(wts, pos, aww)
        return batch

    def csr(self):
        """The current edge set as a row-sorted CSR."""
        return _csr_from_keys(self.n, self.keys, self.wts)


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    n: int
    row_off: np.ndarray
    col: np.ndarray
    w: np.ndarray
    source: int
    stream: BatchStream
    batch_edges: int          # total updates per batch (half del, half add)
    graph_seed: int
    tree_fraction: float = 0.0

    @property
    def m(self) -> int:
        return int(self.col.size)

    def batch(self, k: int, dist=None) -> Batch:
        """Batch k (seed graph_seed*1000+k) drawn against the current edges."""
        n_del = self.batch_edges // 2
        n_add = self.batch_edges - n_del
        return self.stream.next(n_del, n_add, seed=self.graph_seed * 1000 + k,
                                dist=dist, tree_fraction=self.tree_fraction)


def tiny_er(seed: int = 1) -> Workload:
    """ER digraph, n=1,024, m=8,192, w~U[1,100], source 0; batches of 64
    updates (32 deletions of existing edges + 32 new edges, w~U[1,100])."""
    n, m = 1024, 8192
    row_off, col, w = er_digraph(n, m, 1, 100, seed)
    st = BatchStream(n, row_off, col, w, 1, 100, "uniform")
    return Workload("er-1k-8k", n, row_off, col, w, 0, st, 64, seed)


def rmat(scale: int = 20, edge_factor: int = 16, batch_frac: float = 0.01,
         seed: int = 1, m: int | None = None) -> Workload:
    """R-MAT scale ``scale`` (a=.57 b=.19 c=.19 d=.05), m = edge_factor*n
    unique edges, w~U[1,100], source = max out-degree vertex; batches of
    batch_frac*m updates, half deletions (uniform over current edges) and
    half insertions drawn from the same R-MAT distribution."""
    n = 1 << scale
    m = edge_factor * n if m is None else m
    row_off, col, w, sampler = rmat_digraph(scale, m, 1, 100, seed)
    st = BatchStream(n, row_off, col, w, 1, 100, "rmat", sampler=sampler)
    src = max_out_degree_source(row_off)
    b = max(2, int(round(batch_frac * m)))
    return Workload(f"rmat{scale}-ef{edge_factor}", n, row_off, col, w, src,
                    st, b, seed)


def grid(rows: int = 4096, cols: int = 4096, batch_frac: float = 0.01,
         seed: int = 1, insert_kind: str = "local5",
         tree_fraction: float = 0.5) -> Workload:
    """rows x cols 4-neighbour grid, both directions with independent
    weights w~U[1,1000], source at corner (0,0); batches of batch_frac*m
    updates, half deletions (tree_fraction of them on shortest-path-tree
    edges) and half insertions (local 5x5 shortcuts by default)."""
    n = rows * cols
    row_off, col, w = grid_digraph(rows, cols, 1, 1000, seed)
    st = BatchStream(n, row_off, col, w, 1, 1000, insert_kind,
                     grid_shape=(rows, cols))
    b = max(2, int(round(batch_frac * col.size)))
    name = f"grid{rows}x{cols}" + ("" if insert_kind == "local5" else f"-{insert_kind}")
    return Workload(name, n, row_off, col, w, 0, st, b, seed, tree_fraction=tree_fraction)


# --------------------------------------------------------------------------
# symmetric (undirected) graphs for the triangle count
# --------------------------------------------------------------------------

def symmetrize(n: int, row_off: np.ndarray, col: np.ndarray, w: np.ndarray):
    """Every edge in both directions; a pair stored twice keeps the weight of
    its (min, max) orientation, else of the one edge given.  Self-loops are
    dropped."""
    u = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_off))
    v = col.astype(np.int64)
    keep = u != v
    u, v, ww = u[keep], v[keep], np.asarray(w)[keep]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    key = lo * n + hi
    order = np.lexsort((u > v, key))        # the (min, max) orientation first
    key, ww = key[order], ww[order]
    first = np.ones(key.size, bool)
    first[1:] = key[1:] != key[:-1]
    key, ww = key[first], ww[first]
    a, b = key // n, key % n
    both = np.concatenate([a * n + b, b * n + a])
    wb = np.concatenate([ww, ww])
    order = np.argsort(both, kind="stable")
    return _csr_from_keys(n, both[order], wb[order])


class UndirectedStream:
    """Update batches of a symmetric graph: every deleted or inserted pair
    {u, v} appears as both u -> v and v -> u, deletions name present pairs,
    insertions absent ones, and no pair appears twice in a batch."""

    def __init__(self, n, row_off, col, w, wlo, whi, sampler=None):
        self.n = int(n)
        keys = csr_keys(self.n, row_off, col)
        u, v = keys // self.n, keys % self.n
        sel = u < v
        self.keys = np.sort(keys[sel])                 # pairs as u * n + v, u < v
        order = np.argsort(keys[sel], kind="stable")
        self.wts = np.asarray(w, np.int32)[sel][order]
        self.wlo, self.whi = int(wlo), int(whi)
        self.sampler = sampler

    def next(self, n_del: int, n_add: int, seed: int, **_ignored) -> Batch:
        """n_del / n_add directed updates, i.e. n_del // 2 and n_add // 2
        pairs."""
        rng = np.random.default_rng(seed)
        n = self.n
        n_del, n_add = n_del // 2, n_add // 2
        di = rng.choice(self.keys.size, size=n_del, replace=False)
        dkeys = self.keys[di]
        chosen = np.empty(0, np.int64)
        for _ in range(64):
            if chosen.size >= n_add:
                break
            k = int((n_add - chosen.size) * 1.5) + 64
            if self.sampler is not None:
                a, b = self.sampler.draw(rng, k)
            else:
                a = rng.integers(0, n, size=k, dtype=np.int64)
                b = rng.integers(0, n, size=k, dtype=np.int64)
            lo, hi = np.minimum(a, b), np.maximum(a, b)
            cand = (lo * n + hi)[lo != hi]
            pos = np.minimum(np.searchsorted(self.keys, cand), max(self.keys.size - 1, 0))
            cand = cand[~((self.keys.size > 0) & (self.keys[pos] == cand))]
            cand = cand[~np.isin(cand, dkeys)]
            chosen = _first_unique_in_order(np.concatenate([chosen, cand]))
        if chosen.size < n_add:
            raise RuntimeError("could not draw enough new pairs")
        akeys = chosen[:n_add]
        aw = rng.integers(self.wlo, self.whi + 1, size=n_add, dtype=np.int64).astype(np.int32)
        du, dv = dkeys // n, dkeys % n
        au, av = akeys // n, akeys % n
        batch = Batch(
            del_src=np.concatenate([du, dv]).astype(np.int32),
            del_dst=np.concatenate([dv, du]).astype(np.int32),
            add_src=np.concatenate([au, av]).astype(np.int32),
            add_dst=np.concatenate([av, au]).astype(np.int32),
            add_w=np.concatenate([aw, aw]),
        )
        keep = np.ones(self.keys.size, bool)
        keep[di] = False
        keys, wts = self.keys[keep], self.wts[keep]
        order = np.argsort(akeys, kind="stable")
        pos = np.searchsorted(keys, akeys[order])
        self.keys = np.insert(keys, pos, akeys[order])
        self.wts = np.insert(wts, pos, aw[order])
        return batch


def sym_er(n: int = 1024, pairs: int = 4096, batch_pairs: int = 32, seed: int = 1):
    """Symmetric ER graph: `pairs` random unordered pairs, both directions,
    w~U[1,100]; batches of batch_pairs deleted + batch_pairs new pairs."""
    ro, col, w = er_digraph(n, pairs, 1, 100, seed)
    ro, col, w = symmetrize(n, ro, col, w)
    st = UndirectedStream(n, ro, col, w, 1, 100)
    return Workload(f"sym-er{n}", n, ro, col, w, 0, st, 4 * batch_pairs, seed)


def sym_rmat(scale: int = 16, edge_factor: int = 8, batch_frac: float = 0.01, seed: int = 1):
    """Symmetric R-MAT: edge_factor * n R-MAT edges (a=.57 b=.19 c=.19
    d=.05) stored in both directions; batches of batch_frac of the pairs
    deleted and as many new R-MAT pairs inserted, both directions."""
    n = 1 << scale
    ro, col, w, sampler = rmat_digraph(scale, edge_factor * n, 1, 100, seed)
    ro, col, w = symmetrize(n, ro, col, w)
    st = UndirectedStream(n, ro, col, w, 1, 100, sampler=sampler)
    pairs = col.size // 2
    b = max(1, int(round(batch_frac * pairs)))
    return Workload(f"sym-rmat{scale}-ef{edge_factor}", n, ro, col, w,
                    max_out_degree_source(ro), st, 4 * b, seed)


# --------------------------------------------- batched and serving workloads

def batched_rmat(seed: int, k: int = 64):
    """The batched form: k R-MAT graphs, scales ~U{12..18}, edge factor 16,
    w~U[1,100], each with its own source (max out-degree) and its own batch
    of ~U[0.5%, 5%] of its m (50/50)."""
    rng = np.random.default_rng(seed)
    scales = rng.integers(12, 19, size=k)
    fracs = rng.uniform(0.005, 0.05, size=k)
    return [rmat(scale=int(sc), batch_frac=float(fr), seed=seed * 100 + i)
            for i, (sc, fr) in enumerate(zip(scales, fracs))]


def serving_graphs(seed: int, big_scale: int = 22):
    """The serving form's graphs: 2 R-MAT graphs of scale big_scale + 6 of
    scale ~U{16..20}, edge factor 16, w~U[1,100], each with its own source
    (max out-degree vertex)."""
    rng = np.random.default_rng(seed)
    scales = [big_scale, big_scale] + [int(x) for x in rng.integers(16, 21, size=6)]
    return [rmat(scale=sc, batch_frac=0.001, seed=seed * 100 + 50 + i)
            for i, sc in enumerate(scales)]


def serving_requests(ws, count: int, seed: int):
    """`count` batches: graph uniform over ws, size log-uniform in [1e3, 1e6]
    (at most half the graph's edges), 50/50 deletions/insertions; a query of
    1024 random vertices of the same graph after every 4th batch.  Returns
    (graph index, Batch, query vertices or None) triples; the graphs' batch
    streams advance as the batches are drawn."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        gi = int(rng.integers(0, len(ws)))
        W = ws[gi]
        size = int(np.exp(rng.uniform(np.log(1e3), np.log(1e6))))
        size = max(2, min(size, W.m // 2))
        b = W.stream.next(size // 2, size - size // 2, seed=seed * 100000 + i)
        q = (rng.integers(0, W.n, size=1024).astype(np.int32) if i % 4 == 3 else None)
        reqs.append((gi, b, q))
    return reqs
