"""Batched form: many independent graphs in one handle.

The graphs are packed as a disjoint union -- graph i's vertex v becomes
offset[i] + v -- and initialised with one source per graph
(sp_sssp_init_multi), so every component holds exactly its own
single-source distances.  A round of per-graph update batches becomes one
union batch, applied by the same kernels in one pass (one persistent launch
per loop for all graphs), optionally replayed from a captured CUDA graph.
This module only marshals arrays (offsets, concatenation, slicing); all
computation runs in libsp's kernels.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import sp


@dataclasses.dataclass
class Packed:
    n: int
    row_off: np.ndarray
    col: np.ndarray
    w: np.ndarray
    offsets: np.ndarray      # [k+1] vertex offsets
    sources: np.ndarray      # [k] union ids


def pack_graphs(graphs, sources) -> Packed:
    """graphs: list of (n_i, row_off_i, col_i, w_i); sources: per-graph ids."""
    ns = np.array([g[0] for g in graphs], dtype=np.int64)
    offsets = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(ns, out=offsets[1:])
    n = int(offsets[-1])
    if n >= 2 ** 31:
        raise ValueError("union too large")
    ms = [int(g[2].size) for g in graphs]
    eoff = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    row_off = np.empty(n + 1, dtype=np.int64)
    col = np.empty(int(eoff[-1]), dtype=np.int32)
    w = np.empty(int(eoff[-1]), dtype=np.int32)
    for i, (ni, ro, c, ww) in enumerate(graphs):
        row_off[offsets[i]:offsets[i] + ni] = np.asarray(ro[:-1], np.int64) + eoff[i]
        col[eoff[i]:eoff[i + 1]] = np.asarray(c, np.int64) + offsets[i]
        w[eoff[i]:eoff[i + 1]] = ww
    row_off[n] = eoff[-1]
    src = np.array(sources, dtype=np.int64) + offsets[:-1]
    return Packed(n, row_off, col, w, offsets, src.astype(np.int32))


def pack_batches(packed: Packed, batches):
    """Per-graph batches (workloads.Batch-like) -> one union batch of int32
    arrays (del_src, del_dst, add_src, add_dst, add_w)."""
    off = packed.offsets
    cat = lambda f, shift: np.concatenate(
        [np.asarray(getattr(b, f), np.int64) + (off[i] if shift else 0)
         for i, b in enumerate(batches)]).astype(np.int32)
    return (cat("del_src", True), cat("del_dst", True), cat("add_src", True),
            cat("add_dst", True), cat("add_w", False))


class BatchedGraphs:
    """k graphs in one libsp handle."""

    def __init__(self, graphs, sources, slack: float = 0.25, stream=None):
        self.packed = pack_graphs(graphs, sources)
        p = self.packed
        self.g = sp.Graph(p.n, p.row_off, p.col, p.w, slack=slack, stream=stream)
        self.k = len(graphs)

    def init(self, stats: bool = False):
        return self.g.sssp_init_multi(self.packed.sources, stats=stats)

    def apply(self, batches, stats: bool = False):
        return self.g.apply_batch(*pack_batches(self.packed, batches), stats=stats)

    def dist(self, i: int | None = None):
        d = self.g.get_dist()
        off = self.packed.offsets
        if i is not None:
            return d[off[i]:off[i + 1]]
        return [d[off[j]:off[j + 1]] for j in range(self.k)]

    def close(self):
        self.g.close()
