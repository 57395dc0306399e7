"""CPU oracle for dynamic SSSP -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference legs may import this package.  The product path (the CUDA
library and its Python binding) never does.  The oracle and the CUDA path
share no code; both consume the seeded inputs of
``paper_2507_11094_gb300.workloads``.

``OracleGraph`` wraps ``oracle.c``: an edge-set model with the paper's batch
order (deletions, then insertions; DynSSSP listing, Section 3) and a
from-scratch binary-heap Dijkstra after every batch (the plain definition of
the distances the method maintains; Section 3 "Example to Illustrate Dynamic
SSSP").  ``invariants.check_sssp`` checks any dist/parent pair against a graph.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

INF = 2147483647 // 2          # INT_MAX/2, the appendix listing's "infinite"
OK, EINVAL, ENOMEM, ERANGE = 0, -1, -2, -3

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-Wall",
                           "-shared", "-fPIC", src, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    lib.or_graph_new.restype = P
    lib.or_graph_new.argtypes = [i32, P, P, P, ctypes.POINTER(ctypes.c_int)]
    lib.or_graph_free.restype = None
    lib.or_graph_free.argtypes = [P]
    lib.or_num_edges.restype = i64
    lib.or_num_edges.argtypes = [P]
    lib.or_export_csr.restype = None
    lib.or_export_csr.argtypes = [P, P, P, P]
    lib.or_apply_batch.restype = ctypes.c_int
    lib.or_apply_batch.argtypes = [P, i64, P, P, i64, P, P, P, P]
    lib.or_dijkstra.restype = ctypes.c_int
    lib.or_dijkstra.argtypes = [P, i32, P]
    f32 = ctypes.c_float
    lib.or_pr_static.restype = ctypes.c_int
    lib.or_pr_static.argtypes = [P, f32, f32, i32, P, P]
    lib.or_tc_static.restype = ctypes.c_int
    lib.or_tc_static.argtypes = [P, P]
    lib.or_pr_batch.restype = ctypes.c_int
    lib.or_pr_batch.argtypes = [P, i64, P, P, i64, P, P, P, f32, f32, i32, P, P]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


class OracleGraph:
    """Edge-set model of a weighted digraph with batch updates and Dijkstra."""

    def __init__(self, n: int, row_off, col, w):
        lib = _load()
        self.n = int(n)
        self._keep = (np.ascontiguousarray(row_off, dtype=np.int64),
                      np.ascontiguousarray(col, dtype=np.int32),
                      np.ascontiguousarray(w, dtype=np.int32))
        if self._keep[0].size != self.n + 1:
            raise OracleError(EINVAL, "row_off size")
        st = ctypes.c_int(0)
        h = lib.or_graph_new(self.n, *(_ptr(a) for a in self._keep),
                             ctypes.byref(st))
        self._keep = None
        if not h:
            raise OracleError(st.value, "or_graph_new")
        self._h = ctypes.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            _load().or_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def m(self) -> int:
        return int(_load().or_num_edges(self._h))

    def csr(self):
        """Current edge set as a row-sorted CSR (row_off, col, w)."""
        m = self.m
        ro = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(m, 1), dtype=np.int32)
        w = np.empty(max(m, 1), dtype=np.int32)
        _load().or_export_csr(self._h, _ptr(ro), _ptr(col), _ptr(w))
        return ro, col[:m], w[:m]

    def apply_batch(self, del_src, del_dst, add_src, add_dst, add_w):
        """Apply deletions then insertions; returns counters
        (del_applied, del_absent, add_applied, add_present)."""
        a = [np.ascontiguousarray(x, dtype=np.int32)
             for x in (del_src, del_dst, add_src, add_dst, add_w)]
        if a[0].size != a[1].size or not (a[2].size == a[3].size == a[4].size):
            raise OracleError(EINVAL, "batch array sizes")
        cnt = np.zeros(4, dtype=np.int64)
        rc = _load().or_apply_batch(self._h, a[0].size, _ptr(a[0]), _ptr(a[1]),
                                    a[2].size, _ptr(a[2]), _ptr(a[3]), _ptr(a[4]),
                                    _ptr(cnt))
        if rc != OK:
            raise OracleError(rc, "or_apply_batch")
        return tuple(int(x) for x in cnt)

    def apply(self, batch):
        """Apply a ``workloads.Batch``."""
        return self.apply_batch(batch.del_src, batch.del_dst, batch.add_src,
                                batch.add_dst, batch.add_w)

    # -- triangle count (appendix listing "Dynamic TC": staticTC) ----------
    def triangles(self) -> int:
        """staticTC on the current edge set (every triangle once on a
        symmetric graph)."""
        c = ctypes.c_int64(0)
        rc = _load().or_tc_static(self._h, ctypes.byref(c))
        if rc != OK:
            raise OracleError(rc, "or_tc_static")
        return int(c.value)

    # -- PageRank (appendix listing "Dynamic PR": staticPR, DynPR) --------
    def pagerank(self, damping=0.85, beta=1e-6, max_iter=100):
        """staticPR: (ranks float32[n], Jacobi steps)."""
        pr = np.empty(self.n, dtype=np.float32)
        it = ctypes.c_int32(0)
        rc = _load().or_pr_static(self._h, float(damping), float(beta), int(max_iter),
                                  _ptr(pr), ctypes.byref(it))
        if rc != OK:
            raise OracleError(rc, "or_pr_static")
        return pr, int(it.value)

    def pagerank_batch(self, batch, pr, damping=0.85, beta=1e-6, max_iter=100):
        """One DynPR batch on ranks ``pr`` (float32[n], updated in place).
        Returns counters: the four batch counters, vertices flagged for the
        deletions and for the insertions, Jacobi steps of each phase."""
        a = [np.ascontiguousarray(x, dtype=np.int32)
             for x in (batch.del_src, batch.del_dst, batch.add_src, batch.add_dst,
                       batch.add_w)]
        assert pr.dtype == np.float32 and pr.flags.c_contiguous and pr.size == self.n
        cnt = np.zeros(8, dtype=np.int64)
        rc = _load().or_pr_batch(self._h, a[0].size, _ptr(a[0]), _ptr(a[1]), a[2].size,
                                 _ptr(a[2]), _ptr(a[3]), _ptr(a[4]), float(damping),
                                 float(beta), int(max_iter), _ptr(pr), _ptr(cnt))
        if rc != OK:
            raise OracleError(rc, "or_pr_batch")
        return tuple(int(x) for x in cnt)

    def dijkstra(self, src: int, allow_range_error: bool = False) -> np.ndarray:
        """Distances from src (int32; INF for unreachable)."""
        dist = np.empty(self.n, dtype=np.int32)
        rc = _load().or_dijkstra(self._h, int(src), _ptr(dist))
        if rc == ERANGE and allow_range_error:
            return dist
        if rc != OK:
            raise OracleError(rc, "or_dijkstra")
        return dist
