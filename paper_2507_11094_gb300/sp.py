"""ctypes binding of libsp (include/sp.h): argument marshalling only.

Every step of the computation runs in libsp's CUDA kernels.  PyTorch supplies
device memory (its caching allocator, passed as an sp_allocator) and the CUDA
stream.  Arrays may be numpy (host) or CUDA torch tensors (device); the
matching ``*_on_device`` flag is set from the array type.  There is no CPU
fallback: if libsp.so is missing or CUDA is unavailable, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SP_INF = 1073741823
SP_WMAX = 1 << 20
SP_NPHASE = 8
PHASES = ("sort", "count", "merge", "inval", "pull", "add", "push", "finish")

STATUS = {0: "SP_OK", -1: "SP_EINVAL", -2: "SP_ENOMEM", -3: "SP_ERANGE",
          -4: "SP_ESTATE", -5: "SP_ECUDA", -6: "SP_ETIMEOUT",
          -7: "SP_ENOMEM_BUDGET"}
SP_OK, SP_EINVAL, SP_ENOMEM, SP_ERANGE = 0, -1, -2, -3
SP_ESTATE, SP_ECUDA, SP_ETIMEOUT, SP_ENOMEM_BUDGET = -4, -5, -6, -7


class SpError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class BatchStats(ctypes.Structure):
    _fields_ = [
        ("n_del_applied", ctypes.c_int64), ("n_del_absent", ctypes.c_int64),
        ("n_add_applied", ctypes.c_int64), ("n_add_present", ctypes.c_int64),
        ("affected", ctypes.c_int64), ("seeds", ctypes.c_int64),
        ("relaxed_edges", ctypes.c_int64), ("improved", ctypes.c_int64),
        ("rows_touched", ctypes.c_int64), ("rows_relocated", ctypes.c_int64),
        ("rounds_inval", ctypes.c_int32), ("rounds_push", ctypes.c_int32),
        ("n_launches", ctypes.c_int32), ("regrows", ctypes.c_int32),
        ("alg_bytes", ctypes.c_int64 * SP_NPHASE),
        ("ms_phase", ctypes.c_float * SP_NPHASE),
        ("ms_total", ctypes.c_float),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_
             if k not in ("alg_bytes", "ms_phase")}
        d["alg_bytes"] = dict(zip(PHASES, list(self.alg_bytes)))
        d["ms_phase"] = dict(zip(PHASES, list(self.ms_phase)))
        return d


class GraphInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("source", ctypes.c_int32), ("m", ctypes.c_int64),
        ("cap_fwd", ctypes.c_int64), ("cap_rev", ctypes.c_int64),
        ("pool_used_fwd", ctypes.c_int64), ("pool_used_rev", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64), ("state", ctypes.c_int32),
        ("num_sms", ctypes.c_int32), ("pool_step", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                            ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                           ctypes.c_void_p)


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("n_slots", ctypes.c_int32),
                ("loop_blocks", ctypes.c_int32), ("slack", ctypes.c_float),
                ("delta", ctypes.c_int32), ("max_batch_updates", ctypes.c_int64)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("updates", ctypes.c_int64), ("submit_ms", ctypes.c_double),
                ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double),
                ("loaded", ctypes.c_int32), ("gpu_start_ms", ctypes.c_double),
                ("gpu_done_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("resident_bytes", ctypes.c_int64), ("max_resident_bytes", ctypes.c_int64),
                ("loads", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("queries", ctypes.c_int64),
                ("updates", ctypes.c_int64), ("resident_graphs", ctypes.c_int32),
                ("registered_graphs", ctypes.c_int32), ("recoveries", ctypes.c_int64),
                ("restores", ctypes.c_int64), ("load_ms", ctypes.c_double),
                ("evict_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Allocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


# Entry points declared in include/sp.h: name -> (restype, argtypes)
_P, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
SIGNATURES = {
    "sp_graph_create": (ctypes.c_int, [_I32, _I64, _P, _P, _P, ctypes.c_int, ctypes.c_float,
                                       _P, _P, ctypes.POINTER(ctypes.c_void_p)]),
    "sp_graph_destroy": (ctypes.c_int, [_P]),
    "sp_sssp_init": (ctypes.c_int, [_P, _I32, _P]),
    "sp_apply_batch": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _P, ctypes.c_int, _P]),
    "sp_apply_batch_get": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _P, ctypes.c_int,
                                          _P, _P, ctypes.c_int, _P]),
    "sp_get_dist": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "sp_graph_num_edges": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "sp_export_csr": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int]),
    "sp_export_csr_noalloc": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "sp_graph_info_get": (ctypes.c_int, [_P, ctypes.POINTER(GraphInfo)]),
    "sp_set_limits": (ctypes.c_int, [_P, _I32, _I64]),
    "sp_set_push_delta": (ctypes.c_int, [_P, _I32]),
    "sp_set_inval_switch": (ctypes.c_int, [_P, _I32]),
    "sp_set_local_rounds": (ctypes.c_int, [_P, _I32]),
    "sp_set_schedule": (ctypes.c_int, [_P, _I32, _I32]),
    "sp_inject_missed_arrival": (ctypes.c_int, [_P, _I32]),
    "sp_set_dist": (ctypes.c_int, [_P, _I32, _P, _P, ctypes.c_int]),
    "sp_footprint_bound": (ctypes.c_int, [_I32, _I64, ctypes.c_float, _I64,
                                          ctypes.POINTER(ctypes.c_int64)]),
    "sp_set_batch_graphs": (ctypes.c_int, [_P, _I32]),
    "sp_loop_counters": (ctypes.c_int, [_P, _P, _I32]),
    "sp_pr_init": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, _I32, _P]),
    "sp_pr_apply_batch": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _P, ctypes.c_int, _P]),
    "sp_pr_get": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "sp_tc_init": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "sp_tc_apply_batch": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _P, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int64), _P]),
    "sp_sssp_init_multi": (ctypes.c_int, [_P, _P, _I32, ctypes.c_int, _P]),
    "sp_reserve": (ctypes.c_int, [_P, _I64]),
    "sp_async_result_bytes": (ctypes.c_size_t, []),
    "sp_apply_batch_async": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _P, _P]),
    "sp_apply_batch_finish": (ctypes.c_int, [_P, _P, _P]),
    "sp_capture_apply": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _P, _P,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "sp_exec_launch": (ctypes.c_int, [_P]),
    "sp_exec_destroy": (ctypes.c_int, [_P]),
    "sp_sync": (ctypes.c_int, [_P]),
    "sp_query": (ctypes.c_int, [_P, _I32, _P, _P, ctypes.c_int]),
    "sp_set_loop_blocks": (ctypes.c_int, [_P, _I32]),
    "sp_server_create": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_void_p)]),
    "sp_server_destroy": (ctypes.c_int, [_P]),
    "sp_server_add_graph": (ctypes.c_int, [_P, _I32, _I64, _P, _P, _P, _I32,
                                           ctypes.POINTER(ctypes.c_int32)]),
    "sp_server_submit_batch": (ctypes.c_int, [_P, _I32, _I64, _P, _P, _I64, _P, _P, _P,
                                              ctypes.POINTER(ctypes.c_int64)]),
    "sp_server_submit_query": (ctypes.c_int, [_P, _I32, _I32, _P,
                                              ctypes.POINTER(ctypes.c_int64)]),
    "sp_server_wait": (ctypes.c_int, [_P, _I64, _P, _P, _I32]),
    "sp_server_drain": (ctypes.c_int, [_P]),
    "sp_server_stats_get": (ctypes.c_int, [_P, _P]),
    "sp_server_get_dist": (ctypes.c_int, [_P, _I32, _P]),
    "sp_last_cuda_error": (ctypes.c_char_p, [_P]),
    "sp_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "sp_version": (ctypes.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libsp.so (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"{path} is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, what: str, h=None):
    if rc != SP_OK:
        if rc == SP_ETIMEOUT and h is not None:
            # say which device bound ended the call (loop counters 9..11)
            out = np.zeros(12, dtype=np.int64)
            if load().sp_loop_counters(h, out.ctypes.data_as(ctypes.c_void_p), 12) == SP_OK:
                what = (f"{what} (bound {int(out[9])} at site {int(out[10])}, "
                        f"index {int(out[11])}; push rounds {int(out[0])}, "
                        f"single-block {int(out[1])}, invalidation rounds {int(out[5])})")
        raise SpError(rc, what)


def _check_export_targets(g, row_off, col, w):
    """The export writes n+1 int64 offsets and m int32 columns and weights
    through raw device pointers: reject anything else before the call."""
    import torch
    m = g.m
    want = ((row_off, torch.int64, g.n + 1, "row_off"), (col, torch.int32, max(m, 1), "col"),
            (w, torch.int32, max(m, 1), "w"))
    dev = torch.device("cuda", g.device)
    for t, dt, need, name in want:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name}: a torch tensor is required")
        if t.dtype != dt:
            raise ValueError(f"{name}: dtype {t.dtype}, expected {dt}")
        if not t.is_contiguous():
            raise ValueError(f"{name}: must be contiguous")
        if t.numel() < need:
            raise ValueError(f"{name}: {t.numel()} elements, at least {need} needed")
    for t, dt, need, name in want:
        if not t.is_cuda:
            raise ValueError(f"{name}: must be a CUDA tensor")
        if t.device != dev:
            raise ValueError(f"{name}: must be on the graph's device")
    spans = []
    for t, dt, need, name in want:
        lo = t.data_ptr()
        spans.append((lo, lo + need * t.element_size(), name))
    spans.sort()
    for (a0, a1, an), (b0, b1, bn) in zip(spans, spans[1:]):
        if b0 < a1:
            raise ValueError(f"{an} and {bn} overlap")


_TORCH = None


def _torch():
    """torch, once CUDA is known to be there (checked on the first call)."""
    global _TORCH
    if _TORCH is None:
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: libsp has no CPU path")
        _TORCH = torch
    return _TORCH


def _is_cuda_tensor(x) -> bool:
    if _TORCH is not None:   # the common case: one isinstance check
        return isinstance(x, _TORCH.Tensor) and x.is_cuda
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


class _Arrays:
    """Marshal a group of arrays as all-host (numpy) or all-device (torch)."""

    def __init__(self, arrays, dtypes):
        self.keep = []
        self.ptrs = []
        dev = [a is not None and _is_cuda_tensor(a) for a in arrays]
        self.on_device = any(dev)
        if self.on_device and not all(d for d, a in zip(dev, arrays) if a is not None):
            raise TypeError("mix of host and device arrays")
        for a, dt in zip(arrays, dtypes):
            if a is None:
                self.ptrs.append(None)
                continue
            if self.on_device:
                t = _torch()
                tdt = t.int32 if dt is np.int32 else t.int64
                if a.dtype != tdt:   # converted only when needed (each call costs µs)
                    a = a.to(tdt)
                if not a.is_contiguous():
                    a = a.contiguous()
                self.keep.append(a)
                self.ptrs.append(ctypes.c_void_p(a.data_ptr()))
            else:
                a = np.ascontiguousarray(a, dtype=dt)
                self.keep.append(a)
                self.ptrs.append(a.ctypes.data_as(ctypes.c_void_p))


class Graph:
    """A device-resident dynamic graph with SSSP distances (libsp handle)."""

    def __init__(self, n, row_off, col, w, slack: float = 0.25, stream=None,
                 torch_allocator: bool = True, refuse_alloc=None):
        """refuse_alloc: optional callable(nbytes) -> bool; True makes that
        device allocation fail (returns NULL to the library), for tests of the
        SP_ENOMEM paths.  It needs torch_allocator."""
        torch = _torch()
        lib = load()
        self.n = int(n)
        self.device = torch.cuda.current_device()
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        self._alloc = None
        alloc_p = None
        if torch_allocator:
            dev = torch.cuda.current_device()

            def _a(ctx, size, st):
                if refuse_alloc is not None and refuse_alloc(int(size)):
                    return None
                try:
                    return torch.cuda.caching_allocator_alloc(int(size), dev, st or 0)
                except Exception:
                    return None

            def _f(ctx, ptr, size, st):
                try:
                    torch.cuda.caching_allocator_delete(ptr)
                except Exception:
                    pass

            self._alloc = Allocator(None, ALLOC_FN(_a), FREE_FN(_f))
            alloc_p = ctypes.byref(self._alloc)
        arr = _Arrays([row_off, col, w], [np.int64, np.int32, np.int32])
        m = int(arr.keep[1].numel() if arr.on_device else arr.keep[1].size)
        h = ctypes.c_void_p()
        rc = lib.sp_graph_create(self.n, m, arr.ptrs[0], arr.ptrs[1], arr.ptrs[2],
                                 int(arr.on_device), float(slack), alloc_p,
                                 ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h))
        _check(rc, "sp_graph_create")
        self._h = h

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().sp_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls ------------------------------------------------------------
    def sssp_init(self, source: int, stats: bool = False):
        st = BatchStats() if stats else None
        rc = load().sp_sssp_init(self._h, int(source), ctypes.byref(st) if st else None)
        _check(rc, "sp_sssp_init", self._h)
        return st

    def apply_batch(self, del_src, del_dst, add_src, add_dst, add_w, stats: bool = False,
                    raise_on_error: bool = True):
        """Apply deletions then insertions; numpy arrays are host inputs,
        CUDA tensors device inputs.  Returns BatchStats (or None)."""
        arr = _Arrays([del_src, del_dst, add_src, add_dst, add_w], [np.int32] * 5)
        size = (lambda a: int(a.numel())) if arr.on_device else (lambda a: int(a.size))
        nd, na = size(arr.keep[0]), size(arr.keep[2])
        if size(arr.keep[1]) != nd or size(arr.keep[3]) != na or size(arr.keep[4]) != na:
            raise SpError(SP_EINVAL, "batch array sizes")
        st = BatchStats() if stats else None
        rc = load().sp_apply_batch(self._h, nd, arr.ptrs[0], arr.ptrs[1], na, arr.ptrs[2],
                                   arr.ptrs[3], arr.ptrs[4], int(arr.on_device),
                                   ctypes.byref(st) if st else None)
        if raise_on_error:
            _check(rc, "sp_apply_batch", self._h)
            return st
        return rc, st

    def apply_batch_get(self, del_src, del_dst, add_src, add_dst, add_w, dist, parent=None,
                        stats: bool = False):
        """apply_batch, then the distances (and parents) after it into
        ``dist`` / ``parent``, in one call with one synchronisation: CUDA
        tensors or int32 numpy arrays of n entries (page-locked host arrays
        are written in place).  Returns BatchStats (or None)."""
        arr = _Arrays([del_src, del_dst, add_src, add_dst, add_w], [np.int32] * 5)
        size = (lambda a: int(a.numel())) if arr.on_device else (lambda a: int(a.size))
        nd, na = size(arr.keep[0]), size(arr.keep[2])
        if size(arr.keep[1]) != nd or size(arr.keep[3]) != na or size(arr.keep[4]) != na:
            raise SpError(SP_EINVAL, "batch array sizes")
        out_dev = _is_cuda_tensor(dist)
        ptrs = []
        for x in (dist, parent):
            if x is None:
                ptrs.append(None)
                continue
            if out_dev:
                t = _torch()
                if (not _is_cuda_tensor(x) or x.dtype != t.int32 or x.numel() != self.n or
                        not x.is_contiguous() or x.device.index != self.device):
                    raise SpError(SP_EINVAL, "apply_batch_get: outputs must be contiguous "
                                             "int32 CUDA tensors of n entries on the graph's "
                                             "device")
                ptrs.append(ctypes.c_void_p(x.data_ptr()))
            else:
                if (not isinstance(x, np.ndarray) or x.dtype != np.int32 or x.size != self.n or
                        not x.flags.c_contiguous or not x.flags.writeable):
                    raise SpError(SP_EINVAL, "apply_batch_get: outputs must be writable, "
                                             "contiguous int32 arrays of n entries")
                ptrs.append(x.ctypes.data_as(ctypes.c_void_p))
        st = BatchStats() if stats else None
        rc = load().sp_apply_batch_get(self._h, nd, arr.ptrs[0], arr.ptrs[1], na, arr.ptrs[2],
                                       arr.ptrs[3], arr.ptrs[4], int(arr.on_device), ptrs[0],
                                       ptrs[1], int(out_dev), ctypes.byref(st) if st else None)
        _check(rc, "sp_apply_batch_get", self._h)
        return st

    def apply(self, batch, stats: bool = False):
        """Apply a ``workloads.Batch``."""
        return self.apply_batch(batch.del_src, batch.del_dst, batch.add_src,
                                batch.add_dst, batch.add_w, stats=stats)

    def sssp_init_multi(self, sources, stats: bool = False):
        """Distances from the nearest of several sources (batched form)."""
        arr = _Arrays([sources], [np.int32])
        k = int(arr.keep[0].numel() if arr.on_device else arr.keep[0].size)
        st = BatchStats() if stats else None
        rc = load().sp_sssp_init_multi(self._h, arr.ptrs[0], k, int(arr.on_device),
                                       ctypes.byref(st) if st else None)
        _check(rc, "sp_sssp_init_multi", self._h)
        return st

    def reserve(self, max_updates: int):
        """Size per-batch buffers so apply_async never allocates."""
        _check(load().sp_reserve(self._h, int(max_updates)), "sp_reserve")

    def capture(self, del_src, del_dst, add_src, add_dst, add_w):
        """Record one asynchronous batch (CUDA tensors, fixed addresses and
        sizes) into a CUDA graph; returns an Exec to replay it."""
        return Exec(self, del_src, del_dst, add_src, add_dst, add_w)

    def sync(self):
        _check(load().sp_sync(self._h), "sp_sync")

    def query(self, vertices):
        """Distances of the given vertices (numpy in, numpy out)."""
        v = np.ascontiguousarray(vertices, dtype=np.int32)
        out = np.empty(v.size, dtype=np.int32)
        rc = load().sp_query(self._h, v.size, v.ctypes.data_as(ctypes.c_void_p),
                             out.ctypes.data_as(ctypes.c_void_p), 0)
        _check(rc, "sp_query")
        return out

    def set_loop_blocks(self, blocks: int):
        _check(load().sp_set_loop_blocks(self._h, int(blocks)), "sp_set_loop_blocks")

    def get_dist(self, parent: bool = False, out=None):
        """dist (and parent) as numpy arrays, or into ``out`` = (dist,
        parent_or_None): CUDA tensors, or int32 numpy arrays of n entries
        (page-locked ones are written in place by the kernel)."""
        lib = load()
        if out is not None and isinstance(out[0], np.ndarray):
            d, p = out
            for x in (d, p):
                if x is not None and (x.dtype != np.int32 or x.size != self.n or
                                      not x.flags.c_contiguous or not x.flags.writeable):
                    raise SpError(SP_EINVAL, "get_dist: out arrays must be writable, "
                                             "contiguous int32 of n entries")
            rc = lib.sp_get_dist(self._h, d.ctypes.data_as(ctypes.c_void_p),
                                 p.ctypes.data_as(ctypes.c_void_p) if p is not None else None, 0)
            _check(rc, "sp_get_dist")
            return out
        if out is not None:
            d, p = out
            rc = lib.sp_get_dist(self._h, ctypes.c_void_p(d.data_ptr()),
                                 ctypes.c_void_p(p.data_ptr()) if p is not None else None, 1)
            _check(rc, "sp_get_dist")
            return out
        d = np.empty(self.n, dtype=np.int32)
        p = np.empty(self.n, dtype=np.int32) if parent else None
        rc = lib.sp_get_dist(self._h, d.ctypes.data_as(ctypes.c_void_p),
                             p.ctypes.data_as(ctypes.c_void_p) if p is not None else None, 0)
        _check(rc, "sp_get_dist")
        return (d, p) if parent else d

    @property
    def m(self) -> int:
        v = ctypes.c_int64()
        _check(load().sp_graph_num_edges(self._h, ctypes.byref(v)), "sp_graph_num_edges")
        return int(v.value)

    def export_csr(self, reverse: bool = False):
        m = self.m
        ro = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(m, 1), dtype=np.int32)
        w = np.empty(max(m, 1), dtype=np.int32)
        rc = load().sp_export_csr(self._h, int(reverse), ro.ctypes.data_as(ctypes.c_void_p),
                                  col.ctypes.data_as(ctypes.c_void_p),
                                  w.ctypes.data_as(ctypes.c_void_p), 0)
        _check(rc, "sp_export_csr")
        return ro, col[:m], w[:m]

    def export_csr_device(self, row_off, col, w, reverse: bool = False,
                          noalloc: bool = False):
        """Export into caller-owned CUDA tensors (int64 row_off[n+1], int32
        col[m], int32 w[m]).  noalloc=True uses sp_export_csr_noalloc, which
        allocates no device memory during the call."""
        lib = load()
        _check_export_targets(self, row_off, col, w)
        p = [ctypes.c_void_p(t.data_ptr()) for t in (row_off, col, w)]
        if noalloc:
            rc = lib.sp_export_csr_noalloc(self._h, int(reverse), *p)
            _check(rc, "sp_export_csr_noalloc")
        else:
            rc = lib.sp_export_csr(self._h, int(reverse), *p, 1)
            _check(rc, "sp_export_csr")
        return row_off, col, w

    def info(self) -> GraphInfo:
        gi = GraphInfo()
        _check(load().sp_graph_info_get(self._h, ctypes.byref(gi)), "sp_graph_info_get")
        return gi

    def set_delta(self, delta: int):
        """Near-far bucket width of the push loop (0 = plain frontier rounds)."""
        _check(load().sp_set_push_delta(self._h, int(delta)), "sp_set_push_delta")

    def set_inval_switch(self, rounds: int):
        """Frontier rounds of the invalidation before pointer jumping
        (< 0: never, 0: jump at once)."""
        _check(load().sp_set_inval_switch(self._h, int(rounds)), "sp_set_inval_switch")

    # -- PageRank ------------------------------------------------------------
    def pr_init(self, damping: float = 0.85, beta: float = 1e-6, max_iter: int = 100,
                stats: bool = False):
        """staticPR (single precision); returns BatchStats or None."""
        st = BatchStats() if stats else None
        rc = load().sp_pr_init(self._h, float(damping), float(beta), int(max_iter),
                               ctypes.byref(st) if st else None)
        _check(rc, "sp_pr_init", self._h)
        return st

    def pr_apply_batch(self, del_src, del_dst, add_src, add_dst, add_w, stats: bool = False):
        """DynPR for one batch (numpy: host inputs, CUDA tensors: device)."""
        arr = _Arrays([del_src, del_dst, add_src, add_dst, add_w], [np.int32] * 5)
        size = (lambda a: int(a.numel())) if arr.on_device else (lambda a: int(a.size))
        nd, na = size(arr.keep[0]), size(arr.keep[2])
        if size(arr.keep[1]) != nd or size(arr.keep[3]) != na or size(arr.keep[4]) != na:
            raise SpError(SP_EINVAL, "batch array sizes")
        st = BatchStats() if stats else None
        rc = load().sp_pr_apply_batch(self._h, nd, arr.ptrs[0], arr.ptrs[1], na, arr.ptrs[2],
                                      arr.ptrs[3], arr.ptrs[4], int(arr.on_device),
                                      ctypes.byref(st) if st else None)
        _check(rc, "sp_pr_apply_batch", self._h)
        return st

    def pr_apply(self, batch, stats: bool = False):
        return self.pr_apply_batch(batch.del_src, batch.del_dst, batch.add_src, batch.add_dst,
                                   batch.add_w, stats=stats)

    def pr_get(self):
        out = np.empty(self.n, dtype=np.float32)
        _check(load().sp_pr_get(self._h, out.ctypes.data_as(ctypes.c_void_p), 0), "sp_pr_get")
        return out

    # -- triangle count ------------------------------------------------------
    def tc_init(self) -> int:
        """staticTC of a symmetric graph."""
        c = ctypes.c_int64()
        _check(load().sp_tc_init(self._h, ctypes.byref(c)), "sp_tc_init")
        return int(c.value)

    def tc_apply_batch(self, del_src, del_dst, add_src, add_dst, add_w, stats: bool = False):
        """DynTC for one symmetric batch; returns the new count (and stats)."""
        arr = _Arrays([del_src, del_dst, add_src, add_dst, add_w], [np.int32] * 5)
        size = (lambda a: int(a.numel())) if arr.on_device else (lambda a: int(a.size))
        nd, na = size(arr.keep[0]), size(arr.keep[2])
        if size(arr.keep[1]) != nd or size(arr.keep[3]) != na or size(arr.keep[4]) != na:
            raise SpError(SP_EINVAL, "batch array sizes")
        st = BatchStats() if stats else None
        c = ctypes.c_int64()
        rc = load().sp_tc_apply_batch(self._h, nd, arr.ptrs[0], arr.ptrs[1], na, arr.ptrs[2],
                                      arr.ptrs[3], arr.ptrs[4], int(arr.on_device),
                                      ctypes.byref(c), ctypes.byref(st) if st else None)
        _check(rc, "sp_tc_apply_batch", self._h)
        return (int(c.value), st) if stats else int(c.value)

    def tc_apply(self, batch, stats: bool = False):
        return self.tc_apply_batch(batch.del_src, batch.del_dst, batch.add_src, batch.add_dst,
                                   batch.add_w, stats=stats)

    def loop_counters(self) -> dict:
        """Loop counters of the last call (tuning aid)."""
        out = np.zeros(16, dtype=np.int64)
        _check(load().sp_loop_counters(self._h, out.ctypes.data_as(ctypes.c_void_p), 16),
               "sp_loop_counters")
        keys = ("rounds_push", "local_rounds", "local_episodes", "splits", "far_moves",
                "rounds_inval", "jumps", "local_ns", "push_ns", "timeout", "timeout_site",
                "timeout_index", "pool_subrounds", "pool_entries", "pool_ns0",
                "pool_subrounds0")
        return dict(zip(keys, (int(x) for x in out)))

    def last_cuda_error(self) -> str:
        return load().sp_last_cuda_error(self._h).decode()

    def set_batch_graphs(self, on: bool):
        """Replay repeated batch shapes as a cached CUDA graph (default on)."""
        _check(load().sp_set_batch_graphs(self._h, int(bool(on))), "sp_set_batch_graphs")

    def set_local_rounds(self, max_edges: int):
        """Frontier-edge bound of single-block push rounds (0 = off)."""
        _check(load().sp_set_local_rounds(self._h, int(max_edges)), "sp_set_local_rounds")

    def set_schedule(self, small_deg: int = 8, pool_rounds: int = 0):
        """Push schedule: small-list degree bound (thread per vertex up to it,
        warp-wide edge chunks above) and block-local sub-rounds per grid round
        (0 = off)."""
        _check(load().sp_set_schedule(self._h, int(small_deg), int(pool_rounds)),
               "sp_set_schedule")

    def inject_missed_arrival(self, site: int):
        """Test hook: block 0 skips the grid barriers of wait site 2, 4 or 5,
        so their bounded waits run out (0 = off)."""
        _check(load().sp_inject_missed_arrival(self._h, int(site)),
               "sp_inject_missed_arrival")

    def set_dist(self, source: int, dist, parent):
        """Install distances and parents exported by get_dist (checked exact
        on the device; SpError SP_EINVAL otherwise)."""
        d = np.ascontiguousarray(dist, dtype=np.int32)
        p = np.ascontiguousarray(parent, dtype=np.int32)
        if d.size != self.n or p.size != self.n:
            raise SpError(SP_EINVAL, "dist/parent sizes")
        _check(load().sp_set_dist(self._h, int(source), d.ctypes.data_as(ctypes.c_void_p),
                                  p.ctypes.data_as(ctypes.c_void_p), 0), "sp_set_dist")

    def set_limits(self, max_rounds: int = 0, wait_ns: int = 0):
        _check(load().sp_set_limits(self._h, int(max_rounds), int(wait_ns)), "sp_set_limits")


class Exec:
    """A captured batch: launch() replays it on the graph's stream; finish()
    waits and reports the batch status and statistics."""

    def __init__(self, g: Graph, del_src, del_dst, add_src, add_dst, add_w):
        lib = load()
        torch = _torch()
        self.g = g
        self.inputs = (del_src, del_dst, add_src, add_dst, add_w)
        for t in self.inputs:
            if not _is_cuda_tensor(t) or t.dtype != torch.int32 or not t.is_contiguous():
                raise TypeError("capture needs contiguous int32 CUDA tensors")
        self.nd, self.na = int(del_src.numel()), int(add_src.numel())
        nbytes = int(lib.sp_async_result_bytes())
        self.result = torch.zeros(nbytes, dtype=torch.uint8, pin_memory=True)
        h = ctypes.c_void_p()
        p = [ctypes.c_void_p(t.data_ptr()) for t in self.inputs]
        rc = lib.sp_capture_apply(g._h, self.nd, p[0], p[1], self.na, p[2], p[3], p[4],
                                  ctypes.c_void_p(self.result.data_ptr()), ctypes.byref(h))
        _check(rc, "sp_capture_apply")
        self._h = h

    def launch(self):
        _check(load().sp_exec_launch(self._h), "sp_exec_launch")

    def finish(self, stats: bool = False, raise_on_error: bool = True):
        self.g.sync()
        st = BatchStats() if stats else None
        rc = load().sp_apply_batch_finish(self.g._h, ctypes.c_void_p(self.result.data_ptr()),
                                          ctypes.byref(st) if st else None)
        if raise_on_error:
            _check(rc, "sp_apply_batch_finish", self.g._h)
            return st
        return rc, st

    def close(self):
        if getattr(self, "_h", None):
            load().sp_exec_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving runtime (sp_server_*): many graphs, requests submitted
    asynchronously and run by worker slots, graphs admitted under an HBM
    budget with least-recently-used eviction.  All arrays are host (numpy)."""

    def __init__(self, hbm_budget_bytes: int, n_slots: int = 2, loop_blocks: int = 0,
                 slack: float = 0.25, delta: int = 0, max_batch_updates: int = 0):
        _torch()
        cfg = ServerConfig(int(hbm_budget_bytes), int(n_slots), int(loop_blocks),
                           float(slack), int(delta), int(max_batch_updates))
        h = ctypes.c_void_p()
        _check(load().sp_server_create(ctypes.byref(cfg), ctypes.byref(h)), "sp_server_create")
        self._h = h
        self._n = {}
        self._k = {}

    def close(self):
        if getattr(self, "_h", None):
            load().sp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_graph(self, n, row_off, col, w, source: int) -> int:
        ro = np.ascontiguousarray(row_off, dtype=np.int64)
        c = np.ascontiguousarray(col, dtype=np.int32)
        ww = np.ascontiguousarray(w, dtype=np.int32)
        gid = ctypes.c_int32()
        rc = load().sp_server_add_graph(self._h, int(n), int(c.size),
                                        ro.ctypes.data_as(ctypes.c_void_p),
                                        c.ctypes.data_as(ctypes.c_void_p),
                                        ww.ctypes.data_as(ctypes.c_void_p), int(source),
                                        ctypes.byref(gid))
        _check(rc, "sp_server_add_graph")
        self._n[gid.value] = int(n)
        return gid.value

    def submit_batch(self, graph: int, del_src, del_dst, add_src, add_dst, add_w) -> int:
        a = [np.ascontiguousarray(x, dtype=np.int32)
             for x in (del_src, del_dst, add_src, add_dst, add_w)]
        if a[0].size != a[1].size or not (a[2].size == a[3].size == a[4].size):
            raise SpError(SP_EINVAL, "batch array sizes")
        p = [x.ctypes.data_as(ctypes.c_void_p) for x in a]
        rid = ctypes.c_int64()
        rc = load().sp_server_submit_batch(self._h, int(graph), a[0].size, p[0], p[1],
                                           a[2].size, p[2], p[3], p[4], ctypes.byref(rid))
        _check(rc, "sp_server_submit_batch")
        return rid.value

    def submit(self, graph: int, batch) -> int:
        """Submit a ``workloads.Batch``."""
        return self.submit_batch(graph, batch.del_src, batch.del_dst, batch.add_src,
                                 batch.add_dst, batch.add_w)

    def submit_query(self, graph: int, vertices) -> int:
        v = np.ascontiguousarray(vertices, dtype=np.int32)
        rid = ctypes.c_int64()
        rc = load().sp_server_submit_query(self._h, int(graph), v.size,
                                           v.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rid))
        _check(rc, "sp_server_submit_query")
        self._k[rid.value] = v.size
        return rid.value

    def wait(self, request_id: int, timeout_ms: int = -1):
        """(RequestInfo, distances or None); raises on a failed request."""
        info = RequestInfo()
        k = self._k.pop(request_id, None)
        out = np.empty(k, dtype=np.int32) if k is not None else None
        rc = load().sp_server_wait(self._h, int(request_id), ctypes.byref(info),
                                   out.ctypes.data_as(ctypes.c_void_p) if k else None,
                                   int(timeout_ms))
        if rc != SP_OK and k is not None:
            self._k[request_id] = k
        _check(rc, "sp_server_wait")
        return info, out

    def drain(self):
        _check(load().sp_server_drain(self._h), "sp_server_drain")

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(load().sp_server_stats_get(self._h, ctypes.byref(st)), "sp_server_stats_get")
        return st

    def get_dist(self, graph: int):
        d = np.empty(self._n[graph], dtype=np.int32)
        rc = load().sp_server_get_dist(self._h, int(graph), d.ctypes.data_as(ctypes.c_void_p))
        _check(rc, "sp_server_get_dist")
        return d


def footprint_bound(n: int, m: int, slack: float = 0.25, max_updates: int = 0) -> int:
    """Upper bound of a handle's device bytes (sp_footprint_bound)."""
    _torch()
    v = ctypes.c_int64()
    _check(load().sp_footprint_bound(int(n), int(m), float(slack), int(max_updates),
                                     ctypes.byref(v)), "sp_footprint_bound")
    return int(v.value)


def status_str(code: int) -> str:
    return load().sp_status_str(int(code)).decode()
