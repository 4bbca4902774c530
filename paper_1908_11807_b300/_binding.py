"""Thin ctypes binding of ``libarborx_b300.so`` (argument marshalling only).

Every step of the search runs in the library's CUDA kernels; this module only
passes device pointers, sizes and the current torch stream.  Tensors must be
contiguous CUDA tensors on the current device.  If the library has not been
built the import fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import torch

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libarborx_b300.so")

ARBORX_OK = 0
ARBORX_EINVAL = 1
ARBORX_ENOMEM = 2
ARBORX_ECUDA = 3
ARBORX_ETIMEOUT = 4
ARBORX_EOVERFLOW = 5
ARBORX_ESTATE = 6
ARBORX_POINTS = 0
ARBORX_BOXES = 1
ARBORX_BUILD_APETREI = 0
ARBORX_BUILD_KARRAS = 1
ARBORX_MAX_K = 512
ARBORX_QOPT_EMIT_SUBTREES = 1
MLP_PARAMS = 4481

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class arborx_opts(ctypes.Structure):
    _fields_ = [
        ("key_bits", ctypes.c_int32),
        ("sort_queries", ctypes.c_int32),
        ("validate", ctypes.c_int32),
        ("keep_order", ctypes.c_int32),
        ("block_size", ctypes.c_int32),
        ("stack_smem", ctypes.c_int32),
        ("build_method", ctypes.c_int32),
        ("stats", ctypes.c_int32),
        ("sorted_rows", ctypes.c_int32),
        ("knn_anchor", ctypes.c_int32),
        ("queries_per_warp", ctypes.c_int32),
        ("knn_heap_from", ctypes.c_int32),
        ("alloc", _ALLOC_FN),
        ("free", _FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
    ]


class ArborXError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} (status {code})")


_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library (fails loudly if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1908_11807_b300.build_ext` "
                              "(or __graft_entry__.build()); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.arborx_version.restype = ctypes.c_char_p
        L.arborx_error_string.restype = ctypes.c_char_p
        L.arborx_error_string.argtypes = [ctypes.c_int]
        L.arborx_default_opts.argtypes = [ctypes.POINTER(arborx_opts)]
        L.arborx_build.argtypes = [vp, i64, i32, ctypes.POINTER(arborx_opts), vp, ctypes.POINTER(vp)]
        L.arborx_destroy.argtypes = [vp]
        L.arborx_size.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32)]
        L.arborx_check.argtypes = [vp, vp]
        L.arborx_query_spatial_count.argtypes = [vp, vp, i64, ctypes.c_float, vp, vp, vp]
        L.arborx_query_spatial_fill.argtypes = [vp, vp, i64, ctypes.c_float, vp, vp, vp, i64]
        L.arborx_query_spatial.argtypes = [vp, vp, i64, ctypes.c_float, vp, vp, vp, ctypes.POINTER(vp),
                                           ctypes.POINTER(i64)]
        L.arborx_free.argtypes = [vp, vp, ctypes.c_size_t, vp]
        L.arborx_query_nearest.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp, vp]
        L.arborx_query_order.argtypes = [vp, vp, i64, vp, vp]
        L.arborx_mlp_forward.argtypes = [vp, vp, vp, i64, i32, vp, vp]
        L.arborx_mlp_grad.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp]
        L.arborx_mlp_train.argtypes = [vp, vp, i64, i32, i32, i32, ctypes.c_float, ctypes.c_float, vp, vp, vp]
        L.arborx_query_spatial_buffered_count.argtypes = [vp, vp, i64, ctypes.c_float, i32, vp, vp, vp,
                                                          ctypes.POINTER(i64)]
        L.arborx_query_spatial_buffered_fill.argtypes = [vp, vp, i64, ctypes.c_float, vp, vp, vp, i64]
        L.arborx_query_spatial_buffered.argtypes = [vp, vp, i64, ctypes.c_float, i32, vp, vp, vp, vp, i64]
        L.arborx_query_spatial_nearest.argtypes = [vp, vp, i64, ctypes.c_float, i32, i32, vp, vp, vp, vp, i64, vp,
                                                   vp, vp]
        L.arborx_query_order_boxes.argtypes = [vp, vp, i64, vp, vp]
        L.arborx_selftest_bounded_wait.argtypes = [vp]
        L.arborx_selftest_scan_wait.argtypes = [vp]
        L.arborx_rebuild.argtypes = [vp, vp, vp]
        L.arborx_order.argtypes = [vp, i64, i32, ctypes.POINTER(arborx_opts), vp, vp]
        L.arborx_query_intersects.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp, i64]
        L.arborx_batch_create.argtypes = [i64, vp, vp, vp, ctypes.POINTER(arborx_opts), vp, ctypes.POINTER(vp)]
        L.arborx_batch_entries.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.arborx_batch_run.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
        L.arborx_batched.argtypes = [i64, vp, vp, vp, vp, vp, ctypes.POINTER(arborx_opts), vp, vp, vp, vp, i64]
        L.arborx_batch_check.argtypes = [vp, vp]
        L.arborx_batch_destroy.argtypes = [vp]
        L.arborx_query_nearest_bounded.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp, vp, vp,
                                                   ctypes.POINTER(i64)]
        L.arborx_query_nearest_learned.argtypes = [vp, vp, i64, i32, vp, ctypes.c_float, vp, vp, vp, vp, vp,
                                                   ctypes.POINTER(i64)]
        L.arborx_stats.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint64)]
        L.arborx_set_query_option.argtypes = [vp, i32, i64]
        L.arborx_export_tree.argtypes = [vp, vp, vp, vp, vp, vp]
        L.arborx_sort_pairs.argtypes = [vp, vp, i64, i32, vp]
        L.arborx_sort_pairs_noalloc.argtypes = [vp, vp, i64, i32, vp]
        L.arborx_profile_enable.argtypes = [ctypes.c_int]
        L.arborx_profile_report.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
        _lib = L
    return _lib


def error_string(code: int) -> str:
    return lib().arborx_error_string(int(code)).decode()


def version() -> str:
    return lib().arborx_version().decode()


def _check(code: int, where: str) -> None:
    if code != ARBORX_OK:
        raise ArborXError(code, where)


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _as_f32_cuda(x: torch.Tensor, width: int, name: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if x.dim() != 2 or x.shape[1] != width:
        raise ValueError(f"{name} must have shape [n][{width}]")
    return x.contiguous()


def default_opts(**kw) -> arborx_opts:
    o = arborx_opts()
    _check(lib().arborx_default_opts(ctypes.byref(o)), "arborx_default_opts")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class BVH:
    """A linear BVH on the current CUDA device (wraps an ``arborx_handle``)."""

    def __init__(self, prims: torch.Tensor, kind: Optional[int] = None, **opts):
        if kind is None:
            kind = ARBORX_POINTS if prims.dim() == 2 and prims.shape[1] == 3 else ARBORX_BOXES
        width = 3 if kind == ARBORX_POINTS else 6
        self.prims = _as_f32_cuda(prims, width, "prims")
        self.kind = int(kind)
        self.n = int(self.prims.shape[0])
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        _check(lib().arborx_build(_ptr(self.prims), self.n, self.kind, ctypes.byref(self.opts), _stream(),
                                  ctypes.byref(h)), "arborx_build")
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("BVH destroyed")
        return self._h

    def rebuild(self, prims: torch.Tensor) -> None:
        """Rebuild the tree in place over new coordinates of the same primitives (same n and kind);
        with validate=0 the call only enqueues work and can be captured in a CUDA graph."""
        width = 3 if self.kind == ARBORX_POINTS else 6
        p = _as_f32_cuda(prims, width, "prims")
        if p.shape[0] != self.n:
            raise ValueError(f"rebuild needs the same number of primitives ({self.n})")
        _check(lib().arborx_rebuild(self.handle, _ptr(p), _stream()), "arborx_rebuild")
        self.prims = p

    def destroy(self) -> None:
        if getattr(self, "_h", None) is not None:
            lib().arborx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def check(self) -> None:
        """Synchronise and raise if a kernel reported an error on this tree."""
        _check(lib().arborx_check(self.handle, _stream()), "arborx_check")

    # -- spatial (2P)
    def query_order(self, queries: torch.Tensor) -> torch.Tensor:
        """Morton traversal order of a query set (int32 [m]), reusable across query calls."""
        q = _as_f32_cuda(queries, 3, "queries")
        order = torch.empty(q.shape[0], dtype=torch.int32, device=q.device)
        _check(lib().arborx_query_order(self.handle, _ptr(q), q.shape[0], _stream(), _ptr(order)),
               "arborx_query_order")
        return order

    def query_order_boxes(self, boxes: torch.Tensor) -> torch.Tensor:
        """Morton traversal order of a set of query boxes float32 [m, 6] (by box centre)."""
        b = _as_f32_cuda(boxes, 6, "boxes")
        order = torch.empty(b.shape[0], dtype=torch.int32, device=b.device)
        _check(lib().arborx_query_order_boxes(self.handle, _ptr(b), b.shape[0], _stream(), _ptr(order)),
               "arborx_query_order_boxes")
        return order

    def query_intersects_async(self, boxes: torch.Tensor, buffer_size: int = 16,
                               order: Optional[torch.Tensor] = None, capacity: Optional[int] = None,
                               indices: Optional[torch.Tensor] = None) -> Tuple[torch.Tensor, torch.Tensor]:
        """Box-intersection query with no host synchronisation: (offsets int64 [m+1], indices int32
        [capacity]); the first offsets[-1] entries of ``indices`` are the CSR rows.  ``capacity``
        defaults to m * buffer_size; rows beyond it are dropped and ``check()`` raises."""
        b = _as_f32_cuda(boxes, 6, "boxes")
        m = b.shape[0]
        offsets = torch.empty(m + 1, dtype=torch.int64, device=b.device)
        if indices is None:
            cap = int(m * buffer_size if capacity is None else capacity)
            indices = torch.empty(max(cap, 1), dtype=torch.int32, device=b.device)
        else:
            cap = indices.numel() if capacity is None else int(capacity)
            if indices.dtype != torch.int32 or not indices.is_cuda or indices.numel() < cap:
                raise ValueError("indices must be an int32 CUDA tensor of at least `capacity` entries")
        _check(lib().arborx_query_intersects(self.handle, _ptr(b), m, int(buffer_size), _ptr(order), _stream(),
                                             _ptr(offsets), _ptr(indices), cap), "arborx_query_intersects")
        self._async_keep = (b, order)  # inputs stay alive while the stream works
        return offsets, indices

    def query_intersects(self, boxes: torch.Tensor, buffer_size: int = 16,
                         order: Optional[torch.Tensor] = None) -> Tuple[torch.Tensor, torch.Tensor]:
        """Box-intersection query: (offsets int64 [m+1], indices int32 [nnz]).  Reads the total back
        (synchronises) and, when the rows outgrew the first buffer, repeats with the exact size."""
        b = _as_f32_cuda(boxes, 6, "boxes")
        m = b.shape[0]
        cap = max(m * int(buffer_size), 1)
        while True:
            offsets, idx = self.query_intersects_async(b, buffer_size, order=order, capacity=cap)
            total = int(offsets[-1].item()) if m > 0 else 0
            if total <= cap:
                self.check()
                return offsets, idx[:total]
            try:
                self.check()  # clears the overflow flag of the attempt that was too small
            except ArborXError as e:
                if e.code != ARBORX_EOVERFLOW:
                    raise
            cap = total

    def emit_subtrees(self, on: bool = True) -> None:
        """Radius and box queries take wholly contained subtrees from the kept sorted leaf order
        instead of walking them (needs keep_order=1; speed only)."""
        _check(lib().arborx_set_query_option(self.handle, ARBORX_QOPT_EMIT_SUBTREES, int(bool(on))),
               "arborx_set_query_option")
        self._emit = bool(on)

    def stats(self) -> dict:
        """Internal nodes loaded and queries traversed since the last call (needs stats=1)."""
        out = (ctypes.c_uint64 * 4)()
        _check(lib().arborx_stats(self.handle, _stream(), out), "arborx_stats")
        return {"spatial_nodes": out[0], "nearest_nodes": out[1], "spatial_queries": out[2],
                "nearest_queries": out[3]}

    def query_spatial_async(self, queries: torch.Tensor, radius: float, buffer_size: int = 32,
                            order: Optional[torch.Tensor] = None, capacity: Optional[int] = None,
                            indices: Optional[torch.Tensor] = None) -> Tuple[torch.Tensor, torch.Tensor]:
        """One-pass spatial query with no host synchronisation: (offsets int64 [m+1], indices int32
        [capacity]); the first offsets[-1] entries of ``indices`` are the CSR rows.  ``capacity``
        defaults to m * buffer_size; rows beyond it are dropped and ``check()`` raises."""
        q = _as_f32_cuda(queries, 3, "queries")
        m = q.shape[0]
        offsets = torch.empty(m + 1, dtype=torch.int64, device=q.device)
        if indices is None:
            cap = int(m * buffer_size if capacity is None else capacity)
            indices = torch.empty(max(cap, 1), dtype=torch.int32, device=q.device)
        else:
            cap = indices.numel() if capacity is None else int(capacity)
            if indices.dtype != torch.int32 or not indices.is_cuda or indices.numel() < cap:
                raise ValueError("indices must be an int32 CUDA tensor of at least `capacity` entries")
        _check(lib().arborx_query_spatial_buffered(self.handle, _ptr(q), m, ctypes.c_float(radius), int(buffer_size),
                                                   _ptr(order), _stream(), _ptr(offsets), _ptr(indices), cap),
               "arborx_query_spatial_buffered")
        self._async_keep = (q, order)  # inputs stay alive while the stream works
        return offsets, indices

    def query_spatial_nearest(self, queries: torch.Tensor, radius: float, k: int, buffer_size: int = 32,
                              order: Optional[torch.Tensor] = None, capacity: Optional[int] = None,
                              indices: Optional[torch.Tensor] = None, return_dist2: bool = True):
        """The one-pass spatial query of ``query_spatial_async`` and the nearest query of
        ``query_nearest`` over the same queries in one call, the nearest traversal running
        concurrently on a second stream of the handle: (offsets, indices, nearest indices,
        nearest squared distances or None).  No host synchronisation."""
        q = _as_f32_cuda(queries, 3, "queries")
        m = q.shape[0]
        offsets = torch.empty(m + 1, dtype=torch.int64, device=q.device)
        if indices is None:
            cap = int(m * buffer_size if capacity is None else capacity)
            indices = torch.empty(max(cap, 1), dtype=torch.int32, device=q.device)
        else:
            cap = indices.numel() if capacity is None else int(capacity)
            if indices.dtype != torch.int32 or not indices.is_cuda or indices.numel() < cap:
                raise ValueError("indices must be an int32 CUDA tensor of at least `capacity` entries")
        kk = min(int(k), self.n)
        kidx = torch.empty((m, kk), dtype=torch.int32, device=q.device)
        kd2 = torch.empty((m, kk), dtype=torch.float32, device=q.device) if return_dist2 else None
        _check(lib().arborx_query_spatial_nearest(self.handle, _ptr(q), m, ctypes.c_float(radius), int(buffer_size),
                                                  int(k), _ptr(order), _stream(), _ptr(offsets), _ptr(indices), cap,
                                                  None, _ptr(kidx), _ptr(kd2)), "arborx_query_spatial_nearest")
        self._async_keep = (q, order)  # inputs stay alive while the streams work
        return offsets, indices, kidx, kd2

    def query_spatial_count(self, queries: torch.Tensor, radius: float,
                            offsets: Optional[torch.Tensor] = None,
                            order: Optional[torch.Tensor] = None) -> torch.Tensor:
        q = _as_f32_cuda(queries, 3, "queries")
        m = q.shape[0]
        if offsets is None:
            offsets = torch.empty(m + 1, dtype=torch.int64, device=q.device)
        _check(lib().arborx_query_spatial_count(self.handle, _ptr(q), m, ctypes.c_float(radius), _ptr(order),
                                                _stream(), _ptr(offsets)), "arborx_query_spatial_count")
        self._count_q = q
        self._count_order = order  # must stay alive until the fill
        return offsets

    def query_spatial_fill(self, queries: torch.Tensor, radius: float, offsets: torch.Tensor,
                           indices: torch.Tensor) -> torch.Tensor:
        q = getattr(self, "_count_q", None)  # the exact buffer the count pass traversed
        if q is None:
            raise ArborXError(ARBORX_ESTATE, "arborx_query_spatial_fill")
        _check(lib().arborx_query_spatial_fill(self.handle, _ptr(q), q.shape[0], ctypes.c_float(radius),
                                               _stream(), _ptr(offsets), _ptr(indices), indices.numel()),
               "arborx_query_spatial_fill")
        return indices

    def query_spatial(self, queries: torch.Tensor, radius: float, order: Optional[torch.Tensor] = None,
                      buffer_size: int = 0) -> Tuple[torch.Tensor, torch.Tensor]:
        """CSR (offsets int64 [m+1], indices int32 [nnz]) of the primitives within
        ``radius`` of each query.  buffer_size = 0: two traversals (count, read the total
        back, fill); buffer_size > 0: one traversal keeping up to buffer_size results per
        query, a second one only for queries with more."""
        if buffer_size > 0:
            q = _as_f32_cuda(queries, 3, "queries")
            m = q.shape[0]
            offsets = torch.empty(m + 1, dtype=torch.int64, device=q.device)
            nnz = ctypes.c_int64(0)
            _check(lib().arborx_query_spatial_buffered_count(self.handle, _ptr(q), m, ctypes.c_float(radius),
                                                             int(buffer_size), _ptr(order), _stream(),
                                                             _ptr(offsets), ctypes.byref(nnz)),
                   "arborx_query_spatial_buffered_count")
            indices = torch.empty(nnz.value, dtype=torch.int32, device=q.device)
            _check(lib().arborx_query_spatial_buffered_fill(self.handle, _ptr(q), m, ctypes.c_float(radius),
                                                            _stream(), _ptr(offsets), _ptr(indices),
                                                            indices.numel()), "arborx_query_spatial_buffered_fill")
            return offsets, indices
        offsets = self.query_spatial_count(queries, radius, order=order)
        nnz = int(offsets[-1].item())
        self.check()
        indices = torch.empty(nnz, dtype=torch.int32, device=offsets.device)
        self.query_spatial_fill(queries, radius, offsets, indices)
        return offsets, indices

    # -- nearest
    def query_nearest(self, queries: torch.Tensor, k: int, return_dist2: bool = True,
                      with_offsets: bool = False, order: Optional[torch.Tensor] = None):
        """Rows [m][min(k, n)] of neighbour indices (int32) in (d2, index) order,
        and their squared distances (float32) if requested."""
        q = _as_f32_cuda(queries, 3, "queries")
        m = q.shape[0]
        kk = min(int(k), self.n)
        idx = torch.empty((m, kk), dtype=torch.int32, device=q.device)
        d2 = torch.empty((m, kk), dtype=torch.float32, device=q.device) if return_dist2 else None
        off = torch.empty(m + 1, dtype=torch.int64, device=q.device) if with_offsets else None
        _check(lib().arborx_query_nearest(self.handle, _ptr(q), m, int(k), _ptr(order), _stream(), _ptr(off),
                                          _ptr(idx), _ptr(d2)), "arborx_query_nearest")
        out = (idx, d2) if return_dist2 else (idx,)
        if with_offsets:
            out = out + (off,)
        return out if len(out) > 1 else out[0]

    # -- learned initial bound
    def mlp_forward(self, params: torch.Tensor, queries: torch.Tensor, tensor_cores: bool = True) -> torch.Tensor:
        q = _as_f32_cuda(queries, 3, "queries")
        y = torch.empty(q.shape[0], dtype=torch.float32, device=q.device)
        _check(lib().arborx_mlp_forward(self.handle, _ptr(params), _ptr(q), q.shape[0], int(bool(tensor_cores)),
                                        _stream(), _ptr(y)), "arborx_mlp_forward")
        return y

    def mlp_grad(self, params: torch.Tensor, queries: torch.Tensor, labels: torch.Tensor):
        q = _as_f32_cuda(queries, 3, "queries")
        grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=q.device)
        loss = torch.empty(1, dtype=torch.float32, device=q.device)
        _check(lib().arborx_mlp_grad(self.handle, _ptr(params), _ptr(q), _ptr(labels.contiguous()), q.shape[0],
                                     _stream(), _ptr(grad), _ptr(loss)), "arborx_mlp_grad")
        return loss, grad

    def mlp_train(self, params: torch.Tensor, queries: torch.Tensor, k: int, epochs: int = 10, batch: int = 4096,
                  lr: float = 1e-3, lr_final: Optional[float] = None) -> torch.Tensor:
        """Train ``params`` (float32 [4481] CUDA tensor, updated in place); returns the loss per epoch."""
        q = _as_f32_cuda(queries, 3, "queries")
        if params.dtype != torch.float32 or params.numel() != MLP_PARAMS or not params.is_contiguous():
            raise ValueError("params must be a contiguous float32 tensor of 4481 values")
        loss = torch.empty(max(epochs, 1), dtype=torch.float32, device=q.device)
        _check(lib().arborx_mlp_train(self.handle, _ptr(q), q.shape[0], int(k), int(epochs), int(batch),
                                      ctypes.c_float(lr), ctypes.c_float(lr if lr_final is None else lr_final),
                                      _stream(), _ptr(params), _ptr(loss)), "arborx_mlp_train")
        return loss[:epochs]

    def query_nearest_bounded(self, queries: torch.Tensor, k: int, bound2: torch.Tensor,
                              order: Optional[torch.Tensor] = None, return_dist2: bool = True,
                              count_fallbacks: bool = False):
        """Nearest query whose traversal starts from the given squared bounds (float32 [m])."""
        q = _as_f32_cuda(queries, 3, "queries")
        m = q.shape[0]
        kk = min(int(k), self.n)
        idx = torch.empty((m, kk), dtype=torch.int32, device=q.device)
        d2 = torch.empty((m, kk), dtype=torch.float32, device=q.device) if return_dist2 else None
        fb = ctypes.c_int64(0)
        b2 = bound2.contiguous()
        _check(lib().arborx_query_nearest_bounded(self.handle, _ptr(q), m, int(k), _ptr(b2), _ptr(order), _stream(),
                                                  None, _ptr(idx), _ptr(d2),
                                                  ctypes.byref(fb) if count_fallbacks else None),
               "arborx_query_nearest_bounded")
        out = (idx, d2) if return_dist2 else (idx,)
        if count_fallbacks:
            out = out + (int(fb.value),)
        return out if len(out) > 1 else out[0]

    def query_nearest_learned(self, queries: torch.Tensor, k: int, params: torch.Tensor, margin: float,
                              order: Optional[torch.Tensor] = None, return_dist2: bool = True,
                              count_fallbacks: bool = False):
        q = _as_f32_cuda(queries, 3, "queries")
        m = q.shape[0]
        kk = min(int(k), self.n)
        idx = torch.empty((m, kk), dtype=torch.int32, device=q.device)
        d2 = torch.empty((m, kk), dtype=torch.float32, device=q.device) if return_dist2 else None
        fb = ctypes.c_int64(0)
        _check(lib().arborx_query_nearest_learned(self.handle, _ptr(q), m, int(k), _ptr(params),
                                                  ctypes.c_float(margin), _ptr(order), _stream(), None, _ptr(idx),
                                                  _ptr(d2), ctypes.byref(fb) if count_fallbacks else None),
               "arborx_query_nearest_learned")
        out = (idx, d2) if return_dist2 else (idx,)
        if count_fallbacks:
            out = out + (int(fb.value),)
        return out if len(out) > 1 else out[0]

    # -- inspection
    def export_tree(self, order: bool = False):
        """(records float32 [2+2(n-1)][8], scene float32 [6], codes uint64 [n] | None, perm int32 [n] | None)."""
        dev = self.prims.device
        n = self.n
        rec = torch.empty((2 + 2 * max(n - 1, 0), 8), dtype=torch.float32, device=dev) if n > 0 else None
        scene = torch.empty(6, dtype=torch.float32, device=dev)
        codes = torch.empty(n, dtype=torch.int64, device=dev) if order else None
        perm = torch.empty(n, dtype=torch.int32, device=dev) if order else None
        _check(lib().arborx_export_tree(self.handle, _stream(), _ptr(rec), _ptr(scene), _ptr(codes), _ptr(perm)),
               "arborx_export_tree")
        return rec, scene, codes, perm


def arborx_build(prims: torch.Tensor, kind: Optional[int] = None, **opts) -> BVH:
    return BVH(prims, kind, **opts)


def arborx_query_spatial(bvh: BVH, queries: torch.Tensor, radius: float):
    return bvh.query_spatial(queries, radius)


def arborx_query_nearest(bvh: BVH, queries: torch.Tensor, k: int, return_dist2: bool = True):
    return bvh.query_nearest(queries, k, return_dist2)


def arborx_sort_pairs(keys: torch.Tensor, key_bits: int) -> Tuple[torch.Tensor, torch.Tensor]:
    """Stable radix sort of int32/int64 keys (treated as unsigned, key_bits significant
    bits) on the GPU: (sorted keys, permutation int32)."""
    if keys.dtype not in (torch.int32, torch.int64) or not keys.is_cuda:
        raise TypeError("keys must be an int32 or int64 CUDA tensor")
    if (keys.dtype == torch.int32) != (key_bits <= 32):
        raise ValueError("int32 keys need key_bits <= 32, int64 keys key_bits > 32")
    k = keys.contiguous().clone()
    perm = torch.empty(k.numel(), dtype=torch.int32, device=k.device)
    _check(lib().arborx_sort_pairs(_ptr(k), _ptr(perm), k.numel(), int(key_bits), _stream()), "arborx_sort_pairs")
    return k, perm


def order(prims: torch.Tensor, kind: Optional[int] = None) -> torch.Tensor:
    """Morton traversal order (int32 [m]) of points float32 [m, 3] or boxes [m, 6], scaled by the
    set's own bounding box: needs no tree, so it can run on another stream during a build.  Only
    enqueues work on the current stream."""
    if kind is None:
        kind = ARBORX_BOXES if (prims.dim() == 2 and prims.shape[1] == 6) else ARBORX_POINTS
    x = _as_f32_cuda(prims, 6 if kind == ARBORX_BOXES else 3, "prims")
    out = torch.empty(x.shape[0], dtype=torch.int32, device=x.device)
    _check(lib().arborx_order(_ptr(x), x.shape[0], int(kind), None, _stream(), _ptr(out)), "arborx_order")
    return out


def profile_enable(on: bool = True) -> None:
    """Bracket every library kernel launch with CUDA events (process-wide)."""
    _check(lib().arborx_profile_enable(1 if on else 0), "arborx_profile_enable")


def profile_report() -> dict:
    """{kernel name: (launches, total device ms)} since the last report; resets."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().arborx_profile_report(buf, len(buf)), "arborx_profile_report")
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def release_cached_memory() -> None:
    """Return the library's pooled device memory to the driver."""
    _check(lib().arborx_release_cached_memory(), "arborx_release_cached_memory")


def batched(points: torch.Tensor, queries: torch.Tensor, point_offsets, query_offsets, ks, **opts):
    """All clouds built and queried in one synchronous call (``arborx_batched``): (row_offsets int64
    [M+1], indices int32 [entries] local to each cloud, dist2 float32 [entries])."""
    import numpy as np
    p = _as_f32_cuda(points, 3, "points")
    q = _as_f32_cuda(queries, 3, "queries")
    po = np.ascontiguousarray(point_offsets, dtype=np.int64)
    qo = np.ascontiguousarray(query_offsets, dtype=np.int64)
    kv = np.ascontiguousarray(ks, dtype=np.int32)
    c = len(kv)
    if po.shape != (c + 1,) or qo.shape != (c + 1,):
        raise ValueError("offsets must have n_clouds + 1 entries")
    entries = int(sum((qo[i + 1] - qo[i]) * min(int(kv[i]), int(po[i + 1] - po[i])) for i in range(c)))
    row_off = torch.empty(int(qo[-1]) + 1, dtype=torch.int64, device=p.device)
    idx = torch.empty(max(entries, 1), dtype=torch.int32, device=p.device)
    d2 = torch.empty(max(entries, 1), dtype=torch.float32, device=p.device)
    o = default_opts(**opts)
    _check(lib().arborx_batched(c, po.ctypes.data_as(ctypes.c_void_p), qo.ctypes.data_as(ctypes.c_void_p),
                                kv.ctypes.data_as(ctypes.c_void_p), _ptr(p), _ptr(q), ctypes.byref(o), _stream(),
                                _ptr(row_off), _ptr(idx), _ptr(d2), entries), "arborx_batched")
    return row_off, idx[:entries], d2[:entries]


class Batch:
    """Many point clouds built and queried together (wraps an ``arborx_batch``).

    point_offsets / query_offsets: int64 [C+1] host sequences; ks: per-cloud k (1..32)."""

    def __init__(self, point_offsets, query_offsets, ks, **opts):
        import numpy as np
        self.point_offsets = np.ascontiguousarray(point_offsets, dtype=np.int64)
        self.query_offsets = np.ascontiguousarray(query_offsets, dtype=np.int64)
        self.ks = np.ascontiguousarray(ks, dtype=np.int32)
        c = len(self.ks)
        if self.point_offsets.shape != (c + 1,) or self.query_offsets.shape != (c + 1,):
            raise ValueError("offsets must have n_clouds + 1 entries")
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        _check(lib().arborx_batch_create(c, self.point_offsets.ctypes.data_as(ctypes.c_void_p),
                                         self.query_offsets.ctypes.data_as(ctypes.c_void_p),
                                         self.ks.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self.opts),
                                         _stream(), ctypes.byref(h)), "arborx_batch_create")
        self._h = h
        n, m, e = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().arborx_batch_entries(h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(e)), "arborx_batch_entries")
        self.n_points, self.n_queries, self.entries = n.value, m.value, e.value

    def run(self, points: torch.Tensor, queries: torch.Tensor, use_graph: bool = True, out=None,
            return_dist2: bool = True):
        """(row_offsets int64 [M+1], indices int32 [entries] local to each cloud, dist2 float32 [entries])."""
        p = _as_f32_cuda(points, 3, "points")
        q = _as_f32_cuda(queries, 3, "queries")
        if p.shape[0] != self.n_points or q.shape[0] != self.n_queries:
            raise ValueError("points / queries do not match the planned offsets")
        if out is None:
            out = (torch.empty(self.n_queries + 1, dtype=torch.int64, device=p.device),
                   torch.empty(max(self.entries, 1), dtype=torch.int32, device=p.device),
                   torch.empty(max(self.entries, 1), dtype=torch.float32, device=p.device) if return_dist2 else None)
        off, idx, d2 = out
        _check(lib().arborx_batch_run(self._h, _ptr(p), _ptr(q), int(bool(use_graph)), _stream(), _ptr(off),
                                      _ptr(idx), _ptr(d2)), "arborx_batch_run")
        return off, idx[: self.entries], (d2[: self.entries] if d2 is not None else None)

    def check(self) -> None:
        _check(lib().arborx_batch_check(self._h, _stream()), "arborx_batch_check")

    def destroy(self) -> None:
        if getattr(self, "_h", None) is not None:
            lib().arborx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
