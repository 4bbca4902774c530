"""CPU oracle for the LBVH search path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never imports it,
and it never imports the product library: the two share no code.

Contents (ArborX, arXiv 1908.11807):

* ``arborx_oracle.c`` (loaded through ctypes): scene box, Morton codes, brute
  force spatial / box / nearest queries (the definitions written out), a median-split
  CPU BVH (independent accelerated evaluator) and the FP64 checkers.
* ``tree_check``: invariants any LBVH over the given primitives must satisfy.
* ``mlp``: float64 forward / backward / Adam of the k-th-distance regressor.

Each function's docstring names the paper passage it follows.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

from . import build_oracle

POINTS = 0
BOXES = 1

_lib = None


def lib():
    """Load (building if needed) the compiled oracle."""
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        f32p = ctypes.POINTER(ctypes.c_float)
        i64 = ctypes.c_int64
        vp = ctypes.c_void_p
        L.orc_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_scene_box.restype = i64
        L.orc_scene_box.argtypes = [vp, i64, ctypes.c_int, vp]
        L.orc_morton.argtypes = [vp, i64, ctypes.c_int, vp, ctypes.c_int, vp]
        L.orc_spatial_count_brute.argtypes = [vp, i64, ctypes.c_int, vp, i64, ctypes.c_float, vp]
        L.orc_spatial_fill_brute.argtypes = [vp, i64, ctypes.c_int, vp, i64, ctypes.c_float, vp, vp]
        L.orc_nearest_brute.argtypes = [vp, i64, ctypes.c_int, vp, i64, ctypes.c_int, vp, vp]
        L.orc_intersects_count_brute.argtypes = [vp, i64, ctypes.c_int, vp, i64, vp]
        L.orc_intersects_fill_brute.argtypes = [vp, i64, ctypes.c_int, vp, i64, vp, vp]
        L.orc_bvh_intersects_count.argtypes = [vp, vp, i64, vp]
        L.orc_bvh_intersects_fill.argtypes = [vp, vp, i64, vp, vp]
        L.orc_bvh_build.restype = vp
        L.orc_bvh_build.argtypes = [vp, i64, ctypes.c_int]
        L.orc_bvh_free.argtypes = [vp]
        L.orc_bvh_nnodes.restype = i64
        L.orc_bvh_nnodes.argtypes = [vp]
        L.orc_bvh_spatial_count.argtypes = [vp, vp, i64, ctypes.c_float, vp]
        L.orc_bvh_spatial_fill.argtypes = [vp, vp, i64, ctypes.c_float, vp, vp]
        L.orc_bvh_nearest.argtypes = [vp, vp, i64, ctypes.c_int, vp, vp]
        L.orc_fp64_check_spatial.restype = i64
        L.orc_fp64_check_spatial.argtypes = [vp, i64, ctypes.c_int, vp, vp, i64, ctypes.c_float, vp, vp,
                                             ctypes.c_double, vp]
        L.orc_fp64_check_nearest.restype = i64
        L.orc_fp64_check_nearest.argtypes = [vp, i64, ctypes.c_int, vp, vp, i64, ctypes.c_int, vp,
                                             ctypes.c_double, vp]
        del f32p
        _lib = L
    return _lib


def threads() -> int:
    return lib().orc_threads()


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _kind_of(prims: np.ndarray) -> int:
    if prims.ndim != 2 or prims.shape[1] not in (3, 6):
        raise ValueError("primitives must be [n][3] points or [n][6] boxes")
    return POINTS if prims.shape[1] == 3 else BOXES


def scene_box(prims: np.ndarray) -> Tuple[np.ndarray, int]:
    """Scene bounding box (Sec. 2.1): min / max of every box corner.
    Returns (float32[6] = lo.xyz, hi.xyz, number of non-finite coordinates)."""
    prims = _c(prims, np.float32)
    out = np.zeros(6, np.float32)
    bad = lib().orc_scene_box(_p(prims), prims.shape[0], _kind_of(prims), _p(out))
    return out, int(bad)


def morton(prims: np.ndarray, sb: np.ndarray, key_bits: int = 30) -> np.ndarray:
    """Morton codes of the centroids scaled by the scene box (Sec. 2.1, Morton
    code step): 30-bit (10 bits / axis) or 63-bit (21 bits / axis), uint64."""
    prims = _c(prims, np.float32)
    sb = _c(sb, np.float32)
    bits = {30: 10, 63: 21}[key_bits]
    out = np.zeros(prims.shape[0], np.uint64)
    lib().orc_morton(_p(prims), prims.shape[0], _kind_of(prims), _p(sb), bits, _p(out))
    return out


def spatial_brute(prims: np.ndarray, queries: np.ndarray, r: float) -> Tuple[np.ndarray, np.ndarray]:
    """All primitives within distance r of each query (Sec. 2.2, spatial
    queries; closed ball, FP32 d^2 <= fl(r*r)), by brute force, as CSR
    (offsets int64 [m+1], indices int32, rows ascending)."""
    prims = _c(prims, np.float32)
    queries = _c(queries, np.float32).reshape(-1, 3)
    m = queries.shape[0]
    counts = np.zeros(m, np.int64)
    L = lib()
    L.orc_spatial_count_brute(_p(prims), prims.shape[0], _kind_of(prims), _p(queries), m, ctypes.c_float(r),
                              _p(counts))
    offsets = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    indices = np.zeros(int(offsets[-1]), np.int32)
    L.orc_spatial_fill_brute(_p(prims), prims.shape[0], _kind_of(prims), _p(queries), m, ctypes.c_float(r),
                             _p(offsets), _p(indices))
    return offsets, indices


def intersects_brute(prims: np.ndarray, qboxes: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """All primitives whose box meets each query box (lo.xyz, hi.xyz), closed
    intervals on every axis -- the spatial traversal of Sec. 2.2 with the box
    intersection test of Sec. 2 as its predicate -- by brute force, as CSR
    (offsets int64 [m+1], indices int32, rows ascending)."""
    prims = _c(prims, np.float32)
    qboxes = _c(qboxes, np.float32).reshape(-1, 6)
    m = qboxes.shape[0]
    counts = np.zeros(m, np.int64)
    L = lib()
    L.orc_intersects_count_brute(_p(prims), prims.shape[0], _kind_of(prims), _p(qboxes), m, _p(counts))
    offsets = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    indices = np.zeros(int(offsets[-1]), np.int32)
    L.orc_intersects_fill_brute(_p(prims), prims.shape[0], _kind_of(prims), _p(qboxes), m, _p(offsets),
                                _p(indices))
    return offsets, indices


def nearest_brute(prims: np.ndarray, queries: np.ndarray, k: int) -> Tuple[np.ndarray, np.ndarray]:
    """The min(k, n) nearest primitives of each query in (d^2, index) order
    (Sec. 2.2, nearest queries), by brute force: (indices int32 [m][kk],
    dist2 float32 [m][kk])."""
    prims = _c(prims, np.float32)
    queries = _c(queries, np.float32).reshape(-1, 3)
    m = queries.shape[0]
    kk = min(k, prims.shape[0])
    idx = np.full((m, kk), -1, np.int32)
    d2 = np.full((m, kk), np.inf, np.float32)
    if kk > 0 and m > 0:
        lib().orc_nearest_brute(_p(prims), prims.shape[0], _kind_of(prims), _p(queries), m, int(k), _p(idx), _p(d2))
    return idx, d2


class CpuBVH:
    """Median-split CPU BVH (leaf size 4): an evaluator independent of the LBVH,
    used to check large cases.  Results equal the brute-force definitions."""

    def __init__(self, prims: np.ndarray):
        self.prims = _c(prims, np.float32)
        self.n = self.prims.shape[0]
        self.kind = _kind_of(self.prims)
        self._h = lib().orc_bvh_build(_p(self.prims), self.n, self.kind)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_bvh_free(self._h)
            self._h = None

    def nnodes(self) -> int:
        return int(lib().orc_bvh_nnodes(self._h))

    def spatial_count(self, queries: np.ndarray, r: float) -> np.ndarray:
        queries = _c(queries, np.float32).reshape(-1, 3)
        counts = np.zeros(queries.shape[0], np.int64)
        lib().orc_bvh_spatial_count(self._h, _p(queries), queries.shape[0], ctypes.c_float(r), _p(counts))
        return counts

    def spatial(self, queries: np.ndarray, r: float) -> Tuple[np.ndarray, np.ndarray]:
        queries = _c(queries, np.float32).reshape(-1, 3)
        counts = self.spatial_count(queries, r)
        offsets = np.zeros(queries.shape[0] + 1, np.int64)
        np.cumsum(counts, out=offsets[1:])
        indices = np.zeros(int(offsets[-1]), np.int32)
        lib().orc_bvh_spatial_fill(self._h, _p(queries), queries.shape[0], ctypes.c_float(r), _p(offsets),
                                   _p(indices))
        return offsets, indices

    def intersects(self, qboxes: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
        """Box query (as ``intersects_brute``) through the median-split tree."""
        qboxes = _c(qboxes, np.float32).reshape(-1, 6)
        m = qboxes.shape[0]
        counts = np.zeros(m, np.int64)
        lib().orc_bvh_intersects_count(self._h, _p(qboxes), m, _p(counts))
        offsets = np.zeros(m + 1, np.int64)
        np.cumsum(counts, out=offsets[1:])
        indices = np.zeros(int(offsets[-1]), np.int32)
        lib().orc_bvh_intersects_fill(self._h, _p(qboxes), m, _p(offsets), _p(indices))
        return offsets, indices

    def nearest(self, queries: np.ndarray, k: int) -> Tuple[np.ndarray, np.ndarray]:
        queries = _c(queries, np.float32).reshape(-1, 3)
        m = queries.shape[0]
        kk = min(k, self.n)
        idx = np.full((m, kk), -1, np.int32)
        d2 = np.full((m, kk), np.inf, np.float32)
        if kk > 0 and m > 0:
            lib().orc_bvh_nearest(self._h, _p(queries), m, int(k), _p(idx), _p(d2))
        return idx, d2


def fp64_check_spatial(prims, queries, r, offsets, indices, sample, rel=1e-6) -> Tuple[int, int]:
    """FP64 re-check of a spatial result on the sampled queries: returns
    (intolerable disagreements, tolerated ones within rel * r of the radius)."""
    prims = _c(prims, np.float32)
    queries = _c(queries, np.float32).reshape(-1, 3)
    sample = _c(sample, np.int64)
    offsets = _c(offsets, np.int64)
    indices = _c(indices, np.int32)
    tol = np.zeros(1, np.int64)
    bad = lib().orc_fp64_check_spatial(_p(prims), prims.shape[0], _kind_of(prims), _p(queries), _p(sample),
                                       sample.shape[0], ctypes.c_float(r), _p(offsets), _p(indices),
                                       ctypes.c_double(rel), _p(tol))
    return int(bad), int(tol[0])


def fp64_check_nearest(prims, queries, k, indices, sample, rel=1e-6) -> Tuple[int, int]:
    """FP64 re-check of a nearest result [m][min(k,n)] on the sampled queries:
    returns (intolerable disagreements, tolerated ones within rel * d_k)."""
    prims = _c(prims, np.float32)
    queries = _c(queries, np.float32).reshape(-1, 3)
    sample = _c(sample, np.int64)
    indices = _c(indices, np.int32)
    tol = np.zeros(1, np.int64)
    bad = lib().orc_fp64_check_nearest(_p(prims), prims.shape[0], _kind_of(prims), _p(queries), _p(sample),
                                       sample.shape[0], int(k), _p(indices), ctypes.c_double(rel), _p(tol))
    return int(bad), int(tol[0])


def rows_as_sets_equal(off_a, idx_a, off_b, idx_b) -> Optional[int]:
    """None if every CSR row holds the same set of indices, else the first
    differing row.  Rows are compared after sorting (row order is not part of
    the result)."""
    off_a = np.asarray(off_a, np.int64)
    off_b = np.asarray(off_b, np.int64)
    if off_a.shape != off_b.shape:
        return 0
    cnt_a = np.diff(off_a)
    cnt_b = np.diff(off_b)
    diff = np.nonzero(cnt_a != cnt_b)[0]
    if diff.size:
        return int(diff[0])
    m = cnt_a.shape[0]
    row = np.repeat(np.arange(m, dtype=np.int64), cnt_a)
    ka = np.lexsort((np.asarray(idx_a, np.int64), row))
    kb = np.lexsort((np.asarray(idx_b, np.int64), row))
    sa = np.asarray(idx_a, np.int64)[ka]
    sb = np.asarray(idx_b, np.int64)[kb]
    bad = np.nonzero(sa != sb)[0]
    if bad.size:
        return int(row[bad[0]])
    return None
