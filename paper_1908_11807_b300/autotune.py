"""Autotuner for the query launch parameters.

Picks, for a workload class, the traversal block size, the number of stack
entries kept in shared memory, the walk form of the nearest query's tree bound,
the row-buffer estimate of the one-pass spatial query (0 = two passes) and the
margin of the learned bound, by timing the
candidates with CUDA events on a sample of the caller's queries
(``tune``, ``tune_margin``); the row-buffer width for one radius from the
distribution of its hit counts (``pick_buffer``); and the tiles of the batched
many-cloud query: block size, shared stack entries, queries per warp and the
heap/list threshold (``tune_batch``).  Choices of ``tune`` and ``tune_batch`` are cached in JSON
keyed by the workload class, in ``$ARBORX_TUNE_CACHE`` or
``~/.cache/arborx_b300/tune.json``.

Every candidate returns identical results (the launch parameters and the
buffer estimate only change speed), so the tuner times nothing but speed.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Iterable, Optional

import torch

from . import _binding as _b

DEFAULT_BLOCKS = (64, 128, 256)
DEFAULT_STACKS = (4, 8, 16)
DEFAULT_BUFFERS = (0, 16, 24, 32)
DEFAULT_MARGINS = (0.0, 0.1, 0.2, 0.35, 0.5, 0.7, 0.9)
DEFAULT_ANCHORS = (1, 2, 3)  # forms of the nearest query's tree bound (two walks, the first descent)


def cache_path() -> str:
    return os.environ.get("ARBORX_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "arborx_b300", "tune.json"))


def cache_key(n: int, k: int, tag: str) -> str:
    return f"n2^{int(round(math.log2(max(n, 1))))}/k{k}/{tag}"


def _load() -> Dict[str, dict]:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(key: str, value: dict) -> None:
    d = _load()
    d[key] = value
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _time(fn, reps: int = 3) -> float:
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


DEFAULT_ANCHOR = 3     # the library's own tree-bound form (the traversal's first descent)
ANCHOR_MARGIN = 0.01   # another form replaces it only when faster by more than this fraction


def pick_anchor(ms: dict) -> int:
    """The tree-bound form to use given the measured time of each: the library default unless
    another form is faster by more than ANCHOR_MARGIN, so that near-ties (forms within timing
    noise of each other) do not flip the choice from one tuning run to the next."""
    best = min(ms, key=ms.get)
    if DEFAULT_ANCHOR in ms and ms[best] >= (1.0 - ANCHOR_MARGIN) * ms[DEFAULT_ANCHOR]:
        return DEFAULT_ANCHOR
    return best


def tune(points: torch.Tensor, queries: torch.Tensor, radius: float, k: int, tag: str,
         blocks: Iterable[int] = DEFAULT_BLOCKS, stacks: Iterable[int] = DEFAULT_STACKS,
         buffers: Iterable[int] = DEFAULT_BUFFERS, params: Optional[torch.Tensor] = None,
         margins: Iterable[float] = DEFAULT_MARGINS, anchors: Iterable[int] = DEFAULT_ANCHORS,
         use_cache: bool = True) -> dict:
    """Return {"block_size", "stack_smem", "buffer_size", "margin", "knn_anchor", "ms"} for this
    workload class, timing the candidates on (points, queries) unless the cache has them.  The
    row-buffer widths timed are ``buffers`` and the widths ``pick_buffer`` derives from the
    queries' own hit counts."""
    key = cache_key(points.shape[0], k, tag)
    if use_cache:
        hit = _load().get(key)
        if hit is not None:
            return hit
    best = None
    for block in blocks:
        for stack in stacks:
            bvh = _b.BVH(points, block_size=block, stack_smem=stack)
            order = bvh.query_order(queries)
            ms_knn = _time(lambda: bvh.query_nearest(queries, k, order=order))
            ms_sp = _time(lambda: bvh.query_spatial(queries, radius, order=order))
            cand = (ms_knn + ms_sp, block, stack)
            if best is None or cand < best:
                best = cand
            bvh.destroy()
    _, block, stack = best
    # the walk form of the nearest query's tree bound, at the best launch parameters
    anchor_ms = {}
    for anchor in anchors:
        bvh = _b.BVH(points, block_size=block, stack_smem=stack, knn_anchor=anchor)
        order = bvh.query_order(queries)
        anchor_ms[anchor] = _time(lambda: bvh.query_nearest(queries, k, order=order))
        bvh.destroy()
    anchor = pick_anchor(anchor_ms)
    bvh = _b.BVH(points, block_size=block, stack_smem=stack, knn_anchor=anchor)
    order = bvh.query_order(queries)
    # the fixed widths and those of the query set's own hit counts (the median, 99th percentile and
    # largest count of a sample, rounded up to a multiple of 4), each timed in the single-call
    # one-pass form the step runs (0: the two-pass query)
    buf_ms = {}
    for bs in sorted(set(buffers) | buffer_candidates(bvh, queries, radius)):
        if bs == 0:
            buf_ms[bs] = _time(lambda: bvh.query_spatial(queries, radius, order=order))
        else:
            buf_ms[bs] = _time(lambda: bvh.query_spatial_async(queries, radius, buffer_size=bs, order=order))
    buf_best = min(buf_ms, key=buf_ms.get)
    margin = None
    if params is not None:
        margin = min((_time(lambda: bvh.query_nearest_learned(queries, k, params, mg, order=order)), mg)
                     for mg in margins)[1]
    bvh.destroy()
    out = {"block_size": block, "stack_smem": stack, "buffer_size": buf_best, "margin": margin,
           "knn_anchor": anchor, "ms_queries": round(best[0], 4)}
    if use_cache:
        _store(key, out)
    return out


def tune_margin(bvh, queries: torch.Tensor, k: int, params: torch.Tensor,
                margins: Iterable[float] = DEFAULT_MARGINS, objective: str = "time") -> float:
    """Margin of the learned bound that minimises the nearest query's cost on ``queries``, which
    should be a held-out draw of the workload's query distribution (not the queries that are
    then timed or checked).  ``objective`` is "time" (CUDA-event time) or "nodes" (internal nodes
    loaded by all passes, bounded pass and fallbacks together; needs a tree built with stats=1;
    deterministic for a given regressor)."""
    order = bvh.query_order(queries)
    if objective == "time":
        return min((_time(lambda: bvh.query_nearest_learned(queries, k, params, mg, order=order)), mg)
                   for mg in margins)[1]
    if objective != "nodes":
        raise ValueError("objective must be 'time' or 'nodes'")
    best = None
    for mg in margins:
        bvh.stats()
        bvh.query_nearest_learned(queries, k, params, mg, order=order)
        cand = (bvh.stats()["nearest_nodes"], mg)
        if cand[0] == 0:
            raise RuntimeError("objective 'nodes' needs a tree built with stats=1")
        best = cand if best is None or cand < best else best
    return best[1]


MAX_BUFFER_SIZE = 4096  # ARBORX_MAX_BUFFER_SIZE
BUFFER_BYTES_CAP = 1 << 32  # row buffers of at most 4 GB (m * width * 4 bytes)


def _round4(x: float) -> int:
    return max(4, 4 * int(math.ceil(x / 4.0)))


def _hit_stats(bvh, queries: torch.Tensor, radius: float, sample: int = 65536) -> dict:
    """Mean, median, 99th percentile and largest hit count over a strided sample of the queries."""
    step = max(1, int(queries.shape[0]) // sample)
    cnt = torch.diff(bvh.query_spatial_count(queries[::step].contiguous(), radius)).double()
    return {"mean": float(cnt.mean()), "p50": float(cnt.quantile(0.5)), "p99": float(cnt.quantile(0.99)),
            "max": float(cnt.max())}


def buffer_candidates(bvh, queries: torch.Tensor, radius: float, hits: Optional[dict] = None) -> set:
    """Row-buffer widths worth timing for this radius: two passes (0) and the median, 99th
    percentile and largest hit count of a sample, each rounded up to a multiple of 4, at most 4096
    and at most 4 GB of buffer."""
    m = int(queries.shape[0])
    if m == 0:
        return {0}
    hits = hits or _hit_stats(bvh, queries, radius)
    cap = min(MAX_BUFFER_SIZE, (BUFFER_BYTES_CAP // (4 * m)) // 4 * 4)
    cands = {0}
    if cap >= 4:
        cands |= {min(cap, _round4(hits[q])) for q in ("p50", "p99", "max")}
    return cands


def pick_buffer(bvh, queries: torch.Tensor, radius: float, order: Optional[torch.Tensor] = None,
                sample: int = 65536, reps: int = 2) -> dict:
    """Row-buffer width of the one-pass radius query for this radius (0 = two passes).

    A row that fits its buffer is written once; a row that overflows costs a second traversal,
    so the useful widths sit at the top of the hit-count distribution.  The candidates are two
    passes and the median, 99th percentile and largest count of a strided sample of the queries
    (each rounded up to a multiple of 4, at most 4096 and at most 4 GB of buffer); each is timed
    on all the queries and the fastest is returned with the timings and the sample's counts.  On a
    tree built with keep_order=1 the subtree-emitting traversal is timed at that width too, and
    left switched on for the tree (``emit_subtrees``) when it is faster."""
    m = int(queries.shape[0])
    if m == 0:
        return {"buffer_size": 0, "ms": {}, "hits": {}}
    hits = _hit_stats(bvh, queries, radius, sample)
    keep = bool(getattr(bvh.opts, "keep_order", 0))
    if keep:
        bvh.emit_subtrees(False)  # widths are timed with the walking traversal
    cands = buffer_candidates(bvh, queries, radius, hits)
    ms = {}
    for bs in sorted(cands):
        ms[bs] = round(_time(lambda: bvh.query_spatial(queries, radius, order=order, buffer_size=bs), reps), 4)
    best = min(ms, key=ms.get)
    out = {"buffer_size": best, "ms": ms, "hits": {k: round(v, 2) for k, v in hits.items()}, "emit_subtrees": False}
    if keep:
        # a tree that keeps its sorted leaf order can also take contained subtrees whole: timed at
        # the best width, kept on only if faster
        bvh.emit_subtrees(True)
        t = round(_time(lambda: bvh.query_spatial(queries, radius, order=order, buffer_size=best), reps), 4)
        out["emit_ms"] = t
        if t < ms[best]:
            out["emit_subtrees"] = True
        else:
            bvh.emit_subtrees(False)
    return out


DEFAULT_QPW = (32, 64, 128)


def batch_cache_key(n_points: int, ks) -> str:
    mix = "-".join(str(int(k)) for k in sorted(set(int(k) for k in ks)))
    return f"batch/n2^{int(round(math.log2(max(n_points, 1))))}/c{len(ks)}/k{mix}"


DEFAULT_HEAP_FROM = (17, 33)


def tune_batch(point_offsets, query_offsets, ks, points: torch.Tensor, queries: torch.Tensor,
               blocks: Iterable[int] = DEFAULT_BLOCKS, stacks: Iterable[int] = DEFAULT_STACKS,
               qpws: Iterable[int] = DEFAULT_QPW, heap_froms: Iterable[int] = DEFAULT_HEAP_FROM,
               anchors: Iterable[int] = DEFAULT_ANCHORS, use_cache: bool = True) -> dict:
    """Tiles of the batched many-cloud query (block size, shared stack entries, queries per warp,
    and the k from which candidates go to the shared-memory heap instead of a register list) for
    this batch shape, cached by (total points bucket, cloud count, k mix).  Times one graph replay
    of the whole batch per candidate: the heap threshold first (library tiles), then the walk form
    of the tree bound, then block and stack, then queries per warp.  Every candidate returns identical results."""
    key = batch_cache_key(int(points.shape[0]), ks)
    if use_cache:
        hit = _load().get(key)
        if hit is not None:
            return hit

    def run_ms(**opts):
        b = _b.Batch(point_offsets, query_offsets, ks, **opts)
        out = b.run(points, queries, use_graph=True)
        t = _time(lambda: b.run(points, queries, use_graph=True, out=(out[0], out[1], out[2])))
        b.destroy()
        return t

    hf = min((run_ms(knn_heap_from=h), h) for h in heap_froms)[1]
    an = pick_anchor({a: run_ms(knn_heap_from=hf, knn_anchor=a) for a in anchors})
    best = None
    for block in blocks:
        for stack in stacks:
            cand = (run_ms(block_size=block, stack_smem=stack, knn_heap_from=hf, knn_anchor=an), block, stack, 32)
            best = cand if best is None or cand < best else best
    for qpw in qpws:
        if qpw == 32:
            continue
        cand = (run_ms(block_size=best[1], stack_smem=best[2], queries_per_warp=qpw, knn_heap_from=hf,
                       knn_anchor=an), best[1], best[2], qpw)
        best = cand if cand < best else best
    out = {"block_size": best[1], "stack_smem": best[2], "queries_per_warp": best[3], "knn_heap_from": hf,
           "knn_anchor": an, "ms": round(best[0], 4)}
    if use_cache:
        _store(key, out)
    return out
