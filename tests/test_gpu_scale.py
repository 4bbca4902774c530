"""Full-size parity: the paper-scale workloads (1e6 and 1e7 points in a
uniform cube and on a hollow sphere, 1e7 boxes) and the 256^3 lattice, in the
launch configuration the benchmark uses.  Results are checked on sampled
queries against the oracle's CPU BVH (exact rows) and FP64 checker, and at
every query through size-independent properties (closed-form lattice counts,
CSR structure, row order)."""
import functools
import math

import numpy as np
import pytest

import datagen
import oracle
from oracle import tree_check
from tests.gpu_helpers import assert_nearest_equal, assert_spatial_equal, dev, host

pytestmark = pytest.mark.gpu

S2 = datagen.SEED0 + 2
S3 = datagen.SEED0 + 3


def _ab():
    import paper_1908_11807_b300 as ab
    return ab


def _sub_csr(off, idx, rows):
    cnt = off[rows + 1] - off[rows]
    sub_off = np.concatenate([[0], np.cumsum(cnt)])
    sub_idx = np.concatenate([idx[off[j]:off[j + 1]] for j in rows]) if len(rows) else np.zeros(0, np.int32)
    return sub_off, sub_idx


# the benchmark's step: fixed launch parameters (block 64, 16 shared stack entries), asynchronous
# validation, one query order shared by a one-pass spatial query (32-slot rows) and the k-NN query
BENCH_LAUNCH = dict(block_size=64, stack_smem=16, validate=0)
BENCH_BUFFER = 32


@pytest.mark.parametrize("dist,n", [("cube", 1_000_000), ("hollow_sphere", 1_000_000),
                                    ("cube", 10_000_000), ("hollow_sphere", 10_000_000)])
def test_paper_scale_sampled_exact(dist, n):
    ab = _ab()
    m = 1_000_000
    p, q = datagen.workload(dist, n, m, S2)
    r = datagen.radius_for_mean(n, dist)
    bvh = ab.BVH(dev(p), **BENCH_LAUNCH)
    qd = dev(q)
    order = bvh.query_order(qd)
    og, ig = bvh.query_spatial(qd, r, order=order, buffer_size=BENCH_BUFFER)
    kg, dg = bvh.query_nearest(qd, 10, order=order)
    bvh.check()
    # the two-pass scheme returns the same CSR arrays (same traversal order)
    og2, ig2 = bvh.query_spatial(qd, r, order=order)
    assert bool((og2 == og).all()) and bool((ig2 == ig).all())
    # the benchmark step's form (both queries in one call, the k-NN traversal on a second
    # stream) returns the same arrays as the two calls
    oc, ic, kc, dc = bvh.query_spatial_nearest(qd, r, 10, buffer_size=BENCH_BUFFER, order=order,
                                               capacity=int(ig.numel()))
    bvh.check()
    assert bool((oc == og).all()) and bool((ic[:ig.numel()] == ig).all())
    assert bool((kc == kg).all()) and bool((dc == dg).all())
    del oc, ic, kc, dc
    og, ig, kg, dg = host(og), host(ig), host(kg), host(dg)
    # every row: CSR well formed, nearest rows sorted by (d2, index), distinct
    assert og[0] == 0 and np.all(np.diff(og) >= 0) and og[-1] == ig.size
    assert ig.min() >= 0 and ig.max() < n
    assert np.all((np.diff(dg, axis=1) > 0) | ((np.diff(dg, axis=1) == 0) & (np.diff(kg, axis=1) > 0)))
    mean = ig.size / m
    if dist == "cube":
        assert 9.0 < mean < 11.0  # the radius was chosen for a mean of 10 neighbours
    # sampled rows exact against the oracle's CPU BVH
    g = np.random.default_rng(n)
    rows = np.sort(g.choice(m, 20_000, replace=False))
    cpu = oracle.CpuBVH(p)
    oo, io = cpu.spatial(q[rows], r)
    so, si = _sub_csr(og, ig, rows)
    assert_spatial_equal(so, si, oo, io)
    ko, do = cpu.nearest(q[rows], 10)
    assert_nearest_equal(kg[rows], dg[rows], ko, do)
    # FP64 checker on a smaller sample: disagreements only at the 1e-6 edge
    few = rows[:64]
    bad, _ = oracle.fp64_check_spatial(p, q, r, og, ig, few)
    assert bad == 0
    bad, _ = oracle.fp64_check_nearest(p, q, 10, kg, few)
    assert bad == 0


def test_boxes_1e7_build_and_queries():
    ab = _ab()
    n = 10_000_000
    b = datagen.boxes(n, S2)
    bvh = ab.BVH(dev(b), keep_order=1)
    rec, scene, codes, perm = bvh.export_tree(order=True)
    bvh.check()
    sb, _ = oracle.scene_box(b)
    assert np.array_equal(host(scene), sb)
    tree_check.check_lbvh(host(rec), b, host(perm), host(codes).view(np.uint64), sb, check_split=False)
    del rec, codes, perm
    q = datagen.cube(200_000, S2, datagen.STREAM_QUERIES)
    og, ig = bvh.query_spatial(dev(q), 1e-3)
    kg, dg = bvh.query_nearest(dev(q), 10)
    rows = np.arange(0, 200_000, 50)
    cpu = oracle.CpuBVH(b)
    oo, io = cpu.spatial(q[rows], 1e-3)
    so, si = _sub_csr(host(og), host(ig), rows)
    assert_spatial_equal(so, si, oo, io)
    ko, do = cpu.nearest(q[rows], 10)
    assert_nearest_equal(host(kg)[rows], host(dg)[rows], ko, do)


def _lattice_counts(sites, side, r):
    """Closed form with clipping: number of integer offsets in the ball whose
    target stays inside the grid, per site."""
    R = int(math.ceil(r))
    cnt = np.zeros(len(sites), np.int64)
    for dx in range(-R, R + 1):
        for dy in range(-R, R + 1):
            for dz in range(-R, R + 1):
                if dx * dx + dy * dy + dz * dz <= r * r:
                    t = sites + np.array([dx, dy, dz])
                    cnt += np.all((t >= 0) & (t < side), axis=1)
    return cnt


def test_lattice_256_all_sites():
    ab = _ab()
    side = datagen.LATTICE_SIDE
    pts = datagen.lattice(side)
    bvh = ab.BVH(dev(pts))
    idx, q = datagen.lattice_sites(1_000_000, S3)
    sites = q.astype(np.int64)
    qd = dev(q)
    for r, interior_count in ((1.0, 7), (2.5, 81), (4.0, 257)):
        og, ig = bvh.query_spatial(qd, r)
        cnt = np.diff(host(og))
        assert np.array_equal(cnt, _lattice_counts(sites, side, r))
        R = int(math.ceil(r))
        interior = np.all((sites >= R) & (sites <= side - 1 - R), axis=1)
        assert np.all(cnt[interior] == interior_count)
        # index sets of sampled sites equal the enumerated offsets
        og_h, ig_h = host(og), host(ig)
        for j in np.random.default_rng(int(r * 10)).choice(len(q), 300, replace=False):
            sx, sy, sz = sites[j]
            want = sorted(int(x + side * y + side * side * z)
                          for x in range(sx - R, sx + R + 1) for y in range(sy - R, sy + R + 1)
                          for z in range(sz - R, sz + R + 1)
                          if 0 <= x < side and 0 <= y < side and 0 <= z < side
                          and (x - sx) ** 2 + (y - sy) ** 2 + (z - sz) ** 2 <= r * r)
            assert sorted(ig_h[og_h[j]:og_h[j + 1]].tolist()) == want
    kg, dg = bvh.query_nearest(qd, 27)
    kg, dg = host(kg), host(dg)
    interior = np.all((sites >= 1) & (sites <= side - 2), axis=1)
    off3 = np.array([dx + side * dy + side * side * dz for dz in (-1, 0, 1) for dy in (-1, 0, 1)
                     for dx in (-1, 0, 1)])
    want = np.sort(idx[interior, None] + off3[None, :], axis=1)
    assert np.array_equal(np.sort(kg[interior], axis=1), want)
    # boundary sites (ties in the cut shell): exact against brute force
    bnd = np.nonzero(~interior)[0][:150]
    ko, do = oracle.nearest_brute(pts, q[bnd], 27)
    assert_nearest_equal(kg[bnd], dg[bnd], ko, do)


@functools.lru_cache(maxsize=1)
def _mixture_full():
    # the learned-bound workload at its stated size: 1e7 mixture points, 1e7 queries, 1e6 training
    # queries, and a held-out draw of 1e7 queries for the margin
    seed = datagen.SEED0 + 5
    n = m = 10_000_000
    p = datagen.gaussian_mixture(n, seed)
    q = datagen.gaussian_mixture(m, seed, datagen.STREAM_QUERIES)
    qt = datagen.gaussian_mixture(1_000_000, seed, datagen.STREAM_TRAIN)
    qh = datagen.gaussian_mixture(m, seed, datagen.STREAM_HELDOUT)
    return p, q, qt, qh


@functools.lru_cache(maxsize=1)
def _mixture_cpu_bvh():
    return oracle.CpuBVH(_mixture_full()[0])


@pytest.mark.parametrize("k", [10, 50])
def test_learned_full_size_exact_and_faster(k):
    # 1e7 points, all 1e7 queries, the regressor trained by the library on 1e6 exact labels, the
    # margin tuned on a held-out draw: every row equals the plain traversal's, sampled rows equal
    # the oracle's CPU BVH, and the learned query is faster than the plain one
    ab = _ab()
    import torch
    from oracle import mlp
    from paper_1908_11807_b300 import autotune
    p, q, qt, qh = _mixture_full()
    m = q.shape[0]
    bvh = ab.BVH(dev(p), **BENCH_LAUNCH)
    params = dev(mlp.he_init(np.random.default_rng(5)).astype(np.float32))
    loss = host(bvh.mlp_train(params, dev(qt), k, epochs=200, batch=2048, lr=5e-3, lr_final=1e-5))
    assert loss[-1] < 0.5 * loss[0]
    margin = autotune.tune_margin(bvh, dev(qh), k, params)
    qd = dev(q)
    order = bvh.query_order(qd)
    li, ld, fb = bvh.query_nearest_learned(qd, k, params, margin, order=order, count_fallbacks=True)
    pi, pd = bvh.query_nearest(qd, k, order=order)
    bvh.check()
    assert torch.equal(li, pi) and torch.equal(ld, pd)
    assert 0 <= fb < m // 4
    rows = np.sort(np.random.default_rng(7 + k).choice(m, 10_000, replace=False))
    ko, do = _mixture_cpu_bvh().nearest(q[rows], k)
    assert_nearest_equal(host(li)[rows], host(ld)[rows], ko, do)
    del li, ld, pi, pd

    def best_ms(fn):
        fn()
        torch.cuda.synchronize()
        t = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
        return min(t)

    learned_ms = best_ms(lambda: bvh.query_nearest_learned(qd, k, params, margin, order=order))
    plain = {}
    for anchor in (0, 1, 2, 3):  # the paper's unbounded start, and the three forms of the tree bound
        t = ab.BVH(dev(p), knn_anchor=anchor, **BENCH_LAUNCH)
        plain[anchor] = best_ms(lambda: t.query_nearest(qd, k, order=order))
        t.destroy()
    print(f"k={k}: learned {learned_ms:.2f} ms (margin {margin}, fallbacks {fb / m:.4f}); plain from an "
          f"unbounded start {plain[0]:.2f} ms ({plain[0] / learned_ms:.3f}x), with the far-corner tree bound "
          f"{plain[1]:.2f} ms ({plain[1] / learned_ms:.3f}x), with the query-path tree bound {plain[2]:.2f} ms "
          f"({plain[2] / learned_ms:.3f}x), with the first-descent tree bound {plain[3]:.2f} ms "
          f"({plain[3] / learned_ms:.3f}x)")
    # what the trained network gains over the method without it (the paper's traversal, which
    # starts unbounded), at identical results: measured 1.35x (k = 10) and 1.16x (k = 50); the
    # thresholds keep about two thirds of it so that clock noise between best-of-three timings cannot
    # flip the result.  The tree's own bound (knn_anchor = 2 or 3) reaches the same on this workload,
    # which is reported, not asserted.
    assert plain[0] / learned_ms >= {10: 1.2, 50: 1.08}[k]
    bvh.destroy()


@functools.lru_cache(maxsize=1)
def _large_cloud(n, m):
    return datagen.cube(n, S2 + 7), datagen.cube(m, S2 + 7, datagen.STREAM_QUERIES)


@pytest.mark.parametrize("key_bits", [30, 63])
def test_large_n_sampled_exact(key_bits):
    # 2^27 - 3 points (13x the benchmark's tree, a ragged last sort tile and Apetrei chunk):
    # sampled rows of both queries exact against the oracle's brute force
    ab = _ab()
    n, m = (1 << 27) - 3, 100_000
    p, q = _large_cloud(n, m)
    r = datagen.radius_for_mean(n, "cube")
    bvh = ab.BVH(dev(p), key_bits=key_bits, **BENCH_LAUNCH)
    qd = dev(q)
    order = bvh.query_order(qd)
    og, ig = bvh.query_spatial(qd, r, order=order, buffer_size=BENCH_BUFFER)
    kg, dg = bvh.query_nearest(qd, 10, order=order)
    bvh.check()
    og, ig, kg, dg = host(og), host(ig), host(kg), host(dg)
    assert og[0] == 0 and np.all(np.diff(og) >= 0) and og[-1] == ig.size and 9.0 < ig.size / m < 11.0
    rows = np.sort(np.random.default_rng(key_bits).choice(m, 64, replace=False))
    oo, io = oracle.spatial_brute(p, q[rows], r)
    so, si = _sub_csr(og, ig, rows)
    assert_spatial_equal(so, si, oo, io)
    ko, do = oracle.nearest_brute(p, q[rows], 10)
    assert_nearest_equal(kg[rows], dg[rows], ko, do)


def test_more_than_2_31_results():
    # 2.4e9 CSR entries (9.6 GB of indices): 64-bit offsets end to end, rows exact on a sample
    ab = _ab()
    import torch
    n, m = 10_000_000, 200_000
    p = datagen.cube(n, S2 + 8)
    q = datagen.cube(m, S2 + 8, datagen.STREAM_QUERIES)
    r = datagen.radius_for_mean(n, "cube") * (12_000 / 10) ** (1 / 3)  # about 12 000 results per query
    bvh = ab.BVH(dev(p))
    qd = dev(q)
    offsets = bvh.query_spatial_count(qd, r)
    total = int(offsets[-1])
    assert total > (1 << 31)
    indices = torch.empty(total, dtype=torch.int32, device="cuda")
    bvh.query_spatial_fill(qd, r, offsets, indices)
    bvh.check()
    off = host(offsets)
    assert off.dtype == np.int64 and off[0] == 0 and np.all(np.diff(off) >= 0) and off[-1] == total
    rows = np.array([0, 1, m // 2, m - 2, m - 1] + list(np.random.default_rng(8).choice(m, 11, replace=False)))
    oo, io = oracle.spatial_brute(p, q[rows], r)
    got = [host(indices[int(off[j]):int(off[j + 1])]) for j in rows]
    so = np.concatenate([[0], np.cumsum([len(x) for x in got])])
    assert_spatial_equal(so, np.concatenate(got), oo, io)
