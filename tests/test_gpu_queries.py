"""GPU parity of the traversals (Sec. 2.2) against the oracle's brute force:
spatial count-and-fill CSR rows as exact index sets, nearest rows exact in
(d^2, index) order with identical squared distances, edge cases, and the
closed-form lattice pins."""
import math

import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_helpers import assert_nearest_equal, assert_spatial_equal, dev, host

pytestmark = pytest.mark.gpu


def _ab():
    import paper_1908_11807_b300 as ab
    return ab


S1 = datagen.SEED0 + 1
CASES = {
    # small workload: 1e4 cube points, 1e4 queries, r for mean 10, k = 10
    "cube_1e4": lambda: (*datagen.workload("cube", 10_000, 10_000, S1), datagen.radius_for_mean(10_000, "cube")),
    "hollow_sphere_2e4": lambda: (*datagen.workload("hollow_sphere", 20_000, 5000, S1),
                                  datagen.radius_for_mean(20_000, "hollow_sphere")),
    "gaussian_2e4": lambda: (*datagen.workload("gaussian_mixture", 20_000, 5000, S1), 0.01),
    "duplicates": lambda: (np.repeat(datagen.cube(600, 3), 9, 0), datagen.cube(3001, 4), 0.03),
    "flat_plane": lambda: (np.concatenate([datagen.cube(8000, 5)[:, :2], np.full((8000, 1), 0.5, np.float32)], 1),
                           datagen.cube(2999, 6), 0.02),
    "collinear": lambda: (np.stack([np.linspace(0, 1, 5000, dtype=np.float32)] * 3, 1), datagen.cube(1000, 7), 0.01),
    "paper_filled": lambda: (datagen.paper_shape(20_000, "filled_cube", 8),
                             datagen.paper_shape(5000, "filled_sphere", 9), datagen.paper_radius(20_000)),
    "paper_hollow": lambda: (datagen.paper_shape(20_000, "hollow_cube", 10),
                             datagen.paper_shape(5000, "hollow_sphere", 11), datagen.paper_radius(20_000)),
    "boxes": lambda: (datagen.boxes(20_000, 12, half_max=0.01), datagen.cube(5000, 13), 0.01),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_spatial_matches_brute_force(name):
    ab = _ab()
    p, q, r = CASES[name]()
    bvh = ab.BVH(dev(p))
    og, ig = bvh.query_spatial(dev(q), r)
    bvh.check()
    oo, io = oracle.spatial_brute(p, q, r)
    assert_spatial_equal(host(og), host(ig), oo, io)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("k", [1, 10, 27, 50])
def test_nearest_matches_brute_force(name, k):
    ab = _ab()
    p, q, _ = CASES[name]()
    bvh = ab.BVH(dev(p))
    ig, dg = bvh.query_nearest(dev(q), k)
    bvh.check()
    io, do = oracle.nearest_brute(p, q, k)
    assert_nearest_equal(host(ig), host(dg), io, do)


@pytest.mark.parametrize("k", [2, 10, 16])
@pytest.mark.parametrize("shift", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_nearest_rows_into_unaligned_buffers(k, shift):
    # full-width rows go out two entries per store into 8-byte aligned outputs; caller buffers
    # that start 4 bytes off take the one-entry stores (the C interface, with offset pointers)
    ab = _ab()
    import ctypes
    import torch
    p, q = datagen.workload("cube", 3000, 700, 24)
    bvh = ab.BVH(dev(p))
    m = len(q)
    io, do = oracle.nearest_brute(p, q, k)
    idx = torch.full((m * k + 2,), 7, dtype=torch.int32, device="cuda")
    d2 = torch.full((m * k + 2,), 7.0, dtype=torch.float32, device="cuda")
    qd = dev(q)
    st = ab.lib().arborx_query_nearest(bvh.handle, ctypes.c_void_p(qd.data_ptr()), m, k, None, None, None,
                                       ctypes.c_void_p(idx.data_ptr() + 4 * shift[0]),
                                       ctypes.c_void_p(d2.data_ptr() + 4 * shift[1]))
    assert st == 0
    torch.cuda.synchronize()
    bvh.check()
    gi = host(idx)[shift[0]:shift[0] + m * k].reshape(m, k)
    gd = host(d2)[shift[1]:shift[1] + m * k].reshape(m, k)
    assert_nearest_equal(gi, gd, io, do)
    assert host(idx)[shift[0] + m * k] == 7 and (shift[0] == 0 or host(idx)[0] == 7)  # nothing outside
    assert host(d2)[shift[1] + m * k] == 7.0 and (shift[1] == 0 or host(d2)[0] == 7.0)


@pytest.mark.parametrize("k", [2, 3, 4, 5, 8, 9, 16, 17, 31, 32, 33, 64, 100, 256, 512])
def test_nearest_every_list_width(k):
    ab = _ab()
    p, q = datagen.workload("cube", 3000, 700, 21)
    bvh = ab.BVH(dev(p))
    ig, dg = bvh.query_nearest(dev(q), k)
    io, do = oracle.nearest_brute(p, q, k)
    assert_nearest_equal(host(ig), host(dg), io, do)


@pytest.mark.parametrize("build_method", [0, 1])
@pytest.mark.parametrize("name", ["cube_1e4", "duplicates", "flat_plane", "boxes", "paper_hollow"])
def test_subtree_emission_matches_brute_force(name, build_method):
    # radius and box rows with wholly contained subtrees taken from the kept leaf order (both
    # builders' node numberings), through the two-pass, one-pass and one-call forms, at the
    # workload's radius and at a radius holding hundreds of points per row
    ab = _ab()
    p, q, r = CASES[name]()
    bvh = ab.BVH(dev(p), keep_order=1, build_method=build_method)
    bvh.emit_subtrees(True)
    qd = dev(q)
    for rr in (r, 3 * r):
        oo, io = oracle.spatial_brute(p, q, rr)
        og, ig = bvh.query_spatial(qd, rr)
        assert_spatial_equal(host(og), host(ig), oo, io)
        og, ig = bvh.query_spatial(qd, rr, buffer_size=16)
        assert_spatial_equal(host(og), host(ig), oo, io)
        og, ig = bvh.query_spatial_async(qd, rr, buffer_size=8, capacity=max(int(oo[-1]), 1))
        assert_spatial_equal(host(og), host(ig)[:int(host(og)[-1])], oo, io)
        bvh.check()
    qb = np.concatenate([q - 2 * r, q + 2 * r], 1).astype(np.float32)
    ob, ib = oracle.intersects_brute(p, qb)
    og, ig = bvh.query_intersects(dev(qb), buffer_size=16)
    bvh.check()
    assert_spatial_equal(host(og), host(ig), ob, ib)


def test_subtree_emission_lattice_and_whole_tree():
    # lattice rows from integer enumeration, and a radius that contains the whole tree (the root
    # itself is emitted)
    ab = _ab()
    side = 24
    g = np.arange(side, dtype=np.float32)
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    sites = pts[np.random.default_rng(55).integers(0, len(pts), 3000)]
    bvh = ab.BVH(dev(pts), keep_order=1)
    bvh.emit_subtrees(True)
    for r in (1.0, 2.5, 4.0, 100.0):
        oo, io = oracle.spatial_brute(pts, sites, r)
        og, ig = bvh.query_spatial(dev(sites), r, buffer_size=32)
        bvh.check()
        assert_spatial_equal(host(og), host(ig), oo, io)


def test_subtree_emission_needs_the_kept_order():
    ab = _ab()
    bvh = ab.BVH(dev(datagen.cube(100, 56)))
    with pytest.raises(ab.ArborXError):
        bvh.emit_subtrees(True)
    bvh.emit_subtrees(False)


@pytest.mark.parametrize("k", [17, 20, 31, 32, 33])
def test_nearest_register_list_up_to_32(k):
    # knn_heap_from = 33 serves k <= 32 with a 32-entry register list instead of the heap
    ab = _ab()
    p, q = datagen.workload("cube", 3000, 700, 23)
    io, do = oracle.nearest_brute(p, q, k)
    for hf in (17, 33):
        bvh = ab.BVH(dev(p), knn_heap_from=hf)
        ig, dg = bvh.query_nearest(dev(q), k)
        bvh.check()
        assert_nearest_equal(host(ig), host(dg), io, do)


@pytest.mark.parametrize("opts", [dict(sort_queries=0), dict(key_bits=63), dict(build_method=1), dict(stack_smem=1),
                                  dict(stack_smem=64, block_size=64), dict(block_size=256, stack_smem=4),
                                  dict(block_size=32), dict(knn_anchor=0), dict(knn_anchor=0, build_method=1), dict(knn_anchor=2),
                                  dict(knn_anchor=2, build_method=1), dict(knn_anchor=3), dict(knn_anchor=3, stack_smem=1),
                                  dict(knn_anchor=3, build_method=1), dict(knn_anchor=3, stack_smem=2)])
def test_options_do_not_change_results(opts):
    ab = _ab()
    p, q = datagen.workload("hollow_sphere", 30_000, 4000, 22)
    r = datagen.radius_for_mean(30_000, "hollow_sphere") * 3
    bvh = ab.BVH(dev(p), **opts)
    og, ig = bvh.query_spatial(dev(q), r)
    kg, dg = bvh.query_nearest(dev(q), 10)
    bvh.check()
    oo, io = oracle.spatial_brute(p, q, r)
    assert_spatial_equal(host(og), host(ig), oo, io)
    ko, do = oracle.nearest_brute(p, q, 10)
    assert_nearest_equal(host(kg), host(dg), ko, do)


@pytest.mark.parametrize("build_method", [0, 1])
@pytest.mark.parametrize("k", [2, 5, 10, 27, 33])
def test_anchor_bound_with_ties_at_the_bound(k, build_method):
    # The tree's own initial bound (a subtree box's farthest corner) is exact only if a primitive
    # at exactly that distance still wins by index.  Clouds where it lands on ties: 40 copies of
    # each point (queries on and off the points), and an integer lattice whose box corners are
    # lattice points; both builders write the leaf counts the bound needs.  Every form: the two
    # walks, the first-descent form (whose stack compaction drops entries beyond the bound:
    # stack_smem 1 sends them through the local part), and the unbounded start.
    ab = _ab()
    base = datagen.cube(300, 50)
    dup = np.repeat(base, 40, 0)
    q = np.concatenate([base[:200], datagen.cube(500, 51)]).astype(np.float32)
    g = np.arange(12, dtype=np.float32)
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    ql = np.concatenate([lat[::7], lat[::11] + 0.5]).astype(np.float32)
    for p, qq in ((dup, q), (lat, ql)):
        ref_i, ref_d = oracle.nearest_brute(p, qq, k)
        for anchor, stack in ((1, 16), (2, 16), (3, 16), (3, 1), (3, 4), (0, 16)):
            bvh = ab.BVH(dev(p), build_method=build_method, knn_anchor=anchor, stack_smem=stack)
            ig, dg = bvh.query_nearest(dev(qq), k)
            bvh.check()
            assert_nearest_equal(host(ig), host(dg), ref_i, ref_d)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 9, 10, 11])
def test_small_trees_and_k_above_n(n):
    ab = _ab()
    import torch
    p = datagen.cube(n, 30 + n).reshape(n, 3)
    q = datagen.cube(257, 31)
    bvh = ab.BVH(dev(p) if n else torch.zeros((0, 3), device="cuda"))
    og, ig = bvh.query_spatial(dev(q), 0.4)
    oo, io = oracle.spatial_brute(p, q, 0.4)
    assert_spatial_equal(host(og), host(ig), oo, io)
    kg, dg, offs = bvh.query_nearest(dev(q), 10, with_offsets=True)
    ko, do = oracle.nearest_brute(p, q, 10)
    assert_nearest_equal(host(kg), host(dg), ko, do)
    kk = min(10, n)
    assert host(offs).tolist() == [j * kk for j in range(258)]


def test_query_edge_cases():
    ab = _ab()
    p = datagen.cube(5000, 40)
    q = np.concatenate([datagen.cube(1000, 41), np.array([[np.nan, 0, 0], [0, np.inf, 0], [-5, -5, -5],
                                                          [9, 9, 9], p[17], p[4000]], np.float32)])
    bvh = ab.BVH(dev(p))
    for r in (0.0, 1e-7, 0.05, 2.0, float("inf")):
        og, ig = bvh.query_spatial(dev(q), r)
        oo, io = oracle.spatial_brute(p, q, r)
        assert_spatial_equal(host(og), host(ig), oo, io)
    kg, dg = bvh.query_nearest(dev(q), 7)
    ko, do = oracle.nearest_brute(p, q, 7)
    assert_nearest_equal(host(kg), host(dg), ko, do)
    assert host(kg)[1000].tolist() == [-1] * 7
    # empty query set
    import torch
    og, ig = bvh.query_spatial(torch.zeros((0, 3), device="cuda"), 0.1)
    assert host(og).tolist() == [0]
    with pytest.raises(ab.ArborXError):
        bvh.query_spatial(dev(q), -1.0)
    with pytest.raises(ab.ArborXError):
        bvh.query_spatial(dev(q), float("nan"))
    with pytest.raises(ab.ArborXError):
        bvh.query_nearest(dev(q), 0)
    with pytest.raises(ab.ArborXError):
        bvh.query_nearest(dev(q), 513)


def test_adversarial_radius_edge_points():
    # points placed at exactly the FP32 radius from the query and one ulp
    # either side; pruning must never lose a result (conservative node boxes)
    ab = _ab()
    g = np.random.default_rng(50)
    q = np.array([[0.5, 0.5, 0.5]], np.float32)
    r = np.float32(0.1)
    dirs = g.standard_normal((3000, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    p = (0.5 + dirs * float(r)).astype(np.float32)
    p = np.concatenate([p, np.nextafter(p, np.float32(0.5)), np.nextafter(p, np.float32(2.0)),
                        datagen.cube(5000, 51)]).astype(np.float32)
    bvh = ab.BVH(dev(p))
    og, ig = bvh.query_spatial(dev(q), float(r))
    oo, io = oracle.spatial_brute(p, q, float(r))
    assert_spatial_equal(host(og), host(ig), oo, io)
    kg, dg = bvh.query_nearest(dev(q), 200)
    ko, do = oracle.nearest_brute(p, q, 200)
    assert_nearest_equal(host(kg), host(dg), ko, do)


def test_shared_query_order():
    ab = _ab()
    p, q = datagen.workload("cube", 50_000, 7000, 61)
    r = datagen.radius_for_mean(50_000, "cube")
    bvh = ab.BVH(dev(p))
    qd = dev(q)
    order = bvh.query_order(qd)
    og, ig = bvh.query_spatial(qd, r, order=order)
    kg, dg = bvh.query_nearest(qd, 10, order=order)
    oo, io = oracle.spatial_brute(p, q, r)
    assert_spatial_equal(host(og), host(ig), oo, io)
    ko, do = oracle.nearest_brute(p, q, 10)
    assert_nearest_equal(host(kg), host(dg), ko, do)
    # any permutation is a valid traversal order: results do not depend on it
    import torch
    rev = torch.flip(order, [0]).contiguous()
    og2, ig2 = bvh.query_spatial(qd, r, order=rev)
    assert_spatial_equal(host(og2), host(ig2), oo, io)


def test_spatial_split_calls_and_capacity():
    ab = _ab()
    import torch
    p, q = datagen.workload("cube", 20_000, 3000, 60)
    r = datagen.radius_for_mean(20_000, "cube")
    bvh = ab.BVH(dev(p))
    qd = dev(q)
    off = bvh.query_spatial_count(qd, r)
    nnz = int(off[-1].item())
    idx = torch.empty(nnz, dtype=torch.int32, device="cuda")
    bvh.query_spatial_fill(qd, r, off, idx)
    oo, io = oracle.spatial_brute(p, q, r)
    assert_spatial_equal(host(off), host(idx), oo, io)
    # too small a capacity: writes are skipped and reported
    small = torch.empty(nnz // 2, dtype=torch.int32, device="cuda")
    bvh.query_spatial_fill(qd, r, off, small)
    with pytest.raises(ab.ArborXError) as e:
        bvh.check()
    assert e.value.code == 5
    bvh.check()  # cleared


@pytest.mark.parametrize("side", [48])
def test_lattice_closed_form_counts_and_knn27(side):
    ab = _ab()
    pts = datagen.lattice(side)
    bvh = ab.BVH(dev(pts))
    g = np.random.default_rng(70)
    idx = g.integers(0, side ** 3, size=20_000)
    sites = np.stack([idx % side, (idx // side) % side, idx // (side * side)], 1)
    q = sites.astype(np.float32)
    golden = {1.0: 7, 2.5: 81, 4.0: 257}
    for r, want in golden.items():
        og, ig = bvh.query_spatial(dev(q), r)
        cnt = np.diff(host(og))
        R = math.ceil(r)
        interior = np.all((sites >= R) & (sites <= side - 1 - R), axis=1)
        assert np.all(cnt[interior] == want)
        # boundary sites: exact against brute force
        b = np.nonzero(~interior)[0][:2000]
        oo, io = oracle.spatial_brute(pts, q[b], r)
        og_h, ig_h = host(og), host(ig)
        sub_off = np.concatenate([[0], np.cumsum(cnt[b])])
        sub_idx = np.concatenate([ig_h[og_h[j]:og_h[j + 1]] for j in b])
        assert_spatial_equal(sub_off, sub_idx, oo, io)
    kg, dg = bvh.query_nearest(dev(q), 27)
    interior = np.all((sites >= 1) & (sites <= side - 2), axis=1)
    off3 = np.array([dx + side * dy + side * side * dz for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
    want = np.sort(idx[interior, None] + off3[None, :], axis=1)
    assert np.array_equal(np.sort(host(kg)[interior], axis=1), want)
    assert np.array_equal(np.unique(host(dg)[interior]), np.array([0, 1, 2, 3], np.float32))


@pytest.mark.parametrize("name", ["cube_1e4", "paper_hollow", "duplicates", "boxes"])
@pytest.mark.parametrize("bs", [1, 4, 10, 32, 4096])
def test_one_pass_spatial_matches_brute_force(name, bs):
    # 1P: one traversal keeps up to bs results per query; overflowing rows are refilled by a
    # second traversal; results equal the definition for any buffer estimate
    ab = _ab()
    p, q, r = CASES[name]()
    bvh = ab.BVH(dev(p))
    og, ig = bvh.query_spatial(dev(q), r, buffer_size=bs)
    bvh.check()
    oo, io = oracle.spatial_brute(p, q, r)
    assert_spatial_equal(host(og), host(ig), oo, io)


@pytest.mark.parametrize("bs", [80, 84, 128, 130])
@pytest.mark.parametrize("emit", [False, True])
def test_one_pass_wide_rows(bs, emit):
    # row buffers whose width is a multiple of 4 write hits four at a time (a separate kernel
    # form; 130 keeps one store per hit): wide rows that fit, that end in a partial group of 1..3
    # and that overflow into the second traversal, for radius and box rows, with and without
    # subtree emission
    ab = _ab()
    p = datagen.cube(20_000, 64)
    q = datagen.cube(1500, 65)
    r = datagen.radius_for_mean(20_000, "cube") * (100 / 10) ** (1 / 3)  # about 100 hits per row
    bvh = ab.BVH(dev(p), keep_order=int(emit))
    if emit:
        bvh.emit_subtrees(True)
    qd = dev(q)
    oo, io = oracle.spatial_brute(p, q, r)
    counts = np.diff(oo)
    assert (counts < bs).any() and (counts > bs).any()
    assert {int(c) % 4 for c in counts[counts < bs]} == {0, 1, 2, 3}
    og, ig = bvh.query_spatial(qd, r, buffer_size=bs)
    bvh.check()
    assert_spatial_equal(host(og), host(ig), oo, io)
    og, ig = bvh.query_spatial_async(qd, r, buffer_size=bs, capacity=int(oo[-1]))
    bvh.check()
    assert_spatial_equal(host(og), host(ig)[:int(host(og)[-1])], oo, io)
    half = np.float32(0.8 * r)
    qb = np.concatenate([q - half, q + half], 1).astype(np.float32)
    ob, ib = oracle.intersects_brute(p, qb)
    og, ig = bvh.query_intersects(dev(qb), buffer_size=bs)
    bvh.check()
    assert_spatial_equal(host(og), host(ig), ob, ib)


def test_one_pass_spatial_edge_cases():
    ab = _ab()
    import ctypes
    import torch
    p = datagen.cube(3000, 62)
    q = np.concatenate([datagen.cube(500, 63), np.array([[np.nan, 0, 0]], np.float32)])
    bvh = ab.BVH(dev(p))
    for r in (0.0, 0.2, float("inf")):
        og, ig = bvh.query_spatial(dev(q), r, buffer_size=8)
        oo, io = oracle.spatial_brute(p, q, r)
        assert_spatial_equal(host(og), host(ig), oo, io)
    og, ig = bvh.query_spatial(torch.zeros((0, 3), device="cuda"), 0.1, buffer_size=8)
    assert host(og).tolist() == [0] and ig.numel() == 0
    L = ab.lib()
    qd = dev(q)
    off = torch.empty(len(q) + 1, dtype=torch.int64, device="cuda")
    idx = torch.empty(10, dtype=torch.int32, device="cuda")
    # a fill without its count call is refused
    st = L.arborx_query_spatial_buffered_fill(bvh.handle, ctypes.c_void_p(qd.data_ptr()), len(q), ctypes.c_float(0.1),
                                             None, ctypes.c_void_p(off.data_ptr()), ctypes.c_void_p(idx.data_ptr()), 10)
    assert st == 6
    nnz = ctypes.c_int64(0)
    for bad in (0, 4097):
        st = L.arborx_query_spatial_buffered_count(bvh.handle, ctypes.c_void_p(qd.data_ptr()), len(q),
                                                   ctypes.c_float(0.1), bad, None, None,
                                                   ctypes.c_void_p(off.data_ptr()), ctypes.byref(nnz))
        assert st == 1


@pytest.mark.parametrize("name", ["cube_1e4", "paper_hollow", "duplicates", "boxes"])
@pytest.mark.parametrize("bs", [1, 10, 32])
def test_async_one_pass_spatial_matches(name, bs):
    # single-call one-pass query (no host round trip): same CSR as the two-pass query
    ab = _ab()
    p, q, r = CASES[name]()
    bvh = ab.BVH(dev(p))
    qd = dev(q)
    order = bvh.query_order(qd)
    off, idx = bvh.query_spatial_async(qd, r, buffer_size=bs, order=order, capacity=len(q) * 64)
    bvh.check()
    og, ig = bvh.query_spatial(qd, r, order=order)
    nnz = int(off[-1])
    assert np.array_equal(host(off), host(og)) and np.array_equal(host(idx)[:nnz], host(ig))
    oo, io = oracle.spatial_brute(p, q, r)
    assert_spatial_equal(host(off), host(idx)[:nnz], oo, io)


@pytest.mark.parametrize("bs", [10, 28])
def test_async_one_pass_many_scan_tiles(bs):
    # the single-call form scans and compacts in one kernel with a look-back over query tiles
    # (hundreds of them at 300k queries, so look-back windows of 32 tiles are crossed); its CSR
    # must equal the two-pass query's exactly (both bs % 4 forms of the row copy)
    ab = _ab()
    p = datagen.cube(200_000, 66)
    q = datagen.cube(300_000, 67)
    r = datagen.radius_for_mean(200_000, "cube")
    bvh = ab.BVH(dev(p))
    qd = dev(q)
    order = bvh.query_order(qd)
    og, ig = bvh.query_spatial(qd, r, order=order)
    nnz = int(ig.numel())
    off, idx = bvh.query_spatial_async(qd, r, buffer_size=bs, order=order, capacity=nnz)
    bvh.check()
    assert np.array_equal(host(off), host(og))
    assert np.array_equal(host(idx)[:nnz], host(ig))


@pytest.mark.parametrize("m", [1, 31, 2047, 2048, 2049, 4096, 6145])
def test_async_one_pass_scan_tile_edges(m):
    # query counts around the fused scan's 2048-query tiles: one partial tile, exactly full tiles,
    # one query into the next tile; offsets and rows equal the two-pass query's
    ab = _ab()
    p = datagen.cube(50_000, 68)
    q = datagen.cube(m, 69)
    r = datagen.radius_for_mean(50_000, "cube")
    bvh = ab.BVH(dev(p))
    qd = dev(q)
    og, ig = bvh.query_spatial(qd, r)
    nnz = int(ig.numel())
    for bs in (8, 10):
        off, idx = bvh.query_spatial_async(qd, r, buffer_size=bs, capacity=max(nnz, 1))
        bvh.check()
        assert np.array_equal(host(off), host(og))
        assert np.array_equal(host(idx)[:nnz], host(ig))


def test_async_one_pass_spatial_capacity_and_graph():
    ab = _ab()
    import torch
    p, q, r = CASES["cube_1e4"]()
    bvh = ab.BVH(dev(p))
    qd = dev(q)
    og, ig = bvh.query_spatial(qd, r)
    nnz = int(ig.numel())
    # too small a buffer: nothing past it is written, the overflow is reported, offsets stay complete
    off, idx = bvh.query_spatial_async(qd, r, buffer_size=8, capacity=nnz - 1)
    with pytest.raises(ab.ArborXError):
        bvh.check()
    assert np.array_equal(host(off), host(og))
    # exact capacity
    off, idx = bvh.query_spatial_async(qd, r, buffer_size=8, capacity=nnz)
    bvh.check()
    assert np.array_equal(host(idx)[:nnz], host(ig))
    # empty query set
    off0, _ = bvh.query_spatial_async(qd[:0], r, buffer_size=8, capacity=0)
    assert host(off0).tolist() == [0]
    # the call enqueues work only, so it can be captured in a CUDA graph and replayed
    order = bvh.query_order(qd)
    out_idx = torch.empty(len(q) * 16, dtype=torch.int32, device="cuda")
    bvh.query_spatial_async(qd, r, buffer_size=16, order=order, indices=out_idx)  # size the workspaces
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        goff, _ = bvh.query_spatial_async(qd, r, buffer_size=16, order=order, indices=out_idx)
    out_idx.fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    bvh.check()
    assert np.array_equal(host(goff), host(og))
    assert np.array_equal(host(out_idx)[:nnz], host(ig))


@pytest.mark.parametrize("name", ["cube_1e4", "paper_hollow", "duplicates", "boxes", "gaussian_2e4"])
@pytest.mark.parametrize("bs,k,given_order", [(10, 10, True), (32, 1, False), (28, 50, True)])
def test_spatial_nearest_in_one_call(name, bs, k, given_order):
    # the two traversals forked onto two streams give what the two calls give one after the
    # other, and the brute-force rows; later work on the caller's stream sees both results
    import torch
    ab = _ab()
    p, q, r = CASES[name]()
    bvh = ab.BVH(dev(p))
    qd = dev(q)
    order = bvh.query_order(qd) if given_order else None
    off, idx, kidx, kd2 = bvh.query_spatial_nearest(qd, r, k, buffer_size=bs, order=order, capacity=len(q) * 64)
    ksum = kidx.to(torch.int64).sum()  # enqueued on the caller's stream right after the call
    bvh.check()
    off_s, idx_s = bvh.query_spatial_async(qd, r, buffer_size=bs, order=order, capacity=len(q) * 64)
    ki_s, kd_s = bvh.query_nearest(qd, k, order=order)
    nnz = int(off[-1])
    assert np.array_equal(host(off), host(off_s))
    assert np.array_equal(host(idx)[:nnz], host(idx_s)[:nnz])
    assert np.array_equal(host(kidx), host(ki_s)) and np.array_equal(host(kd2), host(kd_s))
    assert int(ksum) == int(ki_s.to(torch.int64).sum())
    oo, io = oracle.spatial_brute(p, q, r)
    assert_spatial_equal(host(off), host(idx)[:nnz], oo, io)
    ko, do = oracle.nearest_brute(p, q, k)
    assert_nearest_equal(host(kidx), host(kd2), ko, do)


def test_spatial_nearest_in_one_call_edges_and_graph():
    import torch
    ab = _ab()
    p, q, r = CASES["cube_1e4"]()
    qd = dev(q)
    # empty query set, and an empty tree
    bvh = ab.BVH(dev(p))
    off, idx, kidx, kd2 = bvh.query_spatial_nearest(qd[:0], r, 10, buffer_size=8, capacity=0)
    assert host(off).tolist() == [0] and kidx.shape == (0, 10)
    empty = ab.BVH(torch.zeros((0, 3), device="cuda"))
    off, idx, kidx, kd2 = empty.query_spatial_nearest(qd, r, 5, buffer_size=8)
    empty.check()
    assert not host(off).any() and kidx.shape == (len(q), 0)
    # argument checks of both queries (buffer size, k), before any work is enqueued
    for bs, kk in ((0, 10), (4097, 10), (8, 0), (8, 513)):
        with pytest.raises(ab.ArborXError):
            bvh.query_spatial_nearest(qd, r, kk, buffer_size=bs)
    # more than n neighbours: rows of n
    small = ab.BVH(dev(p[:7]))
    _, _, kidx, kd2 = small.query_spatial_nearest(qd, r, 12, buffer_size=8)
    ko, do = oracle.nearest_brute(p[:7], q, 12)
    assert_nearest_equal(host(kidx), host(kd2), ko, do)
    # the first call creates the handle's second stream; later calls can be captured and replayed
    order = bvh.query_order(qd)
    out_idx = torch.empty(len(q) * 16, dtype=torch.int32, device="cuda")
    bvh.query_spatial_nearest(qd, r, 10, buffer_size=16, order=order, indices=out_idx)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        goff, _, gki, gkd = bvh.query_spatial_nearest(qd, r, 10, buffer_size=16, order=order, indices=out_idx)
    out_idx.fill_(-7)
    gki.fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    bvh.check()
    og, ig = bvh.query_spatial(qd, r, order=order)
    ki, kd = bvh.query_nearest(qd, 10, order=order)
    assert np.array_equal(host(goff), host(og)) and np.array_equal(host(out_idx)[:ig.numel()], host(ig))
    assert np.array_equal(host(gki), host(ki)) and np.array_equal(host(gkd), host(kd))
