"""GPU parity of the box-intersection query (the spatial traversal of Sec. 2.2 with the
closed-box overlap test as its predicate) against the oracle: exact CSR rows as index sets
on point and box trees, every row-buffer width, both query orders, both hierarchy builders,
the closed-form lattice rows, edge cases (empty inputs, NaN, infinite and inverted bounds,
touching boxes), capacity overflow, graph capture, and the full-size 1e7-box tree."""
import math

import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_helpers import assert_spatial_equal, dev, host

pytestmark = pytest.mark.gpu

S1 = datagen.SEED0 + 1
S2 = datagen.SEED0 + 2


def _ab():
    import paper_1908_11807_b300 as ab
    return ab


def _lattice_boxes(side, m, seed):
    """Query boxes over a side^3 lattice: random real bounds, integer bounds, zero extents."""
    g = np.random.default_rng(seed)
    lo = g.uniform(-3, side + 2, (m, 3))
    qb = np.concatenate([lo, lo + g.uniform(0, 4, (m, 3))], 1)
    ints = g.integers(-1, side + 1, (m // 3, 3)).astype(np.float64)
    qb[: m // 3, :3] = ints
    qb[: m // 3, 3:] = ints + g.integers(0, 2, (m // 3, 3))
    return qb.astype(np.float32)


CASES = {
    # 1e4 cube points, cube queries sized for a mean of 10 hits
    "cube_points_1e4": lambda: (datagen.cube(10_000, S1),
                                datagen.query_cubes(10_000, S1, datagen.box_half_for_mean(10_000, prim_half_max=0.0))),
    # 2e4 boxes (half-widths up to 0.01) met by anisotropic query boxes
    "boxes_2e4": lambda: (datagen.boxes(20_000, S1, half_max=0.01),
                          datagen.boxes(5000, S1, half_max=0.03, stream=datagen.STREAM_QUERIES)),
    "lattice_24": lambda: (datagen.lattice(24), _lattice_boxes(24, 3000, 7)),
    "gaussian_2e4": lambda: (datagen.gaussian_mixture(20_000, S1),
                             datagen.boxes(4000, S1, half_max=0.02, stream=datagen.STREAM_QUERIES)),
    "duplicates": lambda: (np.repeat(datagen.cube(600, 3), 9, 0),
                           datagen.query_cubes(3001, 4, 0.04)),
    "flat_plane": lambda: (np.concatenate([datagen.cube(8000, 5)[:, :2], np.full((8000, 1), 0.5, np.float32)], 1),
                           datagen.query_cubes(2999, 6, 0.02)),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("buffer_size", [1, 16])
def test_intersects_matches_brute_force(name, buffer_size):
    ab = _ab()
    p, qb = CASES[name]()
    bvh = ab.BVH(dev(p))
    og, ig = bvh.query_intersects(dev(qb), buffer_size=buffer_size)
    bvh.check()
    oo, io = oracle.intersects_brute(p, qb)
    assert oo[-1] > 0
    assert_spatial_equal(host(og), host(ig), oo, io)


def test_intersects_lattice_rows_closed_form():
    # rows by integer enumeration (ceil of the low bound to floor of the high bound per axis)
    ab = _ab()
    side = 32
    p = datagen.lattice(side)
    qb = _lattice_boxes(side, 4000, 9)
    og, ig = ab.BVH(dev(p)).query_intersects(dev(qb), buffer_size=8)
    off, idx = host(og), host(ig)
    for j, b in enumerate(qb.astype(np.float64)):
        axes = []
        for a in range(3):
            lo, hi = max(math.ceil(b[a]), 0), min(math.floor(b[3 + a]), side - 1)
            axes.append(range(lo, hi + 1) if lo <= hi else range(0))
        want = sorted(x + side * y + side * side * z for z in axes[2] for y in axes[1] for x in axes[0])
        assert sorted(idx[off[j]:off[j + 1]].tolist()) == want, j


@pytest.mark.parametrize("opts", [dict(sort_queries=0), dict(key_bits=63), dict(build_method=1),
                                  dict(block_size=256, stack_smem=4)])
def test_intersects_options_give_the_same_rows(opts):
    ab = _ab()
    p, qb = CASES["boxes_2e4"]()
    ref = ab.BVH(dev(p))
    o1, i1 = ref.query_intersects(dev(qb))
    bvh = ab.BVH(dev(p), **opts)
    o2, i2 = bvh.query_intersects(dev(qb))
    bvh.check()
    assert_spatial_equal(host(o2), host(i2), host(o1), host(i1))


def test_intersects_order_is_a_permutation_and_optional():
    ab = _ab()
    import torch
    p, qb = CASES["cube_points_1e4"]()
    bvh = ab.BVH(dev(p))
    qd = dev(qb)
    order = bvh.query_order_boxes(qd)
    assert np.array_equal(np.sort(host(order)), np.arange(len(qb)))
    o1, i1 = bvh.query_intersects(qd, order=order)
    o2, i2 = bvh.query_intersects(qd)
    assert_spatial_equal(host(o1), host(i1), host(o2), host(i2))
    # a reversed order is also an order: same rows
    o3, i3 = bvh.query_intersects(qd, order=torch.flip(order, [0]).contiguous())
    assert_spatial_equal(host(o3), host(i3), host(o2), host(i2))
    # n = 0 or m < 2: the identity
    assert host(ab.BVH(dev(p[:0])).query_order_boxes(qd)).tolist() == list(range(len(qb)))
    assert host(bvh.query_order_boxes(qd[:1])).tolist() == [0]


def test_intersects_edge_cases():
    ab = _ab()
    inf, nan = np.inf, np.nan
    pts = datagen.lattice(4)
    qb = np.array([[nan, 0, 0, 3, 3, 3],
                   [-inf, -inf, -inf, inf, inf, inf],
                   [6, -1, -1, 4, 11, 11],
                   [1, 1, 1, 1, 1, 1],
                   [1, 1, 1, 2, 2, 2],
                   [3.5, 0, 0, 9, 9, 9],
                   [-5, -5, -5, -1e-7, 9, 9]], np.float32)
    for prims in (pts, np.array([[0, 0, 0, 10, 10, 10], [20, 20, 20, 30, 30, 30]], np.float32),
                  pts[:1], pts[:2]):
        bvh = ab.BVH(dev(prims))
        og, ig = bvh.query_intersects(dev(qb), buffer_size=2)
        bvh.check()
        oo, io = oracle.intersects_brute(prims, qb)
        assert_spatial_equal(host(og), host(ig), oo, io)
    # empty tree: every row empty; empty query set
    bvh = ab.BVH(dev(pts[:0]))
    og, ig = bvh.query_intersects(dev(qb))
    assert host(og).tolist() == [0] * (len(qb) + 1) and ig.numel() == 0
    bvh = ab.BVH(dev(pts))
    og, ig = bvh.query_intersects(dev(qb[:0]))
    assert host(og).tolist() == [0] and ig.numel() == 0
    with pytest.raises(ValueError):
        bvh.query_intersects(dev(pts))  # points are not boxes


def test_intersects_async_capacity_and_graph():
    ab = _ab()
    import torch
    p, qb = CASES["cube_points_1e4"]()
    bvh = ab.BVH(dev(p))
    qd = dev(qb)
    og, ig = bvh.query_intersects(qd)
    nnz = int(ig.numel())
    # too small a buffer: nothing past it is written, the overflow is reported, offsets stay complete
    off, idx = bvh.query_intersects_async(qd, buffer_size=4, capacity=nnz - 1)
    with pytest.raises(ab.ArborXError) as e:
        bvh.check()
    assert e.value.code == ab.ARBORX_EOVERFLOW
    assert np.array_equal(host(off), host(og))
    off, idx = bvh.query_intersects_async(qd, buffer_size=4, capacity=nnz)
    bvh.check()
    assert np.array_equal(host(idx)[:nnz], host(ig))
    # the call only enqueues work: capture it in a CUDA graph and replay
    order = bvh.query_order_boxes(qd)
    out_idx = torch.empty(len(qb) * 16, dtype=torch.int32, device="cuda")
    bvh.query_intersects_async(qd, buffer_size=16, order=order, indices=out_idx)  # size the workspaces
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        goff, _ = bvh.query_intersects_async(qd, buffer_size=16, order=order, indices=out_idx)
    out_idx.fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    bvh.check()
    assert np.array_equal(host(goff), host(og))
    nnz_g = int(host(goff)[-1])
    assert_spatial_equal(host(goff), host(out_idx)[:nnz_g], host(og), host(ig))


def test_intersects_boxes_1e7_every_row():
    # the 1e7-box tree (centres uniform, half-widths up to 1e-3) and 1e6 cube queries sized for a
    # mean of 10 hits: every row against the oracle's CPU BVH
    ab = _ab()
    n, m = 10_000_000, 1_000_000
    b = datagen.boxes(n, S2)
    qb = datagen.query_cubes(m, S2, datagen.box_half_for_mean(n))
    bvh = ab.BVH(dev(b), block_size=64, stack_smem=16, validate=0)
    og, ig = bvh.query_intersects(dev(qb), buffer_size=32)
    bvh.check()
    oo, io = oracle.CpuBVH(b).intersects(qb)
    assert 8 < oo[-1] / m < 12
    assert_spatial_equal(host(og), host(ig), oo, io)
    rows = np.random.default_rng(3).choice(m, 24, replace=False)  # and a few by brute force
    so, si = oracle.intersects_brute(b, qb[rows])
    go = host(og)
    gi = host(ig)
    for k, j in enumerate(rows):
        assert sorted(gi[go[j]:go[j + 1]].tolist()) == si[so[k]:so[k + 1]].tolist()
