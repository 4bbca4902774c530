"""In-place rebuild (arborx_rebuild): the tree over new coordinates of the same primitives equals
a fresh build over them record for record, queries on it equal the oracle's, its options
(63-bit codes, the Karras hierarchy, boxes) carry over, and a rebuild plus queries captured once
in a CUDA graph follows coordinates that change between replays (a time-stepping loop)."""
import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_helpers import assert_nearest_equal, assert_spatial_equal, dev, host

pytestmark = pytest.mark.gpu


def _ab():
    import paper_1908_11807_b300 as ab
    return ab


@pytest.mark.parametrize("opts", [dict(), dict(key_bits=63), dict(build_method=1), dict(keep_order=1)])
def test_rebuild_equals_a_fresh_build(opts):
    ab = _ab()
    p0 = datagen.cube(20_000, 1)
    p1 = datagen.cube(20_000, 2)
    bvh = ab.BVH(dev(p0), **opts)
    for p in (p1, p0, p1):  # rebuild twice over the same shape, then reuse the kept scratch
        bvh.rebuild(dev(p))
        bvh.check()
        fresh = ab.BVH(dev(p), **opts)
        r1, s1, c1, q1 = bvh.export_tree(order=bool(opts.get("keep_order")))
        r2, s2, c2, q2 = fresh.export_tree(order=bool(opts.get("keep_order")))
        # defined parts of the layout: record 0 and the child records, fields lo.xyz, enc, hi.xyz
        # (record 1 is reserved and aux unspecified)
        a, b = host(r1)[:, :7], host(r2)[:, :7]
        a, b = np.delete(a, 1, axis=0), np.delete(b, 1, axis=0)
        bad = np.nonzero(np.any(a.view(np.int32) != b.view(np.int32), axis=1))[0]
        assert bad.size == 0, (bad[:5], a[bad[:2]], b[bad[:2]])
        assert np.array_equal(host(s1), host(s2))
        if opts.get("keep_order"):
            assert np.array_equal(host(c1), host(c2)) and np.array_equal(host(q1), host(q2))
    q = datagen.cube(2000, 3)
    og, ig = bvh.query_spatial(dev(q), 0.03)
    oo, io = oracle.spatial_brute(p1, q, 0.03)
    assert_spatial_equal(host(og), host(ig), oo, io)


def test_rebuild_boxes_and_bad_arguments():
    ab = _ab()
    b0 = datagen.boxes(5000, 4, half_max=0.01)
    b1 = datagen.boxes(5000, 5, half_max=0.01)
    bvh = ab.BVH(dev(b0))
    bvh.rebuild(dev(b1))
    q = datagen.cube(500, 6)
    ki, kd = bvh.query_nearest(dev(q), 10)
    io, do = oracle.nearest_brute(b1, q, 10)
    assert_nearest_equal(host(ki), host(kd), io, do)
    with pytest.raises(ValueError):
        bvh.rebuild(dev(b1[:10]))  # another number of primitives
    with pytest.raises(ValueError):
        bvh.rebuild(dev(datagen.cube(5000, 7)))  # points for a box tree


def test_rebuild_and_queries_in_one_graph_follow_moving_points():
    ab = _ab()
    import torch
    n, m, r, k = 30_000, 3000, 0.03, 8
    frames = [datagen.cube(n, 10 + t) for t in range(3)]
    q = datagen.cube(m, 20)
    pts = dev(frames[0])
    qd = dev(q)
    bvh = ab.BVH(pts, validate=0)
    rows = torch.empty(m * 64, dtype=torch.int32, device="cuda")
    # first calls size every workspace; the graph then allocates nothing of the library's
    bvh.rebuild(pts)
    order = bvh.query_order(qd)
    bvh.query_spatial_async(qd, r, buffer_size=16, order=order, indices=rows)
    bvh.query_nearest(qd, k, order=order)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bvh.rebuild(pts)
        gorder = bvh.query_order(qd)
        goff, _ = bvh.query_spatial_async(qd, r, buffer_size=16, order=gorder, indices=rows)
        gidx, gd2 = bvh.query_nearest(qd, k, order=gorder)
    for p in frames:  # new coordinates in the same buffer, then one replay per time step
        pts.copy_(dev(p))
        g.replay()
        torch.cuda.synchronize()
        bvh.check()
        oo, io = oracle.spatial_brute(p, q, r)
        off = host(goff)
        assert_spatial_equal(off, host(rows)[:int(off[-1])], oo, io)
        eo, ed = oracle.nearest_brute(p, q, k)
        assert_nearest_equal(host(gidx), host(gd2), eo, ed)


def test_rebuild_rejects_a_non_finite_coordinate_and_recovers():
    ab = _ab()
    p0 = datagen.cube(4000, 30)
    bad = p0.copy()
    bad[1234, 1] = np.nan
    bvh = ab.BVH(dev(p0))
    with pytest.raises(ab.ArborXError) as e:
        bvh.rebuild(dev(bad))
    assert e.value.code == ab.ARBORX_EINVAL
    p1 = datagen.cube(4000, 31)
    bvh.rebuild(dev(p1))  # a successful rebuild makes the tree valid again
    q = datagen.cube(700, 32)
    og, ig = bvh.query_spatial(dev(q), 0.05)
    oo, io = oracle.spatial_brute(p1, q, 0.05)
    assert_spatial_equal(host(og), host(ig), oo, io)
    ki, kd = bvh.query_nearest(dev(q), 5)
    eo, ed = oracle.nearest_brute(p1, q, 5)
    assert_nearest_equal(host(ki), host(kd), eo, ed)
