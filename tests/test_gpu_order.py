"""The tree-free traversal order (arborx_order, Sec. 2.2 query ordering with the set's own
bounding box): the permutation equals the stable argsort of the oracle's Morton keys (top 24 of
30 bits) scaled by the set's own box, for points and box centres; it is a permutation for empty,
single, duplicate, flat and non-finite sets; query rows traversed in it equal the oracle's; it
runs on a second stream while the tree is built, and inside a captured CUDA graph."""
import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_helpers import assert_nearest_equal, assert_spatial_equal, dev, host

pytestmark = pytest.mark.gpu


def _ab():
    import paper_1908_11807_b300 as ab
    return ab


def _expected(prims):
    sb, _ = oracle.scene_box(prims)
    keys = oracle.morton(prims, sb, 30) >> 6
    return np.argsort(keys, kind="stable")


@pytest.mark.parametrize("make", [
    lambda: datagen.cube(100_003, 40),                       # several tiles and a ragged tail
    lambda: datagen.hollow_sphere(50_000, 41),
    lambda: datagen.gaussian_mixture(60_000, 42),
    lambda: np.repeat(datagen.cube(500, 43), 11, 0),         # duplicate keys: ties keep input order
    lambda: np.concatenate([datagen.cube(9000, 44)[:, :2], np.full((9000, 1), 0.5, np.float32)], 1),
    lambda: datagen.boxes(40_000, 45, half_max=0.01),        # box centres
])
def test_order_equals_stable_argsort_of_oracle_keys(make):
    ab = _ab()
    p = make().astype(np.float32)
    got = host(ab.order(dev(p)))
    assert np.array_equal(got, _expected(p))


def test_order_edge_cases_are_permutations():
    ab = _ab()
    assert ab.order(dev(datagen.cube(0, 1))).numel() == 0
    assert host(ab.order(dev(datagen.cube(1, 1)))).tolist() == [0]
    q = datagen.cube(5000, 46)
    q[::7, 1] = np.nan
    q[3, 0] = np.inf
    got = host(ab.order(dev(q)))
    assert np.array_equal(np.sort(got), np.arange(len(q)))
    allnan = np.full((300, 3), np.nan, np.float32)
    assert np.array_equal(np.sort(host(ab.order(dev(allnan)))), np.arange(300))
    with pytest.raises(ValueError):
        ab.order(dev(datagen.cube(10, 1))[:, :2].contiguous())


def test_rows_in_the_tree_free_order_match_the_oracle():
    ab = _ab()
    n, m, k = 200_000, 20_000, 10
    p, q = datagen.cube(n, 47), datagen.cube(m, 48)
    r = datagen.radius_for_mean(n, "cube")
    order = ab.order(dev(q))
    bvh = ab.BVH(dev(p))
    og, ig = bvh.query_spatial(dev(q), r, order=order, buffer_size=16)
    bvh.check()
    oo, io = oracle.spatial_brute(p, q, r)
    assert_spatial_equal(host(og), host(ig), oo, io)
    ki, kd = bvh.query_nearest(dev(q), k, order=order)
    eo, ed = oracle.nearest_brute(p, q, k)
    assert_nearest_equal(host(ki), host(kd), eo, ed)


def test_order_on_a_side_stream_during_the_build_and_in_a_graph():
    ab = _ab()
    import torch
    n, m, k = 300_000, 30_000, 8
    p, q = datagen.gaussian_mixture(n, 49), datagen.gaussian_mixture(m, 50)
    pd, qd = dev(p), dev(q)
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    start = torch.cuda.Event()
    start.record(main)
    with torch.cuda.stream(side):
        side.wait_event(start)
        order = ab.order(qd)
        done = torch.cuda.Event()
        done.record(side)
    bvh = ab.BVH(pd, validate=0)  # on the main stream, concurrently with the order
    main.wait_event(done)
    order.record_stream(main)
    ki, kd = bvh.query_nearest(qd, k, order=order)
    bvh.check()
    eo, ed = oracle.nearest_brute(p, q, k)
    assert_nearest_equal(host(ki), host(kd), eo, ed)
    assert np.array_equal(host(order), _expected(q))
    # the call only enqueues work: capture it and replay
    ab.order(qd)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        gorder = ab.order(qd)
    gorder.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(host(gorder), _expected(q))
