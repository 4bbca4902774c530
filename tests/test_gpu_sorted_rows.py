"""opts.sorted_rows: every spatial or box row in ascending primitive index order, so the CSR
output equals the oracle's brute-force rows exactly, entry by entry (not only as sets), through
every entry point that writes rows, including long rows, empty rows, a row holding every
primitive, a caller buffer larger than the result, and a captured CUDA graph."""
import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_helpers import dev, host

pytestmark = pytest.mark.gpu

S1 = datagen.SEED0 + 1


def _ab():
    import paper_1908_11807_b300 as ab
    return ab


CASES = {
    "cube_1e4": lambda: (datagen.cube(10_000, S1), datagen.cube(10_000, S1, datagen.STREAM_QUERIES),
                         datagen.radius_for_mean(10_000, "cube")),
    # hollow-sphere queries in a hollow cube: rows from 0 to several hundred entries
    "paper_hollow": lambda: (datagen.paper_shape(20_000, "hollow_cube", 10),
                             datagen.paper_shape(5000, "hollow_sphere", 11), datagen.paper_radius(20_000)),
    "duplicates": lambda: (np.repeat(datagen.cube(600, 3), 9, 0), datagen.cube(3001, 4), 0.03),
    "boxes": lambda: (datagen.boxes(20_000, 12, half_max=0.01), datagen.cube(5000, 13), 0.01),
}


def _assert_rows_exact(off_g, idx_g, off_o, idx_o):
    assert np.array_equal(off_g, off_o)
    nnz = int(off_o[-1])
    bad = np.nonzero(idx_g[:nnz] != idx_o)[0]
    assert bad.size == 0, f"entry {bad[0]}: gpu {idx_g[bad[0]]} oracle {idx_o[bad[0]]}"


@pytest.mark.parametrize("name", sorted(CASES))
def test_sorted_rows_two_pass_and_one_pass(name):
    ab = _ab()
    p, q, r = CASES[name]()
    oo, io = oracle.spatial_brute(p, q, r)
    bvh = ab.BVH(dev(p), sorted_rows=1)
    qd = dev(q)
    og, ig = bvh.query_spatial(qd, r)  # two passes
    bvh.check()
    _assert_rows_exact(host(og), host(ig), oo, io)
    og, ig = bvh.query_spatial(qd, r, buffer_size=8)  # one pass, count and fill calls
    bvh.check()
    _assert_rows_exact(host(og), host(ig), oo, io)
    # one call, a buffer larger than the result: the unused tail does not disturb the rows
    og, ig = bvh.query_spatial_async(qd, r, buffer_size=8, capacity=int(oo[-1]) * 2 + 17)
    bvh.check()
    _assert_rows_exact(host(og), host(ig), oo, io)


def test_sorted_rows_box_queries():
    ab = _ab()
    p = datagen.boxes(20_000, S1, half_max=0.01)
    qb = datagen.boxes(5000, S1, half_max=0.03, stream=datagen.STREAM_QUERIES)
    oo, io = oracle.intersects_brute(p, qb)
    bvh = ab.BVH(dev(p), sorted_rows=1)
    og, ig = bvh.query_intersects(dev(qb), buffer_size=4)
    bvh.check()
    _assert_rows_exact(host(og), host(ig), oo, io)


def test_sorted_rows_edge_cases():
    ab = _ab()
    p = datagen.cube(3000, 5)
    q = np.concatenate([datagen.cube(50, 6), np.full((3, 3), 7.0, np.float32)])  # last rows empty
    bvh = ab.BVH(dev(p), sorted_rows=1)
    # a radius that takes every point: one row of n entries per query
    og, ig = bvh.query_spatial(dev(q[:4]), 10.0)
    oo, io = oracle.spatial_brute(p, q[:4], 10.0)
    _assert_rows_exact(host(og), host(ig), oo, io)
    og, ig = bvh.query_spatial(dev(q), 0.05)
    oo, io = oracle.spatial_brute(p, q, 0.05)
    _assert_rows_exact(host(og), host(ig), oo, io)
    og, ig = bvh.query_spatial(dev(q[:0]), 0.05)
    assert host(og).tolist() == [0] and ig.numel() == 0
    with pytest.raises(ab.ArborXError):
        ab.BVH(dev(p), sorted_rows=2)


def test_sorted_rows_in_a_captured_graph():
    ab = _ab()
    import torch
    p, q, r = CASES["cube_1e4"]()
    oo, io = oracle.spatial_brute(p, q, r)
    bvh = ab.BVH(dev(p), sorted_rows=1)
    qd = dev(q)
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
    _assert_rows_exact(host(goff), host(out_idx), oo, io)
