"""Seeded random sweep of small problems through every query form: each case draws a cloud
(uniform, hollow sphere, duplicates, a flat plane, or boxes), its size, the query set, radius, k,
row-buffer width and build/traversal options, and checks the radius rows (two-pass, one-pass and
the one-call form), the nearest rows and the box-query rows against the oracle's brute force."""
import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_helpers import assert_nearest_equal, assert_spatial_equal, dev, host

pytestmark = pytest.mark.gpu


def _case(seed):
    g = np.random.default_rng([20260, seed])
    n = int(g.choice([0, 1, 2, 3, 17, int(g.integers(4, 3000))]))
    m = int(g.choice([0, 1, int(g.integers(2, 600))]))
    kind = g.choice(["cube", "sphere", "dups", "flat", "boxes"])
    if kind == "cube":
        p = datagen.cube(n, seed)
    elif kind == "sphere":
        p = datagen.hollow_sphere(n, seed)
    elif kind == "dups":
        p = np.repeat(datagen.cube(max(n // 7, 1), seed), 7, 0)[:n]
    elif kind == "flat":
        p = np.concatenate([datagen.cube(n, seed)[:, :2], np.full((n, 1), 0.25, np.float32)], 1)
    else:
        p = datagen.boxes(n, seed, half_max=float(g.uniform(0, 0.05)))
    q = (g.random((m, 3)) * 1.4 - 0.2).astype(np.float32)
    opts = dict(sort_queries=int(g.integers(0, 2)), key_bits=int(g.choice([30, 63])),
                build_method=int(g.integers(0, 2)), sorted_rows=int(g.integers(0, 2)),
                block_size=int(g.choice([32, 64, 128, 256])), stack_smem=int(g.choice([0, 1, 4, 16])),
                knn_anchor=int(g.integers(0, 4)), knn_heap_from=int(g.choice([0, 17, 33])),
                keep_order=int(g.integers(0, 2)))
    r = float(g.choice([0.0, g.uniform(0.01, 0.3), 2.0]))
    k = int(g.choice([1, 5, 10, 16, 17, 27, 40]))
    bs = int(g.choice([1, 4, 16, 32, 84]))
    half = float(g.uniform(0.0, 0.2))
    return p.astype(np.float32), q, opts, r, k, bs, half


@pytest.mark.parametrize("seed", range(200))
def test_random_case_matches_brute_force(seed):
    import paper_1908_11807_b300 as ab
    p, q, opts, r, k, bs, half = _case(seed)
    bvh = ab.BVH(dev(p), **opts)
    if opts["keep_order"]:
        bvh.emit_subtrees(True)  # radius and box rows take contained subtrees whole
    qd = dev(q)
    oo, io = oracle.spatial_brute(p, q, r)
    exact_rows = bool(opts["sorted_rows"])

    def check_rows(og, ig, oo, io):
        og, ig = host(og), host(ig)
        if exact_rows:  # ascending rows: entry by entry
            assert np.array_equal(og, oo) and np.array_equal(ig[:int(oo[-1])], io)
        else:
            assert_spatial_equal(og, ig[:int(og[-1])], oo, io)

    og, ig = bvh.query_spatial(qd, r)
    bvh.check()
    check_rows(og, ig, oo, io)
    og, ig = bvh.query_spatial(qd, r, buffer_size=bs)
    bvh.check()
    check_rows(og, ig, oo, io)
    if len(q):
        og, ig = bvh.query_spatial_async(qd, r, buffer_size=bs, capacity=max(int(oo[-1]), 1))
        bvh.check()
        check_rows(og, ig, oo, io)
    ki, kd = bvh.query_nearest(qd, k)
    bvh.check()
    eo, ed = oracle.nearest_brute(p, q, k)
    assert_nearest_equal(host(ki), host(kd), eo, ed)
    qb = np.concatenate([q - half, q + half], 1).astype(np.float32)
    ob, ib = oracle.intersects_brute(p, qb)
    og, ig = bvh.query_intersects(dev(qb), buffer_size=bs)
    bvh.check()
    check_rows(og, ig, ob, ib)
