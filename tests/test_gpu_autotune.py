"""The autotuner: every configuration it returns is a valid one and gives the same results as the
library defaults (launch parameters, row-buffer widths and batch tiles change speed only)."""
import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_helpers import assert_nearest_equal, assert_spatial_equal, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _private_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("ARBORX_TUNE_CACHE", str(tmp_path / "tune.json"))


def test_tune_returns_a_valid_configuration_with_the_default_results():
    import paper_1908_11807_b300 as ab
    from paper_1908_11807_b300 import autotune
    p, q = datagen.workload("cube", 200_000, 20_000, 70)
    r = datagen.radius_for_mean(200_000, "cube")
    pd, qd = dev(p), dev(q)
    t = autotune.tune(pd, qd, r, 10, "cube", use_cache=True)
    assert t["block_size"] in autotune.DEFAULT_BLOCKS and t["stack_smem"] in autotune.DEFAULT_STACKS
    assert t["knn_anchor"] in autotune.DEFAULT_ANCHORS
    assert autotune.tune(pd, qd, r, 10, "cube") == t  # second call: from the cache
    bvh = ab.BVH(pd, block_size=t["block_size"], stack_smem=t["stack_smem"])
    # a fixed width, or one taken from the queries' own hit counts (a multiple of 4)
    assert t["buffer_size"] in set(autotune.DEFAULT_BUFFERS) | autotune.buffer_candidates(bvh, qd, r)
    og, ig = bvh.query_spatial(qd, r, buffer_size=t["buffer_size"])
    kg, dg = bvh.query_nearest(qd, 10)
    bvh.check()
    oo, io = oracle.spatial_brute(p, q, r)
    assert_spatial_equal(host(og), host(ig), oo, io)
    ko, do = oracle.nearest_brute(p, q, 10)
    assert_nearest_equal(host(kg), host(dg), ko, do)


@pytest.mark.parametrize("r", [1.0, 2.5, 4.0])
def test_pick_buffer_per_radius(r):
    import paper_1908_11807_b300 as ab
    from paper_1908_11807_b300 import autotune
    side = 40
    g = np.arange(side, dtype=np.float32)
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    sites = pts[np.random.default_rng(71).integers(0, len(pts), 20_000)]
    bvh = ab.BVH(dev(pts))
    qd = dev(sites)
    pick = autotune.pick_buffer(bvh, qd, r)
    bs = pick["buffer_size"]
    assert bs in pick["ms"] and (bs == 0 or bs % 4 == 0)
    # the candidates cover the largest row of the sample, so a one-pass pick holds every row
    assert max(pick["ms"]) >= pick["hits"]["max"]
    og, ig = bvh.query_spatial(qd, r, buffer_size=bs)
    bvh.check()
    oo, io = oracle.spatial_brute(pts, sites, r)
    assert_spatial_equal(host(og), host(ig), oo, io)


def test_tune_batch_returns_valid_tiles_with_the_default_results():
    import torch
    import paper_1908_11807_b300 as ab
    from paper_1908_11807_b300 import autotune
    g = np.random.default_rng(72)
    sizes = np.floor(10.0 ** g.uniform(2.0, 3.5, 24)).astype(int)
    w = [dict(points=(datagen.cube if c % 2 else datagen.hollow_sphere)(int(n), 72, datagen.STREAM_POINTS, c),
              queries=datagen.cube(int(n), 72, datagen.STREAM_QUERIES, c), k=int(g.choice([1, 10, 32])))
         for c, n in enumerate(sizes)]
    pts = np.concatenate([c["points"] for c in w])
    qs = np.concatenate([c["queries"] for c in w])
    ks = np.array([c["k"] for c in w], np.int32)
    po = np.concatenate([[0], np.cumsum([len(c["points"]) for c in w])]).astype(np.int64)
    qo = np.concatenate([[0], np.cumsum([len(c["queries"]) for c in w])]).astype(np.int64)
    P, Q = dev(pts), dev(qs)
    t = autotune.tune_batch(po, qo, ks, P, Q, blocks=(64, 128), stacks=(4, 16))
    assert t["block_size"] in (64, 128) and t["stack_smem"] in (4, 16)
    assert t["queries_per_warp"] in autotune.DEFAULT_QPW and t["knn_heap_from"] in autotune.DEFAULT_HEAP_FROM
    assert t["knn_anchor"] in autotune.DEFAULT_ANCHORS
    ref = ab.Batch(po, qo, ks)
    o0, i0, d0 = ref.run(P, Q)
    for qpw, hf in ((32, 17), (64, 33), (128, 17), (256, 33)):
        b = ab.Batch(po, qo, ks, block_size=t["block_size"], stack_smem=t["stack_smem"], queries_per_warp=qpw,
                     knn_heap_from=hf)
        o1, i1, d1 = b.run(P, Q, use_graph=True)
        b.check()
        assert torch.equal(o0, o1) and torch.equal(i0, i1) and torch.equal(d0, d1)
        b.destroy()
    # and the default rows are the oracle's, cloud by cloud
    oh, ih, dh = host(o0), host(i0), host(d0)
    for c in range(len(w)):
        k = int(ks[c])
        io, do = oracle.nearest_brute(w[c]["points"], w[c]["queries"], k)
        a, b_ = int(oh[qo[c]]), int(oh[qo[c + 1]])
        kk = io.shape[1]
        assert_nearest_equal(ih[a:b_].reshape(-1, kk), dh[a:b_].reshape(-1, kk), io, do)
    ref.destroy()


def test_batch_rejects_bad_tiles():
    import paper_1908_11807_b300 as ab
    po = np.array([0, 100], np.int64)
    with pytest.raises(ab.ArborXError):
        ab.Batch(po, po, np.array([5], np.int32), queries_per_warp=48)
    with pytest.raises(ab.ArborXError):
        ab.Batch(po, po, np.array([5], np.int32), knn_heap_from=20)
