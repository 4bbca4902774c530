"""GPU parity of the batched many-cloud path: every cloud's rows equal the
oracle's brute-force nearest rows over that cloud alone (indices local to the
cloud), with and without CUDA-graph replay, including empty clouds, one-point
clouds and k above the cloud size; the full 512-cloud workload is checked on
sampled clouds."""
import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_helpers import assert_nearest_equal, dev, host

pytestmark = pytest.mark.gpu


def _ab():
    import paper_1908_11807_b300 as ab
    return ab


def _make(sizes, qsizes, ks, seed):
    pts, qs = [], []
    for c, (n, m) in enumerate(zip(sizes, qsizes)):
        gen = datagen.cube if c % 2 == 0 else datagen.hollow_sphere
        pts.append(gen(n, seed, datagen.STREAM_POINTS, c).reshape(n, 3))
        qs.append(gen(m, seed, datagen.STREAM_QUERIES, c).reshape(m, 3))
    po = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    qo = np.concatenate([[0], np.cumsum(qsizes)]).astype(np.int64)
    return pts, qs, po, qo, np.asarray(ks, np.int32)


def _check_against_oracle(pts, qs, ks, off, idx, d2, clouds):
    for c in clouds:
        m = len(qs[c])
        if m == 0:
            continue
        io, do = oracle.nearest_brute(pts[c], qs[c], int(ks[c]))
        kk = io.shape[1]
        q0 = sum(len(x) for x in qs[:c])
        rows = off[q0:q0 + m + 1]
        assert np.all(np.diff(rows) == kk)
        got_i = idx[rows[0]:rows[-1]].reshape(m, kk)
        got_d = d2[rows[0]:rows[-1]].reshape(m, kk)
        assert_nearest_equal(got_i, got_d, io, do)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_small_matches_per_cloud_oracle(use_graph):
    ab = _ab()
    sizes = [0, 1, 2, 5, 33, 1000, 2500, 3000, 17, 900, 1, 4096, 0, 700]
    qsizes = [10, 7, 0, 20, 40, 1000, 500, 3000, 50, 900, 3, 800, 0, 700]
    ks = [1, 1, 10, 32, 10, 10, 32, 1, 32, 16, 10, 2, 5, 8]
    pts, qs, po, qo, ks = _make(sizes, qsizes, ks, 5)
    b = ab.Batch(po, qo, ks)
    P = dev(np.concatenate(pts).astype(np.float32))
    Q = dev(np.concatenate(qs).astype(np.float32))
    for rep in range(2):  # second call replays the graph
        off, idx, d2 = b.run(P, Q, use_graph=use_graph)
        b.check()
        _check_against_oracle(pts, qs, ks, host(off), host(idx), host(d2), range(len(ks)))


@pytest.mark.parametrize("opts", [dict(knn_anchor=0), dict(knn_anchor=1), dict(knn_anchor=2), dict(knn_anchor=3),
                                  dict(knn_anchor=3, knn_heap_from=33), dict(knn_anchor=3, stack_smem=1),
                                  dict(knn_anchor=3, queries_per_warp=64)])
def test_batch_tree_bound_forms_match_per_cloud_oracle(opts):
    # every form of the tree's own bound, from each cloud's subtree root: the walks, the
    # first-descent form (register lists up to 10; wider classes take the query-path walk) and
    # the unbounded start; stack_smem 1 sends the first descent's compaction through the local part
    ab = _ab()
    sizes = [0, 1, 2, 5, 33, 1000, 2500, 3000, 17, 900, 1, 4096, 0, 700]
    qsizes = [10, 7, 0, 20, 40, 1000, 500, 3000, 50, 900, 3, 800, 0, 700]
    ks = [1, 1, 10, 32, 10, 10, 32, 1, 32, 16, 10, 2, 5, 8]
    pts, qs, po, qo, ks = _make(sizes, qsizes, ks, 6)
    b = ab.Batch(po, qo, ks, **opts)
    P = dev(np.concatenate(pts).astype(np.float32))
    Q = dev(np.concatenate(qs).astype(np.float32))
    off, idx, d2 = b.run(P, Q, use_graph=False)
    b.check()
    _check_against_oracle(pts, qs, ks, host(off), host(idx), host(d2), range(len(ks)))


def test_batch_many_clouds_sampled():
    # 512 clouds, sizes log-uniform in [1e3, 1e5], cube / hollow sphere, k in {1, 10, 32}
    ab = _ab()
    w = datagen.batched_workload(512, datagen.SEED0 + 4)
    pts = [c["points"] for c in w]
    qs = [c["queries"] for c in w]
    ks = np.array([c["k"] for c in w], np.int32)
    po = np.concatenate([[0], np.cumsum([len(p) for p in pts])]).astype(np.int64)
    qo = np.concatenate([[0], np.cumsum([len(q) for q in qs])]).astype(np.int64)
    b = ab.Batch(po, qo, ks)
    P = dev(np.concatenate(pts))
    Q = dev(np.concatenate(qs))
    off, idx, d2 = b.run(P, Q, use_graph=True)
    off, idx, d2 = b.run(P, Q, use_graph=True)
    b.check()
    off, idx, d2 = host(off), host(idx), host(d2)
    assert off[-1] == b.entries
    sample = sorted(set(np.random.default_rng(4).choice(512, 12, replace=False).tolist()) | {int(np.argmin(po[1:] - po[:-1]))})
    for c in sample:  # brute force on a query subsample of each sampled cloud
        m = len(qs[c])
        sub = np.arange(0, m, max(1, m // 300))
        io, do = oracle.nearest_brute(pts[c], qs[c][sub], int(ks[c]))
        kk = io.shape[1]
        q0 = int(qo[c])
        starts = off[q0 + sub]
        got_i = np.stack([idx[s:s + kk] for s in starts])
        got_d = np.stack([d2[s:s + kk] for s in starts])
        assert_nearest_equal(got_i, got_d, io, do)


def test_batch_rejects_bad_plans():
    ab = _ab()
    with pytest.raises(ab.ArborXError):
        ab.Batch([0, 10], [0, 5], [33])
    with pytest.raises(ab.ArborXError):
        ab.Batch([0, 10, 5], [0, 5, 6], [1, 1])
    with pytest.raises(ab.ArborXError):
        ab.Batch([1, 10], [0, 5], [1])


def test_one_call_batched_matches_oracle_and_checks_capacity():
    ab = _ab()
    import ctypes
    import torch
    sizes = [0, 1, 3, 700, 2000, 64, 1500]
    qsizes = [4, 9, 6, 300, 1000, 0, 800]
    ks = [1, 10, 32, 10, 32, 16, 1]
    pts, qs, po, qo, ks = _make(sizes, qsizes, ks, 9)
    P = dev(np.concatenate(pts).astype(np.float32))
    Q = dev(np.concatenate(qs).astype(np.float32))
    off, idx, d2 = ab.batched(P, Q, po, qo, ks)
    _check_against_oracle(pts, qs, ks, host(off), host(idx), host(d2), range(len(ks)))
    # the same rows as the planned batch
    o2, i2, d22 = ab.Batch(po, qo, ks).run(P, Q, use_graph=False)
    assert np.array_equal(host(off), host(o2)) and np.array_equal(host(idx), host(i2))
    # a capacity below the batch's entries is refused before any work
    entries = int(idx.numel())
    rows = torch.empty(int(qo[-1]) + 1, dtype=torch.int64, device="cuda")
    small = torch.empty(entries, dtype=torch.int32, device="cuda")
    o = ab.default_opts()
    st = ab.lib().arborx_batched(len(ks), po.ctypes.data_as(ctypes.c_void_p), qo.ctypes.data_as(ctypes.c_void_p),
                                 ks.ctypes.data_as(ctypes.c_void_p), P.data_ptr(), Q.data_ptr(), ctypes.byref(o),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), rows.data_ptr(),
                                 small.data_ptr(), None, entries - 1)
    assert st == ab.ARBORX_EINVAL
