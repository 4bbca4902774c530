"""Shared helpers of the GPU parity tests (device transfer, result comparison)."""
import numpy as np

import oracle


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def spatial_gpu(bvh, q, r):
    off, idx = bvh.query_spatial(dev(q), r)
    return host(off), host(idx)


def assert_spatial_equal(off_g, idx_g, off_o, idx_o):
    assert off_g.shape == off_o.shape
    bad = oracle.rows_as_sets_equal(off_g, idx_g, off_o, idx_o)
    assert bad is None, f"row {bad}: gpu {sorted(idx_g[off_g[bad]:off_g[bad + 1]].tolist())} " \
                        f"oracle {sorted(idx_o[off_o[bad]:off_o[bad + 1]].tolist())}"


def assert_nearest_equal(ig, dg, io, do):
    assert ig.shape == io.shape, (ig.shape, io.shape)
    rows = np.nonzero(np.any(ig != io, axis=1))[0]
    assert rows.size == 0, f"row {rows[0]}: gpu {ig[rows[0]].tolist()} oracle {io[rows[0]].tolist()}"
    if dg is not None:
        assert np.array_equal(dg, do)
