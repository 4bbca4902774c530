"""Caller-supplied device allocators (arborx_opts.alloc / free): a torch-backed
allocator serves the build and the queries with identical results; an
allocator that fails (returns NULL) makes the call return ARBORX_ENOMEM; one
that returns memory off the 256-byte boundary is refused (released again,
ARBORX_ENOMEM), so no traversal reads a misaligned 32-byte slot."""
import numpy as np
import pytest

import datagen
import oracle
from tests.gpu_helpers import assert_nearest_equal, assert_spatial_equal, dev, host

pytestmark = pytest.mark.gpu


def _allocator(offset=0, fail=False):
    import torch
    from paper_1908_11807_b300 import _binding as b
    live = {}
    calls = {"alloc": 0, "free": 0}

    @b._ALLOC_FN
    def alloc(nbytes, stream, ctx):
        calls["alloc"] += 1
        if fail:
            return None
        t = torch.empty(nbytes + 512, dtype=torch.uint8, device="cuda")
        p = t.data_ptr() + offset
        live[p] = t
        return p

    @b._FREE_FN
    def free(ptr, nbytes, stream, ctx):
        calls["free"] += 1
        live.pop(ptr, None)

    return alloc, free, live, calls


def test_torch_backed_allocator_serves_build_and_queries():
    import paper_1908_11807_b300 as ab
    p, q = datagen.workload("cube", 20_000, 3000, 41)
    r = datagen.radius_for_mean(20_000, "cube")
    alloc, free, live, calls = _allocator()
    bvh = ab.BVH(dev(p), alloc=alloc, free=free)
    og, ig = bvh.query_spatial(dev(q), r, buffer_size=16)
    kg, dg = bvh.query_nearest(dev(q), 10)
    bvh.check()
    oo, io = oracle.spatial_brute(p, q, r)
    assert_spatial_equal(host(og), host(ig), oo, io)
    ko, do = oracle.nearest_brute(p, q, 10)
    assert_nearest_equal(host(kg), host(dg), ko, do)
    assert calls["alloc"] > 0
    bvh.destroy()
    import torch
    torch.cuda.synchronize()
    assert not live and calls["free"] == calls["alloc"]  # every block handed back


@pytest.mark.parametrize("case", ["null", "misaligned"])
def test_failing_or_misaligned_allocator_is_reported(case):
    import paper_1908_11807_b300 as ab
    p = datagen.cube(5000, 42)
    alloc, free, live, calls = _allocator(offset=16 if case == "misaligned" else 0, fail=case == "null")
    with pytest.raises(ab.ArborXError) as e:
        ab.BVH(dev(p), alloc=alloc, free=free)
    from paper_1908_11807_b300 import _binding as b
    assert e.value.code == b.ARBORX_ENOMEM
    assert calls["alloc"] >= 1
    if case == "misaligned":
        assert not live and calls["free"] == calls["alloc"]  # the refused block was released
