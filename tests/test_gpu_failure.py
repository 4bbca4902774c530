"""Failure detection on the GPU without a fault: a bounded wait on a flag that nothing sets gives
up after the look-back's iteration cap, the error reaches the host as ARBORX_ETIMEOUT, and the
device keeps working (a query right after is exact)."""
import ctypes
import time

import pytest

import datagen
import oracle
from tests.gpu_helpers import assert_spatial_equal, dev, host

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_device_stays_usable():
    import torch
    import paper_1908_11807_b300 as ab
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.time()
    st = ab.lib().arborx_selftest_bounded_wait(stream)
    elapsed = time.time() - t0
    assert st == ab.ARBORX_ETIMEOUT
    assert elapsed < 20.0
    p = datagen.cube(5000, 3)
    q = datagen.cube(300, 4)
    bvh = ab.BVH(dev(p))
    og, ig = bvh.query_spatial(dev(q), 0.05)
    bvh.check()
    oo, io = oracle.spatial_brute(p, q, 0.05)
    assert_spatial_equal(host(og), host(ig), oo, io)


def test_scan_look_back_times_out_and_the_device_stays_usable():
    # the one-call spatial query's scan kernel, started on a tile whose predecessor never
    # publishes: its bounded look-back gives up, ARBORX_ETIMEOUT reaches the host, and the
    # one-call query right after is exact
    import torch
    import paper_1908_11807_b300 as ab
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.time()
    st = ab.lib().arborx_selftest_scan_wait(stream)
    assert st == ab.ARBORX_ETIMEOUT
    assert time.time() - t0 < 20.0
    p = datagen.cube(5000, 5)
    q = datagen.cube(3000, 6)
    bvh = ab.BVH(dev(p))
    off, idx = bvh.query_spatial_async(dev(q), 0.05, buffer_size=8, capacity=3000 * 64)
    bvh.check()
    oo, io = oracle.spatial_brute(p, q, 0.05)
    assert_spatial_equal(host(off), host(idx)[:int(host(off)[-1])], oo, io)
