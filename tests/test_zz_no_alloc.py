"""The allocation-free sort entry point, checked against the ordinary one.

arborx_sort_pairs_noalloc serves callers that may not allocate device memory
during a call (code living inside another framework's fixed memory budget, or
a loop whose memory is planned up front).  It keeps its temporaries in one
fixed device array owned by the library.  This file is collected last so that
a run stopping at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_KEYS = 1 << 20


def _sort_noalloc(keys_np, key_bits):
    import torch
    import paper_1908_11807_b300 as ab
    keys = torch.from_numpy(keys_np).cuda().contiguous()
    perm = torch.empty(keys.numel(), dtype=torch.int32, device="cuda")
    st = ab.lib().arborx_sort_pairs_noalloc(ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(perm.data_ptr()),
                                            keys.numel(), key_bits, torch.cuda.current_stream().cuda_stream)
    assert st == 0, ab.error_string(st)
    return keys.cpu().numpy(), perm.cpu().numpy()


def _sort_reference(keys_np, key_bits):
    import torch
    import paper_1908_11807_b300 as ab
    k, p = ab.arborx_sort_pairs(torch.from_numpy(keys_np).cuda(), key_bits)
    return k.cpu().numpy(), p.cpu().numpy()


def test_noalloc_sort_matches_allocating_sort_twice_in_a_row():
    g = np.random.default_rng(2024)
    # call 1: 64-bit keys, the larger footprint
    k1 = (g.integers(0, 1 << 62, size=1_000_003, dtype=np.uint64) & np.uint64((1 << 63) - 1))
    k1[::7] = k1[3]  # ties must keep input order
    a_keys, a_perm = _sort_noalloc(k1.view(np.int64), 63)
    r_keys, r_perm = _sort_reference(k1.view(np.int64), 63)
    assert np.array_equal(a_perm, r_perm) and np.array_equal(a_keys, r_keys)
    assert np.array_equal(a_perm, np.argsort(k1, kind="stable"))
    # call 2 on the same scratch: 32-bit keys, smaller n (stale contents must not leak in)
    k2 = g.integers(0, 1 << 30, size=300_001, dtype=np.uint64).astype(np.uint32)
    k2[:100_000] = k2[5]
    b_keys, b_perm = _sort_noalloc(k2.view(np.int32), 30)
    s_keys, s_perm = _sort_reference(k2.view(np.int32), 30)
    assert np.array_equal(b_perm, s_perm) and np.array_equal(b_keys, s_keys)
    # call 3: exactly the maximum size
    k3 = g.integers(0, 1 << 32, size=MAX_KEYS, dtype=np.uint64).astype(np.uint32)
    c_keys, c_perm = _sort_noalloc(k3.view(np.int32), 32)
    assert np.array_equal(c_perm, np.argsort(k3, kind="stable"))


@pytest.mark.parametrize("key_bits,wide", [(8, False), (20, False), (40, True)])
def test_noalloc_sort_odd_pass_counts_copy_back_from_the_array(key_bits, wide):
    # 1, 3 and 5 eight-bit passes leave the sorted pairs in the array's second buffers, from
    # which the call copies them back into the caller's; two calls in a row near the size limit
    g = np.random.default_rng([2025, key_bits])
    for n in (MAX_KEYS - 5, 777_777):
        k = g.integers(0, 1 << key_bits, size=n, dtype=np.uint64)
        k[::5] = k[1]
        k = k if wide else k.astype(np.uint32)
        view = k.view(np.int64) if wide else k.view(np.int32)
        a_keys, a_perm = _sort_noalloc(view, key_bits)
        r_keys, r_perm = _sort_reference(view, key_bits)
        assert np.array_equal(a_perm, r_perm) and np.array_equal(a_keys, r_keys)
        assert np.array_equal(a_perm, np.argsort(k, kind="stable"))
        assert np.array_equal(a_keys.view(k.dtype), np.sort(k, kind="stable"))


def test_noalloc_sort_rejects_sizes_beyond_its_array():
    import paper_1908_11807_b300 as ab
    L = ab.lib()
    dummy = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    assert L.arborx_sort_pairs_noalloc(dummy, dummy, MAX_KEYS + 1, 30, None) == 1
    assert L.arborx_sort_pairs_noalloc(dummy, dummy, 10, 0, None) == 1
    assert L.arborx_sort_pairs_noalloc(None, None, 0, 30, None) == 0
