"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every declared symbol, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "arborx_b300.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"ARBORX_API\s+[^;(]*?\b(arborx_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    import paper_1908_11807_b300 as ab
    return ab.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("arborx_build", "arborx_destroy", "arborx_query_spatial", "arborx_query_spatial_count",
                 "arborx_query_spatial_fill", "arborx_query_nearest", "arborx_error_string", "arborx_check",
                 "arborx_sort_pairs", "arborx_export_tree"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    raw = ctypes.CDLL(L._name)
    missing = [n for n in _declared() if not hasattr(raw, n)]
    assert not missing, missing


def test_only_declared_symbols_are_exported(L):
    # the library keeps its internals hidden (-fvisibility=hidden)
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", L._name], capture_output=True, text=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if " T " in ln and ln.split()[-1].startswith("arborx_")})
    assert exported == _declared()


def test_error_strings_and_defaults():
    import paper_1908_11807_b300 as ab
    assert ab.error_string(0) == "ok"
    assert ab.error_string(4) == "bounded device wait timed out"
    assert ab.error_string(99) == "unknown"
    o = ab.default_opts()
    assert (o.key_bits, o.sort_queries, o.validate, o.keep_order, o.block_size, o.stack_smem, o.build_method,
            o.stats) == (30, 1, 1, 0, 0, 0, 0, 0)
    assert ab.version().startswith("arborx-b300")


def test_invalid_arguments_rejected_without_device(L):
    import paper_1908_11807_b300._binding as b
    h = ctypes.c_void_p()
    o = b.default_opts()
    # n < 0, bad kind, NULL out, NULL prims with n > 0, bad key_bits / block size
    assert L.arborx_build(None, -1, 0, ctypes.byref(o), None, ctypes.byref(h)) == b.ARBORX_EINVAL
    assert L.arborx_build(None, 10, 2, ctypes.byref(o), None, ctypes.byref(h)) == b.ARBORX_EINVAL
    assert L.arborx_build(None, 10, 0, ctypes.byref(o), None, None) == b.ARBORX_EINVAL
    assert L.arborx_build(None, 10, 0, ctypes.byref(o), None, ctypes.byref(h)) == b.ARBORX_EINVAL
    assert L.arborx_build(None, 1 << 30, 0, ctypes.byref(o), None, ctypes.byref(h)) == b.ARBORX_EINVAL
    for field, val in (("key_bits", 31), ("block_size", 48), ("block_size", 512), ("stack_smem", -1),
                       ("build_method", 2)):
        bad = b.default_opts(**{field: val})
        assert L.arborx_build(ctypes.c_void_p(16), 10, 0, ctypes.byref(bad), None, ctypes.byref(h)) == b.ARBORX_EINVAL
    # NULL handle everywhere
    assert L.arborx_query_nearest(None, None, 0, 10, None, None, None, None, None) == b.ARBORX_EINVAL
    assert L.arborx_query_spatial_count(None, None, 0, ctypes.c_float(1.0), None, None, None) == b.ARBORX_EINVAL
    assert L.arborx_query_order(None, None, 0, None, None) == b.ARBORX_EINVAL
    assert L.arborx_stats(None, None, None) == b.ARBORX_EINVAL
    assert L.arborx_check(None, None) == b.ARBORX_EINVAL
    assert L.arborx_destroy(None) == b.ARBORX_OK
    assert L.arborx_default_opts(None) == b.ARBORX_EINVAL
    # sort: bad key width
    assert L.arborx_sort_pairs(None, None, 10, 0, None) == b.ARBORX_EINVAL
    assert L.arborx_sort_pairs(None, None, 10, 65, None) == b.ARBORX_EINVAL
    assert L.arborx_sort_pairs(None, None, 0, 30, None) == b.ARBORX_OK
    # tree-free order: bad size, null pointers, bad kind; an empty set needs no device
    assert L.arborx_order(None, -1, 0, None, None, None) == b.ARBORX_EINVAL
    assert L.arborx_order(None, 10, 0, None, None, None) == b.ARBORX_EINVAL
    assert L.arborx_order(ctypes.c_void_p(16), 10, 2, None, None, ctypes.c_void_p(16)) == b.ARBORX_EINVAL
    assert L.arborx_order(None, 1 << 30, 0, None, None, None) == b.ARBORX_EINVAL
    assert L.arborx_order(None, 0, 0, None, None, None) == b.ARBORX_OK
    # rebuild needs a handle
    assert L.arborx_rebuild(None, None, None) == b.ARBORX_EINVAL
    # spatial and nearest in one call: a handle, then the checks of both queries
    assert L.arborx_query_spatial_nearest(None, None, 0, ctypes.c_float(1.0), 8, 10, None, None,
                                          ctypes.c_void_p(16), None, 0, None, None, None) == b.ARBORX_EINVAL


def test_binding_refuses_cpu_tensors():
    import torch
    import paper_1908_11807_b300 as ab
    with pytest.raises(TypeError):
        ab.BVH(torch.zeros((10, 3)))


def test_option_struct_matches_the_header(L):
    # the binding's ctypes struct lists the header's fields in the header's order, and the
    # library fills the documented defaults (no GPU needed)
    import paper_1908_11807_b300 as ab
    src = open(HEADER).read()
    body = src[src.index("typedef struct arborx_opts {"):src.index("} arborx_opts;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(\w+)\s*;", body)
    from paper_1908_11807_b300 import _binding
    assert fields == [f for f, _ in _binding.arborx_opts._fields_]
    o = ab.default_opts()
    assert (o.key_bits, o.sort_queries, o.validate, o.knn_anchor, o.queries_per_warp, o.knn_heap_from) == \
        (30, 1, 1, 3, 0, 0)
