"""GPU parity of the LBVH construction (Sec. 2.1): scene box, Morton codes and
the stable sort bit-exact against the oracle, tree invariants of the hierarchy
and the bottom-up fit, error behaviour."""
import numpy as np
import pytest

import datagen
import oracle
from oracle import tree_check
from tests.gpu_helpers import dev, host

pytestmark = pytest.mark.gpu


def _ab():
    import paper_1908_11807_b300 as ab
    return ab


def _cell_edges(n: int, seed: int) -> np.ndarray:
    """Points on and within a few ulps of the 10-bit Morton cell edges L + j (H - L) / 1024 of
    a scene box with extents 1, 3 and fl(0.7) (reciprocals inexact for the last two), and at
    fractions of a cell on both sides of the division-free form's acceptance margin, plus the
    box's two corners, which fix the scene box.  Coordinates near an edge must take the exact
    division and the others the multiply; either way the codes must equal the oracle's."""
    rng = np.random.default_rng(seed)
    lo = np.array([0.0, -1.25, 0.1], np.float32)
    hi = np.array([1.0, 1.75, np.float32(0.1) + np.float32(0.7)], np.float32)
    cols = []
    for a in range(3):
        ext = np.float64(hi[a]) - np.float64(lo[a])
        edges = (np.float64(lo[a]) + np.arange(1025) * ext / 1024).astype(np.float32)
        vals = [edges]
        # inside the cells: on both sides of the division-free form's 2^-11 acceptance margin
        for frac in (2.0 ** -12, 2.0 ** -11, 1.5 * 2.0 ** -11, 2.0 ** -10, 0.5, 1 - 2.0 ** -10, 1 - 1.5 * 2.0 ** -11,
                     1 - 2.0 ** -11, 1 - 2.0 ** -12):
            vals.append((np.float64(lo[a]) + (np.arange(1024) + frac) * ext / 1024).astype(np.float32))
        for s in (1, 2, 3):
            up, dn = edges.copy(), edges.copy()
            for _ in range(s):
                up = np.nextafter(up, np.float32(np.inf))
                dn = np.nextafter(dn, np.float32(-np.inf))
            vals += [up, dn]
        v = np.clip(np.concatenate(vals), lo[a], hi[a]).astype(np.float32)
        cols.append(rng.choice(v, n))
    pts = np.stack(cols, 1).astype(np.float32)
    return np.concatenate([pts, lo[None], hi[None]]).astype(np.float32)


CLOUDS = {
    "cell_edges": lambda: _cell_edges(20_000, 17),
    "cube_1e4": lambda: datagen.cube(10_000, datagen.SEED0 + 1),
    "hollow_sphere_2e4": lambda: datagen.hollow_sphere(20_000, datagen.SEED0 + 2),
    "gaussian_3e4": lambda: datagen.gaussian_mixture(30_000, datagen.SEED0 + 5),
    "ragged_4097": lambda: datagen.cube(4097, 7),  # one full sort tile + 1
    "ragged_12289": lambda: datagen.cube(12289, 8),
    "duplicates": lambda: np.repeat(datagen.cube(700, 9), 13, axis=0),
    "all_equal": lambda: np.full((5000, 3), 0.25, np.float32),
    "flat_plane": lambda: np.concatenate([datagen.cube(6000, 10)[:, :2], np.full((6000, 1), 2.0, np.float32)], 1),
    "collinear": lambda: np.stack([np.linspace(-1, 1, 3001, dtype=np.float32)] * 3, 1),
    "lattice_32": lambda: datagen.lattice(32),
    "tiny_2": lambda: datagen.cube(2, 11),
    "tiny_3": lambda: datagen.cube(3, 12),
    "boxes_2e4": lambda: datagen.boxes(20_000, datagen.SEED0 + 2),
    # runs of 1000 equal codes: subtrees made only of index bits span several 256-leaf chunks
    "dup_runs_1000": lambda: np.repeat(datagen.cube(60, 13), 1000, axis=0),
    "chunk_256": lambda: datagen.cube(256, 14),
    "chunk_257": lambda: datagen.cube(257, 15),
    "chunk_1023": lambda: datagen.cube(1023, 16),
}


@pytest.mark.parametrize("name", sorted(CLOUDS))
@pytest.mark.parametrize("key_bits", [30, 63])
@pytest.mark.parametrize("method", [0, 1], ids=["apetrei", "karras"])
def test_build_bit_exact_and_invariants(name, key_bits, method):
    ab = _ab()
    p = CLOUDS[name]()
    bvh = ab.BVH(dev(p), keep_order=1, key_bits=key_bits, build_method=method)
    rec, scene, codes, perm = bvh.export_tree(order=True)
    bvh.check()
    rec, scene, codes, perm = host(rec), host(scene), host(codes).view(np.uint64), host(perm).astype(np.int64)
    sb, bad = oracle.scene_box(p)
    assert bad == 0
    assert np.array_equal(scene, sb)
    want_codes = oracle.morton(p, sb, key_bits)
    # stable sort by code: ties keep index order (codes augmented with the index)
    want_perm = np.lexsort((np.arange(len(p)), want_codes))
    assert np.array_equal(perm, want_perm)
    assert np.array_equal(codes, want_codes[want_perm])
    tree_check.check_lbvh(rec, p, perm, codes, sb)


@pytest.mark.parametrize("n", [1, 2, 5])
@pytest.mark.parametrize("method", [0, 1], ids=["apetrei", "karras"])
def test_build_tiny_and_single_leaf(n, method):
    ab = _ab()
    p = datagen.cube(n, 40 + n)
    bvh = ab.BVH(dev(p), keep_order=1, build_method=method)
    rec, scene, codes, perm = bvh.export_tree(order=True)
    tree_check.check_lbvh(host(rec), p, host(perm), host(codes).view(np.uint64), host(scene))


def test_empty_tree():
    ab = _ab()
    import torch
    bvh = ab.BVH(torch.zeros((0, 3), device="cuda"))
    q = dev(datagen.cube(100, 1))
    off, idx = bvh.query_spatial(q, 1.0)
    assert host(off).tolist() == [0] * 101 and idx.numel() == 0
    ii, dd = bvh.query_nearest(q, 5)
    assert tuple(ii.shape) == (100, 0)


def test_nonfinite_primitive_rejected():
    ab = _ab()
    p = datagen.cube(1000, 3)
    p[500, 1] = np.nan
    with pytest.raises(ab.ArborXError) as e:
        ab.BVH(dev(p))
    assert e.value.code == 1
    p[500, 1] = np.inf
    with pytest.raises(ab.ArborXError):
        ab.BVH(dev(p))
    # asynchronous build: reported by check()
    bvh = ab.BVH(dev(p), validate=0)
    with pytest.raises(ab.ArborXError) as e:
        bvh.check()
    assert e.value.code == 1


def test_unaligned_input_pointer():
    ab = _ab()
    import torch
    p = datagen.cube(3001, 4)
    buf = torch.zeros(3 * 3001 + 1, dtype=torch.float32, device="cuda")
    buf[1:] = dev(p.ravel())
    view = buf[1:].view(3001, 3)  # 4-byte aligned, not 16
    bvh = ab.BVH(view, keep_order=1)
    rec, scene, codes, perm = bvh.export_tree(order=True)
    sb, _ = oracle.scene_box(p)
    assert np.array_equal(host(scene), sb)
    tree_check.check_lbvh(host(rec), p, host(perm), host(codes).view(np.uint64), sb)


@pytest.mark.parametrize("n", [1, 100, 4096, 4097, 100_003, 1_000_000])
@pytest.mark.parametrize("key_bits", [8, 16, 30, 32])
def test_sort_pairs_u32_matches_stable_argsort(n, key_bits):
    ab = _ab()
    g = np.random.default_rng(n + key_bits)
    hi = 1 << key_bits
    keys = g.integers(0, hi, size=n, dtype=np.uint64).astype(np.uint32)
    keys[: n // 3] = keys[0]  # many ties
    import torch
    sk, perm = ab.arborx_sort_pairs(torch.from_numpy(keys.view(np.int32)).cuda(), key_bits)
    want = np.argsort(keys, kind="stable")
    assert np.array_equal(host(perm), want)
    assert np.array_equal(host(sk).view(np.uint32), keys[want])


@pytest.mark.parametrize("n", [3, 3072, 3073, 500_000])
@pytest.mark.parametrize("key_bits", [40, 63, 64])
def test_sort_pairs_u64_matches_stable_argsort(n, key_bits):
    ab = _ab()
    import torch
    g = np.random.default_rng(n * 7 + key_bits)
    keys = g.integers(0, 1 << 62, size=n, dtype=np.uint64) & np.uint64((1 << key_bits) - 1)
    if key_bits == 64:
        keys |= np.uint64(1 << 63) * (g.integers(0, 2, size=n).astype(np.uint64))
    keys[::5] = keys[1]
    sk, perm = ab.arborx_sort_pairs(torch.from_numpy(keys.view(np.int64)).cuda(), key_bits)
    want = np.argsort(keys, kind="stable")
    assert np.array_equal(host(perm), want)
    assert np.array_equal(host(sk).view(np.uint64), keys[want])


@pytest.mark.parametrize("n", [50_000, 255, 512, 513, 65_539, 400_000])
def test_apetrei_and_karras_build_the_same_tree(n):
    # same binary radix tree up to node numbering: identical sets of (range, box)
    ab = _ab()
    p = datagen.gaussian_mixture(n, 77)
    trees = []
    for method in (0, 1):
        bvh = ab.BVH(dev(p), keep_order=1, build_method=method)
        rec, scene, codes, perm = bvh.export_tree(order=True)
        rec = host(rec)
        st = tree_check.check_lbvh(rec, p, host(perm), host(codes).view(np.uint64), host(scene))
        # child records sorted by content describe the tree independent of numbering
        kids = rec[2:].copy()
        enc = kids[:, 3].view(np.int32)
        kids[:, 3] = np.where(enc < 0, enc, 0).view(np.float32)  # keep leaves, forget internal ids
        trees.append((np.sort(kids.view(np.uint32).view([("", np.uint32)] * 8), axis=0), st["depth"]))
    assert np.array_equal(trees[0][0], trees[1][0])
    assert trees[0][1] == trees[1][1]


@pytest.mark.parametrize("cloud", ["cube", "cell_edges"])
def test_query_order_is_stable_morton_order(cloud):
    ab = _ab()
    if cloud == "cube":
        p = datagen.cube(20_000, 78)
        q = np.concatenate([datagen.cube(5000, 79) * 1.2 - 0.1, p[:100]]).astype(np.float32)  # some outside
    else:
        p = _cell_edges(20_000, 78)
        q = np.concatenate([_cell_edges(20_000, 79), _cell_edges(2000, 80) * 1.1 - 0.05]).astype(np.float32)
    bvh = ab.BVH(dev(p))
    order = host(bvh.query_order(dev(q))).astype(np.int64)
    sb, _ = oracle.scene_box(p)
    codes = oracle.morton(q, sb, 30) >> 6  # clamped into the tree's scene box; top 24 bits order
    assert np.array_equal(order, np.lexsort((np.arange(len(q)), codes)))


def test_traversal_statistics():
    ab = _ab()
    p, q = datagen.workload("cube", 100_000, 10_000, 80)
    bvh = ab.BVH(dev(p), stats=1)
    bvh.query_spatial(dev(q), 0.02)
    bvh.query_nearest(dev(q), 10)
    st = bvh.stats()
    assert st["spatial_queries"] == 10_000 and st["nearest_queries"] == 10_000
    # every query loads at least the root's children, at most every internal node twice (2 passes)
    assert 10_000 * 2 <= st["spatial_nodes"] <= 2 * 10_000 * 99_999
    assert 10_000 <= st["nearest_nodes"] <= 10_000 * 99_999
    assert bvh.stats()["nearest_nodes"] == 0  # reset
