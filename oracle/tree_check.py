"""Invariants of a linear BVH -- TEST INFRASTRUCTURE ONLY.

Checks a tree exported by the library against what the paper's construction
fixes (Sec. 2, Sec. 2.1), independently of how the tree was built:

* a binary tree over n leaves has n - 1 internal nodes, every node reachable
  from the root exactly once (Sec. 2: one internal node fewer than leaves);
* the root box is the scene box (Sec. 2: the root bounds every object);
* every node box is the union of its children's boxes, leaves hold their
  primitive's box (Sec. 2.1, the bottom-up box step);
* the aux word of every record counts the leaves under it (1 for a leaf, n
  for the root record), the library's documented format;
* leaves are ordered by Morton code, the codes of the leaves are
  non-decreasing, the permutation is a permutation, and each internal node
  covers a contiguous range of sorted leaves split at the highest differing
  bit of the index-augmented code (Sec. 2.1, sort and hierarchy steps).

Exported layout being checked (the library's documented format): ``records``
float32 [2 + 2 (n - 1)][8]; a record is (lo.x, lo.y, lo.z, enc, hi.x, hi.y,
hi.z, aux) with ``enc`` an int32 bit pattern: enc >= 0 is an internal node id,
enc < 0 a leaf holding primitive ~enc, and ``aux`` the int32 bit pattern of
the number of leaves under the record.  Record 0 describes the root; the
children of internal node p are records 2 + 2p (left) and 3 + 2p (right).
"""
from __future__ import annotations

import numpy as np


class TreeError(AssertionError):
    pass


def _fail(msg):
    raise TreeError(msg)


def prim_boxes(prims: np.ndarray) -> np.ndarray:
    prims = np.asarray(prims, np.float32)
    if prims.shape[1] == 3:
        return np.concatenate([prims, prims], axis=1)
    return prims


def _delta(codes_aug_hi, codes_aug_lo, i, j):
    """Length of the common prefix of the index-augmented keys (code, position)."""
    hi_i, hi_j = codes_aug_hi[i], codes_aug_hi[j]
    x = hi_i ^ hi_j
    out = np.empty(i.shape, np.int64)
    same = x == 0
    # key part differs: count leading zeros of the 64-bit xor
    xs = x[~same].astype(np.uint64)
    lz = np.full(xs.shape, 64, np.int64)
    for b in range(63, -1, -1):
        hit = ((xs >> np.uint64(b)) & np.uint64(1)).astype(bool) & (lz == 64)
        lz[hit] = 63 - b
    out[~same] = lz
    y = (codes_aug_lo[i[same]] ^ codes_aug_lo[j[same]]).astype(np.uint64)
    lz2 = np.full(y.shape, 64, np.int64)
    for b in range(63, -1, -1):
        hit = ((y >> np.uint64(b)) & np.uint64(1)).astype(bool) & (lz2 == 64)
        lz2[hit] = 63 - b
    out[same] = 64 + lz2
    return out


def check_lbvh(records: np.ndarray, prims: np.ndarray, perm: np.ndarray | None = None,
               codes: np.ndarray | None = None, scene: np.ndarray | None = None,
               check_split: bool = True, check_counts: bool = True) -> dict:
    """Raise TreeError on the first violated invariant; return summary stats."""
    prims = np.asarray(prims, np.float32)
    n = prims.shape[0]
    boxes = prim_boxes(prims)
    rec = np.asarray(records, np.float32).reshape(-1, 8)
    if n == 0:
        return dict(n=0, depth=0)
    n_int = n - 1
    if rec.shape[0] < 2 + 2 * n_int:
        _fail(f"records too short: {rec.shape[0]} < {2 + 2 * n_int}")
    rec = rec[: 2 + 2 * n_int]
    enc = rec[:, 3].view(np.int32)
    lo = rec[:, 0:3]
    hi = rec[:, 4:7]

    # scene box / root box
    if scene is not None:
        scene = np.asarray(scene, np.float32)
        if not (np.array_equal(lo[0], scene[:3]) and np.array_equal(hi[0], scene[3:])):
            _fail(f"root box {lo[0]},{hi[0]} != scene box {scene}")
    true_lo = boxes[:, :3].min(axis=0)
    true_hi = boxes[:, 3:].max(axis=0)
    if not (np.array_equal(lo[0], true_lo) and np.array_equal(hi[0], true_hi)):
        _fail(f"root box {lo[0]},{hi[0]} != union of primitive boxes {true_lo},{true_hi}")

    aux = rec[:, 7].view(np.int32)
    if n == 1:
        if enc[0] != ~0:
            _fail(f"single-leaf root must hold primitive 0, enc={enc[0]}")
        if check_counts and aux[0] != 1:
            _fail(f"single-leaf root record counts {aux[0]} leaves, expected 1")
        return dict(n=1, depth=0)
    root = int(enc[0])
    if root < 0 or root >= n_int:
        _fail(f"root record must point at an internal node, enc={root}")

    child = enc[2:].reshape(n_int, 2)
    # every internal id other than the root appears exactly once as a child
    internal_children = child[child >= 0]
    if internal_children.size != n_int - 1:
        _fail(f"{internal_children.size} internal child slots, expected {n_int - 1}")
    if np.any(internal_children == root) or np.any(internal_children >= n_int):
        _fail("internal child id out of range or pointing at the root")
    if np.unique(internal_children).size != internal_children.size:
        _fail("an internal node has two parents")
    leaf_prims = ~child[child < 0]
    if leaf_prims.size != n or np.unique(leaf_prims).size != n or leaf_prims.min() < 0 or leaf_prims.max() >= n:
        _fail("leaves do not hold each primitive exactly once")

    # BFS from the root: reachability, depth, parent links
    parent = np.full(n_int, -1, np.int64)
    slot_of = np.full(n_int, -1, np.int64)  # record slot holding the node's own box
    slot_of[root] = 0
    frontier = np.array([root], np.int64)
    seen = 1
    depth = 0
    while frontier.size:
        depth += 1
        kids = np.stack([2 + 2 * frontier, 3 + 2 * frontier], axis=1).ravel()
        kid_enc = enc[kids]
        is_int = kid_enc >= 0
        nxt = kid_enc[is_int].astype(np.int64)
        parent[nxt] = np.repeat(frontier, 2)[is_int]
        slot_of[nxt] = kids[is_int]
        seen += nxt.size
        frontier = nxt
        if depth > 4 * 64 + 8:
            _fail("tree deeper than any LBVH over these keys can be (cycle?)")
    if seen != n_int:
        _fail(f"{seen} internal nodes reachable from the root, expected {n_int}")

    # node box = union of child boxes (exact); leaf record = primitive box
    node_lo = lo[slot_of]
    node_hi = hi[slot_of]
    lchild = 2 + 2 * np.arange(n_int)
    rchild = lchild + 1
    ulo = np.minimum(lo[lchild], lo[rchild])
    uhi = np.maximum(hi[lchild], hi[rchild])
    badn = np.nonzero(~(np.all(ulo == node_lo, axis=1) & np.all(uhi == node_hi, axis=1)))[0]
    if badn.size:
        p = int(badn[0])
        _fail(f"node {p} box {node_lo[p]},{node_hi[p]} != union of children {ulo[p]},{uhi[p]}")
    leaf_slots = np.nonzero(enc[2:] < 0)[0] + 2
    lp = ~enc[leaf_slots]
    if not (np.array_equal(lo[leaf_slots], boxes[lp, :3]) and np.array_equal(hi[leaf_slots], boxes[lp, 3:])):
        _fail("a leaf record does not hold its primitive's box")

    if check_counts:
        # leaves under each internal node, bottom-up over the BFS levels
        levels = []
        fr = np.array([root], np.int64)
        while fr.size:
            levels.append(fr)
            kids = enc[np.stack([2 + 2 * fr, 3 + 2 * fr], axis=1).ravel()]
            fr = kids[kids >= 0].astype(np.int64)
        under = np.zeros(n_int, np.int64)
        for lev in reversed(levels):
            for side in (2, 3):
                e = enc[side + 2 * lev].astype(np.int64)
                under[lev] += np.where(e < 0, 1, under[np.where(e < 0, 0, e)])
        want = np.where(enc[2:] < 0, 1, under[np.where(enc[2:] < 0, 0, enc[2:])])
        bad = np.nonzero(aux[2:] != want)[0]
        if bad.size:
            r = int(bad[0]) + 2
            _fail(f"record {r} counts {aux[r]} leaves, expected {want[bad[0]]}")
        if aux[0] != n:
            _fail(f"root record counts {aux[0]} leaves, expected {n}")

    stats = dict(n=n, depth=depth)
    if perm is None:
        return stats

    perm = np.asarray(perm).astype(np.int64)
    if perm.shape != (n,) or not np.array_equal(np.sort(perm), np.arange(n)):
        _fail("perm is not a permutation of 0..n-1")
    pos = np.empty(n, np.int64)
    pos[perm] = np.arange(n)
    if codes is not None:
        codes = np.asarray(codes).astype(np.uint64)
        if np.any(codes[1:] < codes[:-1]):
            _fail("sorted codes decrease")
        eq = codes[1:] == codes[:-1]
        if np.any(eq & (perm[1:] < perm[:-1])):
            _fail("equal codes not in index order (sort not stable)")

    # leaf-position range per internal node, bottom-up by reverse BFS order
    order = []
    frontier = np.array([root], np.int64)
    while frontier.size:
        order.append(frontier)
        kids = enc[np.stack([2 + 2 * frontier, 3 + 2 * frontier], axis=1).ravel()]
        frontier = kids[kids >= 0].astype(np.int64)
    rmin = np.zeros(n_int, np.int64)
    rmax = np.zeros(n_int, np.int64)
    cnt = np.zeros(n_int, np.int64)
    for level in reversed(order):
        le = enc[2 + 2 * level].astype(np.int64)
        re = enc[3 + 2 * level].astype(np.int64)

        def rng_of(e):
            leaf = e < 0
            pmn = np.where(leaf, pos[np.where(leaf, ~e, 0)], rmin[np.where(leaf, 0, e)])
            pmx = np.where(leaf, pos[np.where(leaf, ~e, 0)], rmax[np.where(leaf, 0, e)])
            c = np.where(leaf, 1, cnt[np.where(leaf, 0, e)])
            return pmn, pmx, c

        a0, a1, ac = rng_of(le)
        b0, b1, bc = rng_of(re)
        if np.any(a1 + 1 != b0):
            _fail("left child range does not end right before the right child range")
        rmin[level] = a0
        rmax[level] = b1
        cnt[level] = ac + bc
    if np.any(rmax - rmin + 1 != cnt):
        _fail("an internal node covers a non-contiguous leaf range")
    if rmin[root] != 0 or rmax[root] != n - 1:
        _fail("root does not cover all leaves")

    if check_split and codes is not None:
        # split at the highest differing bit of (code, position): the split
        # boundary has the smallest common prefix of all adjacent pairs in range
        idx = np.arange(n_int)
        le = enc[2 + 2 * idx].astype(np.int64)
        split = np.where(le < 0, pos[np.where(le < 0, ~le, 0)], rmax[np.where(le < 0, 0, le)])
        codes_hi = codes
        codes_lo = np.arange(n, dtype=np.uint64)
        d_split = _delta(codes_hi, codes_lo, split, split + 1)
        d_range = _delta(codes_hi, codes_lo, rmin, rmax)
        if np.any(d_split != d_range):
            p = int(np.nonzero(d_split != d_range)[0][0])
            _fail(f"node {p} is not split at the highest differing bit of its range")
    return stats
