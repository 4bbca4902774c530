"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed-form lattice counts, hand-derived Morton codes, integer enumeration,
scipy's k-d tree in float64, brute force on tiny inputs, and planted mistakes
that each pin must catch."""
import itertools
import math
import os

import numpy as np
import pytest

import datagen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ lattice

def _lattice(side):
    return datagen.lattice(side)


def test_lattice_golden_counts_by_integer_enumeration():
    # the stored counts are arithmetic facts: recount them with integers only
    for r, cnt, strict in _read_golden("lattice_counts.txt"):
        r = float(r)
        R = int(math.ceil(r))
        pts = itertools.product(range(-R, R + 1), repeat=3)
        sq = [x * x + y * y + z * z for x, y, z in pts]
        assert sum(s <= r * r for s in sq) == int(cnt)
        assert sum(s < r * r for s in sq) == int(strict)


@pytest.mark.parametrize("evaluator", ["brute", "bvh"])
def test_lattice_interior_counts(evaluator):
    side = 14
    pts = _lattice(side)
    bvh = oracle.CpuBVH(pts) if evaluator == "bvh" else None
    for r, cnt, _ in _read_golden("lattice_counts.txt"):
        r = float(r)
        R = int(math.ceil(r))
        ax = np.arange(R, side - R)
        z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
        sites = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.float32)
        if evaluator == "brute":
            off, _ = oracle.spatial_brute(pts, sites, r)
            counts = np.diff(off)
        else:
            counts = bvh.spatial_count(sites, r)
        assert np.all(counts == int(cnt)), (r, np.unique(counts))


def test_lattice_boundary_counts_match_clipped_enumeration():
    side = 9
    pts = _lattice(side)
    g = np.random.default_rng(3)
    sites = g.integers(0, side, size=(200, 3))
    for r in (1.0, 2.5, 4.0):
        off, idx = oracle.spatial_brute(pts, sites.astype(np.float32), r)
        for j, (sx, sy, sz) in enumerate(sites):
            R = int(math.ceil(r))
            want = sorted(
                int(x + side * y + side * side * z)
                for x in range(sx - R, sx + R + 1) for y in range(sy - R, sy + R + 1) for z in range(sz - R, sz + R + 1)
                if 0 <= x < side and 0 <= y < side and 0 <= z < side
                and (x - sx) ** 2 + (y - sy) ** 2 + (z - sz) ** 2 <= r * r)
            assert sorted(idx[off[j]:off[j + 1]].tolist()) == want


@pytest.mark.parametrize("evaluator", ["brute", "bvh"])
def test_lattice_knn27_is_the_3x3x3_block(evaluator):
    side = 10
    pts = _lattice(side)
    ax = np.arange(1, side - 1)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    sites = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    q = sites.astype(np.float32)
    if evaluator == "brute":
        idx, d2 = oracle.nearest_brute(pts, q, 27)
    else:
        idx, d2 = oracle.CpuBVH(pts).nearest(q, 27)
    off = np.array([dx + side * dy + side * side * dz for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
    base = sites[:, 0] + side * sites[:, 1] + side * side * sites[:, 2]
    want = np.sort(base[:, None] + off[None, :], axis=1)
    assert np.array_equal(np.sort(idx, axis=1), want)
    # rows are in (d2, index) order and distances are the shells 0,1,2,3
    assert np.all(np.diff(d2, axis=1) >= 0)
    assert np.array_equal(np.unique(d2), np.array([0, 1, 2, 3], np.float32))


def test_lattice_knn_tie_break_at_boundary_shell():
    # k = 7 cuts inside the d2 = 1 shell? no: 1 + 6 = 7 exactly.  k = 10 cuts
    # inside the d2 = 2 shell (12 ties): the 3 lowest indices of that shell win.
    side = 7
    pts = _lattice(side)
    s = np.array([[3, 3, 3]])
    idx, d2 = oracle.nearest_brute(pts, s.astype(np.float32), 10)
    c = 3 + side * 3 + side * side * 3
    shell2 = sorted(c + dx + side * dy + side * side * dz
                    for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3) if dx * dx + dy * dy + dz * dz == 2)
    assert idx[0, 7:].tolist() == shell2[:3]
    assert np.all(d2[0, 7:] == 2)


# ------------------------------------------------------------------ Morton

def test_morton_golden():
    for kb, x, y, z, code in _read_golden("morton.txt"):
        prims = np.array([[0, 0, 0], [1, 1, 1], [float(x), float(y), float(z)]], np.float32)
        sb, bad = oracle.scene_box(prims)
        assert bad == 0 and np.array_equal(sb, [0, 0, 0, 1, 1, 1])
        got = oracle.morton(prims, sb, int(kb))[2]
        assert int(got) == int(code, 16), (kb, x, y, z, hex(int(got)))


def test_morton_bits_deinterleave():
    # decode each code with string manipulation and compare with the integer
    # quantisation floor(u * 1024) computed in float64 (exact for these inputs)
    g = np.random.default_rng(5)
    qi = g.integers(0, 1024, size=(500, 3))
    u = (qi + 0.5) / 1024.0
    prims = np.concatenate([np.array([[0, 0, 0], [1, 1, 1]]), u]).astype(np.float32)
    sb, _ = oracle.scene_box(prims)
    codes = oracle.morton(prims, sb, 30)[2:]
    for c, (a, b, d) in zip(codes, qi):
        s = format(int(c), "030b")
        assert int(s[0::3], 2) == a and int(s[1::3], 2) == b and int(s[2::3], 2) == d


def test_morton_planted_axis_swap_is_caught():
    # a transposed operand (x and y swapped) must fail the golden values
    prims = np.array([[0, 0, 0], [1, 1, 1], [1, 0, 0]], np.float32)
    sb, _ = oracle.scene_box(prims)
    swapped = prims[:, [1, 0, 2]]
    assert int(oracle.morton(swapped, sb, 30)[2]) != 0x24924924


def test_morton_boxes_use_centroid_and_flat_axis():
    boxes = np.array([[0, 5, 0, 0, 5, 0], [1, 5, 1, 1, 5, 1], [0.25, 5, 0.5, 0.75, 5, 0.5]], np.float32)
    sb, _ = oracle.scene_box(boxes)
    assert np.array_equal(sb, [0, 5, 0, 1, 5, 1])
    # centroid (0.5, 5, 0.5): y axis is flat (u = 0): x = z = 512
    code = int(oracle.morton(boxes, sb, 30)[2])
    assert code == (1 << 29) | (1 << 27)


def test_scene_box_matches_numpy_and_flags_nonfinite():
    p = datagen.cube(1000, 7)
    sb, bad = oracle.scene_box(p)
    assert bad == 0
    assert np.array_equal(sb[:3], p.min(0)) and np.array_equal(sb[3:], p.max(0))
    b = datagen.boxes(1000, 7)
    sb, _ = oracle.scene_box(b)
    assert np.array_equal(sb[:3], np.minimum(b[:, :3].min(0), b[:, 3:].min(0)))
    assert np.array_equal(sb[3:], np.maximum(b[:, :3].max(0), b[:, 3:].max(0)))
    p[17, 1] = np.nan
    p[18, 2] = np.inf
    assert oracle.scene_box(p)[1] == 2


# --------------------------------------------------- brute force vs library

def test_spatial_brute_vs_scipy_kdtree_float64():
    from scipy.spatial import cKDTree
    p, q = datagen.workload("cube", 3000, 500, 11)
    r = datagen.radius_for_mean(3000, "cube")
    off, idx = oracle.spatial_brute(p, q, r)
    tree = cKDTree(p.astype(np.float64))
    ref = tree.query_ball_point(q.astype(np.float64), r)
    for j in range(len(q)):
        a = set(idx[off[j]:off[j + 1]].tolist())
        b = set(ref[j])
        for i in a ^ b:  # disagreement only at the rounding edge of the radius
            d = np.linalg.norm(q[j].astype(np.float64) - p[i].astype(np.float64))
            assert abs(d - r) <= 1e-6 * r


def test_nearest_brute_vs_scipy_kdtree_float64():
    from scipy.spatial import cKDTree
    p, q = datagen.workload("hollow_sphere", 4000, 400, 12)
    idx, d2 = oracle.nearest_brute(p, q, 10)
    dd, ii = cKDTree(p.astype(np.float64)).query(q.astype(np.float64), 10)
    assert np.allclose(np.sqrt(d2.astype(np.float64)), dd, rtol=1e-6, atol=0)
    same = idx == ii
    assert same.mean() > 0.99  # any difference is a tie or a last-ulp swap
    for j, t in zip(*np.nonzero(~same)):
        assert abs(math.sqrt(d2[j, t]) - dd[j, t]) <= 1e-6 * dd[j, t]


# ------------------------------------------------ brute force vs CPU BVH

CLOUDS = {
    "cube": lambda: datagen.workload("cube", 20000, 3000, 21),
    "hollow_sphere": lambda: datagen.workload("hollow_sphere", 20000, 3000, 22),
    "gaussian_mixture": lambda: datagen.workload("gaussian_mixture", 20000, 3000, 23),
    "duplicates": lambda: (np.repeat(datagen.cube(500, 24), 8, axis=0), datagen.cube(800, 25)),
    "flat_plane": lambda: (np.concatenate([datagen.cube(5000, 26)[:, :2], np.full((5000, 1), 0.5, np.float32)], 1),
                           datagen.cube(800, 27)),
    "collinear": lambda: (np.stack([np.linspace(0, 1, 3000, dtype=np.float32)] * 3, 1), datagen.cube(500, 28)),
}


@pytest.mark.parametrize("name", sorted(CLOUDS))
def test_bvh_equals_brute_spatial(name):
    p, q = CLOUDS[name]()
    r = 0.05
    ob, ib = oracle.spatial_brute(p, q, r)
    ot, it = oracle.CpuBVH(p).spatial(q, r)
    assert oracle.rows_as_sets_equal(ob, ib, ot, it) is None


@pytest.mark.parametrize("name", sorted(CLOUDS))
@pytest.mark.parametrize("k", [1, 10, 27])
def test_bvh_equals_brute_nearest(name, k):
    p, q = CLOUDS[name]()
    ib, db = oracle.nearest_brute(p, q, k)
    it, dt = oracle.CpuBVH(p).nearest(q, k)
    assert np.array_equal(ib, it)
    assert np.array_equal(db, dt)


def test_boxes_bvh_equals_brute():
    b = datagen.boxes(20000, 31, half_max=0.01)
    q = datagen.cube(2000, 32)
    ob, ib = oracle.spatial_brute(b, q, 0.02)
    ot, it = oracle.CpuBVH(b).spatial(q, 0.02)
    assert oracle.rows_as_sets_equal(ob, ib, ot, it) is None
    assert np.array_equal(oracle.nearest_brute(b, q, 10)[0], oracle.CpuBVH(b).nearest(q, 10)[0])


def test_box_distance_zero_inside_and_gap_outside():
    b = np.array([[0, 0, 0, 1, 1, 1]], np.float32)
    q = np.array([[0.5, 0.5, 0.5], [2, 0.5, 0.5], [2, 3, 0.5], [-1, -1, -1]], np.float32)
    _, d2 = oracle.nearest_brute(b, q, 1)
    assert d2[:, 0].tolist() == [0.0, 1.0, 5.0, 3.0]


# -------------------------------------------------------------- edge cases

def test_empty_and_tiny_inputs():
    q = datagen.cube(50, 41)
    for n in (0, 1, 2):
        p = datagen.cube(n, 42).reshape(n, 3)
        off, idx = oracle.spatial_brute(p, q, 0.7)
        ot, it = oracle.CpuBVH(p).spatial(q, 0.7)
        assert oracle.rows_as_sets_equal(off, idx, ot, it) is None
        ib, db = oracle.nearest_brute(p, q, 5)
        assert ib.shape == (50, min(5, n))
        it, dt = oracle.CpuBVH(p).nearest(q, 5)
        assert np.array_equal(ib, it)
        if n:
            full = np.sum((q[:, None, :].astype(np.float64) - p[None].astype(np.float64)) ** 2, -1)
            assert np.array_equal(np.argsort(full, axis=1, kind="stable")[:, :n], ib)
    off, idx = oracle.spatial_brute(datagen.cube(10, 43), np.zeros((0, 3), np.float32), 1.0)
    assert off.tolist() == [0] and idx.size == 0


def test_ties_lower_index_wins_and_duplicates_all_returned():
    p = np.zeros((6, 3), np.float32)
    p[3] = [1, 0, 0]
    q = np.zeros((1, 3), np.float32)
    idx, d2 = oracle.nearest_brute(p, q, 3)
    assert idx.tolist() == [[0, 1, 2]]
    off, ind = oracle.spatial_brute(p, q, 0.0)  # self-matches at d = 0 are returned
    assert sorted(ind.tolist()) == [0, 1, 2, 4, 5]
    it, _ = oracle.CpuBVH(p).nearest(q, 3)
    assert it.tolist() == [[0, 1, 2]]


def test_nonfinite_query_has_no_neighbours():
    p = datagen.cube(100, 44)
    q = np.array([[np.nan, 0, 0], [0.5, 0.5, 0.5], [np.inf, 0, 0]], np.float32)
    off, idx = oracle.spatial_brute(p, q, 10.0)
    assert np.diff(off).tolist() == [0, 100, 0]
    ib, db = oracle.nearest_brute(p, q, 4)
    assert ib[0].tolist() == [-1] * 4 and ib[2].tolist() == [-1] * 4 and np.all(np.isinf(db[0]))
    it, _ = oracle.CpuBVH(p).nearest(q, 4)
    assert np.array_equal(ib, it)


# ---------------------------------------------------------- FP64 checker

def test_fp64_checker_accepts_fp32_results_and_catches_planted_errors():
    p, q = datagen.workload("cube", 5000, 300, 51)
    r = datagen.radius_for_mean(5000, "cube")
    off, idx = oracle.spatial_brute(p, q, r)
    sample = np.arange(300)
    bad, tol = oracle.fp64_check_spatial(p, q, r, off, idx, sample)
    assert bad == 0
    # plant: drop the last index of a non-empty row
    j = int(np.nonzero(np.diff(off) > 0)[0][0])
    keep = np.ones(idx.size, bool)
    keep[off[j + 1] - 1] = False
    off2 = off.copy()
    off2[j + 1:] -= 1
    assert oracle.fp64_check_spatial(p, q, r, off2, idx[keep], sample)[0] >= 1
    # plant: a wrong neighbour
    idx3 = idx.copy()
    idx3[off[j]] = (idx3[off[j]] + 2500) % 5000
    assert oracle.fp64_check_spatial(p, q, r, off, idx3, sample)[0] >= 1

    ik, _ = oracle.nearest_brute(p, q, 10)
    assert oracle.fp64_check_nearest(p, q, 10, ik, sample)[0] == 0
    ik2 = ik.copy()
    ik2[5, 9] = ik2[6, 9] if ik2[6, 9] not in ik2[5] else (ik2[5, 9] + 1) % 5000
    assert oracle.fp64_check_nearest(p, q, 10, ik2, sample)[0] >= 1


def test_fp64_checker_tolerates_only_radius_edge():
    # a point exactly at the FP32 radius edge: FP32 and FP64 may disagree, tolerated
    p = np.array([[0.1, 0.2, 0.3], [0.5, 0.5, 0.5]], np.float32)
    q = np.zeros((1, 3), np.float32)
    r = float(np.sqrt(np.float32(0.1) ** 2 + np.float32(0.2) ** 2 + np.float32(0.3) ** 2))
    off, idx = oracle.spatial_brute(p, q, r)
    bad, tol = oracle.fp64_check_spatial(p, q, r, off, idx, np.array([0]))
    assert bad == 0


def test_strict_radius_reading_would_fail_lattice_pin():
    # planted mistake: treat the ball as open (shrink r by one ulp) -> 1 / 81 / 251
    side = 12
    pts = _lattice(side)
    site = np.array([[6, 6, 6]], np.float32)
    for r, cnt, strict in _read_golden("lattice_counts.txt"):
        r_open = float(np.nextafter(np.float32(float(r)), np.float32(0)))
        off, _ = oracle.spatial_brute(pts, site, r_open)
        assert int(np.diff(off)[0]) == int(strict) != int(cnt) or int(strict) == int(cnt)


def test_paper_shapes_count_statistics():
    # sanity of the paper-shapes generator (Sec. 3.1), not a parity pin: with the radius for a mean
    # of 10 neighbours in the filled cube, filled-sphere queries find about 10 on average (fewer
    # near the cube faces, none beyond), while hollow-sphere queries against the hollow cube mostly
    # find few points and a long tail near the face centres
    import datagen
    p = 10_000
    r = datagen.paper_radius(p)
    o, _ = oracle.spatial_brute(datagen.paper_shape(p, "filled_cube", 8), datagen.paper_shape(p, "filled_sphere", 9), r)
    c = np.diff(o)
    assert 9.5 < c.mean() < 10.5 and c.min() == 0 and 15 <= c.max() <= 40
    o, _ = oracle.spatial_brute(datagen.paper_shape(p, "hollow_cube", 10), datagen.paper_shape(p, "hollow_sphere", 11), r)
    c = np.diff(o)
    assert 1.5 < c.mean() < 4.5 and c.min() == 0 and c.max() >= 8 * c.mean()


# ------------------------------------------------------------------ box queries

def _lattice_box_rows(side, qboxes):
    """Rows of box queries over the side^3 lattice by integer enumeration: per axis the sites
    from ceil(lo) to floor(hi), clipped to the grid (exact: the float32 bounds are exact in float64
    and the sites are integers)."""
    rows = []
    for b in np.asarray(qboxes, np.float64):
        axes = []
        for a in range(3):
            lo, hi = max(math.ceil(b[a]), 0), min(math.floor(b[3 + a]), side - 1)
            axes.append(range(lo, hi + 1) if lo <= hi else range(0))
        rows.append(sorted(x + side * y + side * side * z for z in axes[2] for y in axes[1] for x in axes[0]))
    return rows


def _lattice_query_boxes(side, m, seed):
    g = np.random.default_rng(seed)
    lo = g.uniform(-3, side + 2, (m, 3))
    ext = g.uniform(0, 5, (m, 3)) * (g.random((m, 3)) < 0.9)  # some axes flat
    qb = np.concatenate([lo, lo + ext], 1)
    # integer bounds and zero-extent boxes at sites: every boundary case of the closed reading
    ints = g.integers(-1, side + 1, (m // 4, 3)).astype(np.float64)
    qb[: m // 4, :3] = ints
    qb[: m // 4, 3:] = ints + g.integers(0, 3, (m // 4, 3)) * (g.random((m // 4, 1)) < 0.7)
    return qb.astype(np.float32)


@pytest.mark.parametrize("evaluator", ["brute", "bvh"])
def test_box_query_lattice_rows_by_integer_enumeration(evaluator):
    side = 16
    pts = _lattice(side)
    qb = _lattice_query_boxes(side, 600, 11)
    want = _lattice_box_rows(side, qb)
    off, idx = oracle.intersects_brute(pts, qb) if evaluator == "brute" else oracle.CpuBVH(pts).intersects(qb)
    assert sum(len(r) for r in want) > 1000
    for j, row in enumerate(want):
        assert sorted(idx[off[j]:off[j + 1]].tolist()) == row, j


def test_box_query_lattice_pin_catches_planted_mistakes():
    # open intervals or a swapped axis pair give other rows on the same cases
    side = 16
    qb = _lattice_query_boxes(side, 600, 11)
    want = _lattice_box_rows(side, qb)
    strict = []
    for b in np.asarray(qb, np.float64):
        axes = [range(max(math.floor(b[a]) + 1, 0), min(math.ceil(b[3 + a]) - 1, side - 1) + 1) for a in range(3)]
        strict.append(sorted(x + side * y + side * side * z for z in axes[2] for y in axes[1] for x in axes[0]))
    assert strict != want
    swapped = _lattice_box_rows(side, qb[:, [1, 0, 2, 4, 3, 5]])
    assert swapped != want


def test_box_query_unit_boxes_on_a_line_closed_form():
    # boxes [i, i+1] x [0,1] x [0,1]: a query [a, b] on x meets box i iff i <= b and i + 1 >= a
    n = 50
    i = np.arange(n, dtype=np.float64)
    prims = np.stack([i, 0 * i, 0 * i, i + 1, 0 * i + 1, 0 * i + 1], 1).astype(np.float32)
    g = np.random.default_rng(5)
    ab = np.sort(g.integers(-6, 2 * n + 6, (300, 2)) / 2.0, axis=1)
    qb = np.stack([ab[:, 0], np.full(300, 0.25), np.full(300, 0.25), ab[:, 1], np.full(300, 0.75),
                   np.full(300, 0.75)], 1).astype(np.float32)
    for off, idx in (oracle.intersects_brute(prims, qb), oracle.CpuBVH(prims).intersects(qb)):
        for j, (a, b) in enumerate(ab):
            lo, hi = max(math.ceil(a) - 1, 0), min(math.floor(b), n - 1)
            assert sorted(idx[off[j]:off[j + 1]].tolist()) == list(range(lo, hi + 1)), (a, b)


def test_box_query_holds_the_ball_results():
    # a point within distance r of q lies in the cube [q - r, q + r] (widened by 1e-3 r for the
    # rounding of d^2): the box rows contain the radius rows
    p = datagen.cube(4000, 3)
    q = datagen.cube(500, 3, datagen.STREAM_QUERIES)
    r = 0.06
    off_s, idx_s = oracle.spatial_brute(p, q, r)
    h = r * 1.001
    qb = np.concatenate([q.astype(np.float64) - h, q.astype(np.float64) + h], 1).astype(np.float32)
    off_b, idx_b = oracle.intersects_brute(p, qb)
    assert np.all(np.diff(off_b) >= np.diff(off_s))
    for j in range(500):
        assert set(idx_s[off_s[j]:off_s[j + 1]].tolist()) <= set(idx_b[off_b[j]:off_b[j + 1]].tolist())
    assert np.diff(off_b).sum() > np.diff(off_s).sum()  # the cube's corners hold more


def test_box_query_nan_infinite_and_inverted_bounds():
    inf = np.inf
    pts = _lattice(4)
    boxes = np.array([[0, 0, 0, 10, 10, 10], [20, 20, 20, 30, 30, 30]], np.float32)
    qb = np.array([[np.nan, 0, 0, 3, 3, 3],        # NaN bound: nothing
                   [-inf, -inf, -inf, inf, inf, inf],  # everything
                   [6, -1, -1, 4, 11, 11],           # x inverted: the test alone decides
                   [1, 1, 1, 1, 1, 1]], np.float32)  # a zero-extent box
    off, idx = oracle.intersects_brute(pts, qb)
    assert np.diff(off).tolist() == [0, 64, 0, 1] and idx[off[3]] == 1 + 4 + 16
    off, idx = oracle.intersects_brute(boxes, qb)
    # box [0,10]^3 meets the inverted x-interval [6, 4] (0 <= 4 and 10 >= 6); [20,30]^3 does not
    assert [sorted(idx[off[j]:off[j + 1]].tolist()) for j in range(4)] == [[], [0, 1], [0], [0]]
