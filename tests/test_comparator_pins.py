"""Pins of the comparators behind every parity assertion.

Spatial rows (Sec. 2.2.1) are sets: the traversal order inside a row is not
part of the result, so ``oracle.rows_as_sets_equal`` compares each CSR row as a
sorted set.  Nearest rows (Sec. 2.2.2) are ordered by (d^2, index), so
``tests.gpu_helpers.assert_nearest_equal`` compares them entry by entry, with
the distances bit for bit.  Each test below plants one mistake that a plausible
GPU bug would make and checks that the comparator reports the row it sits in;
a comparator that compared only counts, sorted across rows instead of within
them, or ignored the distances would fail here.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_helpers import assert_nearest_equal, assert_spatial_equal

# five rows: [3, 1, 2] [] [7] [4, 9, 5, 6] [0, 8]
OFF = np.array([0, 3, 3, 4, 8, 10], np.int64)
IDX = np.array([3, 1, 2, 7, 4, 9, 5, 6, 0, 8], np.int32)


def _rows(off, idx):
    return [sorted(idx[off[i]:off[i + 1]].tolist()) for i in range(len(off) - 1)]


def _csr(rows):
    off = np.zeros(len(rows) + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    idx = np.array([v for r in rows for v in r], np.int32)
    return off, idx


def test_equal_rows_compare_equal_in_any_order_inside_a_row():
    rows = [list(reversed(r)) for r in _rows(OFF, IDX)]
    off, idx = _csr(rows)
    assert oracle.rows_as_sets_equal(off, idx, OFF, IDX) is None
    assert oracle.rows_as_sets_equal(OFF, IDX, off, idx) is None
    # a within-row permutation that is not a reversal either
    perm = IDX.copy()
    perm[4:8] = [6, 4, 5, 9]
    assert oracle.rows_as_sets_equal(OFF, perm, OFF, IDX) is None


def test_one_index_swapped_for_another_in_a_middle_row():
    idx = IDX.copy()
    idx[5] = 11  # row 3 holds 11 instead of 9; every count unchanged
    assert oracle.rows_as_sets_equal(OFF, idx, OFF, IDX) == 3
    assert oracle.rows_as_sets_equal(OFF, IDX, OFF, idx) == 3


def test_counts_equal_in_total_but_shifted_between_rows():
    # rows 0 and 2 trade one entry: [3, 1] [] [2, 7] -- same total, same multiset
    off = np.array([0, 2, 2, 4, 8, 10], np.int64)
    idx = np.array([3, 1, 2, 7, 4, 9, 5, 6, 0, 8], np.int32)
    assert np.array_equal(np.sort(idx), np.sort(IDX))
    assert oracle.rows_as_sets_equal(off, idx, OFF, IDX) == 0


def test_entries_traded_between_rows_with_counts_kept():
    # row 0 gets 7, row 2 gets 2: counts and the global multiset are unchanged, so only a
    # per-row comparison sees it (a sort keyed on the index alone, across rows, would not)
    idx = IDX.copy()
    idx[2], idx[3] = 7, 2
    assert oracle.rows_as_sets_equal(OFF, idx, OFF, IDX) == 0
    # the same trade between rows 3 and 4 (the first differing row is reported)
    idx = IDX.copy()
    idx[4], idx[8] = 0, 4
    assert oracle.rows_as_sets_equal(OFF, idx, OFF, IDX) == 3


def test_a_duplicate_in_place_of_a_distinct_index():
    idx = IDX.copy()
    idx[6] = 4  # row 3: [4, 9, 4, 6] against [4, 9, 5, 6]
    assert oracle.rows_as_sets_equal(OFF, idx, OFF, IDX) == 3
    # a duplicated entry in the row that lacks one of its own, both sides of the call
    assert oracle.rows_as_sets_equal(OFF, IDX, OFF, idx) == 3


def test_an_extra_index_in_the_last_row():
    off = np.append(OFF[:-1], OFF[-1] + 1)
    idx = np.append(IDX, np.int32(12))
    assert oracle.rows_as_sets_equal(off, idx, OFF, IDX) == 4
    assert oracle.rows_as_sets_equal(OFF, IDX, off, idx) == 4


def test_an_extra_row_or_a_missing_row():
    off = np.append(OFF, OFF[-1])
    assert oracle.rows_as_sets_equal(off, IDX, OFF, IDX) is not None
    assert oracle.rows_as_sets_equal(OFF[:-1], IDX[:8], OFF, IDX) is not None


def test_an_index_off_by_one_in_the_first_row():
    idx = IDX.copy()
    idx[0] += 1  # [4, 1, 2]
    assert oracle.rows_as_sets_equal(OFF, idx, OFF, IDX) == 0


def test_random_rows_with_one_planted_difference():
    g = np.random.default_rng(7)
    for trial in range(200):
        m = int(g.integers(1, 40))
        rows = [sorted(g.choice(1000, size=int(g.integers(0, 12)), replace=False).tolist()) for _ in range(m)]
        off, idx = _csr(rows)
        shuffled = [list(g.permutation(r)) for r in rows]
        off2, idx2 = _csr(shuffled)
        assert oracle.rows_as_sets_equal(off2, idx2, off, idx) is None
        nonempty = [i for i, r in enumerate(rows) if r]
        if not nonempty:
            continue
        bad = int(g.choice(nonempty))
        planted = [list(r) for r in shuffled]
        j = int(g.integers(0, len(planted[bad])))
        planted[bad][j] = 1000 + trial  # never in any row
        off3, idx3 = _csr(planted)
        assert oracle.rows_as_sets_equal(off3, idx3, off, idx) == bad


def test_assert_spatial_equal_names_the_row():
    idx = IDX.copy()
    idx[3] = 13
    assert_spatial_equal(OFF, IDX, OFF, IDX)
    with pytest.raises(AssertionError, match="row 2"):
        assert_spatial_equal(OFF, idx, OFF, IDX)


# ------------------------------------------------------------- nearest rows

KI = np.array([[4, 2, 9], [0, 1, 3], [7, 7 + 1, 5]], np.int32)
KD = np.array([[0.0, 0.25, 0.25], [0.5, 1.0, 1.0], [0.125, 2.0, 3.0]], np.float32)


def test_nearest_equal_rows_pass():
    assert_nearest_equal(KI.copy(), KD.copy(), KI, KD)
    assert_nearest_equal(KI.copy(), None, KI, KD)


def test_nearest_swapped_pair_is_caught():
    # two entries at the same distance swapped: the (d^2, index) order says the lower index first
    ki = KI.copy()
    ki[0, 1], ki[0, 2] = ki[0, 2], ki[0, 1]
    with pytest.raises(AssertionError, match="row 0"):
        assert_nearest_equal(ki, KD, KI, KD)
    ki = KI.copy()
    ki[1, 1], ki[1, 2] = ki[1, 2], ki[1, 1]
    with pytest.raises(AssertionError, match="row 1"):
        assert_nearest_equal(ki, KD, KI, KD)


def test_nearest_wrong_neighbour_is_caught():
    ki = KI.copy()
    ki[2, 2] = 6
    with pytest.raises(AssertionError, match="row 2"):
        assert_nearest_equal(ki, KD, KI, KD)


def test_nearest_distance_one_ulp_off_is_caught():
    for r, c in [(0, 0), (1, 2), (2, 1)]:
        kd = KD.copy()
        kd[r, c] = np.nextafter(kd[r, c], np.float32(np.inf))
        with pytest.raises(AssertionError):
            assert_nearest_equal(KI, kd, KI, KD)
        kd = KD.copy()
        kd[r, c] = np.nextafter(kd[r, c], np.float32(-np.inf))
        with pytest.raises(AssertionError):
            assert_nearest_equal(KI, kd, KI, KD)


def test_nearest_row_length_mismatch_is_caught():
    with pytest.raises(AssertionError):
        assert_nearest_equal(KI[:, :2], KD[:, :2], KI, KD)
    with pytest.raises(AssertionError):
        assert_nearest_equal(KI[:2], KD[:2], KI, KD)
