"""Pins of the modified-CMRS arrangement oracle (Section 6.6) against what
any valid arrangement must satisfy, independent of how the oracle builds it:
strips padded to multiples of 32 items; inside each 32-item warp pass the
items of one row are one contiguous run of at most M (so lanes that add into
slot lane mod M of a row never collide); the real items are exactly the
strip's items, each row's items in their original order; zero items change
no product; and the number of passes per strip meets its lower bound
max(ceil(items / 32), ceil(longest row / M))."""
import numpy as np
import pytest

import oracle
from paper_1203_2946_gb300 import inputs

M = 8


def check_arrangement(rows, h, cm, pad, slots=M):
    sp0, pk0 = cm["strip_ptr"], cm["packed"]
    sp1, pk1, src = pad["strip_ptr"], pad["packed"], pad["src"]
    bits = oracle.bits_for_height(h)
    mask = (1 << bits) - 1
    strips = (rows + h - 1) // h
    assert sp1.size == strips + 1 and sp1[0] == 0
    assert np.all(sp1 % 32 == 0)
    assert pk1.size == sp1[-1] == src.size
    for s in range(strips):
        a0, b0, a1, b1 = sp0[s], sp0[s + 1], sp1[s], sp1[s + 1]
        items = src[a1:b1]
        real = items[items >= 0]
        # real items: exactly this strip's items, once each
        assert np.array_equal(np.sort(real), np.arange(a0, b0))
        # packed words of real items are the source words; zero items carry column 0
        assert np.array_equal(pk1[a1:b1][items >= 0], pk0[real])
        assert np.all(pk1[a1:b1][items < 0] >> bits == 0)
        ris = pk1[a1:b1] & mask
        assert np.all(ris < h)
        # each row's real items keep their original order
        for r in range(h):
            mine = real[(pk0[real] & mask) == r]
            assert np.all(np.diff(mine) > 0)
        # per 32-item pass: each row is one contiguous run of at most `slots` items
        for c in range(a1, b1, 32):
            rr = ris[c - a1:c - a1 + 32]
            seen = set()
            run_start = 0
            for j in range(1, 33):
                if j == 32 or rr[j] != rr[j - 1]:
                    r = int(rr[j - 1])
                    assert r not in seen, "row %d has two runs in one pass" % r
                    seen.add(r)
                    assert j - run_start <= slots
                    run_start = j
        # lower bound on passes
        T = b0 - a0
        Lmax = int(np.bincount(pk0[a0:b0] & mask, minlength=h).max()) if T else 0
        assert (b1 - a1) // 32 == max(-(-T // 32), -(-Lmax // slots))


def arrange(a, h, slots=M):
    cm = oracle.csr_to_cmrs(a.row_ptr, a.col_ind, a.val, a.cols, h)
    return cm, oracle.pad_arrange(a.rows, h, cm["strip_ptr"], cm["packed"], slots)


@pytest.mark.parametrize("h,slots", [(4, 8), (5, 8), (8, 8), (16, 8), (17, 8), (32, 8), (8, 4), (16, 2),
                                     (17, 2), (32, 1)])
def test_random_strips(h, slots):
    rng = np.random.default_rng(h * 10 + slots)
    for trial in range(6):
        L = rng.integers(0, [3, 12, 40, 120][trial % 4], 300)
        L[rng.integers(0, 300, 3)] = rng.integers(0, 200, 3)  # a few long rows
        a = inputs.from_lengths(L, 500, seed=trial)
        cm, pad = arrange(a, h, slots)
        check_arrangement(a.rows, h, cm, pad, slots)


def test_one_slot_is_row_per_lane():
    """M = 1 at height 32: every pass holds one item of each row, row r at
    position r -- the layout in which the kernel keeps row sums in registers."""
    L = np.random.default_rng(9).integers(0, 40, 320)
    a = inputs.from_lengths(L, 500, seed=9)
    cm, pad = arrange(a, 32, 1)
    check_arrangement(a.rows, 32, cm, pad, 1)
    ris = pad["packed"] & 31
    assert np.array_equal(ris.reshape(-1, 32), np.tile(np.arange(32, dtype=np.uint32), (ris.size // 32, 1)))


def test_spmv_unchanged():
    """Algorithm 1 on the arranged strips gives the CRS product exactly: each
    row's items keep their order and zero items add +0.0."""
    L = np.random.default_rng(3).integers(0, 30, 1000)
    L[7] = 400
    a = inputs.from_lengths(L, 800, seed=4)
    x = np.random.default_rng(5).uniform(-1, 1, a.cols)
    y_ref, _ = oracle.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    for h in (4, 16, 32):
        cm, pad = arrange(a, h)
        v = np.where(pad["src"] >= 0, cm["val"][np.maximum(pad["src"], 0)], 0.0)
        y = oracle.cmrs_spmv(a.rows, h, pad["strip_ptr"], pad["packed"], v, x)
        assert np.array_equal(y, y_ref)


def test_degenerate():
    # empty matrix, empty strips, a ragged last strip, one row holding everything
    for L in (np.zeros(10, int), np.array([0, 0, 0, 0, 5]), np.r_[np.zeros(31, int), 100]):
        a = inputs.from_lengths(L, 200, seed=1)
        for h in (4, 16):
            cm, pad = arrange(a, h)
            check_arrangement(a.rows, h, cm, pad)
    a = inputs.from_lengths(np.zeros(10, int), 5, seed=1)
    cm, pad = arrange(a, 16)
    assert pad["strip_ptr"].tolist() == [0] and pad["packed"].size == 0 or pad["strip_ptr"][-1] == 0


def test_slot_count_too_small():
    a = inputs.from_lengths(np.ones(8, int), 8, seed=1)
    cm = oracle.csr_to_cmrs(a.row_ptr, a.col_ind, a.val, a.cols, 2)
    with pytest.raises(oracle.OracleError):
        oracle.pad_arrange(a.rows, 2, cm["strip_ptr"], cm["packed"], 8)  # 2 x 8 < 32 lanes


def test_catches_a_planted_mistake():
    """The checker rejects arrangements with a row split into two runs or
    with an item dropped (mistakes planted in the oracle's output)."""
    a = inputs.from_lengths(np.array([5, 3, 9, 2]), 40, seed=2)
    cm, pad = arrange(a, 4)
    bad = dict(pad)
    bad["src"] = pad["src"].copy()
    bad["src"][np.flatnonzero(bad["src"] >= 0)[0]] = -1
    with pytest.raises(AssertionError):
        check_arrangement(a.rows, 4, cm, bad)
    bad = dict(pad)
    bad["packed"] = pad["packed"].copy()
    bad["packed"][[0, 9]] = bad["packed"][[9, 0]]
    bad["src"] = pad["src"].copy()
    bad["src"][[0, 9]] = bad["src"][[9, 0]]
    with pytest.raises(AssertionError):
        check_arrangement(a.rows, 4, cm, bad)
