"""Pins of the row-reordering oracle against what the order must satisfy,
independent of how the oracle builds it: a permutation that moves rows only
inside their window; inside a window, lengths non-increasing and equal lengths
in their original order; P A has the original rows; the product is the same
up to the permutation; and, for windows that are whole strips, the modified
CMRS of Section 6.6 (height 32, one slot) of P A needs no more passes than
that of A (sorted groups of 32 minimise the sum of group maxima)."""
import numpy as np
import pytest

import oracle
from paper_1203_2946_gb300 import inputs


def check_order(row_ptr, window, perm):
    L = np.diff(row_ptr)
    n = L.size
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.all(perm // window == np.arange(n) // window)
    for w0 in range(0, n, window):
        p = perm[w0:w0 + window]
        lp = L[p]
        assert np.all(np.diff(lp) <= 0)
        same = np.diff(lp) == 0
        assert np.all(np.diff(p)[same] > 0)


@pytest.mark.parametrize("window", [1, 7, 32, 64, 4096])
def test_order_properties(window):
    rng = np.random.default_rng(window)
    for trial in range(4):
        L = rng.integers(0, [2, 5, 60, 300][trial], 5000)
        rp = np.r_[0, np.cumsum(L)].astype(np.int32)
        check_order(rp, window, oracle.row_order(rp, window))


def test_permuted_rows_and_product():
    a = inputs.from_lengths(np.random.default_rng(2).integers(0, 20, 700), 300, seed=3)
    perm = oracle.row_order(a.row_ptr, 64)
    rp, ci, v = oracle.permute_csr(a.row_ptr, a.col_ind, a.val, perm)
    dense = np.zeros((a.rows, a.cols))
    for i in range(a.rows):
        dense[i, a.col_ind[a.row_ptr[i]:a.row_ptr[i + 1]]] = a.val[a.row_ptr[i]:a.row_ptr[i + 1]]
    dense_p = np.zeros_like(dense)
    for i in range(a.rows):
        dense_p[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    assert np.array_equal(dense_p, dense[perm])
    x = np.random.default_rng(4).uniform(-1, 1, a.cols)
    y, _ = oracle.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    yp, _ = oracle.csr_spmv(rp, ci, v, x)
    assert np.array_equal(yp, y[perm])


def test_fewer_passes_after_reordering():
    rng = np.random.default_rng(5)
    for lo, hi in ((4, 60), (0, 12), (20, 21)):
        a = inputs.from_lengths(rng.integers(lo, hi, 8192), 10000, seed=6)
        perm = oracle.row_order(a.row_ptr, 4096)
        rp, ci, v = oracle.permute_csr(a.row_ptr, a.col_ind, a.val, perm)
        counts = []
        for r_, c_, v_ in ((a.row_ptr, a.col_ind, a.val), (rp, ci, v)):
            cm = oracle.csr_to_cmrs(r_, c_, v_, a.cols, 32)
            counts.append(oracle.pad_arrange(a.rows, 32, cm["strip_ptr"], cm["packed"], 1)["strip_ptr"][-1])
        assert counts[1] <= counts[0]
        # the sorted strips need exactly 32 x (their longest row) items each
        Ls = np.diff(rp)
        assert counts[1] == 32 * sum(int(Ls[s:s + 32].max()) for s in range(0, a.rows, 32))


def test_checker_catches_a_planted_mistake():
    L = np.array([3, 5, 5, 1, 0, 5])
    rp = np.r_[0, np.cumsum(L)].astype(np.int32)
    perm = oracle.row_order(rp, 6)
    assert perm.tolist() == [1, 2, 5, 0, 3, 4]
    bad = perm.copy()
    bad[[0, 1]] = bad[[1, 0]]  # equal lengths out of original order
    with pytest.raises(AssertionError):
        check_order(rp, 6, bad)
    bad = perm.copy()
    bad[[2, 3]] = bad[[3, 2]]  # a shorter row before a longer one
    with pytest.raises(AssertionError):
        check_order(rp, 6, bad)
