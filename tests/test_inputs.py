"""Structure checks on the seeded generators (shapes, sortedness, determinism)."""
import numpy as np

from paper_1203_2946_gb300 import inputs


def _valid(a):
    assert a.row_ptr[0] == 0 and a.row_ptr[-1] == a.nnz
    assert (np.diff(a.row_ptr) >= 0).all()
    assert a.col_ind.min(initial=0) >= 0 and a.col_ind.max(initial=0) < a.cols
    for i in range(0, a.rows, max(1, a.rows // 200)):
        c = a.col_ind[a.row_ptr[i]:a.row_ptr[i + 1]]
        assert (np.diff(c) > 0).all()


def test_stencil27_structure_small():
    a = inputs.stencil_3d_27pt(16, 16, 16, seed=1)
    _valid(a)
    assert a.nnz == (3 * 16 - 2) ** 3
    r = np.repeat(np.arange(a.rows), np.diff(a.row_ptr))
    diag = a.val[a.col_ind == r]
    off = a.col_ind != r
    assert np.all(np.abs(a.val[off]) <= 1)
    assert np.allclose(diag, np.bincount(r[off], np.abs(a.val[off]), a.rows) + 1)


def test_powerlaw_stats_small():
    a = inputs.powerlaw_rows(20000, 2.1, 1000, seed=0)
    _valid(a)
    L = np.diff(a.row_ptr)
    assert L.min() >= 1 and L.max() <= 1000
    assert 3.0 < L.mean() < 7.0
    assert a.val.dtype == np.float32


def test_banded_window_and_determinism():
    a = inputs.banded_random(5000, 300, 10, 60, seed=3)
    b = inputs.banded_random(5000, 300, 10, 60, seed=3)
    assert np.array_equal(a.col_ind, b.col_ind) and np.array_equal(a.val, b.val)
    _valid(a)
    L = np.diff(a.row_ptr)
    assert L.min() >= 10 and L.max() <= 60
    r = np.repeat(np.arange(a.rows), L)
    lo = np.clip(r - 150, 0, 5000 - 300)
    assert ((a.col_ind >= lo) & (a.col_ind < lo + 300)).all()


def test_batched_specs():
    s = inputs.batched_banded_specs()
    assert len(s) == 256
    assert all(1000 <= t["n"] <= 200000 and 64 <= t["width"] <= 2048 and t["k"] in (1, 4, 8, 32) for t in s)


def test_selector_specs_cover_families():
    s = inputs.selector_family_specs(200)
    fams = {t["family"] for t in s}
    assert fams == {"stencil2d", "stencil3d", "banded", "blockdiag", "powerlaw", "uniform"}
    a = inputs.selector_matrix(dict(family="blockdiag", n=1000, block=7, seed=1, mu=7.0))
    _valid(a)
    assert a.nnz == 142 * 49 + 6 * 6
