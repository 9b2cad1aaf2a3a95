"""Pins for the CPU oracle: each check ties it to something other than itself
(the paper's printed example, dense algebra, closed forms, brute force)."""
import itertools
import math
import struct

import numpy as np
import pytest

from paper_1203_2946_gb300 import inputs


# ----------------------------------------------------------------------------- Section 2.3 / 3 / 4 example
def _golden_csr(g):
    return (g["crs_rowptr"].astype(np.int32), g["crs_colind"].astype(np.int32), g["crs_val"])


def test_golden_coo_crs_consistent_with_dense(golden5):
    M = np.stack([golden5["dense_row%d" % i] for i in range(5)])
    r, c, v = golden5["coo_rowind"].astype(int), golden5["coo_colind"].astype(int), golden5["coo_val"]
    D = np.zeros((5, 5))
    D[r, c] = v
    assert np.array_equal(D, M)
    rp, ci, vv = _golden_csr(golden5)
    assert np.array_equal(np.diff(rp), np.bincount(r, minlength=5))
    assert np.array_equal(ci, c) and np.array_equal(vv, v)


def test_golden_cmrs_h2(orc, golden5):
    rp, ci, v = _golden_csr(golden5)
    out = orc.csr_to_cmrs(rp, ci, v, 5, 2)
    assert out["bits"] == 4
    assert np.array_equal(out["strip_ptr"], golden5["cmrs_h2_stripptr"])
    assert np.array_equal(out["row_in_strip"], golden5["cmrs_h2_rowinstrip"])
    assert np.array_equal(out["val"], golden5["cmrs_h2_val"])
    assert np.array_equal(out["packed"] >> 4, golden5["cmrs_h2_colind"])
    assert np.array_equal(out["packed"] & 15, golden5["cmrs_h2_rowinstrip"])


def test_golden_sorted_cmrs_h2(orc, golden5):
    rp, ci, v = _golden_csr(golden5)
    out = orc.csr_to_cmrs(rp, ci, v, 5, 2, sorted_=True)
    assert np.array_equal(out["strip_ptr"], golden5["sorted_h2_stripptr"])
    assert np.array_equal(out["row_in_strip"], golden5["sorted_h2_rowinstrip"])
    assert np.array_equal(out["val"], golden5["sorted_h2_val"])
    assert np.array_equal(out["packed"] >> 4, golden5["sorted_h2_colind"])


def test_golden_inverse(orc, golden5):
    rp, ci, v = _golden_csr(golden5)
    for sorted_ in (False, True):
        cm = orc.csr_to_cmrs(rp, ci, v, 5, 2, sorted_=sorted_)
        back = orc.cmrs_to_csr(5, 2, cm["strip_ptr"], cm["packed"], cm["val"])
        assert np.array_equal(back["row_ptr"], rp)
        assert np.array_equal(back["col_ind"], ci)
        assert np.array_equal(back["val"], v)


def test_golden_spmv_ones(orc, golden5):
    M = np.stack([golden5["dense_row%d" % i] for i in range(5)])
    rp, ci, v = _golden_csr(golden5)
    x = np.ones(5)
    y_dense = M @ x  # = [3, 7, 11, 24, 10] by hand
    assert np.array_equal(y_dense, [3, 7, 11, 24, 10])
    y, a = orc.csr_spmv(rp, ci, v, x)
    assert np.array_equal(y, y_dense) and np.array_equal(a, y_dense)
    for sorted_ in (False, True):
        cm = orc.csr_to_cmrs(rp, ci, v, 5, 2, sorted_=sorted_)
        assert np.array_equal(orc.cmrs_spmv(5, 2, cm["strip_ptr"], cm["packed"], cm["val"], x), y_dense)


# ----------------------------------------------------------------------------- h = 1 is CRS (Section 3)
def test_height_one_is_crs(orc):
    a = inputs.random_csr(37, 23, 0.2, seed=3, empty_row_frac=0.2)
    cm = orc.csr_to_cmrs(a.row_ptr, a.col_ind, a.val, a.cols, 1)
    assert np.array_equal(cm["strip_ptr"], a.row_ptr)
    assert not cm["row_in_strip"].any()
    assert np.array_equal(cm["packed"] >> 4, a.col_ind)


# ----------------------------------------------------------------------------- bits (Section 4 packing)
def test_bits_for_height(orc):
    for h in range(1, 17):
        assert orc.bits_for_height(h) == 4
    for h in range(17, 33):
        assert orc.bits_for_height(h) == 5
    for h in (0, -1, 33, 64):
        assert orc.bits_for_height(h) == -1


# ----------------------------------------------------------------------------- SpMV against dense algebra
@pytest.mark.parametrize("seed", range(6))
def test_csr_spmv_matches_dense(orc, seed):
    rng = np.random.default_rng(seed)
    rows, cols = int(rng.integers(1, 60)), int(rng.integers(1, 60))
    a = inputs.random_csr(rows, cols, float(rng.uniform(0.02, 0.6)), seed=seed, empty_row_frac=0.15)
    x = rng.uniform(-1, 1, cols)
    y, absy = orc.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    D = a.dense()
    assert np.allclose(y, D @ x, rtol=0, atol=1e-14 * max(1.0, np.abs(D).sum()))
    assert np.allclose(absy, np.abs(D) @ np.abs(x), rtol=1e-15, atol=0)
    assert np.array_equal(orc.dense_matvec(D, x), D @ x) or np.allclose(orc.dense_matvec(D, x), D @ x, atol=1e-14)


@pytest.mark.parametrize("h", [1, 2, 3, 4, 5, 8, 13, 16, 17, 32])
def test_cmrs_spmv_reaches_crs_result(orc, h):
    a = inputs.random_csr(75, 50, 0.15, seed=h, empty_row_frac=0.1)
    x = np.random.default_rng(h).uniform(-1, 1, a.cols)
    y_crs, absy = orc.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    cm = orc.csr_to_cmrs(a.row_ptr, a.col_ind, a.val, a.cols, h)
    # unsorted CMRS keeps each row's CRS order: the sums are the same sums
    assert np.array_equal(orc.cmrs_spmv(a.rows, h, cm["strip_ptr"], cm["packed"], cm["val"], x), y_crs)
    cs = orc.csr_to_cmrs(a.row_ptr, a.col_ind, a.val, a.cols, h, sorted_=True)
    ys = orc.cmrs_spmv(a.rows, h, cs["strip_ptr"], cs["packed"], cs["val"], x)
    # rows are column-sorted already, so the in-strip sort keeps each row's order too
    assert np.array_equal(ys, y_crs)
    assert np.allclose(ys, a.dense() @ x, rtol=0, atol=1e-13 * (1 + absy.max()))


def test_identity_and_diagonal(orc):
    n = 97
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    x = np.random.default_rng(0).uniform(-1, 1, n)
    d = np.random.default_rng(1).uniform(-2, 2, n)
    for h in (1, 4, 7, 32):
        cm = orc.csr_to_cmrs(rp, ci, np.ones(n), n, h)
        assert np.array_equal(orc.cmrs_spmv(n, h, cm["strip_ptr"], cm["packed"], cm["val"], x), x)
        cm = orc.csr_to_cmrs(rp, ci, d, n, h)
        assert np.array_equal(orc.cmrs_spmv(n, h, cm["strip_ptr"], cm["packed"], cm["val"], x), d * x)


def test_laplacian_row_sums(orc):
    a, _ = inputs.workload_laplacian_64()
    assert a.rows == 4096 and a.nnz == 20224
    y, _ = orc.csr_spmv(a.row_ptr, a.col_ind, a.val, np.ones(a.cols))
    g = y.reshape(64, 64)
    assert (g[1:-1, 1:-1] == 0).all()
    corners = [g[0, 0], g[0, -1], g[-1, 0], g[-1, -1]]
    assert corners == [2.0, 2.0, 2.0, 2.0]
    edges = np.concatenate([g[0, 1:-1], g[-1, 1:-1], g[1:-1, 0], g[1:-1, -1]])
    assert (edges == 1.0).all()


def test_stencil27_small_row_sums(orc):
    a = inputs.stencil_3d_27pt(6, 5, 4, seed=1)
    n = a.rows
    counts = np.diff(a.row_ptr)
    # interior rows have 27 entries; corners 8
    assert counts.max() == 27 and counts.min() == 8
    assert a.nnz == (3 * 6 - 2) * (3 * 5 - 2) * (3 * 4 - 2)
    y, _ = orc.csr_spmv(a.row_ptr, a.col_ind, a.val, np.ones(n))
    # closed form from the generator: y_i = diag_i + sum off = sum |off| + 1 + sum off
    r = np.repeat(np.arange(n), counts)
    off = a.col_ind != r
    s_abs = np.bincount(r[off], np.abs(a.val[off]), n)
    s_off = np.bincount(r[off], a.val[off], n)
    assert np.allclose(y, s_abs + 1 + s_off, rtol=0, atol=1e-13)


def test_stencil27_full_size_count():
    # 27-point, 128^3, Dirichlet truncation: (3*128-2)^3 entries
    assert (3 * 128 - 2) ** 3 == 55_742_968


# ----------------------------------------------------------------------------- conversions
@pytest.mark.parametrize("h", [1, 2, 3, 4, 8, 16, 31, 32])
def test_round_trip_bit_exact(orc, h):
    a = inputs.random_csr(203, 77, 0.08, seed=100 + h, empty_row_frac=0.3)
    for sorted_ in (False, True):
        cm = orc.csr_to_cmrs(a.row_ptr, a.col_ind, a.val, a.cols, h, sorted_=sorted_)
        # StripPtr definition of Section 3
        S = (a.rows + h - 1) // h
        assert np.array_equal(cm["strip_ptr"][:S], a.row_ptr[np.arange(S) * h])
        assert cm["strip_ptr"][S] == a.nnz
        back = orc.cmrs_to_csr(a.rows, h, cm["strip_ptr"], cm["packed"], cm["val"])
        assert np.array_equal(back["row_ptr"], a.row_ptr)
        assert np.array_equal(back["col_ind"], a.col_ind)
        assert np.array_equal(back["val"], a.val)


def test_sorted_strips_are_sorted_and_a_permutation(orc):
    a = inputs.random_csr(120, 300, 0.05, seed=9)
    h = 8
    cm = orc.csr_to_cmrs(a.row_ptr, a.col_ind, a.val, a.cols, h, sorted_=True)
    sp, col = cm["strip_ptr"], (cm["packed"] >> cm["bits"]).astype(np.int64)
    for s in range(len(sp) - 1):
        seg = col[sp[s]:sp[s + 1]]
        assert (np.diff(seg) >= 0).all()
        src = cm["src"][sp[s]:sp[s + 1]]
        # stable: equal columns keep CRS order
        for c in np.unique(seg):
            assert (np.diff(src[seg == c]) > 0).all()
    assert np.array_equal(np.sort(cm["src"]), np.arange(a.nnz))


def test_unsorted_row_in_strip_is_nondecreasing(orc):
    a = inputs.random_csr(64, 64, 0.2, seed=5, empty_row_frac=0.2)
    for h in (2, 5, 16):
        cm = orc.csr_to_cmrs(a.row_ptr, a.col_ind, a.val, a.cols, h)
        sp, ris = cm["strip_ptr"], cm["row_in_strip"]
        for s in range(len(sp) - 1):
            assert (np.diff(ris[sp[s]:sp[s + 1]]) >= 0).all()


def test_conversion_errors(orc):
    rp = np.array([0, 2, 1, 3], np.int32)
    ci = np.array([0, 1, 2], np.int32)
    with pytest.raises(orc.OracleError) as e:
        orc.csr_to_cmrs(rp, ci, np.ones(3), 3, 2)
    assert e.value.code == orc.ORC_BAD_CSR
    with pytest.raises(orc.OracleError) as e:
        orc.csr_to_cmrs(np.array([0, 1], np.int32), np.array([5], np.int32), np.ones(1), 3, 2)
    assert e.value.code == orc.ORC_BAD_CSR
    with pytest.raises(orc.OracleError) as e:
        orc.csr_to_cmrs(np.array([0, 1], np.int32), np.array([0], np.int32), np.ones(1), 1, 0)
    assert e.value.code == orc.ORC_BAD_HEIGHT
    # 28 column bits for h <= 16 (Section 4): 2^28 columns fit, one more does not
    ok = orc.csr_to_cmrs(np.array([0, 1], np.int32), np.array([2**28 - 1], np.int32), np.ones(1), 2**28, 16)
    assert (ok["packed"][0] >> 4) == 2**28 - 1
    with pytest.raises(orc.OracleError) as e:
        orc.csr_to_cmrs(np.array([0, 1], np.int32), np.array([0], np.int32), np.ones(1), 2**28 + 1, 16)
    assert e.value.code == orc.ORC_COL_OVERFLOW


def test_tail_strip_and_single_dense_row(orc):
    # rows not a multiple of h; every entry in one row
    rows, cols, h = 10, 40, 4
    lengths = np.zeros(rows, int)
    lengths[9] = 40
    a = inputs.from_lengths(lengths, cols, seed=1)
    cm = orc.csr_to_cmrs(a.row_ptr, a.col_ind, a.val, cols, h)
    assert np.array_equal(cm["strip_ptr"], [0, 0, 0, 40])
    assert (cm["row_in_strip"] == 1).all()
    x = np.random.default_rng(2).uniform(-1, 1, cols)
    y = orc.cmrs_spmv(rows, h, cm["strip_ptr"], cm["packed"], cm["val"], x)
    assert np.allclose(y, a.dense() @ x, atol=1e-14) and (y[:9] == 0).all()


# ----------------------------------------------------------------------------- value forms
def _nearest_bf16_bruteforce(f):
    """Nearest BF16 to the float f, ties to even mantissa, by exact comparison
    of the two candidates that bracket it."""
    u = struct.unpack("<I", struct.pack("<f", f))[0]
    lo = u >> 16
    hi_ = lo + 1
    def val(h):
        return struct.unpack("<f", struct.pack("<I", (h << 16) & 0xFFFFFFFF))[0]
    a, b, x = val(lo), val(hi_), float(f)
    da, db = abs(x - a), abs(b - x)
    if da < db:
        return lo
    if db < da:
        return hi_
    return lo if lo % 2 == 0 else hi_


def test_bf16_rne_against_bruteforce(orc):
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.standard_normal(3000).astype(np.float32),
                           (rng.standard_normal(1000) * 1e-30).astype(np.float32),
                           np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, -1.0 - 2**-8, 0.0, -0.0,
                                     3.0e38, 1e-40], np.float32)])
    for f in vals:
        assert orc.bf16_from_f32(f) == _nearest_bf16_bruteforce(float(f)) & 0xFFFF, f
    assert orc.bf16_from_f32(1.0) == 0x3F80
    assert orc.bf16_from_f32(1.0 + 2**-8) == 0x3F80  # tie, even stays
    assert orc.bf16_from_f32(1.0 + 3 * 2**-8) == 0x3F82  # tie, odd rounds up


def test_encode_forms(orc):
    rng = np.random.default_rng(1)
    v = rng.uniform(-1, 1, 2000)
    f32 = orc.encode(v, orc.F32)
    assert np.array_equal(f32, v.astype(np.float32))
    b = orc.encode(v, orc.BF16)
    bb = orc.decode(b, orc.BF16, v.size)
    assert np.all(np.abs(bb - v) <= 2.0**-8 * np.abs(v) + 1e-300)
    s = orc.encode(v, orc.BF16X2)
    hi, lo = s[:v.size], s[v.size:]
    assert np.array_equal(hi, b)
    rec = orc.decode(s, orc.BF16X2, v.size)
    # hi + lo keeps about 16 significant bits
    assert np.all(np.abs(rec - v) <= 2.0**-15 * np.abs(v) + 1e-300)
    assert np.median(np.abs(rec - v) / np.abs(v)) < 2.0**-16
    f = rng.standard_normal(500).astype(np.float32)
    assert np.array_equal(orc.encode(f, orc.F64), f.astype(np.float64))
    assert np.array_equal(orc.encode(f, orc.BF16), orc.encode(f.astype(np.float64), orc.BF16))


# ----------------------------------------------------------------------------- Section 5 model, Eq. (6.1)
def test_model_printed_values(orc):
    # Section 5: h=1, lambda=128, b=4, mu=2 gives f = 16.5; h=16 brings it to about 2
    assert orc.model_f(1, 2, 128, 4) == 16.5
    assert abs(orc.model_f(16, 2, 128, 4) - 2.0) < 0.05
    for h, mu in itertools.product([1, 2, 4, 8, 16], [1, 2, 5, 20, 100]):
        exact = orc.model_a(h, mu, 128, 4)
        assert exact == pytest.approx(orc.model_f(1, mu, 128, 4) / orc.model_f(h, mu, 128, 4))
        approx = 1 + (h - 1) / (1 + h * mu * 4 / 128)  # Eq. (5.2) with lambda - b ~ lambda
        assert abs(exact - approx) / approx < 0.04


@pytest.mark.parametrize("lam,b", [(128, 4), (128, 8), (256, 8), (32, 4)])
def test_segments_closed_form_by_bruteforce(orc, lam, b):
    # appendix: a chunk of n bytes at a uniformly random b-aligned offset touches
    # 1 + (n - b)/lambda segments on average
    for n in range(b, 4 * lam + 1, b):
        mean = np.mean([orc.segments_at(n, lam, s) for s in range(0, lam, b)])
        assert mean == pytest.approx(orc.model_segments(n, lam, b), rel=1e-12)


def test_beta_identity(orc):
    for nnz, rows, strips, sv in [(55742968, 2097152, 524288, 8), (20224, 4096, 1024, 8), (100, 7, 2, 4)]:
        bm, bp = orc.beta(nnz, rows, strips, sv)
        assert bp - bm == -sv * (nnz - rows)
    # the 5-point Laplacian, h = 4: 12*20224 + 4*1024 + 16*4096 = 242688 + 4096 + 65536
    assert orc.beta(20224, 4096, 1024, 8)[1] == 312320


# ----------------------------------------------------------------------------- selector features
def test_features_closed_form_laplacian(orc):
    a, _ = inputs.workload_laplacian_64()
    f = orc.features(a.row_ptr, a.col_ind)
    assert f[0] == 12.0
    assert f[2] == pytest.approx(math.log2(1 + 20224 / 4096))
    assert f[5] == 0.0
    # lengths: 4 corners of 3, 248 edge rows of 4, 3844 interior rows of 5
    assert f[6] == 0 and f[7] == pytest.approx(4 / 4096) and f[8] == pytest.approx(4092 / 4096)
    assert f[4] == pytest.approx(math.log2(6))
    assert f[15] == pytest.approx(math.log2(65))  # max |col - row| = nx
    assert f[16] == 1.0
    # mean |col-row|: each interior row has 0,1,1,64,64; total over all entries
    tot = 2 * (64 * 63) * 1 + 2 * (64 * 63) * 64
    assert f[14] == pytest.approx(math.log2(1 + tot / 20224))
    # h = 1 strip spread = max-min within a row
    r = np.repeat(np.arange(4096), np.diff(a.row_ptr))
    spread = np.array([a.col_ind[r == i].max() - a.col_ind[r == i].min() for i in range(4096)])
    assert f[18] == pytest.approx(math.log2(1 + spread.mean()))


def test_features_bruteforce_random(orc):
    a = inputs.random_csr(90, 90, 0.07, seed=4, empty_row_frac=0.2)
    f = orc.features(a.row_ptr, a.col_ind)
    L = np.diff(a.row_ptr)
    assert f[3] == pytest.approx(L.std() / max(L.mean(), 1))
    assert f[5] == pytest.approx((L == 0).mean())
    edges = [1, 2, 4, 8, 16, 32, 64, 128, 10**9]
    for b in range(8):
        assert f[6 + b] == pytest.approx(((L >= edges[b]) & (L < edges[b + 1])).mean())
    for e, h in enumerate([1, 2, 4, 8, 16, 32]):
        sp = []
        for s in range(0, 90, h):
            c = a.col_ind[a.row_ptr[s]:a.row_ptr[min(s + h, 90)]]
            if c.size:
                sp.append(c.max() - c.min())
        assert f[18 + e] == pytest.approx(math.log2(1 + np.mean(sp)))


def test_features_modified_cmrs_and_strip_sizes_laplacian(orc):
    """f24..f31 on the 5-point 64x64 Laplacian, worked by hand: rows of 5
    entries, 4 on a grid edge, 3 at a corner; a strip of 32 rows is half a grid
    line (159 entries inside the grid, 127 on its first and last lines), a
    strip of 16 rows a quarter (80 or 79; 64 or 63)."""
    a, _ = inputs.workload_laplacian_64()
    f = orc.features(a.row_ptr, a.col_ind)
    # (32, 1): passes = longest row: 124 strips of 5, 4 strips of 4
    assert f[24] == pytest.approx(math.log2(32 * (124 * 5 + 4 * 4) / 20224), abs=1e-15)
    # (32, 2): max(ceil(159/32), ceil(5/2)) = 5 and max(ceil(127/32), 2) = 4: as (32, 1)
    assert f[25] == f[24]
    # (16, 8): 248 strips of ceil(80/32) = 3 passes, 8 on the first and last lines of 2
    assert f[26] == pytest.approx(math.log2(32 * (248 * 3 + 8 * 2) / 20224), abs=1e-15)
    assert f[27] == f[28] == f[29] == 0.0
    # 32-row strips: 124 of 159 entries, 4 of 127; mean 158, variance 31
    assert f[30] == pytest.approx(math.sqrt(31) / 158, rel=1e-12)
    assert f[31] == pytest.approx(math.log2(1 + 159 / 158), rel=1e-12)


def test_features_padded_counts_match_the_arrangement(orc):
    """f24..f26 against the item counts of the Section 6.6 arrangement itself
    (orc_pad_arrange, pinned on its own), on matrices with skewed rows."""
    for seed, maker in enumerate([lambda s: inputs.powerlaw_rows(3000, 1.9, 400, seed=s),
                                  lambda s: inputs.random_csr(700, 900, 0.02, seed=s, empty_row_frac=0.3),
                                  lambda s: inputs.banded_random(2000, 300, 1, 90, seed=s)]):
        a = maker(seed)
        f = orc.features(a.row_ptr, a.col_ind)
        for q, (h, m) in enumerate([(32, 1), (32, 2), (16, 8)]):
            c = orc.csr_to_cmrs(a.row_ptr, a.col_ind, a.val, a.cols, h)
            arr = orc.pad_arrange(a.rows, h, c["strip_ptr"], c["packed"], m)
            assert f[24 + q] == pytest.approx(math.log2(int(arr["strip_ptr"][-1]) / a.nnz), abs=1e-14)


def test_features_entry_weighted_lengths(orc):
    lengths = [0, 5, 31, 32, 511, 512, 8191, 8192, 9000, 3]
    a = inputs.from_lengths(lengths, 20000, seed=1)
    f = orc.features(a.row_ptr, a.col_ind)
    z = sum(lengths)
    assert f[27] == pytest.approx((32 + 511 + 512 + 8191 + 8192 + 9000) / z, rel=1e-14)
    assert f[28] == pytest.approx((512 + 8191 + 8192 + 9000) / z, rel=1e-14)
    assert f[29] == pytest.approx((8192 + 9000) / z, rel=1e-14)
    # one strip of 32 rows holds everything: no spread, the max is the mean
    assert f[30] == 0.0 and f[31] == 1.0


# ----------------------------------------------------------------------------- selector network (textbook MLP, Adam)
def _net(rng, nin=24, nh=64, nout=18, scale=0.3):
    return dict(W1=rng.normal(0, scale, (nh, nin)), b1=rng.normal(0, 0.1, nh),
                W2=rng.normal(0, scale / 2, (nh, nh)), b2=rng.normal(0, 0.1, nh),
                W3=rng.normal(0, scale / 2, (nout, nh)), b3=rng.normal(0, 0.1, nout))


def test_mlp_linear_regime_matches_matmul(orc):
    rng = np.random.default_rng(0)
    p = _net(rng)
    p["b1"] += 100.0  # every hidden unit active: the network is affine
    p["b2"] += 1.0e4  # dominates |W2 h1| (about 1e2 here)
    X = rng.normal(0, 1, (7, 24))
    O = orc.mlp_forward(X, **p)["O"]
    ref = ((X @ p["W1"].T + p["b1"]) @ p["W2"].T + p["b2"]) @ p["W3"].T + p["b3"]
    assert np.allclose(O, ref, rtol=1e-12, atol=1e-10)
    # and with all hidden units dead the output is b3
    p["b1"] -= 1e6
    p["b2"] -= 1e6
    assert np.array_equal(orc.mlp_forward(X, **p)["O"], np.tile(p["b3"], (7, 1)))


def test_mlp_gradient_finite_differences(orc):
    rng = np.random.default_rng(1)
    p = _net(rng, nin=6, nh=9, nout=4)
    X = rng.normal(0, 1, (5, 6))
    T = rng.normal(0, 1, (5, 4))
    loss, g, _ = orc.mlp_loss_grad(X, T, **p)
    O = orc.mlp_forward(X, **p)["O"]
    assert loss == pytest.approx(0.5 * np.mean((O - T) ** 2))
    eps = 1e-6
    for name in p:
        arr = p[name]
        for idx in itertools.islice(np.ndindex(arr.shape), 0, None, 3):
            old = arr[idx]
            arr[idx] = old + eps
            lp = orc.mlp_loss_grad(X, T, **p)[0]
            arr[idx] = old - eps
            lm = orc.mlp_loss_grad(X, T, **p)[0]
            arr[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name][idx]) <= 1e-7 + 1e-5 * abs(fd), (name, idx)


def test_adam_closed_form(orc):
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.1, -0.3, 0.0])
    m, v = np.zeros(3), np.zeros(3)
    orc.adam_step(p, g, m, v, 1, 0.01)
    # first step with zero moments moves each parameter by lr * sign(g) (up to eps)
    assert np.allclose(p, [1.0 - 0.01, -2.0 + 0.01, 0.5], atol=1e-9)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
