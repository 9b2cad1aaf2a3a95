"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Bars: conversions and every index array bit-exact; stored values bit-exact
against the oracle's encoders; FP64 SpMV |y - y*| <= 1e-12 * (|A||x|)_i
(exactly 0 where that scale is 0); FP32-accumulated forms within
(len_i + 2) * 2^-24 * (|A_q||x_q|)_i of the quantised-input oracle (values as
stored, x as FP32, FP64 sums), which bounds any summation order of len_i
exact products in FP32."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1203_2946_gb300 import inputs

pytestmark = pytest.mark.gpu

DTYPES = [0, 1, 2, 3]
VARIANTS = [0, 1, 2]


@pytest.fixture(scope="module")
def b():
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding
    assert torch.cuda.is_available()
    return binding


def dev(a):
    return (torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col_ind).cuda(),
            torch.from_numpy(np.ascontiguousarray(a.val)).cuda())


def stored_np(b, M):
    t = b.stored_values(M).cpu().numpy()
    return t.view(np.uint16) if t.dtype == np.int16 else t


def convert(b, a, h, sorted_=False, dtype=0):
    rp, ci, v = dev(a)
    M = b.cmrs_from_csr(rp, ci, v, a.cols, h, flags=1 if sorted_ else 0, dtype=dtype)
    torch.cuda.synchronize()
    return M


def check_conversion(b, a, h, sorted_=False, dtype=0):
    M = convert(b, a, h, sorted_, dtype)
    ref = orc.csr_to_cmrs(a.row_ptr, a.col_ind, a.val.astype(np.float64), a.cols, h, sorted_)
    assert np.array_equal(M.strip_ptr.cpu().numpy(), ref["strip_ptr"])
    assert np.array_equal(M.col_packed.cpu().numpy()[:a.nnz].view(np.uint32), ref["packed"])
    assert np.array_equal(stored_np(b, M), orc.encode(a.val[ref["src"]], dtype))
    lens = np.diff(ref["strip_ptr"])
    assert M.struct.max_strip_nnz == (int(lens.max()) if lens.size else 0)
    return M


def xvec(a, dtype, seed=5):
    x = np.random.default_rng(seed).uniform(-1, 1, a.cols)
    return x if dtype == 0 else x.astype(np.float32)


def check_spmv(b, M, a, x, variant, dtype):
    y = b.cmrs_spmv(M, torch.from_numpy(x).cuda(), variant=variant).cpu().numpy()
    assert y.shape == (a.rows,)
    if dtype == 0:
        yref, absy = orc.csr_spmv(a.row_ptr, a.col_ind, a.val.astype(np.float64), x)
        err = np.abs(y - yref)
        bad = err > 1e-12 * absy
        assert not bad.any(), (variant, np.nonzero(bad)[0][:10], err[bad][:5], absy[bad][:5])
        return err
    vq = orc.decode(orc.encode(a.val, dtype), dtype, a.nnz)
    yq, aq = orc.csr_spmv(a.row_ptr, a.col_ind, vq, x.astype(np.float64))
    L = np.diff(a.row_ptr)
    tol = (L + 2) * 2.0**-24 * aq
    err = np.abs(y.astype(np.float64) - yq)
    bad = err > tol
    assert not bad.any(), (variant, dtype, np.nonzero(bad)[0][:10], err[bad][:5], tol[bad][:5])
    return err


# ------------------------------------------------------------------ the paper's worked example
def test_golden_5x5(b, golden5):
    rp, ci, v = (golden5["crs_rowptr"].astype(np.int32), golden5["crs_colind"].astype(np.int32), golden5["crs_val"])
    a = inputs.CSR(5, 5, rp, ci, v)
    M = convert(b, a, 2)
    assert np.array_equal(M.strip_ptr.cpu().numpy(), golden5["cmrs_h2_stripptr"])
    pk = M.col_packed.cpu().numpy()[:10].view(np.uint32)
    assert np.array_equal(pk >> 4, golden5["cmrs_h2_colind"]) and np.array_equal(pk & 15, golden5["cmrs_h2_rowinstrip"])
    S = convert(b, a, 2, sorted_=True)
    pk = S.col_packed.cpu().numpy()[:10].view(np.uint32)
    assert np.array_equal(pk >> 4, golden5["sorted_h2_colind"])
    assert np.array_equal(pk & 15, golden5["sorted_h2_rowinstrip"])
    assert np.array_equal(stored_np(b, S), golden5["sorted_h2_val"])
    ones = torch.ones(5, dtype=torch.float64, device="cuda")
    for var in VARIANTS:
        assert b.cmrs_spmv(M, ones, variant=var).cpu().numpy().tolist() == [3, 7, 11, 24, 10]
    assert b.cmrs_spmv(S, ones, variant=1).cpu().numpy().tolist() == [3, 7, 11, 24, 10]
    for sorted_ in (0, 1):
        X = convert(b, a, 2, sorted_=bool(sorted_))
        rp2, ci2, vo = b.cmrs_to_csr(X)
        assert np.array_equal(rp2.cpu().numpy(), rp) and np.array_equal(ci2.cpu().numpy(), ci)
        assert np.array_equal(vo.view(torch.float64)[:10].cpu().numpy(), v)


# ------------------------------------------------------------------ conversions
@pytest.mark.parametrize("h", [1, 2, 3, 4, 5, 8, 16, 17, 32])
@pytest.mark.parametrize("sorted_", [False, True])
def test_conversion_bit_exact(b, h, sorted_):
    a = inputs.random_csr(1500, 900, 0.01, seed=h, empty_row_frac=0.2)
    for dtype in DTYPES:
        check_conversion(b, a, h, sorted_, dtype)


def test_conversion_f32_input_forms(b):
    a = inputs.powerlaw_rows(30000, 2.1, 3000, seed=2)
    for h in (1, 4, 32):
        for dtype in DTYPES:
            check_conversion(b, a, h, False, dtype)
        check_conversion(b, a, h, True, 1)


@pytest.mark.parametrize("h", [1, 4, 8, 32])
def test_round_trip(b, h):
    a = inputs.random_csr(3001, 700, 0.02, seed=40 + h, empty_row_frac=0.3)
    for sorted_ in (False, True):
        for dtype in DTYPES:
            M = convert(b, a, h, sorted_, dtype)
            rp, ci, vo = b.cmrs_to_csr(M)
            assert np.array_equal(rp.cpu().numpy(), a.row_ptr)
            assert np.array_equal(ci.cpu().numpy(), a.col_ind)
            nb = b.lib().cmrs_val_bytes(a.nnz, dtype)
            ref = orc.encode(a.val, dtype)
            got = vo.cpu().numpy()
            if dtype == 3:
                pad = b.lib().cmrs_pad8(a.nnz)
                got16 = got.view(np.uint16)
                got = np.concatenate([got16[:a.nnz], got16[pad:pad + a.nnz]])
            else:
                got = got[:nb].view(ref.dtype)
            assert np.array_equal(got, ref)


def test_long_strips_sort_and_round_trip(b):
    # one 9000-entry row and one 2500-entry row put strips past the 1024-entry
    # shared-memory sort into the radix path
    L = np.full(3000, 3)
    L[7] = 9000
    L[2050] = 2500
    L[100:130] = 0
    a = inputs.from_lengths(L, 20000, seed=3)
    for h in (4, 32):
        for dtype in (0, 3):
            M = check_conversion(b, a, h, True, dtype)
            rp, ci, _ = b.cmrs_to_csr(M)
            assert np.array_equal(rp.cpu().numpy(), a.row_ptr) and np.array_equal(ci.cpu().numpy(), a.col_ind)


def test_invalid_csr_reported(b):
    a = inputs.random_csr(50, 50, 0.1, seed=1)
    rp, ci, v = dev(a)
    bad = ci.clone()
    bad[3] = 50
    with pytest.raises(b.CmrsError) as e:
        b.cmrs_from_csr(rp, bad, v, 50, 4)
    assert e.value.code == 4
    rpb = rp.clone()
    rpb[10] = rpb[11] + 1
    with pytest.raises(b.CmrsError) as e:
        b.cmrs_from_csr(rpb, ci, v, 50, 4)
    assert e.value.code == 4
    rpb = rp.clone()
    rpb[-1] = rpb[-1] - 1
    with pytest.raises(b.CmrsError) as e:
        b.cmrs_from_csr(rpb, ci, v, 50, 4)
    assert e.value.code == 4
    with pytest.raises(b.CmrsError) as e:
        b.cmrs_from_csr(rp, ci, v, 50, 33)
    assert e.value.code == 2


# ------------------------------------------------------------------ SpMV
@pytest.mark.parametrize("h", [1, 2, 3, 4, 8, 16, 32])
@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv_random(b, h, dtype):
    a = inputs.random_csr(6007, 5000, 0.004, seed=h + 10 * dtype, empty_row_frac=0.1)
    M = convert(b, a, h, False, dtype)
    x = xvec(a, dtype)
    for var in VARIANTS:
        check_spmv(b, M, a, x, var, dtype)
    S = convert(b, a, h, True, dtype)
    check_spmv(b, S, a, x, 1, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv_skewed_rows(b, dtype):
    # rows longer than a MERGE tile (1920) and a ROW stage (4096), empty rows,
    # empty strips, a ragged tail strip
    L = np.random.default_rng(1).integers(0, 12, 20001)
    L[5] = 7000
    L[777] = 1930
    L[778] = 1919
    L[5000:5400] = 0
    L[-1] = 2
    a = inputs.from_lengths(L, 30000, seed=9, dtype=np.float64)
    x = xvec(a, dtype)
    for h in (1, 4, 7, 32):
        M = convert(b, a, h, False, dtype)
        for var in VARIANTS:
            check_spmv(b, M, a, x, var, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv_row_lane_long_units(b, dtype):
    """ROW on plain CMRS with one, two or four lanes per row (mean rows up to
    28, 56, 112 entries; heights dividing the unit of 32, 16, 8 rows), each
    unit staged in the warp's shared memory: rows of 1..8, 40..60 and
    70..100 entries, tails that are not a multiple of the unit, and h = 32
    where the wider units fall back to the share-per-thread kernel."""
    long_rows = inputs.banded_random(20_003, 900, 40, 60, seed=5)
    longer_rows = inputs.banded_random(9_001, 1200, 70, 100, seed=7)
    short_rows = inputs.banded_random(20_011, 200, 1, 8, seed=6)
    for a in (long_rows, longer_rows, short_rows):
        a = inputs.CSR(a.rows, a.cols, a.row_ptr, a.col_ind, a.val.astype(np.float64))
        x = xvec(a, dtype)
        for h in (1, 8, 32):
            check_spmv(b, convert(b, a, h, False, dtype), a, x, 0, dtype)


def test_spmv_degenerate(b):
    # nnz = 0 with rows > 0: y = 0
    a = inputs.from_lengths(np.zeros(100, int), 10, seed=1)
    for var in VARIANTS:
        M = convert(b, a, 4)
        y = b.cmrs_spmv(M, torch.ones(10, dtype=torch.float64, device="cuda"), variant=var)
        assert (y == 0).all()
    # one row holding every entry, at the end; everything before it empty
    L = np.zeros(333, int)
    L[-1] = 5000
    a = inputs.from_lengths(L, 6000, seed=2)
    for h in (1, 4, 32):
        M = convert(b, a, h)
        for var in VARIANTS:
            check_spmv(b, M, a, xvec(a, 0), var, 0)
    # a single entry at the very first row; identity; diagonal
    a = inputs.from_lengths(np.array([1] + [0] * 50), 3, seed=3)
    M = convert(b, a, 4)
    for var in VARIANTS:
        check_spmv(b, M, a, xvec(a, 0), var, 0)
    n = 10007
    ident = inputs.CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    x = xvec(ident, 0)
    for h in (1, 3, 32):
        M = convert(b, ident, h)
        for var in VARIANTS:
            assert np.array_equal(b.cmrs_spmv(M, torch.from_numpy(x).cuda(), variant=var).cpu().numpy(), x)
    # rows = 0
    a = inputs.CSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    M = convert(b, a, 4)
    assert b.cmrs_spmv(M, torch.ones(5, dtype=torch.float64, device="cuda")).numel() == 0


@pytest.mark.parametrize("dtype", DTYPES)
def test_merge_tile_sets_either_side_of_the_row_length_bound(b, dtype):
    """MERGE launches 9- (FP64) or 11-entry tiles where rows average fewer
    than 16 entries and 15-entry tiles from 16 on: rows of exactly 16 and
    just under, with empty rows, a row longer than several tiles and a ragged
    tail, both sides of the bound, against the oracle."""
    rng = np.random.default_rng(40 + dtype)
    for target in (15.9, 16.0):
        L = rng.integers(0, 32, 30011)
        L[100:140] = 0
        L[7] = 5000
        L[-1] = 3
        L[8] += int(round(target * L.size)) - int(L.sum())  # mean exactly `target` (to rounding)
        assert L[8] >= 0
        a = inputs.from_lengths(L, 40000, seed=11 + dtype, dtype=np.float64)
        assert (a.nnz >= 16 * a.rows) == (target >= 16.0)
        x = xvec(a, dtype)
        for h in (1, 32):
            check_spmv(b, convert(b, a, h, False, dtype), a, x, 2, dtype)


def test_binding_rejects_mismatched_operands(b):
    """x or y of another value type, too short, or strided: refused by the
    binding before any pointer reaches the library (an FP32 x given to an
    FP64 matrix would be read as half as many doubles, past its end)."""
    a = inputs.random_csr(300, 200, 0.05, seed=1)
    M = convert(b, a, 4)  # FP64
    x64 = torch.ones(a.cols, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        b.cmrs_spmv(M, x64.float())
    with pytest.raises(ValueError):
        b.cmrs_spmv(M, x64[:-1])
    with pytest.raises(ValueError):
        b.cmrs_spmv(M, torch.ones(2 * a.cols, dtype=torch.float64, device="cuda")[::2])
    with pytest.raises(TypeError):
        b.cmrs_spmv(M, x64, torch.empty(a.rows, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        b.cmrs_spmv(M, x64, torch.empty(a.rows - 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        b.cmrs_spmv_noalloc(M, x64.float())
    y = b.cmrs_spmv(M, x64)  # the well-formed call still runs
    assert y.shape == (a.rows,)


def test_spmv_repeatable(b):
    a = inputs.powerlaw_rows(50000, 2.1, 20000, seed=4)
    x = xvec(a, 1)
    xs = torch.from_numpy(x).cuda()
    for h in (4, 16):
        M = convert(b, a, h, False, 1)
        for var in VARIANTS:
            y1 = b.cmrs_spmv(M, xs, variant=var)
            y2 = b.cmrs_spmv(M, xs, variant=var)
            assert torch.equal(y1, y2)
            b.cmrs_spmv_check(M, var)


def test_wait_timeout_reported_and_context_usable(b):
    """A bounded in-kernel mbarrier wait that nothing completes gives up, the
    timeout bit reaches the host as CMRS_ERR_TIMEOUT once (the check clears
    it), and the context still computes correct products afterwards.  Also
    measures how long one failed try takes, hence how long the kernels'
    2^18-try limit lets a wait last (about a second is the aim)."""
    a, x = inputs.workload_laplacian_64()
    M = convert(b, a, 4)
    var = b.CMRS_VARIANT_MERGE
    ws = M.spmv_workspace(var)
    # the phase completed by the probe's own arrival: no timeout
    b.cmrs_wait_probe(ws, 64, arrive=True)
    b.cmrs_spmv_check(M, var)
    # left open: the wait gives up after `tries` tries; the probe grows
    # `tries` only while the time per try keeps a probe under ~0.2 s
    per_try, tries = None, 16
    while True:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.cmrs_wait_probe(ws, tries, arrive=False)
        e1.record()
        torch.cuda.synchronize()
        per_try = e0.elapsed_time(e1) * 1e-3 / tries
        with pytest.raises(b.CmrsError) as ei:
            b.cmrs_spmv_check(M, var)
        assert ei.value.code == 8  # CMRS_ERR_TIMEOUT
        b.cmrs_spmv_check(M, var)  # cleared by the first check
        if tries >= 65536 or per_try * tries * 16 > 0.2:
            break
        tries *= 16
    limit_s = per_try * (1 << 18)
    print("\nbounded wait: %d tries in %.3f ms, %.3f us per try; the kernels' 2^18 tries: %.2f s"
          % (tries, per_try * tries * 1e3, per_try * 1e6, limit_s))
    assert 0.01 < limit_s < 10
    # the context is intact: the product still matches the oracle
    for v in VARIANTS:
        check_spmv(b, M, a, x, v, 0)
    with pytest.raises(b.CmrsError):
        b.cmrs_wait_probe(ws, 0, arrive=False)
    with pytest.raises(b.CmrsError):
        b.cmrs_wait_probe(ws, 65537, arrive=False)


def test_laplacian_64_config(b):
    """5-point Laplacian 64x64, FP64, h = 4: conversion + SpMV against the oracle."""
    a, x = inputs.workload_laplacian_64()
    M = check_conversion(b, a, 4)
    for var in VARIANTS:
        check_spmv(b, M, a, x, var, 0)
    ones = torch.ones(a.cols, dtype=torch.float64, device="cuda")
    g = b.cmrs_spmv(M, ones).cpu().numpy().reshape(64, 64)
    assert (g[1:-1, 1:-1] == 0).all() and g[0, 0] == 2 and g[0, 5] == 1


# ------------------------------------------------------------------ full-size workloads
@pytest.fixture(scope="module")
def stencil27():
    return inputs.workload_stencil27_128()


@pytest.mark.parametrize("h", [4, 16, 32])
def test_stencil27_full_fp64(b, stencil27, h):
    a, x = stencil27
    assert a.nnz == 55_742_968
    M = check_conversion(b, a, h)
    for var in VARIANTS:
        check_spmv(b, M, a, x, var, 0)


def test_stencil27_full_reduced(b, stencil27):
    a, x = stencil27
    for dtype in (1, 2, 3):
        M = convert(b, a, 4, False, dtype)
        check_spmv(b, M, a, x.astype(np.float32), 0, dtype)


def test_stencil27_full_sorted(b, stencil27):
    a, x = stencil27
    M = check_conversion(b, a, 4, True, 0)
    check_spmv(b, M, a, x, 1, 0)


def test_powerlaw_full(b):
    a, x = inputs.workload_powerlaw_4m()
    assert a.rows == 4_194_304
    for h in (4, 32):
        M = check_conversion(b, a, h, False, 1)
        for var in VARIANTS:
            check_spmv(b, M, a, x, var, 1)
    M = convert(b, a, 4, False, 2)
    check_spmv(b, M, a, x, 2, 2)


@pytest.mark.parametrize("which", ["p7", "dense4"])
def test_paper_extra_matrices(b, which):
    """The two synthetic matrices of Section 6.1: a 10^7 random permutation and
    a 10^4 x 10^4 dense matrix stored as sparse (full comparison)."""
    a = inputs.permutation_matrix() if which == "p7" else inputs.dense_as_sparse()
    x = xvec(a, 0)
    for h in (1, 4, 32):
        M = convert(b, a, h)
        for var in VARIANTS:
            check_spmv(b, M, a, x, var, 0)
    # the bench's forms: p7 at height 32, one slot (one pass per strip); dense4 at height 4, 8 slots
    P = b.cmrs_pad(convert(b, a, 32 if which == "p7" else 4), 1 if which == "p7" else 8)
    check_spmv(b, P, a, x, b.CMRS_VARIANT_PADDED, 0)


@pytest.mark.parametrize("case", ["stencil", "short", "long", "very_long", "skewed", "sorted"])
def test_auto_variant(b, case):
    """CMRS_VARIANT_AUTO runs the variant cmrs_spmv_variant names: its y is
    bit-identical to that variant's and passes the oracle bar."""
    rng = np.random.default_rng(21)
    if case == "stencil":
        a, want = inputs.stencil_3d_27pt(20, 20, 20, seed=3), b.CMRS_VARIANT_ROW
    elif case == "short":
        a, want = inputs.from_lengths(rng.integers(0, 3, 30000), 30000, seed=4), b.CMRS_VARIANT_MERGE
    elif case == "long":  # four lanes per row at h = 4
        a, want = inputs.from_lengths(np.full(300, 100), 5000, seed=5), b.CMRS_VARIANT_ROW
    elif case == "very_long":
        a, want = inputs.from_lengths(np.full(300, 150), 5000, seed=5), b.CMRS_VARIANT_MERGE
    elif case == "skewed":
        L = rng.integers(4, 9, 20000)
        L[100] = 5000
        a, want = inputs.from_lengths(L, 20000, seed=6), b.CMRS_VARIANT_MERGE
    else:
        a, want = inputs.from_lengths(rng.integers(4, 9, 20000), 20000, seed=7), b.CMRS_VARIANT_STRIP
    M = convert(b, a, 4, sorted_=(case == "sorted"))
    assert b.cmrs_spmv_variant(M) == want
    x = xvec(a, 0)
    xs = torch.from_numpy(x).cuda()
    y_auto = b.cmrs_spmv(M, xs, variant=b.CMRS_VARIANT_AUTO)
    assert torch.equal(y_auto, b.cmrs_spmv(M, xs, variant=want))
    check_spmv(b, M, a, x, b.CMRS_VARIANT_AUTO, 0)


def test_largest_column_index(b):
    """Columns up to 2^27 - 1 at height 32 (5 RowInStrip bits leave 27 column
    bits in the packed word): conversions bit-exact, products within the bar."""
    cols = 1 << 27
    rng = np.random.default_rng(31)
    L = rng.integers(0, 24, 5000)
    L[0] = 3
    a = inputs.from_lengths(L, cols, seed=32)
    a.col_ind[0:3] = [0, cols // 2, cols - 1]  # row 0: first, middle and last column
    x = inputs.uniform_vector(cols, 33)
    xs = torch.from_numpy(x).cuda()
    yref, absy = orc.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    for sorted_ in (False, True):
        M = check_conversion(b, a, 32, sorted_)
        for var in (VARIANTS if not sorted_ else [b.CMRS_VARIANT_STRIP]):
            y = b.cmrs_spmv(M, xs, variant=var).cpu().numpy()
            assert np.all(np.abs(y - yref) <= 1e-12 * absy), var
    P = b.cmrs_pad(convert(b, a, 32), 1)
    assert int(P.col_packed.cpu().numpy()[:P.nnz].view(np.uint32).max() >> 5) == cols - 1
    y = b.cmrs_spmv(P, xs).cpu().numpy()
    assert np.all(np.abs(y - yref) <= 1e-12 * absy)
    with pytest.raises(b.CmrsError):  # one column more does not fit
        rp, ci = torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col_ind).cuda()
        b.cmrs_from_csr(rp, ci, torch.from_numpy(a.val).cuda(), cols + 1, 32)


@pytest.mark.parametrize("h", [1, 2, 4, 8, 16])
def test_sorted_conversion_of_unordered_rows(b, h):
    """In-strip sort when CRS rows are not in column order (some rows shuffled,
    columns repeated across the rows of a strip): the stable column order of
    the oracle, bit for bit, whichever path the kernel takes."""
    rng = np.random.default_rng(40 + h)
    a = inputs.from_lengths(rng.integers(0, 40, 3000), 64, seed=41)  # 64 columns: many equal columns per strip
    ci = a.col_ind.copy()
    for i in rng.choice(a.rows, 700, replace=False):
        s, e = a.row_ptr[i], a.row_ptr[i + 1]
        ci[s:e] = rng.permutation(ci[s:e])
    a = inputs.CSR(a.rows, a.cols, a.row_ptr, ci, a.val)
    for dtype in (0, 3):
        check_conversion(b, a, h, True, dtype)
    # rows all in order: the merge path; the same oracle order
    a2 = inputs.from_lengths(rng.integers(0, 40, 3000), 64, seed=42)
    check_conversion(b, a2, h, True, 0)
