"""GPU parity of the modified CMRS of Section 6.6 (CMRS_PADDED): the padded
arrangement bit-exact against the oracle's, and the Section 6.6 SpMV kernel
(and Algorithm 1 on padded strips) against the CRS oracle."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1203_2946_gb300 import inputs

pytestmark = pytest.mark.gpu
DTYPES = [0, 1, 2, 3]


@pytest.fixture(scope="module")
def b():
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding
    return binding


def convert(b, a, h, dtype=0):
    rp, ci = torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col_ind).cuda()
    va = torch.from_numpy(np.ascontiguousarray(a.val, dtype=np.float64)).cuda()
    return b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=dtype)


def check_arrangement(b, M, P, a, h, slots=8):
    """Padded StripPtr and packed words equal the oracle's; values are the
    source values moved by the oracle's src map, +0 in zero items."""
    sp = M.strip_ptr.cpu().numpy()
    pk = M.col_packed.cpu().numpy()[:M.nnz].view(np.uint32)
    ref = orc.pad_arrange(a.rows, h, sp, pk, slots)
    log2m = {1: 0, 2: 1, 4: 2, 8: 3}[slots]
    assert P.struct.flags == b.CMRS_PADDED | (log2m << b.CMRS_PAD_SLOTS_SHIFT)
    assert P.nnz == ref["strip_ptr"][-1]
    assert np.array_equal(P.strip_ptr.cpu().numpy(), ref["strip_ptr"])
    assert np.array_equal(P.col_packed.cpu().numpy()[:P.nnz].view(np.uint32), ref["packed"])
    src = ref["src"]
    v0 = b.stored_values(M).cpu().numpy()
    v1 = b.stored_values(P).cpu().numpy()
    halves = 2 if M.dtype == b.CMRS_BF16X2 else 1
    for part in range(halves):
        s0 = v0[part * M.nnz:(part + 1) * M.nnz]
        s1 = v1[part * P.nnz:(part + 1) * P.nnz]
        want = np.zeros_like(s1)
        want[src >= 0] = s0[src[src >= 0]]
        assert np.array_equal(s1.view(np.uint8), want.view(np.uint8))


def xvec(a, dtype, seed=5):
    x = inputs.uniform_vector(a.cols, seed)
    return x if dtype == 0 else x.astype(np.float32)


def check_spmv(b, P, a, x, variant, dtype):
    y = b.cmrs_spmv(P, torch.from_numpy(x).cuda(), variant=variant).cpu().numpy()
    if dtype == 0:
        yref, absy = orc.csr_spmv(a.row_ptr, a.col_ind, a.val.astype(np.float64), x)
        bad = np.abs(y - yref) > 1e-12 * absy
        assert not bad.any(), (variant, np.nonzero(bad)[0][:10])
        return
    vq = orc.decode(orc.encode(a.val, dtype), dtype, a.nnz)
    yq, aq = orc.csr_spmv(a.row_ptr, a.col_ind, vq, x.astype(np.float64))
    tol = (np.diff(a.row_ptr) + 2) * 2.0**-24 * aq
    bad = np.abs(y.astype(np.float64) - yq) > tol
    assert not bad.any(), (variant, dtype, np.nonzero(bad)[0][:10])


def skewed(seed=1, n=20001):
    L = np.random.default_rng(seed).integers(0, 30, n)
    L[5] = 7000
    L[777:790] = 0
    L[4000:4400] = 0
    L[-1] = 3
    return inputs.from_lengths(L, 30000, seed=seed + 10)


HM = [(4, 8), (5, 8), (16, 8), (17, 8), (32, 8), (8, 4), (16, 2), (32, 2), (32, 1)]


@pytest.mark.parametrize("h,slots", HM)
@pytest.mark.parametrize("dtype", DTYPES)
def test_pad_arrangement_bit_exact(b, h, slots, dtype):
    a = skewed()
    M = convert(b, a, h, dtype)
    P = b.cmrs_pad(M, slots)
    check_arrangement(b, M, P, a, h, slots)


@pytest.mark.parametrize("h,slots", HM)
@pytest.mark.parametrize("dtype", DTYPES)
def test_padded_spmv(b, h, slots, dtype):
    a = skewed(2)
    P = b.cmrs_pad(convert(b, a, h, dtype), slots)
    x = xvec(a, dtype)
    for var in (b.CMRS_VARIANT_PADDED, b.CMRS_VARIANT_STRIP, b.CMRS_VARIANT_AUTO):
        check_spmv(b, P, a, x, var, dtype)
    assert b.cmrs_spmv_variant(P) == b.CMRS_VARIANT_PADDED


@pytest.mark.parametrize("h,slots", [(16, 8), (32, 1), (32, 2)])
def test_padded_stencil27_full(b, h, slots):
    """The 27-point 128^3 matrix at the paper's height 16 and M = 8 (Section
    6.6), and at height 32 with one or two slots per row."""
    a, x = inputs.workload_stencil27_128()
    M = convert(b, a, h)
    P = b.cmrs_pad(M, slots)
    sp = P.strip_ptr.cpu().numpy()
    assert np.all(sp % 32 == 0)
    # a 27-point strip of 16 interior rows (432 items) needs 14 passes
    assert P.nnz < 1.05 * a.nnz
    check_spmv(b, P, a, x, b.CMRS_VARIANT_PADDED, 0)


def test_padded_degenerate(b):
    # no entries at all; empty leading strips; one long last row; identity
    for L, cols in ((np.zeros(50, int), 7), (np.r_[np.zeros(40, int), [9000]], 9500), (np.array([1]), 1)):
        a = inputs.from_lengths(L, cols, seed=3)
        for h, slots in ((4, 8), (16, 8), (32, 1)):
            M = convert(b, a, h)
            P = b.cmrs_pad(M, slots)
            check_arrangement(b, M, P, a, h, slots)
            y = b.cmrs_spmv(P, torch.from_numpy(xvec(a, 0)).cuda()).cpu().numpy()
            yref, _ = orc.csr_spmv(a.row_ptr, a.col_ind, a.val, xvec(a, 0))
            assert np.allclose(y, yref, rtol=1e-12, atol=0)
    n = 10007
    ident = inputs.CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    x = xvec(ident, 0)
    for h, slots in ((16, 8), (32, 1)):
        P = b.cmrs_pad(convert(b, ident, h), slots)
        assert np.array_equal(b.cmrs_spmv(P, torch.from_numpy(x).cuda()).cpu().numpy(), x)


@pytest.mark.parametrize("dtype", DTYPES)
def test_padded_short_strips(b, dtype):
    """M = 1 matrices of one or two passes per strip on average (like the
    paper's p7): rows of 0..2 entries, runs of empty strips, one longer row, a
    ragged last strip; also reordered and written back through a row map."""
    L = np.random.default_rng(dtype).integers(0, 2, 70001)
    L[::97] = 2
    L[100:300] = 0
    L[5000] = 90
    a = inputs.from_lengths(L, 80000, seed=dtype + 20)
    P = b.cmrs_pad(convert(b, a, 32, dtype), 1)
    assert P.nnz <= 64 * P.struct.strips
    x = xvec(a, dtype)
    check_spmv(b, P, a, x, b.CMRS_VARIANT_PADDED, dtype)
    rp = torch.from_numpy(a.row_ptr).cuda()
    perm = b.cmrs_row_order(rp, 1024)
    rp2, ci2, v2 = b.cmrs_permute_csr(rp, torch.from_numpy(a.col_ind).cuda(), torch.from_numpy(a.val).cuda(), perm)
    Q = b.cmrs_pad(b.cmrs_from_csr(rp2, ci2, v2, a.cols, 32, dtype=dtype), 1)
    y = b.cmrs_spmv_rows(Q, torch.from_numpy(x).cuda(), perm).cpu().numpy().astype(np.float64)
    vq = orc.decode(orc.encode(a.val, dtype), dtype, a.nnz) if dtype else a.val.astype(np.float64)
    yref, absy = orc.csr_spmv(a.row_ptr, a.col_ind, vq, x.astype(np.float64))
    tol = 1e-12 * absy if dtype == 0 else (np.diff(a.row_ptr) + 2) * 2.0**-24 * absy
    assert np.all(np.abs(y - yref) <= tol)


def long_rows(seed, n=1000, cols=60000):
    """Few long rows (1,500..2,500 entries): few strips of many passes, so
    the padded product splits each strip over several warps; a ragged last
    strip and some empty rows."""
    L = np.random.default_rng(seed).integers(1500, 2500, n)
    L[7:12] = 0
    L[-3:] = 0
    return inputs.from_lengths(L, cols, seed=seed + 30)


@pytest.mark.parametrize("h,slots", HM)
@pytest.mark.parametrize("dtype", DTYPES)
def test_padded_split_strips(b, h, slots, dtype):
    a = long_rows(dtype + h)
    P = b.cmrs_pad(convert(b, a, h, dtype), slots)
    ws = P.spmv_workspace(b.CMRS_VARIANT_PADDED)
    assert ws.numel() > 256  # the workspace holds the partial sums of the split walk
    x = xvec(a, dtype)
    check_spmv(b, P, a, x, b.CMRS_VARIANT_PADDED, dtype)
    y1 = b.cmrs_spmv(P, torch.from_numpy(x).cuda(), variant=b.CMRS_VARIANT_PADDED)
    y2 = b.cmrs_spmv(P, torch.from_numpy(x).cuda(), variant=b.CMRS_VARIANT_PADDED)
    assert torch.equal(y1, y2)  # partials are added in part order: the same result every call
    # a workspace too small for the partial sums runs the one-warp-per-strip walk
    small = b.workspace(256, "cuda")
    y3 = b.cmrs_spmv(P, torch.from_numpy(x).cuda(), variant=b.CMRS_VARIANT_PADDED, workspace_tensor=small)
    check_spmv_result(y3, a, x, dtype)


def check_spmv_result(y, a, x, dtype):
    y = y.cpu().numpy().astype(np.float64)
    if dtype == 0:
        yref, absy = orc.csr_spmv(a.row_ptr, a.col_ind, a.val.astype(np.float64), x)
        assert np.all(np.abs(y - yref) <= 1e-12 * absy)
    else:
        vq = orc.decode(orc.encode(a.val, dtype), dtype, a.nnz)
        yq, aq = orc.csr_spmv(a.row_ptr, a.col_ind, vq, x.astype(np.float64))
        assert np.all(np.abs(y - yq) <= (np.diff(a.row_ptr) + 2) * 2.0**-24 * aq)


def test_padded_split_with_row_map(b):
    a = long_rows(5, n=1500)
    rp = torch.from_numpy(a.row_ptr).cuda()
    perm = b.cmrs_row_order(rp, 512)
    rp2, ci2, v2 = b.cmrs_permute_csr(rp, torch.from_numpy(a.col_ind).cuda(), torch.from_numpy(a.val).cuda(), perm)
    x = xvec(a, 0)
    for h, slots in ((32, 1), (16, 8), (4, 8)):
        Q = b.cmrs_pad(b.cmrs_from_csr(rp2, ci2, v2, a.cols, h), slots)
        y = b.cmrs_spmv_rows(Q, torch.from_numpy(x).cuda(), perm)
        check_spmv_result(y, a, x, 0)


def test_padded_rejections(b):
    a = skewed(3, 2000)
    M = convert(b, a, 16)
    P = b.cmrs_pad(M)
    with pytest.raises(b.CmrsError):
        b.cmrs_spmv(P, torch.from_numpy(xvec(a, 0)).cuda(), variant=b.CMRS_VARIANT_ROW)
    with pytest.raises(b.CmrsError):
        b.cmrs_spmv(M, torch.from_numpy(xvec(a, 0)).cuda(), variant=b.CMRS_VARIANT_PADDED)
    with pytest.raises(b.CmrsError):
        b.cmrs_pad(P)  # already padded
    with pytest.raises(b.CmrsError):
        b.cmrs_to_csr(P)
    with pytest.raises(b.CmrsError):
        rp, ci = torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col_ind).cuda()
        va = torch.from_numpy(a.val).cuda()
        b.cmrs_pad(b.cmrs_from_csr(rp, ci, va, a.cols, 16, flags=b.CMRS_SORTED))
    with pytest.raises(b.CmrsError):
        b.cmrs_pad(convert(b, a, 2))  # 2 rows x 8 slots cannot fill a 32-lane pass
    with pytest.raises(b.CmrsError):
        b.cmrs_pad(M, 1)  # one slot needs height 32
    with pytest.raises(b.CmrsError):
        b.cmrs_pad(M, 3)


def test_padded_repeatable(b):
    a = inputs.powerlaw_rows(30000, 2.1, 5000, seed=4)
    for h, slots in ((16, 8), (32, 1)):
        P = b.cmrs_pad(convert(b, a, h, 1), slots)
        x = torch.from_numpy(xvec(a, 1)).cuda()
        y1 = b.cmrs_spmv(P, x)
        y2 = b.cmrs_spmv(P, x)
        assert torch.equal(y1, y2)
