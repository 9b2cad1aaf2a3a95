"""GPU parity of row reordering: the order and the permuted CRS bit-exact
against the oracle, and the product of the reordered matrix written back in
the original order (cmrs_spmv_rows) against the CRS oracle of the original."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1203_2946_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding
    return binding


def lengths_matrix(seed, n=20011, lo=0, hi=60, cols=30000):
    L = np.random.default_rng(seed).integers(lo, hi, n)
    L[17] = 3000
    L[100:140] = 0
    return inputs.from_lengths(L, cols, seed=seed + 1)


@pytest.mark.parametrize("window", [1, 7, 32, 100, 1024, 4096])
def test_row_order_bit_exact(b, window):
    for seed, (lo, hi) in enumerate(((0, 60), (5, 6), (0, 3))):
        a = lengths_matrix(seed, lo=lo, hi=hi)
        perm = b.cmrs_row_order(torch.from_numpy(a.row_ptr).cuda(), window).cpu().numpy()
        assert np.array_equal(perm, orc.row_order(a.row_ptr, window))


def test_permute_csr_bit_exact(b):
    a = lengths_matrix(4)
    rp, ci = torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col_ind).cuda()
    perm = b.cmrs_row_order(rp, 4096)
    ref = orc.permute_csr(a.row_ptr, a.col_ind, a.val, perm.cpu().numpy())
    for val in (torch.from_numpy(a.val).cuda(), torch.from_numpy(a.val.astype(np.float32)).cuda(), None):
        rp2, ci2, v2 = b.cmrs_permute_csr(rp, ci, val, perm)
        assert np.array_equal(rp2.cpu().numpy(), ref[0])
        assert np.array_equal(ci2.cpu().numpy(), ref[1])
        if val is not None:
            want = ref[2] if val.dtype == torch.float64 else a.val.astype(np.float32)[np.concatenate(
                [np.arange(a.row_ptr[r], a.row_ptr[r + 1]) for r in perm.cpu().numpy()])]
            assert np.array_equal(v2.cpu().numpy(), want)


def test_permute_csr_rejects_bad_perm(b):
    a = lengths_matrix(5, n=500)
    rp, ci, va = (torch.from_numpy(t).cuda() for t in (a.row_ptr, a.col_ind, a.val))
    perm = torch.arange(a.rows, dtype=torch.int32, device="cuda")
    dup = perm.clone()
    dup[3] = 4  # row 3 missing, row 4 twice
    with pytest.raises(b.CmrsError):
        b.cmrs_permute_csr(rp, ci, va, dup)
    out = perm.clone()
    out[0] = a.rows  # outside 0..rows-1
    with pytest.raises(b.CmrsError):
        b.cmrs_permute_csr(rp, ci, va, out)
    with pytest.raises(b.CmrsError):
        b.cmrs_row_order(rp, 5000)


def reordered(b, a, window, h, dtype=0):
    rp, ci = torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col_ind).cuda()
    va = torch.from_numpy(a.val).cuda()
    perm = b.cmrs_row_order(rp, window)
    rp2, ci2, v2 = b.cmrs_permute_csr(rp, ci, va, perm)
    return perm, b.cmrs_from_csr(rp2, ci2, v2, a.cols, h, dtype=dtype)


@pytest.mark.parametrize("dtype", [0, 1])
def test_spmv_rows_matches_original(b, dtype):
    a = lengths_matrix(6, lo=4, hi=60)
    x = inputs.uniform_vector(a.cols, 7)
    if dtype:
        x = x.astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yref, absy = orc.csr_spmv(a.row_ptr, a.col_ind, a.val, x.astype(np.float64))
    vq = orc.decode(orc.encode(a.val, dtype), dtype, a.nnz)
    yq, aq = orc.csr_spmv(a.row_ptr, a.col_ind, vq, x.astype(np.float64))
    tol = (np.diff(a.row_ptr) + 2) * 2.0**-24 * aq

    def check(y):
        y = y.cpu().numpy().astype(np.float64)
        if dtype == 0:
            assert np.all(np.abs(y - yref) <= 1e-12 * absy)
        else:
            assert np.all(np.abs(y - yq) <= tol)

    perm, M = reordered(b, a, 4096, 32, dtype)
    for var in (b.CMRS_VARIANT_ROW, b.CMRS_VARIANT_STRIP, b.CMRS_VARIANT_AUTO):
        check(b.cmrs_spmv_rows(M, xd, perm, variant=var))
    with pytest.raises(b.CmrsError):
        b.cmrs_spmv_rows(M, xd, perm, variant=b.CMRS_VARIANT_MERGE)
    for slots in (1, 8):
        P = b.cmrs_pad(M, slots)
        check(b.cmrs_spmv_rows(P, xd, perm, variant=b.CMRS_VARIANT_PADDED))
        check(b.cmrs_spmv_rows(P, xd, perm))


def test_reordering_cuts_zero_items(b):
    a = lengths_matrix(8, n=65536, lo=4, hi=60)
    rp = torch.from_numpy(a.row_ptr).cuda()
    M0 = b.cmrs_from_csr(rp, torch.from_numpy(a.col_ind).cuda(), torch.from_numpy(a.val).cuda(), a.cols, 32)
    perm, M1 = reordered(b, a, 4096, 32)
    n0, n1 = b.cmrs_pad(M0, 1).nnz, b.cmrs_pad(M1, 1).nnz
    rp2, _, _ = orc.permute_csr(a.row_ptr, a.col_ind, a.val, perm.cpu().numpy())
    Ls = np.diff(rp2)
    assert n1 == 32 * sum(int(Ls[s:s + 32].max()) for s in range(0, a.rows, 32))
    assert n1 - a.nnz < 0.2 * (n0 - a.nnz)  # most of the zero items are gone
