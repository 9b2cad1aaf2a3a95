"""cmrs_spmv_noalloc: the SpMV entry point for callers that cannot allocate
device memory (allocator callbacks, pools that forbid growth, runtimes that
own every buffer).  It takes its scratch from the library's fixed array, so
it is called here straight through the C ABI and compared with cmrs_spmv
(MERGE, caller workspace) on two calls in a row, within the parity
tolerances of the other GPU tests."""
import ctypes

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
    f = binding.lib().cmrs_spmv_noalloc
    f.argtypes = [ctypes.POINTER(binding.cmrs_matrix), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return binding


def call_c_abi(b, M, x, y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return b.lib().cmrs_spmv_noalloc(ctypes.byref(M.struct), ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(y.data_ptr()), stream)


@pytest.mark.parametrize("dtype", [0, 1])
def test_noalloc_matches_workspace_entry_point(b, dtype):
    a = inputs.powerlaw_rows(120_000, 2.1, 20_000, seed=6)
    vals = a.val.astype(np.float64) if dtype == 0 else a.val
    x = np.random.default_rng(2).uniform(-1, 1, a.cols)
    x = x if dtype == 0 else x.astype(np.float32)
    M = b.cmrs_from_csr(torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col_ind).cuda(),
                        torch.from_numpy(np.ascontiguousarray(vals)).cuda(), a.cols, 4, dtype=dtype)
    xd = torch.from_numpy(x).cuda()
    y_ref = b.cmrs_spmv(M, xd, variant=b.CMRS_VARIANT_MERGE).cpu().numpy().astype(np.float64)
    _, scale = orc.csr_spmv(a.row_ptr, a.col_ind, vals.astype(np.float64), x.astype(np.float64))
    L = np.diff(a.row_ptr)
    tol = 1e-12 * scale if dtype == 0 else (L + 2) * 2.0**-24 * scale
    y = torch.empty(a.rows, dtype=xd.dtype, device="cuda")
    for _ in range(2):
        y.fill_(float("nan"))
        assert call_c_abi(b, M, xd, y) == 0
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - y_ref) <= tol)


def test_noalloc_rejects_matrix_past_its_limit(b):
    m = b.cmrs_matrix()
    m.rows, m.cols, m.height, m.bits, m.dtype = 1 << 20, 1 << 20, 4, 4, 0
    m.strips = (m.rows + 3) // 4
    m.nnz = 111_820_801  # one tile more than the fixed scratch holds
    m.strip_ptr = m.col_packed = m.val = 256
    x = torch.empty(1, device="cuda")
    assert b.lib().cmrs_spmv_noalloc(ctypes.byref(m), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                     None) == 7
