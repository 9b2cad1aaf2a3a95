"""CPU-side checks of the C ABI: libcmrs loads, exports every entry point that
include/cmrs.h declares, and its host-only paths (argument checks that return
before any CUDA call) behave as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "cmrs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cmrs_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding
    return binding.lib()


def test_exports_every_declared_symbol(L):
    names = declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n


def test_bits_rule(L):
    # Section 4: 4 bits for heights up to 16; a fifth bit for 17..32
    assert [L.cmrs_bits_for_height(h) for h in (1, 2, 4, 8, 16)] == [4] * 5
    assert [L.cmrs_bits_for_height(h) for h in (17, 31, 32)] == [5] * 3
    assert L.cmrs_bits_for_height(0) == -1 and L.cmrs_bits_for_height(33) == -1


def test_error_strings_and_sizes(L):
    for code in range(0, 9):
        assert L.cmrs_error_string(code).startswith(b"CMRS_")
    assert L.cmrs_val_bytes(10, 0) == 80 and L.cmrs_val_bytes(10, 1) == 40
    assert L.cmrs_val_bytes(10, 2) == 20 and L.cmrs_val_bytes(10, 3) == 2 * 16 + 20
    assert L.cmrs_pad8(0) == 0 and L.cmrs_pad8(9) == 16


def test_host_validation_paths(L):
    from paper_1203_2946_gb300 import binding as b
    p = ctypes.c_void_p(16)
    m = b.cmrs_matrix()
    # height out of range, column overflow: rejected before any device work
    rc = L.cmrs_from_csr(4, 4, 0, p, p, p, 0, 0, 0, 0, p, p, p, p, 1 << 20, None, None)
    assert rc == 2
    rc = L.cmrs_from_csr(4, (1 << 28) + 1, 0, p, p, p, 0, 16, 0, 0, p, p, p, p, 1 << 20, None, None)
    assert rc == 3
    rc = L.cmrs_from_csr(4, 1 << 27, 0, p, p, p, 0, 32, 0, 0, p, p, p, p, 1 << 20, None, None)
    assert rc == 0 or rc == 5 or rc == 7  # 27 column bits fit at h = 32; later steps need a device
    rc = L.cmrs_from_csr(4, 4, 0, p, p, p, 7, 4, 0, 0, p, p, p, p, 1 << 20, None, None)
    assert rc == 1  # bad input value type
    n = ctypes.c_size_t()
    m.rows, m.cols, m.nnz, m.height, m.strips, m.bits, m.dtype = 10, 10, 5, 4, 3, 4, 0
    m.strip_ptr = m.col_packed = m.val = 256  # never dereferenced by the size query
    assert L.cmrs_spmv_workspace(ctypes.byref(m), 0, ctypes.byref(n)) == 0 and n.value >= 256
    assert L.cmrs_spmv_workspace(ctypes.byref(m), 2, ctypes.byref(n)) == 0 and n.value > 256
    m.flags = 1
    assert L.cmrs_spmv_workspace(ctypes.byref(m), 0, ctypes.byref(n)) == 6  # ROW needs unsorted strips
    m.flags = 0
    m.strips = 2
    assert L.cmrs_spmv_workspace(ctypes.byref(m), 0, ctypes.byref(n)) == 1
    m.strips, m.bits = 3, 5
    assert L.cmrs_spmv_workspace(ctypes.byref(m), 0, ctypes.byref(n)) == 1
    # MERGE's workspace at the no-alloc entry point's stated limits: exactly
    # its 2 MiB fixed array, one entry more needs another tile
    m.rows, m.cols, m.height, m.bits = 1 << 20, 1 << 20, 4, 4
    m.strips = (m.rows + 3) // 4
    for dtype, limit in ((0, 67_092_480), (1, 82_001_920), (2, 82_001_920), (3, 82_001_920)):
        m.dtype = dtype
        m.nnz = limit
        assert L.cmrs_spmv_workspace(ctypes.byref(m), 2, ctypes.byref(n)) == 0 and n.value == 2 << 20
        m.nnz = limit + 1
        assert L.cmrs_spmv_workspace(ctypes.byref(m), 2, ctypes.byref(n)) == 0 and n.value > 2 << 20
    # the wait probe checks its workspace and try count before any launch
    assert L.cmrs_wait_probe(None, 0, 0, None) == 1  # tries checked before the fixed array is looked up
    assert L.cmrs_wait_probe(ctypes.c_void_p(4096 + 16), 16, 0, None) == 1
    assert L.cmrs_wait_probe(ctypes.c_void_p(4096), 0, 0, None) == 1
    assert L.cmrs_wait_probe(ctypes.c_void_p(4096), 65537, 0, None) == 1


def test_argument_checks_before_device_work(L):
    """Conversion, SpMM, feature, network and selector entry points: bad
    arguments are rejected, and the size queries answer, on the host alone
    (no device pointer is dereferenced on these paths)."""
    from paper_1203_2946_gb300 import binding as b
    n = ctypes.c_size_t()
    # CRS -> CMRS size query: (rows, nnz, height, flags, dtype, bytes)
    assert L.cmrs_from_csr_workspace(10, 5, 4, 0, 0, None) == 1
    assert L.cmrs_from_csr_workspace(-1, 5, 4, 0, 0, ctypes.byref(n)) == 1
    assert L.cmrs_from_csr_workspace(10, 5, 4, 0, 9, ctypes.byref(n)) == 1
    assert L.cmrs_from_csr_workspace(10, 5, 0, 0, 0, ctypes.byref(n)) == 2
    assert L.cmrs_from_csr_workspace(10, 5, 33, 0, 0, ctypes.byref(n)) == 2
    assert L.cmrs_from_csr_workspace(10, 5, 4, 0, 0, ctypes.byref(n)) == 0 and n.value > 0
    assert L.cmrs_to_csr_workspace(None, ctypes.byref(n)) == 1
    # SpMM: FP32 unsorted, unpadded strips only
    m = b.cmrs_matrix()
    m.rows, m.cols, m.nnz, m.height, m.strips, m.bits, m.dtype, m.flags = 10, 10, 5, 4, 3, 4, 1, 0
    m.strip_ptr = m.col_packed = m.val = 256  # never dereferenced on these paths
    p = ctypes.c_void_p(256)
    assert L.cmrs_spmm(None, 4, p, p, None) == 1
    assert L.cmrs_spmm(ctypes.byref(m), 0, p, p, None) == 1
    m.dtype = 0
    assert L.cmrs_spmm(ctypes.byref(m), 4, p, p, None) == 6  # FP64
    m.dtype, m.flags = 1, 1
    assert L.cmrs_spmm(ctypes.byref(m), 4, p, p, None) == 6  # sorted strips
    m.flags, m.bits = 0, 5
    assert L.cmrs_spmm(ctypes.byref(m), 4, p, p, None) == 2  # bits do not match the height
    m.bits, m.strips = 4, 2
    assert L.cmrs_spmm(ctypes.byref(m), 4, p, p, None) == 1  # strips != ceil(rows / height)
    m.strips = 3
    assert L.cmrs_spmm(ctypes.byref(m), 4, None, p, None) == 1  # X missing
    z = b.cmrs_matrix()
    z.rows, z.cols, z.nnz, z.height, z.strips, z.bits, z.dtype = 0, 10, 0, 4, 0, 4, 1
    assert L.cmrs_spmm(ctypes.byref(z), 4, None, None, None) == 0  # no rows: nothing to do
    # batched plan size query
    A = (ctypes.c_void_p * 1)(ctypes.addressof(m))
    k = (ctypes.c_int32 * 1)(4)
    assert L.cmrs_spmm_plan_workspace(-1, A, k, 1024, ctypes.byref(n)) == 1
    assert L.cmrs_spmm_plan_workspace(1, A, k, 0, ctypes.byref(n)) == 1
    assert L.cmrs_spmm_plan_workspace(1, None, k, 1024, ctypes.byref(n)) == 1
    k0 = (ctypes.c_int32 * 1)(0)
    assert L.cmrs_spmm_plan_workspace(1, A, k0, 1024, ctypes.byref(n)) == 1
    assert L.cmrs_spmm_plan_workspace(1, A, k, 1024, ctypes.byref(n)) == 0 and n.value > 0 and n.value % 256 == 0
    # training data of the network: sizes and pointers checked before any launch
    assert L.cmrs_feature_norm(0, 4, p, p, p, None, None) == 1
    assert L.cmrs_feature_norm(4, 4, None, p, p, None, None) == 1
    assert L.cmrs_feature_apply(4, 4, p, p, p, None, None) == 1
    assert L.cmrs_cost_targets(4, 21, p, ctypes.c_float(0.0), p, None) == 1
    assert L.cmrs_cost_targets(0, 21, p, ctypes.c_float(1.0), p, None) == 1
    # features, network, selector
    assert L.cmrs_features_workspace(-1, ctypes.byref(n)) == 1
    assert L.cmrs_features_workspace(10, None) == 1
    assert L.cmrs_features_workspace(10, ctypes.byref(n)) == 0 and n.value > 0
    assert L.cmrs_features(0, 5, p, p, p, p, 1 << 20, None) == 1
    assert L.cmrs_features(10, 5, p, p, p, None, 1 << 20, None) == 7  # no workspace
    assert L.cmrs_features(10, 5, p, p, p, ctypes.c_void_p(256 + 16), 1 << 20, None) == 7  # misaligned
    assert L.cmrs_mlp_param_count(0, 64, 21) == -1
    # two hidden layers: nin*nh + nh, nh*nh + nh, nh*nout + nout
    assert L.cmrs_mlp_param_count(24, 64, 21) == 24 * 64 + 64 + 64 * 64 + 64 + 64 * 21 + 21
    assert L.cmrs_mlp_forward(0, 24, 64, 21, p, p, p, None) == 1
    assert L.cmrs_mlp_forward(4, 24, 64, 21, None, p, p, None) == 1
    assert L.cmrs_select_strip_workspace(0, 10, 5, 0, ctypes.byref(n)) == 1
    assert L.cmrs_select_strip_workspace(10, 10, 5, 0, None) == 1
    assert L.cmrs_select_strip_workspace(10, 10, 5, 0, ctypes.byref(n)) == 0 and n.value > 0


def test_auto_variant_rule(L):
    """CMRS_VARIANT_AUTO: STRIP on sorted strips; otherwise MERGE for mean row
    length < 2, or > 32 where ROW's two- or four-lanes-per-row mapping does
    not apply (mean up to 56 at heights dividing 16, 112 at heights dividing
    8), or a strip above 8 x height x mean (or unknown); ROW for the rest.
    Host only: the device pointers are never read."""
    from paper_1203_2946_gb300 import binding as b

    def resolve(rows, nnz, height, max_strip, flags=0, variant=-1):
        m = b.cmrs_matrix()
        m.rows, m.cols, m.nnz, m.height = rows, rows, nnz, height
        m.strips, m.bits, m.dtype, m.flags = -(-rows // height), L.cmrs_bits_for_height(height), 0, flags
        m.max_strip_nnz = max_strip
        m.strip_ptr = m.col_packed = m.val = 256
        out = ctypes.c_int(-7)
        rc = L.cmrs_spmv_variant(ctypes.byref(m), variant, ctypes.byref(out))
        return rc, out.value

    ROW, STRIP, MERGE = 0, 1, 2
    assert resolve(1000, 27000, 4, 108) == (0, ROW)            # 27-point stencil shape
    assert resolve(1000, 2000, 4, 8) == (0, ROW)               # mean exactly 2
    assert resolve(1000, 1999, 4, 8) == (0, MERGE)             # mean below 2
    assert resolve(1000, 32000, 4, 128) == (0, ROW)            # mean exactly 32
    assert resolve(1000, 32001, 32, 1025) == (0, MERGE)        # mean above 32, no lanes mapping at h = 32
    assert resolve(1000, 32001, 16, 513) == (0, ROW)           # two lanes per row (h divides 16)
    assert resolve(1000, 56000, 16, 896) == (0, ROW)           # mean exactly 56
    assert resolve(1000, 56001, 16, 897) == (0, MERGE)         # mean above 56, h does not divide 8
    assert resolve(1000, 56001, 4, 225) == (0, ROW)            # four lanes per row (h divides 8)
    assert resolve(1000, 112000, 8, 896) == (0, ROW)           # mean exactly 112
    assert resolve(1000, 112001, 8, 897) == (0, MERGE)         # mean above 112
    assert resolve(1000, 10000, 4, 320) == (0, ROW)            # strip exactly 8 x 4 x 10
    assert resolve(1000, 10000, 4, 321) == (0, MERGE)          # skewed strip
    assert resolve(1000, 10000, 4, -1) == (0, MERGE)           # unknown longest strip
    assert resolve(1000, 10000, 4, 40, flags=1) == (0, STRIP)  # sorted strips
    assert resolve(1000, 10000, 4, 40, flags=1, variant=ROW) == (6, -7)
    assert resolve(1000, 10000, 4, 40, variant=STRIP) == (0, STRIP)
    assert resolve(1000, 10000, 4, 40, variant=3) == (6, -7)   # PADDED needs padded strips
    assert resolve(1000, 10000, 4, 40, variant=4)[0] == 1
    PADDED, P8, P1 = 3, 2 | (3 << 8), 2 | (0 << 8)                    # padded, M = 8 / M = 1
    assert resolve(1000, 10016, 16, -1, flags=P8) == (0, PADDED)       # padded strips (Section 6.6)
    assert resolve(1000, 10016, 32, -1, flags=P1) == (0, PADDED)
    assert resolve(1000, 10016, 16, -1, flags=P8, variant=STRIP) == (0, STRIP)
    assert resolve(1000, 10016, 16, -1, flags=P8, variant=ROW) == (6, -7)
    assert resolve(1000, 10016, 16, -1, flags=P8, variant=MERGE) == (6, -7)
    assert resolve(1000, 10016, 16, -1, flags=P8 | 1)[0] == 1          # sorted and padded
    assert resolve(1000, 10000, 16, -1, flags=P8)[0] == 1              # padded count not a multiple of 32
    assert resolve(1000, 10016, 2, -1, flags=P8)[0] == 1               # 2 rows x 8 slots < 32 lanes
    assert resolve(1000, 10016, 16, -1, flags=P1)[0] == 1              # 16 rows x 1 slot < 32 lanes
    assert resolve(1000, 10016, 16, -1, flags=2 | (4 << 8))[0] == 1    # 16 slots: not a padded form
    assert resolve(1000, 10000, 16, -1, flags=3 << 8)[0] == 1          # slot bits without the padded flag
    assert resolve(0, 0, 4, 0) == (0, MERGE)                   # empty: no rows


def test_pad_host_validation(L):
    """cmrs_pad_workspace: host-only checks of the Section 6.6 conversion input."""
    from paper_1203_2946_gb300 import binding as b
    m = b.cmrs_matrix()
    m.rows, m.cols, m.nnz, m.height, m.strips, m.bits, m.dtype = 100, 100, 500, 16, 7, 4, 0
    m.strip_ptr = m.col_packed = m.val = 256
    n = ctypes.c_size_t()
    assert L.cmrs_pad_workspace(ctypes.byref(m), 8, ctypes.byref(n)) == 0 and n.value >= 256
    assert L.cmrs_pad_workspace(ctypes.byref(m), 2, ctypes.byref(n)) == 0
    assert L.cmrs_pad_workspace(ctypes.byref(m), 1, ctypes.byref(n)) == 2   # 16 rows x 1 slot < 32 lanes
    assert L.cmrs_pad_workspace(ctypes.byref(m), 3, ctypes.byref(n)) == 1   # slots not a power of 2
    assert L.cmrs_pad_workspace(ctypes.byref(m), 16, ctypes.byref(n)) == 1  # slots above 8
    m.flags = 1
    assert L.cmrs_pad_workspace(ctypes.byref(m), 8, ctypes.byref(n)) == 6   # sorted strips
    m.flags = 2 | (3 << 8)
    assert L.cmrs_pad_workspace(ctypes.byref(m), 8, ctypes.byref(n)) == 6   # already padded
    m.flags, m.height, m.strips = 0, 2, 50
    assert L.cmrs_pad_workspace(ctypes.byref(m), 8, ctypes.byref(n)) == 2   # 2 x 8 slots < 32 lanes
    assert L.cmrs_pad_workspace(None, 8, ctypes.byref(n)) == 1


def test_reorder_host_validation(L):
    """Row reordering entry points: argument checks made on the host."""
    p = ctypes.c_void_p(256)
    assert L.cmrs_row_order(10, p, 0, p, None) == 1       # window below 1
    assert L.cmrs_row_order(10, p, 4097, p, None) == 1    # window above 4096
    assert L.cmrs_row_order(0, None, 32, None, None) == 0  # nothing to order
    n = ctypes.c_size_t()
    assert L.cmrs_permute_csr_workspace(1000, ctypes.byref(n)) == 0 and n.value >= 256 + 4000
    assert L.cmrs_permute_csr(10, 5, p, p, p, 2, p, p, p, p, p, 1 << 20, None) == 1   # BF16 input values
    assert L.cmrs_permute_csr(10, 5, p, p, None, 0, p, p, p, None, None, 0, None) == 7  # no workspace
    from paper_1203_2946_gb300 import binding as b
    m = b.cmrs_matrix()
    m.rows, m.cols, m.nnz, m.height, m.strips, m.bits, m.dtype = 10, 10, 5, 4, 3, 4, 0
    m.strip_ptr = m.col_packed = m.val = 256
    assert L.cmrs_spmv_rows(ctypes.byref(m), p, p, None, -1, p, 1 << 20, None) == 1   # no row map


def test_padded_split_workspace(L):
    """cmrs_spmv_workspace for padded matrices: few strips of many passes get
    room for per-part row sums past the 256-byte status block (the split
    walk); many short strips, or plain CMRS, need the status block only.
    Host only: the device pointers are never read."""
    from paper_1203_2946_gb300 import binding as b

    def ws(strips, passes, height=16, slots=8, dtype=0, flags=None):
        m = b.cmrs_matrix()
        m.rows, m.cols, m.height, m.strips = strips * height, 1000, height, strips
        m.nnz, m.bits, m.dtype = strips * passes * 32, L.cmrs_bits_for_height(height), dtype
        m.flags = (2 | ({1: 0, 2: 1, 4: 2, 8: 3}[slots] << 8)) if flags is None else flags
        m.max_strip_nnz = -1
        m.strip_ptr = m.col_packed = m.val = 256
        n = ctypes.c_size_t()
        assert L.cmrs_spmv_workspace(ctypes.byref(m), 3 if flags is None else 0, ctypes.byref(n)) == 0
        return n.value

    few_long = ws(strips=10, passes=4096)
    assert few_long > 256 and (few_long - 256) % 256 == 0
    assert few_long - 256 >= 10 * 2 * 16 * 8            # at least two parts of 16 FP64 row sums per strip
    assert ws(strips=10, passes=4096, dtype=1) < few_long  # FP32 sums take half the room
    assert ws(strips=10, passes=40) == 256                # short strips: one warp per strip
    assert ws(strips=200000, passes=64) == 256            # more strips than two per resident warp
    assert ws(strips=10, passes=4096, flags=0) == 256     # plain CMRS, ROW


def test_binding_checks_tensor_operands_on_the_host():
    """The C ABI takes bare pointers; the Python binding checks each tensor
    (device, value type, contiguity, length) before its pointer goes."""
    import torch
    from paper_1203_2946_gb300 import binding as b
    with pytest.raises(TypeError):
        b._operand(torch.zeros(4, dtype=torch.float64), torch.float64, 4, "x")  # host memory
    with pytest.raises(TypeError):
        b._operand(None, torch.float64, 4, "x")
