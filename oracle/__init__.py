"""CMRS oracle: TEST INFRASTRUCTURE, not part of the product.

A ctypes/numpy front end to cmrs_oracle.c, the plain single-threaded FP64 CPU
restatement of the CMRS method (arXiv:1203.2946).  Only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may import this package.  It
imports nothing from paper_1203_2946_gb300 and the CUDA library imports nothing
from it.
"""
import ctypes
import numpy as np

from .build_oracle import build as _build

_lib = None

ORC_OK, ORC_BAD_HEIGHT, ORC_BAD_CSR, ORC_COL_OVERFLOW, ORC_BAD_ARG = 0, 1, 2, 3, 4
F64, F32, BF16, BF16X2 = 0, 1, 2, 3
NFEAT = 32


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build())
        d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        _lib.orc_bits_for_height.argtypes = [i]
        _lib.orc_bits_for_height.restype = i
        _lib.orc_csr_spmv.argtypes = [i, vp, vp, vp, vp, vp, vp]
        _lib.orc_dense_matvec.argtypes = [i, i, vp, vp, vp]
        _lib.orc_csr_to_cmrs.argtypes = [i, i, i, vp, vp, vp, i, i, vp, vp, vp, vp, vp]
        _lib.orc_csr_to_cmrs.restype = i
        _lib.orc_cmrs_to_csr.argtypes = [i, i, i, vp, vp, vp, vp, vp, vp, vp]
        _lib.orc_cmrs_to_csr.restype = i
        _lib.orc_cmrs_spmv.argtypes = [i, i, vp, vp, vp, vp, vp]
        _lib.orc_bf16_from_f32.argtypes = [ctypes.c_float]
        _lib.orc_bf16_from_f32.restype = ctypes.c_uint16
        _lib.orc_f32_from_bf16.argtypes = [ctypes.c_uint16]
        _lib.orc_f32_from_bf16.restype = ctypes.c_float
        _lib.orc_encode_f64.argtypes = [i, vp, i, vp]
        _lib.orc_encode_f64.restype = i
        _lib.orc_encode_f32.argtypes = [i, vp, i, vp]
        _lib.orc_encode_f32.restype = i
        _lib.orc_decode_to_f64.argtypes = [i, vp, i, vp]
        _lib.orc_decode_to_f64.restype = i
        for name in ("orc_model_segments",):
            getattr(_lib, name).argtypes = [d, d, d]
            getattr(_lib, name).restype = d
        for name in ("orc_model_f", "orc_model_a"):
            getattr(_lib, name).argtypes = [d, d, d, d]
            getattr(_lib, name).restype = d
        _lib.orc_segments_at.argtypes = [ctypes.c_long, ctypes.c_long, ctypes.c_long]
        _lib.orc_segments_at.restype = d
        _lib.orc_beta.argtypes = [d, d, d, d, d, vp, vp]
        _lib.orc_features.argtypes = [i, i, vp, vp, vp]
        _lib.orc_mlp_forward.argtypes = [i, i, i, i] + [vp] * 12
        _lib.orc_mlp_backward.argtypes = [i, i, i, i] + [vp] * 15
        _lib.orc_mlp_backward.restype = d
        _lib.orc_adam_step.argtypes = [i, vp, vp, vp, vp, i, d, d, d, d]
        _lib.orc_pad_arrange.argtypes = [i, i, i, vp, vp, vp, vp, vp]
        _lib.orc_pad_arrange.restype = i
        _lib.orc_row_order.argtypes = [i, vp, i, vp]
        _lib.orc_row_order.restype = i
        _lib.orc_permute_csr.argtypes = [i, vp, vp, vp, vp, vp, vp, vp]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__("oracle status %d" % code)
        self.code = code


def bits_for_height(h):
    return lib().orc_bits_for_height(int(h))


def csr_spmv(row_ptr, col_ind, val, x):
    """y = A x and a = |A||x| in FP64, CRS order (Sections 2.1, 2.3)."""
    rp, ci = _c(row_ptr, np.int32), _c(col_ind, np.int32)
    v, xx = _c(val, np.float64), _c(x, np.float64)
    rows = rp.size - 1
    y = np.empty(rows, np.float64)
    a = np.empty(rows, np.float64)
    lib().orc_csr_spmv(rows, _p(rp), _p(ci), _p(v), _p(xx), _p(y), _p(a))
    return y, a


def dense_matvec(A, x):
    A = _c(A, np.float64)
    xx = _c(x, np.float64)
    y = np.empty(A.shape[0], np.float64)
    lib().orc_dense_matvec(A.shape[0], A.shape[1], _p(A), _p(xx), _p(y))
    return y


def csr_to_cmrs(row_ptr, col_ind, val, cols, height, sorted_=False):
    """Section 3 conversion (+ Section 4 packing and optional in-strip sort).
    Returns dict(strip_ptr, packed, row_in_strip, val, src, bits)."""
    rp, ci, v = _c(row_ptr, np.int32), _c(col_ind, np.int32), _c(val, np.float64)
    rows, nnz = rp.size - 1, ci.size
    h = int(height)
    strips = (rows + h - 1) // h if h > 0 else 0
    sp = np.empty(strips + 1, np.int32)
    pk = np.empty(nnz, np.uint32)
    ris = np.empty(nnz, np.int32)
    vo = np.empty(nnz, np.float64)
    src = np.empty(nnz, np.int32)
    rc = lib().orc_csr_to_cmrs(rows, int(cols), nnz, _p(rp), _p(ci), _p(v), h, int(bool(sorted_)),
                               _p(sp), _p(pk), _p(ris), _p(vo), _p(src))
    if rc:
        raise OracleError(rc)
    return dict(strip_ptr=sp, packed=pk, row_in_strip=ris, val=vo, src=src, bits=bits_for_height(h))


def cmrs_to_csr(rows, height, strip_ptr, packed, val):
    sp, pk, v = _c(strip_ptr, np.int32), _c(packed, np.uint32), _c(val, np.float64)
    nnz = pk.size
    rp = np.empty(rows + 1, np.int32)
    ci = np.empty(nnz, np.int32)
    vo = np.empty(nnz, np.float64)
    src = np.empty(nnz, np.int32)
    rc = lib().orc_cmrs_to_csr(int(rows), nnz, int(height), _p(sp), _p(pk), _p(v), _p(rp), _p(ci), _p(vo), _p(src))
    if rc:
        raise OracleError(rc)
    return dict(row_ptr=rp, col_ind=ci, val=vo, src=src)


def cmrs_spmv(rows, height, strip_ptr, packed, val, x):
    """Algorithm 1 (Section 4) evaluated sequentially in FP64."""
    sp, pk = _c(strip_ptr, np.int32), _c(packed, np.uint32)
    v, xx = _c(val, np.float64), _c(x, np.float64)
    y = np.empty(int(rows), np.float64)
    lib().orc_cmrs_spmv(int(rows), int(height), _p(sp), _p(pk), _p(v), _p(xx), _p(y))
    return y


def pad_arrange(rows, height, strip_ptr, packed, slots=8):
    """Section 6.6 modified CMRS: strips rearranged into 32-item chunks with at
    most `slots` contiguous items per row per chunk, zero-filled.  Returns
    dict(strip_ptr, packed, src) with src[i] = source position or -1 (zero)."""
    sp, pk = _c(strip_ptr, np.int32), _c(packed, np.uint32)
    h = int(height)
    out_sp = np.empty(sp.size, np.int32)
    rc = lib().orc_pad_arrange(int(rows), h, int(slots), _p(sp), _p(pk), _p(out_sp), None, None)
    if rc:
        raise OracleError(rc)
    n = int(out_sp[-1])
    out_pk = np.empty(n, np.uint32)
    src = np.empty(n, np.int64)
    rc = lib().orc_pad_arrange(int(rows), h, int(slots), _p(sp), _p(pk), _p(out_sp), _p(out_pk), _p(src))
    if rc:
        raise OracleError(rc)
    return dict(strip_ptr=out_sp, packed=out_pk, src=src)


def row_order(row_ptr, window):
    """Row reordering: windows of `window` rows, each by length (longest
    first, ties in original order).  perm[i] = original row at position i."""
    rp = _c(row_ptr, np.int32)
    perm = np.empty(rp.size - 1, np.int32)
    rc = lib().orc_row_order(rp.size - 1, _p(rp), int(window), _p(perm))
    if rc:
        raise OracleError(rc)
    return perm


def permute_csr(row_ptr, col_ind, val, perm):
    """CRS of P A: row i is the original row perm[i]."""
    rp, ci, v, pm = _c(row_ptr, np.int32), _c(col_ind, np.int32), _c(val, np.float64), _c(perm, np.int32)
    rows = rp.size - 1
    rpo = np.empty(rows + 1, np.int32)
    cio = np.empty(ci.size, np.int32)
    vo = np.empty(ci.size, np.float64)
    lib().orc_permute_csr(rows, _p(rp), _p(ci), _p(v), _p(pm), _p(rpo), _p(cio), _p(vo))
    return rpo, cio, vo


_STORE_DT = {F64: (np.float64, 1), F32: (np.float32, 1), BF16: (np.uint16, 1), BF16X2: (np.uint16, 2)}


def encode(val, dtype):
    """Stored bits of each value form (F64/F32/BF16/BF16X2 = hi[n] then lo[n])."""
    src = np.asarray(val)
    dt, mult = _STORE_DT[dtype]
    n = src.size
    out = np.empty(n * mult, dt)
    if src.dtype == np.float32:
        s = _c(src, np.float32)
        rc = lib().orc_encode_f32(n, _p(s), int(dtype), _p(out))
    else:
        s = _c(src, np.float64)
        rc = lib().orc_encode_f64(n, _p(s), int(dtype), _p(out))
    if rc:
        raise OracleError(rc)
    return out


def decode(stored, dtype, n):
    """Value each stored form represents, in FP64 (quantised-input oracle)."""
    dt, _ = _STORE_DT[dtype]
    s = _c(stored, dt)
    out = np.empty(n, np.float64)
    rc = lib().orc_decode_to_f64(int(n), _p(s), int(dtype), _p(out))
    if rc:
        raise OracleError(rc)
    return out


def bf16_from_f32(f):
    return lib().orc_bf16_from_f32(float(f))


def f32_from_bf16(h):
    return lib().orc_f32_from_bf16(int(h))


def model_f(h, mu, lam=128.0, b=4.0):
    return lib().orc_model_f(h, mu, lam, b)


def model_a(h, mu, lam=128.0, b=4.0):
    return lib().orc_model_a(h, mu, lam, b)


def model_segments(n, lam, b):
    return lib().orc_model_segments(n, lam, b)


def segments_at(n, lam, start):
    return lib().orc_segments_at(int(n), int(lam), int(start))


def beta(nnz, rows, strips, s_v, s_i=4.0):
    bm, bp = ctypes.c_double(), ctypes.c_double()
    lib().orc_beta(float(nnz), float(rows), float(strips), float(s_v), float(s_i),
                   ctypes.byref(bm), ctypes.byref(bp))
    return bm.value, bp.value


def features(row_ptr, col_ind):
    rp, ci = _c(row_ptr, np.int32), _c(col_ind, np.int32)
    f = np.empty(NFEAT, np.float64)
    lib().orc_features(rp.size - 1, ci.size, _p(rp), _p(ci), _p(f))
    return f


def mlp_forward(X, W1, b1, W2, b2, W3, b3):
    X = _c(X, np.float64)
    B, nin = X.shape
    nh, nout = W1.shape[0], W3.shape[0]
    W1, b1, W2, b2, W3, b3 = (_c(a, np.float64) for a in (W1, b1, W2, b2, W3, b3))
    Z1, H1, Z2, H2 = (np.empty((B, nh)) for _ in range(4))
    O = np.empty((B, nout))
    lib().orc_mlp_forward(B, nin, nh, nout, _p(X), _p(W1), _p(b1), _p(W2), _p(b2), _p(W3), _p(b3),
                          _p(Z1), _p(H1), _p(Z2), _p(H2), _p(O))
    return dict(Z1=Z1, H1=H1, Z2=Z2, H2=H2, O=O)


def mlp_loss_grad(X, T, W1, b1, W2, b2, W3, b3):
    """Loss 1/(2 B nout) sum (O-T)^2 and its gradients (dict)."""
    fw = mlp_forward(X, W1, b1, W2, b2, W3, b3)
    X, T = _c(X, np.float64), _c(T, np.float64)
    B, nin = X.shape
    nh, nout = W1.shape[0], W3.shape[0]
    W2, W3 = _c(W2, np.float64), _c(W3, np.float64)
    g = dict(W1=np.empty((nh, nin)), b1=np.empty(nh), W2=np.empty((nh, nh)), b2=np.empty(nh),
             W3=np.empty((nout, nh)), b3=np.empty(nout))
    loss = lib().orc_mlp_backward(B, nin, nh, nout, _p(X), _p(W2), _p(W3), _p(fw["Z1"]), _p(fw["H1"]),
                                  _p(fw["Z2"]), _p(fw["H2"]), _p(fw["O"]), _p(T),
                                  _p(g["W1"]), _p(g["b1"]), _p(g["W2"]), _p(g["b2"]), _p(g["W3"]), _p(g["b3"]))
    return loss, g, fw


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on FP64 arrays p, m, v."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gg = _c(g, np.float64)
    lib().orc_adam_step(p.size, _p(p), _p(gg), _p(m), _p(v), int(t), float(lr), float(b1), float(b2), float(eps))
