"""Thin ctypes binding of libcmrs (include/cmrs.h), same entry-point names.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device arrays are torch CUDA tensors (torch supplies device memory
and streams); `stream=None` means torch's current stream.  Importing this
module loads libcmrs.so and raises if it is missing: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcmrs.so")

CMRS_OK = 0
CMRS_F64, CMRS_F32, CMRS_BF16, CMRS_BF16X2 = 0, 1, 2, 3
CMRS_SORTED, CMRS_PADDED = 1, 2
CMRS_PAD_SLOTS = 8  # the paper's M
CMRS_PAD_SLOTS_SHIFT = 8
CMRS_VARIANT_AUTO, CMRS_VARIANT_ROW, CMRS_VARIANT_STRIP, CMRS_VARIANT_MERGE = -1, 0, 1, 2
CMRS_VARIANT_PADDED = 3
VARIANTS = {"row": 0, "strip": 1, "merge": 2}
DTYPES = {"f64": 0, "f32": 1, "bf16": 2, "bf16x2": 3}
_STORED = {0: torch.float64, 1: torch.float32, 2: torch.int16, 3: torch.int16}
_XTYPE = {0: torch.float64, 1: torch.float32, 2: torch.float32, 3: torch.float32}


class CmrsError(RuntimeError):
    def __init__(self, code, where=""):
        msg = lib().cmrs_error_string(code).decode()
        if code == 5:
            msg += " (cudaError %d)" % lib().cmrs_last_cuda_error()
        super().__init__("%s: %s" % (where, msg) if where else msg)
        self.code = code


class cmrs_matrix(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("height", ctypes.c_int32), ("strips", ctypes.c_int32), ("bits", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("dtype", ctypes.c_int32), ("max_strip_nnz", ctypes.c_int32),
                ("strip_ptr", ctypes.c_void_p), ("col_packed", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class cmrs_selector(ctypes.Structure):
    _fields_ = [("nin", ctypes.c_int32), ("nh", ctypes.c_int32), ("nout", ctypes.c_int32),
                ("params", ctypes.c_void_p), ("feat_mean", ctypes.c_void_p), ("feat_scale", ctypes.c_void_p)]


NFEAT = 32
SEL_HEIGHTS = (1, 2, 4, 8, 16, 32)
SEL_PADDED = ((32, 1), (32, 2), (16, 8))  # choices 18..20: modified CMRS (height, slots)
SEL_CHOICES = 18 + len(SEL_PADDED)

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcmrs.so is not built (run __graft_entry__.build() or "
                               "python paper_1203_2946_gb300/build.py); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, u, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_size_t
        M = ctypes.POINTER(cmrs_matrix)
        sig = {
            "cmrs_error_string": ([i], ctypes.c_char_p),
            "cmrs_last_cuda_error": ([], i),
            "cmrs_bits_for_height": ([i], i),
            "cmrs_pad8": ([ctypes.c_int64], ctypes.c_int64),
            "cmrs_val_bytes": ([ctypes.c_int64, i], ctypes.c_int64),
            "cmrs_from_csr_workspace": ([i, i, i, u, i, ctypes.POINTER(sz)], i),
            "cmrs_from_csr": ([i, i, i, vp, vp, vp, i, i, u, i, vp, vp, vp, vp, sz, vp, M], i),
            "cmrs_to_csr_workspace": ([M, ctypes.POINTER(sz)], i),
            "cmrs_to_csr": ([M, vp, vp, vp, vp, sz, vp], i),
            "cmrs_spmv_workspace": ([M, i, ctypes.POINTER(sz)], i),
            "cmrs_spmv_variant": ([M, i, ctypes.POINTER(ctypes.c_int)], i),
            "cmrs_pad_workspace": ([M, i, ctypes.POINTER(sz)], i),
            "cmrs_row_order": ([i, vp, i, vp, vp], i),
            "cmrs_permute_csr_workspace": ([i, ctypes.POINTER(sz)], i),
            "cmrs_permute_csr": ([i, i, vp, vp, vp, i, vp, vp, vp, vp, vp, sz, vp], i),
            "cmrs_spmv_rows": ([M, vp, vp, vp, i, vp, sz, vp], i),
            "cmrs_pad_layout": ([M, i, vp, ctypes.POINTER(ctypes.c_int32), vp, sz, vp], i),
            "cmrs_pad_fill": ([M, i, vp, ctypes.c_int32, vp, vp, vp, M], i),
            "cmrs_spmv": ([M, vp, vp, i, vp, sz, vp], i),
            "cmrs_spmv_check": ([M, i, vp, vp], i),
            "cmrs_wait_probe": ([vp, u, i, vp], i),
            "cmrs_spmv_noalloc": ([M, vp, vp, vp], i),
            "cmrs_spmv_noalloc_check": ([vp], i),
            "cmrs_gather_probe": ([i, i, vp, vp, vp, vp, vp], i),
            "cmrs_shard_rows": ([i, vp, i, i, vp], i),
            "cmrs_spmm": ([M, i, vp, vp, vp], i),
            "cmrs_spmm_plan_workspace": ([i, vp, vp, i, ctypes.POINTER(sz)], i),
            "cmrs_spmm_plan_create": ([i, vp, vp, vp, vp, i, i, vp, sz, vp, ctypes.POINTER(vp)], i),
            "cmrs_spmm_batched": ([vp, vp], i),
            "cmrs_spmm_plan_info": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)], i),
            "cmrs_spmm_plan_destroy": ([vp], i),
            "cmrs_spmm_autotune": ([i, vp, vp, vp, vp, vp, i, i, vp, sz, vp, ctypes.POINTER(i),
                                    ctypes.POINTER(ctypes.c_float)], i),
            "cmrs_features_workspace": ([i, ctypes.POINTER(sz)], i),
            "cmrs_features": ([i, i, vp, vp, vp, vp, sz, vp], i),
            "cmrs_mlp_param_count": ([i, i, i], ctypes.c_int64),
            "cmrs_mlp_forward": ([i, i, i, i, vp, vp, vp, vp], i),
            "cmrs_mlp_backward": ([i, i, i, i, vp, vp, vp, vp, vp, vp, vp, vp], i),
            "cmrs_mlp_adam": ([i, vp, vp, vp, vp, i, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, vp], i),
            "cmrs_feature_norm": ([i, i, vp, vp, vp, vp, vp], i),
            "cmrs_feature_apply": ([i, i, vp, vp, vp, vp, vp], i),
            "cmrs_cost_targets": ([i, i, vp, ctypes.c_float, vp, vp], i),
            "cmrs_select_strip_workspace": ([i, i, i, i, ctypes.POINTER(sz)], i),
            "cmrs_select_strip": ([i, i, i, vp, vp, ctypes.POINTER(cmrs_selector), ctypes.POINTER(i),
                                   ctypes.POINTER(i), ctypes.POINTER(i), vp, sz, vp], i),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def declared_symbols():
    """Entry points this binding expects libcmrs to export."""
    lib()
    return sorted(n for n in dir(_lib) if n.startswith("cmrs_"))


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def _operand(t, dtype, n, name):
    """The C ABI takes bare device pointers and reads or writes n elements of
    the matrix's value type there: check the tensor before its pointer goes."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s is %s; this matrix's value form takes %s" % (name, t.dtype, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() < n:
        raise ValueError("%s holds %d elements; the product needs %d" % (name, t.numel(), n))


def _check(rc, where):
    if rc != CMRS_OK:
        raise CmrsError(rc, where)


def workspace(nbytes, device="cuda"):
    """A 256-byte aligned device workspace (torch allocations are) whose first
    256 bytes -- the status block every entry point keeps there -- start at
    zero; the library initialises whatever else it reads."""
    t = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    assert t.data_ptr() % 256 == 0
    t[:256].zero_()
    return t


class Matrix:
    """A CMRS matrix whose arrays are torch tensors kept alive with the struct."""

    def __init__(self, struct, strip_ptr, col_packed, val):
        self.struct = struct
        self.strip_ptr = strip_ptr
        self.col_packed = col_packed
        self.val = val
        self._spmv_ws = {}

    @property
    def rows(self):
        return self.struct.rows

    @property
    def cols(self):
        return self.struct.cols

    @property
    def nnz(self):
        return self.struct.nnz

    @property
    def height(self):
        return self.struct.height

    @property
    def dtype(self):
        return self.struct.dtype

    @property
    def x_dtype(self):
        return _XTYPE[self.struct.dtype]

    def ref(self):
        return ctypes.byref(self.struct)

    def spmv_workspace(self, variant):
        if variant not in self._spmv_ws:
            n = ctypes.c_size_t()
            _check(lib().cmrs_spmv_workspace(self.ref(), variant, ctypes.byref(n)), "cmrs_spmv_workspace")
            self._spmv_ws[variant] = workspace(n.value, self.col_packed.device)
        return self._spmv_ws[variant]


def cmrs_from_csr(row_ptr, col_ind, val, cols, height, flags=0, dtype=CMRS_F64, stream=None):
    """CRS (device int32 row_ptr, col_ind; float64 or float32 val) -> Matrix."""
    dev = row_ptr.device
    rows = row_ptr.numel() - 1
    nnz = col_ind.numel()
    assert row_ptr.dtype == torch.int32 and col_ind.dtype == torch.int32
    in_dt = {torch.float64: CMRS_F64, torch.float32: CMRS_F32}[val.dtype]
    strips = (rows + height - 1) // height if height > 0 else 0
    sp = torch.empty(strips + 1, dtype=torch.int32, device=dev)
    pk = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    vb = lib().cmrs_val_bytes(nnz, dtype)
    if vb < 0:
        raise CmrsError(1, "cmrs_val_bytes")
    vout = torch.empty(max(vb, 16), dtype=torch.uint8, device=dev)
    n = ctypes.c_size_t()
    _check(lib().cmrs_from_csr_workspace(rows, nnz, height, flags, dtype, ctypes.byref(n)), "cmrs_from_csr_workspace")
    ws = workspace(n.value, dev)
    m = cmrs_matrix()
    rc = lib().cmrs_from_csr(rows, cols, nnz, _ptr(row_ptr), _ptr(col_ind), _ptr(val), in_dt, height, flags, dtype,
                             _ptr(sp), _ptr(pk), _ptr(vout), _ptr(ws), n.value, _stream(stream), ctypes.byref(m))
    _check(rc, "cmrs_from_csr")
    return Matrix(m, sp, pk, vout)


def cmrs_pad(A: Matrix, slots=CMRS_PAD_SLOTS, stream=None):
    """Section 6.6 modified CMRS of an unsorted matrix with M = slots (1, 2, 4
    or 8): a new Matrix with CMRS_PADDED set (cmrs_pad_layout, then
    cmrs_pad_fill)."""
    dev = A.col_packed.device
    n = ctypes.c_size_t()
    _check(lib().cmrs_pad_workspace(A.ref(), slots, ctypes.byref(n)), "cmrs_pad_workspace")
    ws = workspace(n.value, dev)
    sp = torch.empty(A.struct.strips + 1, dtype=torch.int32, device=dev)
    nnz_p = ctypes.c_int32()
    _check(lib().cmrs_pad_layout(A.ref(), slots, _ptr(sp), ctypes.byref(nnz_p), _ptr(ws), n.value,
                                 _stream(stream)), "cmrs_pad_layout")
    npad = nnz_p.value
    pk = torch.empty(max(npad, 1), dtype=torch.int32, device=dev)
    vb = lib().cmrs_val_bytes(npad, A.dtype)
    vout = torch.empty(max(vb, 16), dtype=torch.uint8, device=dev)
    m = cmrs_matrix()
    _check(lib().cmrs_pad_fill(A.ref(), slots, _ptr(sp), npad, _ptr(pk), _ptr(vout), _stream(stream),
                               ctypes.byref(m)), "cmrs_pad_fill")
    return Matrix(m, sp, pk, vout)


def cmrs_row_order(row_ptr, window, stream=None):
    """Row reordering: perm[i] = original row at position i; rows sorted by
    length (longest first, ties in order) inside windows of `window` rows."""
    rows = row_ptr.numel() - 1
    perm = torch.empty(max(rows, 1), dtype=torch.int32, device=row_ptr.device)
    _check(lib().cmrs_row_order(rows, _ptr(row_ptr), int(window), _ptr(perm), _stream(stream)), "cmrs_row_order")
    return perm[:rows]


def cmrs_permute_csr(row_ptr, col_ind, val, perm, stream=None):
    """CRS of P A (row i = original row perm[i]); val float64/float32 or None."""
    dev = row_ptr.device
    rows, nnz = row_ptr.numel() - 1, col_ind.numel()
    rp = torch.empty(rows + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    vo = torch.empty(max(nnz, 1), dtype=val.dtype, device=dev) if val is not None else None
    vdt = {torch.float64: CMRS_F64, torch.float32: CMRS_F32}[val.dtype] if val is not None else CMRS_F64
    n = ctypes.c_size_t()
    _check(lib().cmrs_permute_csr_workspace(rows, ctypes.byref(n)), "cmrs_permute_csr_workspace")
    ws = workspace(n.value, dev)
    _check(lib().cmrs_permute_csr(rows, nnz, _ptr(row_ptr), _ptr(col_ind), _ptr(val) if val is not None else None,
                                  vdt, _ptr(perm), _ptr(rp), _ptr(ci), _ptr(vo) if vo is not None else None,
                                  _ptr(ws), n.value, _stream(stream)), "cmrs_permute_csr")
    return rp, ci[:nnz], (vo[:nnz] if vo is not None else None)


def cmrs_spmv_rows(A: Matrix, x, row_map, y=None, variant=CMRS_VARIANT_AUTO, workspace_tensor=None, stream=None):
    """y[row_map[i]] = (A x)_i: the product of a row-reordered matrix in the original order."""
    _operand(x, A.x_dtype, A.cols, "x")
    if y is None:
        y = torch.empty(A.rows, dtype=A.x_dtype, device=x.device)
    _operand(y, A.x_dtype, A.rows, "y")
    _operand(row_map, torch.int32, A.rows, "row_map")
    v = variant
    ws = workspace_tensor if workspace_tensor is not None else A.spmv_workspace(
        CMRS_VARIANT_ROW if v == CMRS_VARIANT_AUTO and cmrs_spmv_variant(A, v) == CMRS_VARIANT_MERGE else v)
    rc = lib().cmrs_spmv_rows(A.ref(), _ptr(x), _ptr(y), _ptr(row_map), variant, _ptr(ws), ws.numel(),
                              _stream(stream))
    _check(rc, "cmrs_spmv_rows")
    return y


def cmrs_spmv(A: Matrix, x, y=None, variant=CMRS_VARIANT_AUTO, workspace_tensor=None, stream=None):
    """y = A x on the device; y is allocated if not given and returned."""
    _operand(x, A.x_dtype, A.cols, "x")
    if y is None:
        y = torch.empty(A.rows, dtype=A.x_dtype, device=x.device)
    _operand(y, A.x_dtype, A.rows, "y")
    ws = workspace_tensor if workspace_tensor is not None else A.spmv_workspace(variant)
    rc = lib().cmrs_spmv(A.ref(), _ptr(x), _ptr(y), variant, _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "cmrs_spmv")
    return y


def cmrs_spmv_variant(A: Matrix, variant=CMRS_VARIANT_AUTO):
    """The kernel variant (CMRS_VARIANT_ROW/_STRIP/_MERGE) cmrs_spmv runs."""
    out = ctypes.c_int(-1)
    _check(lib().cmrs_spmv_variant(A.ref(), variant, ctypes.byref(out)), "cmrs_spmv_variant")
    return out.value


def cmrs_spmv_noalloc(A: Matrix, x, y=None, stream=None):
    """y = A x with no workspace and no device allocation by the library (the
    library's fixed scratch array; see cmrs.h for its limit and sharing)."""
    _operand(x, A.x_dtype, A.cols, "x")
    if y is None:
        y = torch.empty(A.rows, dtype=A.x_dtype, device=x.device)
    _operand(y, A.x_dtype, A.rows, "y")
    _check(lib().cmrs_spmv_noalloc(A.ref(), _ptr(x), _ptr(y), _stream(stream)), "cmrs_spmv_noalloc")
    return y


def cmrs_spmv_noalloc_check(stream=None):
    """Reads and clears the status word of cmrs_spmv_noalloc's fixed array on
    the current device; raises CmrsError(CMRS_ERR_TIMEOUT) if a call since the
    last check gave up a bounded wait."""
    _check(lib().cmrs_spmv_noalloc_check(_stream(stream)), "cmrs_spmv_noalloc_check")


def cmrs_spmv_check(A: Matrix, variant=CMRS_VARIANT_AUTO, stream=None):
    ws = A.spmv_workspace(variant)
    _check(lib().cmrs_spmv_check(A.ref(), variant, _ptr(ws), _stream(stream)), "cmrs_spmv_check")


def cmrs_gather_probe(col, val, x, out=None, stream=None):
    """Streams col (int32) and val (float32 or None), gathers x[col] and sums
    the products into out (device float32 [1]): the gather floor of a matrix."""
    if out is None:
        out = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(lib().cmrs_gather_probe(col.numel(), x.numel(), _ptr(col), _ptr(val), _ptr(x), _ptr(out),
                                   _stream(stream)), "cmrs_gather_probe")
    return out


def cmrs_shard_rows(row_ptr, height, parts):
    """Row bounds of `parts` contiguous ranges of whole strips, balanced by
    entries plus rows (host numpy int32 RowPtr in, numpy int32 [parts + 1])."""
    import numpy as np
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    out = np.empty(parts + 1, dtype=np.int32)
    _check(lib().cmrs_shard_rows(rp.size - 1, rp.ctypes.data, int(height), int(parts), out.ctypes.data),
           "cmrs_shard_rows")
    return out


def cmrs_feature_norm(F, stream=None):
    """Per-feature mean and scale (1 / std, 0 if constant) of the rows of F
    (device float64 [B][nin]) and the normalised FP32 inputs; returns
    (mean, scale, X) as device tensors."""
    F = F.contiguous()
    B, nin = F.shape
    mean = torch.empty(nin, dtype=torch.float32, device=F.device)
    scale = torch.empty_like(mean)
    X = torch.empty((B, nin), dtype=torch.float32, device=F.device)
    _check(lib().cmrs_feature_norm(B, nin, _ptr(F), _ptr(mean), _ptr(scale), _ptr(X), _stream(stream)),
           "cmrs_feature_norm")
    return mean, scale, X


def cmrs_feature_apply(F, mean, scale, stream=None):
    """(F - mean) * scale as device float32 [B][nin] (F device float64)."""
    F = F.contiguous()
    B, nin = F.shape
    X = torch.empty((B, nin), dtype=torch.float32, device=F.device)
    _check(lib().cmrs_feature_apply(B, nin, _ptr(F), _ptr(mean), _ptr(scale), _ptr(X), _stream(stream)),
           "cmrs_feature_apply")
    return X


def cmrs_cost_targets(times, cap, stream=None):
    """min(log2(t / row minimum), cap) as device float32 (times device float64 [B][nout])."""
    times = times.contiguous()
    B, nout = times.shape
    T = torch.empty((B, nout), dtype=torch.float32, device=times.device)
    _check(lib().cmrs_cost_targets(B, nout, _ptr(times), float(cap), _ptr(T), _stream(stream)), "cmrs_cost_targets")
    return T


def cmrs_wait_probe(ws, tries, arrive, stream=None):
    """Bounded in-kernel wait on a phase that completes only if `arrive`;
    leaves the timeout bit in the status word of `ws` when it gives up."""
    _check(lib().cmrs_wait_probe(_ptr(ws), int(tries), int(bool(arrive)), _stream(stream)), "cmrs_wait_probe")


def cmrs_to_csr(A: Matrix, with_values=True, stream=None):
    dev = A.col_packed.device
    rp = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=dev)
    vb = lib().cmrs_val_bytes(A.nnz, A.dtype)
    vo = torch.empty(max(vb, 16), dtype=torch.uint8, device=dev) if with_values else None
    n = ctypes.c_size_t()
    _check(lib().cmrs_to_csr_workspace(A.ref(), ctypes.byref(n)), "cmrs_to_csr_workspace")
    ws = workspace(n.value, dev)
    rc = lib().cmrs_to_csr(A.ref(), _ptr(rp), _ptr(ci), _ptr(vo) if with_values else ctypes.c_void_p(0), _ptr(ws),
                           n.value, _stream(stream))
    _check(rc, "cmrs_to_csr")
    return rp, ci[:A.nnz], vo


def stored_values(A: Matrix):
    """The value array viewed as its storage type (BF16X2: hi then lo halves, int16 bits)."""
    nnz = A.nnz
    dt = _STORED[A.dtype]
    if A.dtype == CMRS_BF16X2:
        pad = lib().cmrs_pad8(nnz)
        w = A.val.view(torch.int16)
        return torch.cat([w[:nnz], w[pad:pad + nnz]])
    return A.val.view(dt)[:nnz]


# ----------------------------------------------------------------------------- SpMM
def cmrs_spmm(A: Matrix, X, Y=None, stream=None):
    """Y = A X for one CMRS_F32 matrix; X [cols][k] row-major float32."""
    k = X.shape[1]
    _operand(X, torch.float32, A.cols * k, "X")
    if Y is None:
        Y = torch.empty((A.rows, k), dtype=torch.float32, device=X.device)
    _operand(Y, torch.float32, A.rows * k, "Y")
    _check(lib().cmrs_spmm(A.ref(), k, _ptr(X), _ptr(Y), _stream(stream)), "cmrs_spmm")
    return Y


def _batch_arrays(mats, Xs, Ys):
    n = len(mats)
    if not (len(Xs) == n and len(Ys) == n):
        raise ValueError("one X and one Y per matrix")
    for M, X, Y in zip(mats, Xs, Ys):
        _operand(X, torch.float32, M.cols * X.shape[1], "X")
        _operand(Y, torch.float32, M.rows * X.shape[1], "Y")
    A = (ctypes.POINTER(cmrs_matrix) * n)(*[ctypes.pointer(m.struct) for m in mats])
    k = (ctypes.c_int32 * n)(*[int(X.shape[1]) for X in Xs])
    Xp = (ctypes.c_void_p * n)(*[X.data_ptr() for X in Xs])
    Yp = (ctypes.c_void_p * n)(*[Y.data_ptr() for Y in Ys])
    return A, k, Xp, Yp


class SpmmPlan:
    """A batched SpMM plan: schedule in a device workspace + captured graph."""

    def __init__(self, mats, Xs, Ys, work_target=8192, use_graph=True, stream=None):
        self._keep = (mats, Xs, Ys)
        A, k, Xp, Yp = _batch_arrays(mats, Xs, Ys)
        n = ctypes.c_size_t()
        _check(lib().cmrs_spmm_plan_workspace(len(mats), A, k, int(work_target), ctypes.byref(n)),
               "cmrs_spmm_plan_workspace")
        self.ws = workspace(n.value, Xs[0].device)
        self.handle = ctypes.c_void_p()
        _check(lib().cmrs_spmm_plan_create(len(mats), A, k, Xp, Yp, int(work_target), int(bool(use_graph)),
                                           _ptr(self.ws), n.value, _stream(stream), ctypes.byref(self.handle)),
               "cmrs_spmm_plan_create")

    def info(self):
        a, b_, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().cmrs_spmm_plan_info(self.handle, ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c)),
               "cmrs_spmm_plan_info")
        return {"units": a.value, "grid": b_.value, "work_target": c.value}

    def close(self):
        if self.handle:
            lib().cmrs_spmm_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cmrs_spmm_batched(plan: SpmmPlan, stream=None):
    _check(lib().cmrs_spmm_batched(plan.handle, _stream(stream)), "cmrs_spmm_batched")


def cmrs_spmm_autotune(mats, Xs, Ys, candidates=(1024, 4096, 16384, 65536), reps=5, stream=None):
    A, k, Xp, Yp = _batch_arrays(mats, Xs, Ys)
    need = 0
    for c in candidates:
        n = ctypes.c_size_t()
        _check(lib().cmrs_spmm_plan_workspace(len(mats), A, k, int(c), ctypes.byref(n)), "cmrs_spmm_plan_workspace")
        need = max(need, n.value)
    ws = workspace(need, Xs[0].device)
    cand = (ctypes.c_int * len(candidates))(*candidates)
    best, ms = ctypes.c_int(), ctypes.c_float()
    _check(lib().cmrs_spmm_autotune(len(mats), A, k, Xp, Yp, cand, len(candidates), int(reps), _ptr(ws), need,
                                    _stream(stream), ctypes.byref(best), ctypes.byref(ms)), "cmrs_spmm_autotune")
    return best.value, ms.value


# ----------------------------------------------------------------------------- selector
def cmrs_features(row_ptr, col_ind, stream=None):
    rows = row_ptr.numel() - 1
    n = ctypes.c_size_t()
    _check(lib().cmrs_features_workspace(rows, ctypes.byref(n)), "cmrs_features_workspace")
    ws = workspace(n.value, row_ptr.device)
    f = torch.empty(NFEAT, dtype=torch.float64, device=row_ptr.device)
    _check(lib().cmrs_features(rows, col_ind.numel(), _ptr(row_ptr), _ptr(col_ind), _ptr(f), _ptr(ws), n.value,
                               _stream(stream)), "cmrs_features")
    return f


def mlp_param_count(nin, nh, nout):
    return int(lib().cmrs_mlp_param_count(nin, nh, nout))


def cmrs_mlp_forward(X, params, nh, nout, acts=None, stream=None):
    B, nin = X.shape
    if acts is None:
        acts = torch.empty(B * (4 * nh + nout), dtype=torch.float32, device=X.device)
    _check(lib().cmrs_mlp_forward(B, nin, nh, nout, _ptr(X), _ptr(params), _ptr(acts), _stream(stream)),
           "cmrs_mlp_forward")
    return acts


def mlp_output(acts, B, nh, nout):
    return acts[4 * B * nh:4 * B * nh + B * nout].view(B, nout)


def cmrs_mlp_backward(X, T, params, acts, nh, nout, grads=None, scratch=None, loss=None, stream=None):
    B, nin = X.shape
    dev = X.device
    if grads is None:
        grads = torch.empty_like(params)
    if scratch is None:
        scratch = torch.empty(B * (nout + 2 * nh), dtype=torch.float32, device=dev)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=dev)
    _check(lib().cmrs_mlp_backward(B, nin, nh, nout, _ptr(X), _ptr(T), _ptr(params), _ptr(acts), _ptr(grads),
                                   _ptr(scratch), _ptr(loss), _stream(stream)), "cmrs_mlp_backward")
    return grads, loss


def cmrs_mlp_adam(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().cmrs_mlp_adam(params.numel(), _ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(step), float(lr),
                               float(beta1), float(beta2), float(eps), _stream(stream)), "cmrs_mlp_adam")


def cmrs_select_strip(row_ptr, col_ind, cols, model=None, stream=None):
    """(height, variant, slots) for a CRS matrix (slots 0: plain CMRS);
    model: dict(params, mean, scale, nh) of device tensors, or None for the
    exhaustive autotune."""
    rows = row_ptr.numel() - 1
    nnz = col_ind.numel()
    n = ctypes.c_size_t()
    _check(lib().cmrs_select_strip_workspace(rows, cols, nnz, int(model is None), ctypes.byref(n)),
           "cmrs_select_strip_workspace")
    ws = workspace(n.value, row_ptr.device)
    sel = None
    if model is not None:
        sel = cmrs_selector(NFEAT, int(model["nh"]), SEL_CHOICES, model["params"].data_ptr(),
                            model["mean"].data_ptr(), model["scale"].data_ptr())
    h, v, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().cmrs_select_strip(rows, cols, nnz, _ptr(row_ptr), _ptr(col_ind),
                                   ctypes.byref(sel) if sel is not None else None, ctypes.byref(h), ctypes.byref(v),
                                   ctypes.byref(m), _ptr(ws), n.value, _stream(stream)), "cmrs_select_strip")
    return h.value, v.value, m.value
