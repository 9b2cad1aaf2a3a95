"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

Every generator returns a CRS matrix (int32 RowPtr, int32 ColInd with columns
strictly increasing inside each row, values) and, where a workload fixes one,
the dense input vector.  Nothing here computes any part of the CMRS method:
no strips, no packing, no products.  The stand-ins replace the University of
Florida collection the paper measured on (Section 6.1), which is not available
here; their shapes follow the five workloads this library is measured on.

Random streams: numpy's default_rng (PCG64) seeded through SeedSequence; each
independent quantity (row lengths, columns, values, x) draws from its own
spawned child so that changing one recipe never shifts another.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSR:
    rows: int
    cols: int
    row_ptr: np.ndarray  # int32 [rows + 1]
    col_ind: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 or float32 [nnz]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col_ind.size)

    def dense(self) -> np.ndarray:
        a = np.zeros((self.rows, self.cols), np.float64)
        r = np.repeat(np.arange(self.rows), np.diff(self.row_ptr))
        np.add.at(a, (r, self.col_ind.astype(np.int64)), self.val.astype(np.float64))
        return a


def _streams(seed: int, k: int):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(k)]


def _finish(rows, cols, lengths, col_ind, val, name, **meta):
    rp = np.zeros(rows + 1, np.int64)
    np.cumsum(lengths, out=rp[1:])
    assert rp[-1] < 2**31
    return CSR(rows, cols, rp.astype(np.int32), np.ascontiguousarray(col_ind, np.int32),
               np.ascontiguousarray(val), name, meta)


# --------------------------------------------------------------------------- stencils
def _stencil(dims, offsets, name):
    """Rows in natural order (last dimension fastest); `offsets` are tuples in
    the same dimension order, listed so that their column offsets increase.
    Out-of-grid neighbours are dropped (Dirichlet truncation, no wrap)."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    coords = np.indices(dims).reshape(len(dims), -1)
    strides = [int(np.prod(dims[i + 1:])) for i in range(len(dims))]
    valid = []
    for off in offsets:
        ok = np.ones(n, bool)
        for d, o in enumerate(off):
            if o:
                c = coords[d] + o
                ok &= (c >= 0) & (c < dims[d])
        valid.append(ok)
    valid = np.stack(valid)  # [noff, n]
    lengths = valid.sum(0)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(lengths, out=rp[1:])
    nnz = int(rp[-1])
    col = np.empty(nnz, np.int32)
    is_diag = np.zeros(nnz, bool)
    before = np.zeros(n, np.int64)
    rows = np.arange(n, dtype=np.int64)
    for k, off in enumerate(offsets):
        ok = valid[k]
        dcol = sum(o * s for o, s in zip(off, strides))
        pos = rp[:-1][ok] + before[ok]
        col[pos] = (rows[ok] + dcol).astype(np.int32)
        if not any(off):
            is_diag[pos] = True
        before += ok
    return n, lengths, col, is_diag, rp


def laplacian_2d_5pt(nx: int = 64, ny: int = 64) -> CSR:
    """2-D 5-point Laplacian on an nx-by-ny grid, natural order, non-periodic:
    4 on the diagonal, -1 for each in-grid neighbour (FP64)."""
    offs = [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
    n, lengths, col, is_diag, _ = _stencil((ny, nx), offs, "lap2d")
    val = np.where(is_diag, 4.0, -1.0)
    return _finish(n, n, lengths, col, val, "laplacian_2d_5pt_%dx%d" % (nx, ny), grid=(nx, ny))


def stencil_2d_9pt(nx, ny, seed=1, dtype=np.float64) -> CSR:
    offs = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return _valued_stencil((ny, nx), offs, seed, dtype, "stencil_2d_9pt")


def stencil_3d_7pt(nx, ny, nz, seed=1, dtype=np.float64) -> CSR:
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    return _valued_stencil((nz, ny, nx), offs, seed, dtype, "stencil_3d_7pt")


def stencil_3d_27pt(nx: int = 128, ny: int = 128, nz: int = 128, seed: int = 1, dtype=np.float64) -> CSR:
    """3-D 27-point stencil, natural (z, y, x) order, non-periodic.  Off-diagonal
    values U[-1, 1]; the diagonal is the row's sum of |off-diagonal| plus 1
    (strict diagonal dominance).  128^3 gives 55,742,968 entries."""
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return _valued_stencil((nz, ny, nx), offs, seed, dtype, "stencil_3d_27pt")


def _valued_stencil(dims, offs, seed, dtype, name):
    n, lengths, col, is_diag, rp = _stencil(dims, offs, name)
    (rv,) = _streams(seed, 1)
    val = rv.uniform(-1.0, 1.0, size=col.size)
    val[is_diag] = 0.0
    absrow = np.add.reduceat(np.abs(val), rp[:-1].astype(np.int64)) if col.size else np.zeros(n)
    absrow[lengths == 0] = 0.0
    row_of_diag = np.repeat(np.arange(n), lengths)[is_diag]
    val[is_diag] = absrow[row_of_diag] + 1.0
    csr = _finish(n, n, lengths, col, val.astype(dtype), "%s_%s" % (name, "x".join(map(str, dims[::-1]))),
                  grid=tuple(dims[::-1]))
    return csr


def uniform_vector(n: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """x ~ U[-1, 1] from default_rng(seed)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n).astype(dtype)


def normal_vector(n: int, seed: int = 0, dtype=np.float32) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n).astype(dtype)


# --------------------------------------------------------------------------- random structures
def _distinct_sorted_columns(lengths, lo, width, rng):
    """For each row i, lengths[i] distinct columns drawn uniformly from
    [lo[i], lo[i] + width[i]), sorted.  Draw iid, then redraw every repeated
    column until none is left; the procedure commutes with any relabelling of
    the column range, so each row's set is a uniform random subset."""
    rows = lengths.size
    row_of = np.repeat(np.arange(rows, dtype=np.int64), lengths)
    lo_e = np.repeat(np.asarray(lo, np.int64), lengths)
    w_e = np.repeat(np.asarray(width, np.int64), lengths)
    col = lo_e + rng.integers(0, w_e)
    span = int(np.max(lo_e + w_e)) + 1 if col.size else 1
    while True:
        key = row_of * span + col
        order = np.argsort(key, kind="stable")
        key = key[order]
        col = col[order]
        dup = np.zeros(col.size, bool)
        dup[1:] = key[1:] == key[:-1]
        if not dup.any():
            return col
        idx = np.nonzero(dup)[0]
        col[idx] = lo_e[idx] + rng.integers(0, w_e[idx])


def powerlaw_rows(n: int = 4_194_304, alpha: float = 2.1, kmax: int = 100_000, seed: int = 0) -> CSR:
    """Row lengths Zipf(alpha) (numpy semantics, support k >= 1) clipped to
    [1, kmax]; columns uniformly random and distinct within the row; values
    N(0, 1) in FP32."""
    r_len, r_col, r_val = _streams(seed, 3)
    lengths = np.minimum(r_len.zipf(alpha, n), kmax).astype(np.int64)
    col = _distinct_sorted_columns(lengths, np.zeros(n, np.int64), np.full(n, n, np.int64), r_col)
    val = r_val.standard_normal(col.size).astype(np.float32)
    return _finish(n, n, lengths, col, val, "powerlaw_n%d_a%g" % (n, alpha), alpha=alpha, kmax=kmax)


def banded_random(n: int, width: int, nnz_lo: int = 10, nnz_hi: int = 60, seed: int = 0) -> CSR:
    """Banded random matrix.  Row i has L_i ~ U{nnz_lo..nnz_hi} entries inside
    the window [lo_i, lo_i + w), lo_i = clamp(i - w/2, 0, n - w), w = min(width,
    n); the window is shifted, never clipped, so the row always fits.  The
    window is cut into L_i strata [floor(j w / L), floor((j+1) w / L)) and one
    column is drawn uniformly in each, which keeps the columns distinct and
    sorted without a sort.  Values N(0, 1) in FP32."""
    r_len, r_col, r_val = _streams(seed, 3)
    w = min(int(width), n)
    hi = min(nnz_hi, w)
    lengths = r_len.integers(min(nnz_lo, hi), hi + 1, size=n).astype(np.int64)
    i = np.arange(n, dtype=np.int64)
    lo = np.clip(i - w // 2, 0, n - w)
    row_of = np.repeat(i, lengths)
    starts = np.zeros(n + 1, np.int64)
    np.cumsum(lengths, out=starts[1:])
    j = np.arange(row_of.size, dtype=np.int64) - starts[row_of]
    L = lengths[row_of]
    b0 = (j * w) // L
    b1 = ((j + 1) * w) // L
    col = lo[row_of] + b0 + np.floor(r_col.random(row_of.size) * (b1 - b0)).astype(np.int64)
    val = r_val.standard_normal(col.size).astype(np.float32)
    return _finish(n, n, lengths, col, val, "banded_n%d_w%d" % (n, w), width=w)


def uniform_random(n: int, mu: float, seed: int = 0, dtype=np.float32) -> CSR:
    """Each row draws Poisson(mu) (at least 1, at most n) distinct uniform columns."""
    r_len, r_col, r_val = _streams(seed, 3)
    lengths = np.clip(r_len.poisson(mu, n), 1, n).astype(np.int64)
    col = _distinct_sorted_columns(lengths, np.zeros(n, np.int64), np.full(n, n, np.int64), r_col)
    val = r_val.standard_normal(col.size).astype(dtype)
    return _finish(n, n, lengths, col, val, "uniform_n%d_mu%g" % (n, mu), mu=mu)


def block_diagonal(n: int, block: int, seed: int = 0, dtype=np.float32) -> CSR:
    """Dense block x block blocks on the diagonal (the last block may be
    smaller); values N(0, 1)."""
    (r_val,) = _streams(seed, 1)
    i = np.arange(n, dtype=np.int64)
    b0 = (i // block) * block
    b1 = np.minimum(b0 + block, n)
    lengths = b1 - b0
    row_of = np.repeat(i, lengths)
    starts = np.zeros(n + 1, np.int64)
    np.cumsum(lengths, out=starts[1:])
    col = b0[row_of] + (np.arange(row_of.size, dtype=np.int64) - starts[row_of])
    val = r_val.standard_normal(col.size).astype(dtype)
    return _finish(n, n, lengths, col, val, "blockdiag_n%d_b%d" % (n, block), block=block)


def random_csr(rows: int, cols: int, density: float, seed: int = 0, empty_row_frac: float = 0.0,
               dtype=np.float64) -> CSR:
    """Small general matrices for edge cases: Bernoulli(density) pattern, a
    fraction of rows forced empty, values U[-1, 1]."""
    r_pat, r_empty, r_val = _streams(seed, 3)
    mask = r_pat.random((rows, cols)) < density
    if empty_row_frac > 0:
        mask[r_empty.random(rows) < empty_row_frac] = False
    lengths = mask.sum(1).astype(np.int64)
    col = np.nonzero(mask)[1].astype(np.int32)
    val = r_val.uniform(-1.0, 1.0, col.size).astype(dtype)
    return _finish(rows, cols, lengths, col, val, "random_%dx%d_d%g" % (rows, cols, density))


def from_lengths(lengths, cols: int, seed: int = 0, dtype=np.float64) -> CSR:
    """Rows with prescribed lengths (may be 0), distinct uniform columns."""
    r_col, r_val = _streams(seed, 2)
    lengths = np.asarray(lengths, np.int64)
    rows = lengths.size
    col = _distinct_sorted_columns(lengths, np.zeros(rows, np.int64), np.full(rows, cols, np.int64), r_col)
    val = r_val.uniform(-1.0, 1.0, col.size).astype(dtype)
    return _finish(rows, cols, lengths, col, val, "lengths_%d" % rows)


def random_lengths_exact_nnz(nnz: int, max_len: int, cols: int, seed: int = 0) -> CSR:
    """Rows of U{1..max_len} entries, as many as it takes to hold exactly
    `nnz` entries (the last row shortened to fit); row i's j-th of L columns
    is drawn uniformly from the stratum [j cols / L, (j + 1) cols / L), so the
    columns are distinct and increasing.  Values U[-1, 1] FP32."""
    r_len, r_col, r_val = _streams(seed, 3)
    lengths = r_len.integers(1, max_len + 1, size=4 * nnz // (max_len + 1) + 64)
    cum = np.cumsum(lengths)
    rows = int(np.searchsorted(cum, nnz)) + 1
    lengths = lengths[:rows].astype(np.int64)
    lengths[-1] -= int(cum[rows - 1]) - nnz
    L = np.repeat(lengths, lengths)
    start = np.repeat(np.cumsum(lengths) - lengths, lengths)
    j = np.arange(nnz, dtype=np.int64) - start
    lo = j * cols // L
    hi = (j + 1) * cols // L
    col = lo + (r_col.random(nnz) * (hi - lo)).astype(np.int64)
    val = r_val.uniform(-1.0, 1.0, nnz).astype(np.float32)
    return _finish(rows, cols, lengths, col, val, "lengths_exact_%d" % nnz)


# --------------------------------------------------------------------------- named workloads
def workload_laplacian_64():
    """5-point Laplacian 64x64 (n=4,096, nnz=20,224), FP64, x U[-1,1] seed 0."""
    a = laplacian_2d_5pt(64, 64)
    return a, uniform_vector(a.cols, 0)


def workload_stencil27_128(dtype=np.float64):
    """27-point stencil 128^3 (n=2,097,152, nnz=55,742,968), matrix seed 1,
    x U[-1,1] seed 0."""
    a = stencil_3d_27pt(128, 128, 128, seed=1, dtype=dtype)
    return a, uniform_vector(a.cols, 0)


def workload_powerlaw_4m():
    """Zipf(2.1) rows clipped to [1, 100000], n = 4,194,304, FP32 N(0,1) values
    (seed 0), x N(0,1) FP32 (seed 1)."""
    a = powerlaw_rows(4_194_304, 2.1, 100_000, seed=0)
    return a, normal_vector(a.cols, 1)


def batched_banded_specs(count: int = 256, seed: int = 7):
    """Sizes of the batched workload: n ~ U{1000..200000}, bandwidth ~
    U{64..2048}, k (right-hand sides) uniform in {1, 4, 8, 32}, matrix seed."""
    rng = np.random.default_rng(seed)
    n = rng.integers(1000, 200_001, size=count)
    w = rng.integers(64, 2049, size=count)
    k = rng.choice(np.array([1, 4, 8, 32]), size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [dict(n=int(n[i]), width=int(w[i]), k=int(k[i]), seed=int(seeds[i])) for i in range(count)]


def batched_banded(spec) -> tuple:
    a = banded_random(spec["n"], spec["width"], 10, 60, seed=spec["seed"])
    X = np.random.default_rng(spec["seed"] + 1).standard_normal((a.cols, spec["k"])).astype(np.float32)
    return a, X


def selector_family_specs(count: int = 2000, seed: int = 11, max_nnz: int | None = None):
    """The selector corpus: families {stencil2d, stencil3d, banded, blockdiag,
    powerlaw, uniform}; n log-uniform in [1e4, 2e6]; target nnz/row
    log-uniform in [2, 200] where the family lets it vary (up to 4e8 entries);
    with max_nnz set, specs whose expected nnz exceeds it shrink n to fit."""
    rng = np.random.default_rng(seed)
    fams = ["stencil2d", "stencil3d", "banded", "blockdiag", "powerlaw", "uniform"]
    specs = []
    for i in range(count):
        fam = fams[int(rng.integers(0, len(fams)))]
        n = int(round(math.exp(rng.uniform(math.log(1e4), math.log(2e6)))))
        mu = float(math.exp(rng.uniform(math.log(2.0), math.log(200.0))))
        s = dict(family=fam, n=n, mu=mu, seed=int(rng.integers(0, 2**31 - 1)))
        if fam == "stencil2d":
            s["points"] = int(rng.choice([5, 9]))
            s["mu"] = float(s["points"])
        elif fam == "stencil3d":
            s["points"] = int(rng.choice([7, 27]))
            s["mu"] = float(s["points"])
        elif fam == "blockdiag":
            s["block"] = int(rng.integers(4, 33))
            s["mu"] = float(s["block"])
        elif fam == "banded":
            s["width"] = int(rng.integers(max(64, int(2 * mu) + 2), 2049))
            s["mu"] = min(mu, 60.0 * 3)
        elif fam == "powerlaw":
            s["alpha"] = float(rng.uniform(1.8, 2.6))
        if max_nnz is not None and s["n"] * s["mu"] > max_nnz:
            s["n"] = max(10_000, int(max_nnz / s["mu"]))
        specs.append(s)
    return specs


def selector_matrix(spec) -> CSR:
    fam, n, seed = spec["family"], spec["n"], spec["seed"]
    if fam == "stencil2d":
        nx = max(3, int(round(math.sqrt(n))))
        return (laplacian_2d_5pt(nx, nx) if spec["points"] == 5 else stencil_2d_9pt(nx, nx, seed, np.float32))
    if fam == "stencil3d":
        m = max(3, int(round(n ** (1.0 / 3.0))))
        if spec["points"] == 7:
            return stencil_3d_7pt(m, m, m, seed, np.float32)
        return stencil_3d_27pt(m, m, m, seed, np.float32)
    if fam == "banded":
        mu = spec["mu"]
        lo = max(2, int(round(mu * 0.5)))
        hi = max(lo, min(int(round(mu * 1.5)), spec["width"]))
        return banded_random(n, spec["width"], lo, hi, seed)
    if fam == "blockdiag":
        return block_diagonal(n, spec["block"], seed)
    if fam == "powerlaw":
        kmax = int(min(n // 4, 20 * spec["mu"] * 50))
        return powerlaw_rows(n, spec["alpha"], max(kmax, 2), seed)
    return uniform_random(n, spec["mu"], seed)


def selector_matrix_arrays(spec):
    """selector_matrix as plain arrays (rows, cols, row_ptr, col_ind, FP32
    values), for worker processes."""
    a = selector_matrix(spec)
    return a.rows, a.cols, a.row_ptr, a.col_ind, np.ascontiguousarray(a.val, dtype=np.float32)


def permutation_matrix(n: int = 10_000_000, seed: int = 7) -> CSR:
    """The paper's p7 (Section 6.1): an n x n random permutation matrix, one
    entry per row (FP64 ones), x ~ U[-1, 1] is drawn separately."""
    (r,) = _streams(seed, 1)
    col = r.permutation(n).astype(np.int32)
    return _finish(n, n, np.ones(n, np.int64), col, np.ones(n), "p%d" % n)


def dense_as_sparse(n: int = 10_000, seed: int = 8) -> CSR:
    """The paper's dense4 (Section 6.1): an n x n dense matrix stored as a
    sparse one, values U[-1, 1] (FP64)."""
    (r,) = _streams(seed, 1)
    col = np.tile(np.arange(n, dtype=np.int32), n)
    return _finish(n, n, np.full(n, n, np.int64), col, r.uniform(-1.0, 1.0, n * n), "dense%d" % n)


def workload_irregular(n: int = 2_097_152, seed: int = 3):
    """Moderately irregular rows for row reordering: banded random, window
    2048, lengths U{4..60} (mean 32), values N(0, 1) as FP64, x ~ U[-1, 1]
    (seed 0)."""
    a = banded_random(n, 2048, 4, 60, seed)
    a = CSR(a.rows, a.cols, a.row_ptr, a.col_ind, a.val.astype(np.float64), "irregular_n%d" % n)
    return a, uniform_vector(a.cols, 0)
