"""Device-side generators of the selector's timing corpus.

The corpus spans matrices of up to 2M rows and 200 entries per row (up to
400M entries), too large to build on the host and copy in.  These generators
follow the family recipes of inputs.selector_family_specs / selector_matrix
(the same spec fields) but draw on the GPU: row lengths with numpy on the host
(at most 2M numbers), columns and values with a seeded torch generator on the
device.  Nothing here computes any part of the CMRS method: no strips, no
packing, no products.

Columns of the random families are drawn one per stratum: a row of L entries
spread over a column range of width W takes one uniform column in each of
[floor(j W / L), floor((j + 1) W / L)), j < L, which keeps them distinct and
increasing without a sort (the banded family of inputs.py draws the same way;
its uniform and power-law families draw uniform subsets on the host instead).
Values are N(0, 1) FP32: timing does not depend on them.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    return g


def _csr(rows, cols, lengths, col, g, device):
    """Row pointer from lengths (int64 device), int32 arrays, N(0,1) values."""
    rp = torch.zeros(rows + 1, dtype=torch.int64, device=device)
    torch.cumsum(lengths, 0, out=rp[1:])
    nnz = int(rp[-1].item())
    if nnz >= 2**31:
        raise ValueError("matrix of %d entries does not fit int32 indices" % nnz)
    val = torch.randn(nnz, generator=g, device=device, dtype=torch.float32)
    return rows, cols, rp.to(torch.int32), col.to(torch.int32), val


def _stratified(lengths, lo, width, g, device):
    """One uniform column per stratum of [lo_i, lo_i + width_i) for row i of
    lengths[i] entries (all device int64)."""
    rows = lengths.numel()
    row_of = torch.repeat_interleave(torch.arange(rows, device=device), lengths)
    start = torch.cumsum(lengths, 0) - lengths
    j = torch.arange(row_of.numel(), device=device, dtype=torch.int64) - start[row_of]
    L = lengths[row_of]
    w = width[row_of]
    b0 = (j * w) // L
    b1 = ((j + 1) * w) // L
    u = torch.rand(row_of.numel(), generator=g, device=device, dtype=torch.float64)
    off = torch.minimum((u * (b1 - b0)).to(torch.int64), b1 - b0 - 1)
    return lo[row_of] + b0 + off


def _stencil(dims, offsets, g, device):
    """Natural order (last dimension fastest), Dirichlet truncation."""
    n = int(np.prod(dims))
    idx = torch.arange(n, device=device, dtype=torch.int64)
    coords, rem = [], idx
    strides = [int(np.prod(dims[i + 1:])) for i in range(len(dims))]
    for s in strides:
        coords.append(rem // s)
        rem = rem % s
    valid = []
    for off in offsets:
        ok = torch.ones(n, dtype=torch.bool, device=device)
        for d, o in enumerate(off):
            if o:
                c = coords[d] + o
                ok &= (c >= 0) & (c < dims[d])
        valid.append(ok)
    valid = torch.stack(valid)  # [noff, n]
    lengths = valid.sum(0).to(torch.int64)
    # entries row by row, offsets in increasing column order
    dcol = torch.tensor([sum(o * s for o, s in zip(off, strides)) for off in offsets], device=device)
    cols = idx[None, :] + dcol[:, None]  # [noff, n]
    col = cols.t()[valid.t()]
    return _csr(n, n, lengths, col, g, device)


def device_matrix(spec, device="cuda"):
    """(rows, cols, row_ptr, col_ind, val) on `device` for one corpus spec."""
    fam, n, seed = spec["family"], int(spec["n"]), int(spec["seed"])
    g = _gen(seed, device)
    host = np.random.default_rng(seed)
    if fam == "stencil2d":
        nx = max(3, int(round(math.sqrt(n))))
        offs = ([(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)] if spec["points"] == 5 else
                [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
        return _stencil((nx, nx), offs, g, device)
    if fam == "stencil3d":
        m = max(3, int(round(n ** (1.0 / 3.0))))
        offs = ([(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
                if spec["points"] == 7 else
                [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
        return _stencil((m, m, m), offs, g, device)
    if fam == "blockdiag":
        blk = int(spec["block"])
        i = torch.arange(n, device=device, dtype=torch.int64)
        b0 = (i // blk) * blk
        lengths = torch.minimum(b0 + blk, torch.full_like(b0, n)) - b0
        return _csr(n, n, lengths, _stratified(lengths, b0, lengths, g, device), g, device)
    if fam == "banded":
        mu, w = spec["mu"], min(int(spec["width"]), n)
        lo = max(2, int(round(mu * 0.5)))
        hi = max(lo, min(int(round(mu * 1.5)), w))
        lengths = torch.from_numpy(host.integers(min(lo, hi), hi + 1, size=n).astype(np.int64)).to(device)
        i = torch.arange(n, device=device, dtype=torch.int64)
        start = torch.clamp(i - w // 2, 0, n - w)
        return _csr(n, n, lengths, _stratified(lengths, start, torch.full_like(i, w), g, device), g, device)
    if fam == "powerlaw":
        kmax = max(2, int(min(n // 4, 20 * spec["mu"] * 50)))
        lens = np.minimum(host.zipf(spec["alpha"], n), kmax).astype(np.int64)
    else:  # uniform
        lens = np.clip(host.poisson(spec["mu"], n), 1, n).astype(np.int64)
    lengths = torch.from_numpy(lens).to(device)
    zeros = torch.zeros(n, dtype=torch.int64, device=device)
    return _csr(n, n, lengths, _stratified(lengths, zeros, torch.full_like(zeros, n), g, device), g, device)
