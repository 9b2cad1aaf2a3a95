"""One product split over several GPUs by strips.

Strips are independent (Section 4: a strip's warp reads only its own entries
and writes only its own rows of y), so each rank owns a contiguous range of
whole strips (cmrs_shard_rows: balanced by entries plus rows), converts its
rows of the CRS matrix to CMRS on its own device, and multiplies them with
cmrs_spmv.  The only exchange is x: rank p owns x[bounds[p]:bounds[p+1]] (a
square matrix: x is split like the rows of y), and before each product every
rank receives the other ranks' pieces into its full copy of x, one broadcast
per rank on the process group (NCCL between GPUs, gloo on CPUs).  y needs no
reduction: each rank's rows are its own.  Every load of the product reads the
local device's memory; no remote memory is a kernel operand.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as b


def local_rows(row_ptr, col_ind, val, r0, r1):
    """Rows [r0, r1) of a host CRS matrix as a CRS matrix of their own (the
    row pointer rebased to 0; columns unchanged)."""
    k0, k1 = int(row_ptr[r0]), int(row_ptr[r1])
    rp = (np.asarray(row_ptr[r0:r1 + 1], dtype=np.int64) - k0).astype(np.int32)
    return rp, np.ascontiguousarray(col_ind[k0:k1]), np.ascontiguousarray(val[k0:k1])


def exchange_x(x_full, bounds, group=None):
    """Every rank sends its piece x_full[bounds[p]:bounds[p+1]] to all others:
    one broadcast per non-empty piece, in rank order."""
    import torch.distributed as dist
    for p in range(len(bounds) - 1):
        a, c = int(bounds[p]), int(bounds[p + 1])
        if c > a:
            dist.broadcast(x_full[a:c], src=p, group=group)


class ShardedSpmv:
    """This rank's share of y = A x for a square host CRS matrix `a`
    (inputs.CSR): its strips in CMRS (padded with `slots` if given) on
    `device`, a full copy of x and its rows of y."""

    def __init__(self, a, rank, world, height, dtype=b.CMRS_F64, slots=None, device="cuda", group=None):
        if a.rows != a.cols:
            raise ValueError("strip sharding splits x like y: the matrix must be square")
        self.rank, self.world, self.group = rank, world, group
        self.bounds = b.cmrs_shard_rows(a.row_ptr, height, world)
        self.r0, self.r1 = int(self.bounds[rank]), int(self.bounds[rank + 1])
        rp, ci, va = local_rows(a.row_ptr, a.col_ind, a.val, self.r0, self.r1)
        self.rows = self.r1 - self.r0
        self.nnz = int(ci.size)
        xt = torch.float64 if dtype == b.CMRS_F64 else torch.float32
        self.x_full = torch.zeros(a.cols, dtype=xt, device=device)
        self.y = torch.empty(self.rows, dtype=xt, device=device)
        self.M = None
        if self.rows > 0:
            M = b.cmrs_from_csr(torch.from_numpy(rp).to(device), torch.from_numpy(ci).to(device),
                                torch.from_numpy(va).to(device), a.cols, height, dtype=dtype)
            self.variant = b.CMRS_VARIANT_AUTO
            if slots:
                M, self.variant = b.cmrs_pad(M, slots), b.CMRS_VARIANT_PADDED
            self.M = M
            self.ws = M.spmv_workspace(self.variant)

    def x_local(self):
        """This rank's piece of x (a view of the full copy): write it before step()."""
        return self.x_full[self.r0:self.r1]

    def product(self):
        """y (this rank's rows) = A x_full on the local device."""
        if self.M is not None:
            b.cmrs_spmv(self.M, self.x_full, self.y, self.variant, self.ws)
        return self.y

    def step(self):
        """Exchange of x, then the local product."""
        if self.world > 1:
            exchange_x(self.x_full, self.bounds, self.group)
        return self.product()
