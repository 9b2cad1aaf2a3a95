"""Schedule autotuner of the batched multi-right-hand-side SpMM.

The batch runs as one persistent launch over work units (matrix, row range)
of about `work_target` entry-columns each.  Its schedule has two parts, both
chosen here by timing the library's own kernels:

1. the strip height of each matrix: every matrix is converted to CMRS at each
   candidate height (cmrs_from_csr) and its product with its k right-hand
   sides (cmrs_spmm, one launch) timed with CUDA events, the L2 flushed
   before each call; the fastest height is kept;
2. the work-unit size of the whole batch (cmrs_spmm_autotune, graph replays
   of each candidate plan).

Every numeric step runs in libcmrs; this module only orchestrates.
"""
from __future__ import annotations

import statistics

import torch

from . import binding as b

HEIGHTS = (1, 2, 4, 8, 16, 32)
WORK_TARGETS = (2048, 8192, 32768, 131072)


class _Flush:
    """256 MiB written, then 256 MiB read: nothing of the timed call's
    operands stays in the L2, and no dirty line is left for it to write back."""

    def __init__(self, device):
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device=device)
        self.r = torch.ones(32 << 20, dtype=torch.int64, device=device)
        self.acc = torch.zeros(1, dtype=torch.int64, device=device)
        self.n = 0

    def __call__(self):
        self.n += 1
        self.w.fill_(self.n & 0xFF)
        torch.sum(self.r, dim=0, keepdim=True, out=self.acc)


def _time(fn, flush, reps):
    fn()
    st = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    torch.cuda._sleep(2_000_000)  # the calls start on a busy GPU
    for i in range(reps):
        flush()
        st[i].record()
        fn()
        en[i].record()
    torch.cuda.synchronize()
    return statistics.median(s.elapsed_time(e) for s, e in zip(st, en))


def tune_heights(csrs, Xs, Ys, heights=HEIGHTS, reps=3):
    """csrs: list of (row_ptr, col_ind, val) device tensors (int32, int32,
    float32) with Xs[i] [cols][k] and Ys[i] [rows][k].  Returns the CMRS
    matrices at their fastest heights, the heights, and the table of ms per
    matrix and height."""
    flush = _Flush(Xs[0].device)
    mats, chosen, table = [], [], []
    for (rp, ci, va), X, Y in zip(csrs, Xs, Ys):
        best, row = None, []
        for h in heights:
            M = b.cmrs_from_csr(rp, ci, va, X.shape[0], h, dtype=b.CMRS_F32)
            ms = _time(lambda: b.cmrs_spmm(M, X, Y), flush, reps)
            row.append(ms)
            if best is None or ms < best[0]:
                best = (ms, h, M)
            del M
        mats.append(best[2])
        chosen.append(best[1])
        table.append(row)
    return mats, chosen, table


def tune(csrs, Xs, Ys, heights=HEIGHTS, work_targets=WORK_TARGETS, reps=3):
    """The whole schedule: heights per matrix, then the work-unit size.
    Returns (mats, heights, work_target, ms_per_batch_at_tuning, table)."""
    mats, chosen, table = tune_heights(csrs, Xs, Ys, heights, reps)
    best, ms = b.cmrs_spmm_autotune(mats, Xs, Ys, candidates=work_targets, reps=reps)
    return mats, chosen, best, ms, table
