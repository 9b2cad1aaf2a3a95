#!/usr/bin/env python3
"""CMRS SpMV benchmark on GB300.

Workload (default): 27-point stencil on a 128^3 grid, non-periodic
(n = 2,097,152 rows, nnz = 55,742,968), FP64 values, x ~ U[-1, 1], stored as
the modified CMRS of Section 6.6 (strip height 32, one slot per row per
pass), SpMV kernel PADDED.  One step = one y = A x through cmrs_spmv.  Inputs
are resident in HBM before the timed region; the L2 is flushed between steps
(256 MiB write, then a 256 MiB read so that the write's dirty lines are not
written back inside the step) and every step is timed by its own pair of CUDA
events on the launching stream.

Metric: GB/s = beta_plus / t with beta_plus = (s_v + s_i) nnz + s_i strips +
2 s_v rows (Eq. 6.1: matrix, x and y moved once), also GFLOP/s = 2 nnz / t and
the paper's (2 nnz - rows) / t.  e2e: the same metric through the C ABI with x
copied from pinned host memory and y copied back inside the timed region,
every step, neighbouring steps' copies overlapping the product on two
buffer pairs.

  python bench.py [--steps K] [--warmup W] [--height H] [--variant row|strip|merge|padded|auto] [--slots M]
  python bench.py --impl reference      # the CPU oracle on the same workload
  torchrun --nproc-per-node N bench.py --gpus N   # the headline split over N GPUs by strips
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "SpMV GB/s (% of GB300 HBM peak) and GFLOP/s; speedup vs plain FP64 CMRS"
FALLBACK_HBM_GBS = 6800.0


def args_parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--height", type=int, default=None,
                   help="strip height (default: 32 for the 27-point headline, power-law and p7; else 4)")
    p.add_argument("--slots", type=int, default=None, help="padded variant: slots per row per warp pass (M of "
                   "Section 6.6; 1, 2, 4 or 8; default 1, irregular 2, dense4 4)")
    p.add_argument("--variant", default=None, choices=["row", "strip", "merge", "auto", "padded"],
                   help="SpMV kernel variant (default: padded for the 27-point headline, p7 and dense4; "
                        "power-law merge; else row)")
    p.add_argument("--workload", default="stencil27",
                   choices=["stencil27", "powerlaw", "batched", "laplacian", "p7", "dense4", "irregular"],
                   help="stencil27 is the headline; the others print the same JSON schema for their workload")
    p.add_argument("--batch-count", type=int, default=256, help="batched workload: matrices (256 = full size)")
    p.add_argument("--window", type=int, default=0, help="irregular workload: row-reordering window (0: none)")
    p.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16", "bf16x2"],
                   help="stencil27: stored value form of the measured line (x and y FP32 unless f64)")
    p.add_argument("--grid", type=int, default=128, help="stencil27: grid edge (128 = the full workload)")
    p.add_argument("--no-extras", action="store_true", help="skip the secondary storage-form measurements")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--shard", action="store_true",
                   help="run the strip-sharded path even on one GPU (it is the default for N > 1)")
    return p.parse_args()


def beta_plus(nnz, rows, strips, s_v, s_i=4):
    return (s_v + s_i) * nnz + s_i * strips + 2 * s_v * rows


def beta_minus(nnz, rows, strips, s_v, s_i=4):
    """Eq. 6.1, input vector not cached: one x read per nonzero."""
    return (2 * s_v + s_i) * nnz + s_i * strips + s_v * rows


def eta(nnz, rows, strips, s_v, ms, peak):
    """beta_-/t, and eta_+- = beta_+-/t / B (B = the measured copy bandwidth)."""
    t = ms / 1e3
    bm = beta_minus(nnz, rows, strips, s_v) / t / 1e9
    return {"beta_minus_gbs": bm, "eta_plus": beta_plus(nnz, rows, strips, s_v) / t / 1e9 / peak,
            "eta_minus": bm / peak}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# --------------------------------------------------------------------------- clocks (NVML, read only)
class ClockSampler:
    """Polls SM clock and clock-event reasons through NVML while the timed
    region runs (read-only queries)."""

    REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
               0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
               0x100: "display_clock_setting"}

    def __init__(self, pci_bus_id: str | None):
        self.samples, self.reasons, self.ok = [], 0, False
        self.max_mhz = None
        try:
            self.nv = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nv.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            rc = 1
            if pci_bus_id:
                rc = self.nv.nvmlDeviceGetHandleByPciBusId_v2(pci_bus_id.encode(), ctypes.byref(self.h))
            if rc != 0:
                rc = self.nv.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(self.h))
            if rc != 0:
                return
            m = ctypes.c_uint()
            if self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(m)) == 0:
                self.max_mhz = m.value
            self.ok = True
        except OSError:
            pass

    def _poll(self):
        c, r = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(c)) == 0:
                self.samples.append(c.value)
            if self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.h, ctypes.byref(r)) == 0:
                self.reasons |= r.value & ~0x1
            time.sleep(0.002)

    def __enter__(self):
        self._stop = threading.Event()
        if self.ok:
            self._t = threading.Thread(target=self._poll, daemon=True)
            self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self.ok:
            self._t.join()

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0, "source": "nvml"}
        return {"sm_mhz": float(statistics.median(self.samples)), "sm_max_mhz": self.max_mhz,
                "reasons": [n for bit, n in self.REASONS.items() if self.reasons & bit],
                "samples": len(self.samples), "source": "nvml"}


# --------------------------------------------------------------------------- distributed helpers
def dist_setup(n_gpus):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- CPU oracle legs
def cpu_oracle_rate(a, x, strips, budget_s=12.0, max_reps=200):
    """Times the oracle's plain FP64 CRS SpMV on the host, single thread."""
    import oracle
    rows = a.rows
    bp = beta_plus(a.nnz, rows, strips, 8)
    t0 = time.perf_counter()
    oracle.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    one = time.perf_counter() - t0
    reps = max(1, min(max_reps, int(budget_s / max(one, 1e-6))))
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
        ts.append(time.perf_counter() - t0)
    t = statistics.mean(ts)
    return {"value": bp / t / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "full matrix, %d timed repetitions after 1 warm-up (%.1f s of CPU work)" % (reps, sum(ts)),
            "ms_per_spmv": t * 1e3, "gflops": 2 * a.nnz / t / 1e9}


def cpu_oracle_rate_all_cores(a, x, strips, runs=11):
    """The same oracle on every core this process may use: the rows split into
    one contiguous slice per core, each slice's plain C loop called from its own
    Python thread (the call releases the interpreter lock), so every row's sum
    is the single-thread oracle's.  11 runs, the slowest dropped, the mean of
    the other 10.  A reported baseline only."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    cores = max(1, len(os.sched_getaffinity(0)))
    lib = oracle.lib()
    rp = np.ascontiguousarray(a.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(a.col_ind, dtype=np.int32)
    va = np.ascontiguousarray(a.val, dtype=np.float64)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(a.rows)
    cuts = [a.rows * i // cores for i in range(cores + 1)]
    parts = [(cuts[i], cuts[i + 1]) for i in range(cores) if cuts[i + 1] > cuts[i]]

    def one(r):
        r0, r1 = r
        lib.orc_csr_spmv(r1 - r0, oracle._p(rp[r0:]), oracle._p(ci), oracle._p(va), oracle._p(xv),
                         oracle._p(y[r0:]), None)

    ts = []
    with ThreadPoolExecutor(len(parts)) as pool:
        list(pool.map(one, parts))  # warm-up
        for _ in range(runs):
            t0 = time.perf_counter()
            list(pool.map(one, parts))
            ts.append(time.perf_counter() - t0)
    ref = oracle.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    same = bool(np.array_equal(y, ref[0] if isinstance(ref, tuple) else ref))
    t = statistics.mean(sorted(ts)[:-1])
    return {"value": beta_plus(a.nnz, a.rows, strips, 8) / t / 1e9, "unit": "GB/s", "cores": len(parts),
            "kind": "oracle, rows split over threads", "sample": "full matrix, %d runs, slowest dropped" % runs,
            "ms_per_spmv": t * 1e3, "same_y_as_single_thread": same}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1203_2946_gb300 import inputs
    if args.workload in ("stencil27", None):
        a, x = inputs.workload_stencil27_128()
        wl = "27-point stencil 128^3 (n=2097152, nnz=55742968), FP64, CRS order"
    elif args.workload == "powerlaw":
        a, x = inputs.workload_powerlaw_4m()
        a = inputs.CSR(a.rows, a.cols, a.row_ptr, a.col_ind, a.val.astype(np.float64))
        x = x.astype(np.float64)
        wl = "power-law rows n=4194304, FP32 values widened to FP64, CRS order"
    elif args.workload == "p7":
        a = inputs.permutation_matrix()
        x = inputs.uniform_vector(a.cols, 0)
        wl = "p7: 10^7 x 10^7 random permutation, FP64, CRS order"
    elif args.workload == "dense4":
        a = inputs.dense_as_sparse()
        x = inputs.uniform_vector(a.cols, 0)
        wl = "dense4: 10^4 x 10^4 dense matrix stored as sparse, FP64, CRS order"
    elif args.workload == "irregular":
        a, x = inputs.workload_irregular()
        wl = "banded rows of 4..60 entries, n=2097152, FP64, CRS order"
    elif args.workload == "batched":
        # a bounded sample of the batch: the first 8 matrices, one CRS product per right-hand side
        specs = inputs.batched_banded_specs()[:8]
        mats = []
        for sp in specs:  # FP64 copies, X by column, made before any timing
            a, X = inputs.batched_banded(sp)
            mats.append((a, np.ascontiguousarray(a.val, dtype=np.float64), np.ascontiguousarray(X.T, dtype=np.float64)))
        lib = oracle.lib()
        ts, bytes_ = [], []
        t_end = time.perf_counter() + 60.0
        for i in range(args.steps + args.warmup):
            a, vd, XT = mats[i % len(mats)]
            k = XT.shape[0]
            y = np.empty(a.rows)
            t0 = time.perf_counter()
            for c in range(k):
                lib.orc_csr_spmv(a.rows, oracle._p(a.row_ptr), oracle._p(a.col_ind), oracle._p(vd), oracle._p(XT[c]),
                                 oracle._p(y), None)
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                ts.append(dt)
                S = (a.rows + args.height - 1) // args.height
                bytes_.append((4 + 4) * a.nnz + 4 * S + 4 * k * (a.rows + a.cols))  # the GPU line's beta+, FP32
            if time.perf_counter() > t_end and len(ts) >= 1:
                break
        value = sum(bytes_) / sum(ts) / 1e9
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
                "steps": len(ts), "warmup": args.warmup, "ms_per_step": sum(ts) / len(ts) * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": "batched banded-random SpMM, the first %d of the 256 matrices in turn, one "
                                       "CRS product per right-hand side (FP32 values and X widened to FP64)" % len(mats)},
                "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                 "sample": "one matrix with all its right-hand sides per step, %d steps" % len(ts)},
                "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    else:
        a, x = inputs.workload_laplacian_64()
        wl = "5-point Laplacian 64x64, FP64, CRS order"
    h = args.height
    strips = (a.rows + h - 1) // h
    # each step is a bounded row slice of the workload, sized from one full call
    t0 = time.perf_counter()
    oracle.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    t_full = time.perf_counter() - t0
    total = args.steps + args.warmup
    frac = min(1.0, 90.0 / max(total * t_full, 1e-9))
    nrow = max(1024, int(a.rows * frac))
    ts, bytes_ = [], []
    lib = oracle.lib()
    for i in range(total):
        r0 = (i * nrow) % max(1, a.rows - nrow + 1)
        rp = np.ascontiguousarray(a.row_ptr[r0:r0 + nrow + 1])
        y = np.empty(nrow)
        t0 = time.perf_counter()
        lib.orc_csr_spmv(nrow, oracle._p(rp), oracle._p(a.col_ind), oracle._p(a.val), oracle._p(x), oracle._p(y), None)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            ts.append(dt)
            nz = int(rp[-1] - rp[0])
            bytes_.append(beta_plus(nz, nrow, (nrow + h - 1) // h, 8))
    t = sum(ts)
    value = sum(bytes_) / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / len(ts) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl + "; each step a slice of %d rows" % nrow},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "%d consecutive rows per step (%.3f of the matrix), %d steps" % (
                                 nrow, nrow / a.rows, len(ts))},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU leg
def kernel_section_sha1(begin, end, source="spmv.cu"):
    """sha1 of the source text of one kernel section of a csrc file (from the
    line holding `begin` up to the line holding `end`)."""
    src = open(os.path.join(ROOT, "paper_1203_2946_gb300", "csrc", source)).read()
    a = src.index(begin)
    b = src.index(end, a + len(begin))
    return hashlib.sha1(src[a:b].encode()).hexdigest()


def traffic_record(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, valid only while
    the kernel's source section is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)[kernel][workload]
        h = kernel_section_sha1(*rec["section"], source=rec.get("source_file", "spmv.cu"))
        return rec["bytes_per_launch"] if rec.get("section_sha1") == h else None
    except Exception:
        return None


def e2e_pipelined_sets(run, copy_in, copy_out, steps, warm=3):
    """End-to-end rate through host buffers over two device buffer sets:
    every step copies its inputs from pinned host memory (copy_in(s), on an
    H2D stream), runs the product (run(s), on the launching stream) and copies
    its results back to pinned host memory (copy_out(s), on a D2H stream), s
    alternating between the sets, so one step's copy-in and the previous
    step's copy-out overlap a product; event waits keep each set's reuse in
    order.  Returns ms per step from CUDA events spanning the first copy-in to
    the last copy-out.  No L2 flush: the resident operands are larger than L2."""
    import torch
    comp = torch.cuda.current_stream()
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    k_done = [torch.cuda.Event() for _ in range(2)]
    in_done = [torch.cuda.Event() for _ in range(2)]
    out_done = [torch.cuda.Event() for _ in range(2)]
    count = [0]

    def one():
        i = count[0]
        count[0] += 1
        s = i & 1
        if i >= 2:
            h2d.wait_event(k_done[s])      # the product two steps back has read set s
        with torch.cuda.stream(h2d):
            copy_in(s)
        in_done[s].record(h2d)
        comp.wait_event(in_done[s])
        if i >= 2:
            comp.wait_event(out_done[s])   # set s's results were copied out two steps back
        run(s)
        k_done[s].record(comp)
        d2h.wait_event(k_done[s])
        with torch.cuda.stream(d2h):
            copy_out(s)
        out_done[s].record(d2h)

    for _ in range(warm):
        one()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(h2d)
    for _ in range(steps):
        one()
    comp.wait_event(out_done[(count[0] - 1) & 1])
    comp.wait_event(out_done[count[0] & 1])
    end.record(comp)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / steps


def e2e_pipelined(run, xh, xds, yds, yhs, steps, warm=3):
    """e2e_pipelined_sets for one input vector x and one result vector y."""
    return e2e_pipelined_sets(lambda s: run(xds[s], yds[s]), lambda s: xds[s].copy_(xh, non_blocking=True),
                              lambda s: yhs[s].copy_(yds[s], non_blocking=True), steps, warm)


L2_NOTE = ("flushed between steps (256 MiB write, then a 256 MiB read so that the dirty lines the write leaves "
           "are written back before the step, not inside it), each step timed by its own CUDA events")


class L2Flush:
    """Between timed steps: write a 256 MiB buffer, which evicts every line of
    the step's operands from the L2 (about 126 MB), then read a second 256 MiB
    buffer.  A write alone leaves the L2 full of dirty lines that the next
    kernel pays to write back to HBM (about 5 us for the FP64 headline, 8 us
    for split BF16); after the read the L2 holds only clean lines of neither
    the matrix nor x nor y."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        self.r = torch.ones(32 << 20, dtype=torch.int64, device=dev)
        self.acc = torch.zeros(1, dtype=torch.int64, device=dev)

    def __call__(self, i):
        import torch
        self.w.fill_(i & 0xFF)
        torch.sum(self.r, dim=0, keepdim=True, out=self.acc)


def time_steps(fn, steps, flush, stream, warm_steps=3, warm_s=0.05):
    """Times `steps` steps, each {flush, fn} with fn bracketed by CUDA events
    on `stream`.  Before them, at least `warm_steps` untimed steps of the same
    {flush, fn} pattern, for at least `warm_s` seconds: the first product
    after the GPU has idled (a matrix built on the host, a synchronising read)
    measured up to twice its steady time (228.6 vs 112.6 us for the 27-point
    headline).  The warm-up is left running on the GPU and a short spin
    kernel follows it, so the timed steps start on a busy GPU and the host
    enqueues them ahead of it."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    t0 = time.perf_counter()
    i = 0
    while i < warm_steps or time.perf_counter() - t0 < warm_s:
        flush(i)
        fn()
        i += 1
        if i % 32 == 0:
            torch.cuda.synchronize()  # keeps the launch queue short
    with torch.cuda.stream(stream):
        torch.cuda._sleep(int(min(steps, 256) * 30e-6 * 2.0e9))  # ~30 us of GPU time per step to enqueue
    for i in range(steps):
        flush(i)
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def run_sharded(args, rank, world, dist):
    """N > 1: the headline matrix split over the ranks by strips (one
    contiguous range of whole strips per GPU, balanced by entries plus rows);
    a step is the exchange of x (one NCCL broadcast per rank's piece) and the
    rank's local product.  Total work is fixed: strong scaling."""
    import torch
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding as b, inputs, shard
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    g = args.grid
    if g == 128:
        a, x = inputs.workload_stencil27_128()
    else:
        a = inputs.stencil_3d_27pt(g, g, g, seed=1)
        x = inputs.uniform_vector(a.cols, 0)
    h = args.height
    slots = args.slots if args.variant == "padded" else None
    S = shard.ShardedSpmv(a, rank, world, h, dtype=b.CMRS_F64, slots=slots, device=dev)
    S.x_local().copy_(torch.from_numpy(x[S.r0:S.r1]))
    flush = L2Flush(dev)
    peak, peak_kind = measured_peaks()
    bp = beta_plus(a.nnz, a.rows, (a.rows + h - 1) // h, 8)
    for _ in range(max(3, args.warmup)):
        S.step()
    pci = getattr(torch.cuda.get_device_properties(dev), "pci_bus_id", None)
    sampler = ClockSampler(pci)
    barrier(dist)
    torch.cuda.synchronize()
    # every rank must run the same number of steps (each holds collectives):
    # a warm-up counted in steps, not in seconds
    warm = max(16, args.warmup)
    with sampler:
        times = time_steps(S.step, args.steps, flush, stream, warm_steps=warm, warm_s=0.0)
    barrier(dist)
    total_ms = max_over_ranks(dist, sum(times))
    per_ms = total_ms / args.steps
    local_ms = max_over_ranks(dist, statistics.mean(time_steps(S.product, 20, flush, stream, warm_steps=warm,
                                                               warm_s=0.0)))
    # e2e: this rank's piece of x in from pinned host memory, exchange, product, its rows of y out
    xh = torch.from_numpy(np.ascontiguousarray(x[S.r0:S.r1])).pin_memory()
    yh = torch.empty(S.rows, dtype=torch.float64).pin_memory()

    def e2e_step():
        S.x_local().copy_(xh, non_blocking=True)
        S.step()
        yh.copy_(S.y, non_blocking=True)
    e_ms = max_over_ranks(dist, statistics.mean(time_steps(e2e_step, 20, lambda i: None, stream, warm_steps=warm,
                                                           warm_s=0.0)))
    # this rank's rows against the FP64 oracle (its rows of A times the whole x)
    import oracle
    S.step()
    from paper_1203_2946_gb300.shard import local_rows
    lrp, lci, lva = local_rows(a.row_ptr, a.col_ind, a.val, S.r0, S.r1)
    err = 0.0
    if S.rows > 0:
        yref, scale = oracle.csr_spmv(lrp, lci, lva, x)
        err = float(np.max(np.abs(S.y.cpu().numpy() - yref) / np.where(scale > 0, scale, 1)))
    err = max_over_ranks(dist, err)
    gbs = bp / (per_ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "27-point stencil %d^3 (n=%d, nnz=%d), FP64, %s, split over %d GPUs by strips"
                                   % (g, a.rows, a.nnz, ("modified CMRS h=%d, M=%d" % (h, slots)) if slots else
                                      "CMRS h=%d" % h, world),
                       "height": h, "slots": slots, "bytes_per_step": bp, "row_bounds": [int(v) for v in S.bounds],
                       "l2": L2_NOTE, "parallelism": "strip shards x%d, x exchanged by NCCL broadcasts" % world},
            "roofline": {"bound": "hbm", "achieved": gbs / world, "peak": peak, "unit": "GB/s",
                         "frac": gbs / world / peak, "peak_kind": peak_kind + " (hbm_gbs), per GPU",
                         "traffic": None, "kernel": "k_spmv_padded" if slots else row_kernel(S.M)},
            "local_product_ms_max_over_ranks": local_ms,
            "err_vs_f64_oracle_max_over_ranks": err,
            "e2e": {"value": bp / (e_ms / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": e_ms,
                    "h2d_bytes_per_step": int(xh.numel() * 8), "d2h_bytes_per_step": int(yh.numel() * 8),
                    "note": "per rank: its piece of x in, exchange, product, its rows of y out (max over ranks)"},
            "gpu_launches": args.steps, "clocks": sampler.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_ours(args):
    import numpy as np
    import torch
    rank, world, dist = dist_setup(args.gpus)
    if world > 1 or args.shard:
        return run_sharded(args, rank, world, dist)
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding as b, inputs
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    variant = binding_variant = dict(b.VARIANTS, auto=b.CMRS_VARIANT_AUTO,
                                     padded=b.CMRS_VARIANT_PADDED)[args.variant]
    g = args.grid
    if g == 128:
        a, x = inputs.workload_stencil27_128()
    else:
        a = inputs.stencil_3d_27pt(g, g, g, seed=1)
        x = inputs.uniform_vector(a.cols, 0)
    dt = {"f64": b.CMRS_F64, "f32": b.CMRS_F32, "bf16": b.CMRS_BF16, "bf16x2": b.CMRS_BF16X2}[args.dtype]
    s_v = {b.CMRS_F64: 8, b.CMRS_F32: 4, b.CMRS_BF16: 2, b.CMRS_BF16X2: 4}[dt]  # stored value bytes
    s_x = 8 if dt == b.CMRS_F64 else 4                                          # x and y element bytes
    h = args.height
    strips = (a.rows + h - 1) // h
    rp = torch.from_numpy(a.row_ptr).to(dev)
    ci = torch.from_numpy(a.col_ind).to(dev)
    va = torch.from_numpy(a.val).to(dev)
    M = b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=dt)
    M_csr = M
    if args.variant == "padded":
        M = b.cmrs_pad(M, args.slots)  # Section 6.6 arrangement; bytes_per_step stays the unpadded beta+
    variant = b.cmrs_spmv_variant(M, binding_variant)
    xv = x if dt == b.CMRS_F64 else x.astype(np.float32)
    xd = torch.from_numpy(xv).to(dev)
    yd = torch.empty(a.rows, dtype=torch.float64 if dt == b.CMRS_F64 else torch.float32, device=dev)
    ws = M.spmv_workspace(variant)
    flush = L2Flush(dev)

    def step():
        b.cmrs_spmv(M, xd, yd, binding_variant, ws)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    bp = (s_v + 4) * a.nnz + 4 * strips + 2 * s_x * a.rows  # beta+ (Eq. 6.1), x and y in their own width
    peak, peak_kind = measured_peaks()
    pci = None
    try:
        pci = torch.cuda.get_device_properties(dev).pci_bus_id if hasattr(torch.cuda.get_device_properties(dev), "pci_bus_id") else None
    except Exception:
        pci = None
    sampler = ClockSampler(pci)
    barrier(dist)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with sampler:
        times = time_steps(step, args.steps, flush, stream, warm_steps=max(3, args.warmup), warm_s=0.25)
    barrier(dist)
    wall = time.perf_counter() - wall0
    total_ms = max_over_ranks(dist, sum(times))
    per_ms = total_ms / args.steps
    value = world * bp * args.steps / (total_ms / 1e3) / 1e9
    b.cmrs_spmv_check(M, variant)

    # e2e through the C ABI with host buffers (x in, y out every step, pipelined)
    xh = torch.from_numpy(xv).pin_memory()
    yhs = [torch.empty(a.rows, dtype=yd.dtype).pin_memory() for _ in range(2)]
    xds = [xd, torch.empty_like(xd)]
    yds = [yd, torch.empty_like(yd)]
    e2e_steps = max(20, min(args.steps, 200))
    e2e_ms = max_over_ranks(dist, e2e_pipelined(lambda xv, yv: b.cmrs_spmv(M, xv, yv, binding_variant, ws), xh, xds,
                                                yds, yhs, e2e_steps))

    kname = {0: row_kernel(M), 1: "k_spmv_strip", 2: "k_spmv_merge", 3: "k_spmv_padded"}[variant]
    split = variant == 3 and ws.numel() > 256  # a padded workspace past the status word: strips split over warps
    if split:
        kname = "k_spmv_padded_split"  # + k_pad_combine
    elif variant == 3 and args.slots == 1 and dt != b.CMRS_F64:
        kname = "k_spmv_padded_bulk"  # the library stages the narrow forms' M = 1 walk through shared memory
    form = {"f64": "FP64 values and x", "f32": "FP32 values, x and y", "bf16": "BF16 values, FP32 x and y",
            "bf16x2": "split-BF16 values, FP32 x and y"}[args.dtype]
    trimmed = sorted(times)[:-1] if len(times) > 1 else times
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": "27-point stencil %d^3 (n=%d, nnz=%d), %s, " % (g, a.rows, a.nnz, form)
                               + ("modified CMRS (Section 6.6) h=%d, M=%d slot(s) per row per pass" % (h, args.slots)
                                  if args.variant == "padded" else "CMRS h=%d, variant %s" % (h, args.variant)),
                   "height": h, "variant": args.variant, "bytes_per_step": bp,
                   "slots": args.slots if args.variant == "padded" else None,
                   "stored_items_per_nnz": M.nnz / a.nnz,
                   "l2": L2_NOTE,
                   "parallelism": "single GPU"},
        "gflops": 2 * a.nnz / (per_ms / 1e3) / 1e9,
        "gflops_paper": (2 * a.nnz - a.rows) / (per_ms / 1e3) / 1e9,
        "eta": eta(a.nnz, a.rows, strips, 8, per_ms, peak) if dt == b.CMRS_F64 else None,
        "pct_of_hbm_peak": 100.0 * (value / world) / peak,
        "pct_of_nominal_8tbs": 100.0 * (value / world) / 8000.0,
        "paper_protocol": {"mean_ms": statistics.mean(trimmed), "std_ms": statistics.pstdev(trimmed),
                           "min_ms": min(times)},
        "roofline": {"bound": "hbm", "achieved": bp / (per_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": bp / (per_ms / 1e3) / 1e9 / peak, "peak_kind": peak_kind + " (hbm_gbs)",
                     "traffic": traffic_record(kname, "stencil27_%d_%s_h%d" % (g, args.dtype, h) + (
                         "_m%d" % args.slots if args.variant == "padded" else "")), "kernel": kname},
        "e2e": {"value": world * bp / (e2e_ms / 1e3) / 1e9, "unit": "GB/s",
                "h2d_bytes_per_step": int(xv.nbytes), "d2h_bytes_per_step": int(a.rows * s_x),
                "ms_per_step": e2e_ms, "note": "x host->device, cmrs_spmv, y device->host every step, "
                "pipelined over two buffer pairs (copy-in, product and copy-out of neighbouring steps overlap); "
                "matrix resident"},
        "gpu_launches": args.steps * (3 if variant == 2 else 2 if split else 1),
        "clocks": sampler.summary(),
        "wall_s_timed_region": wall,
    }
    if rank == 0 and not args.no_extras and world == 1 and dt == b.CMRS_F64 and g == 128:
        line["forms"] = storage_forms(b, a, x, rp, ci, va, h, flush, stream, per_ms,
                                      args.slots if args.variant == "padded" else None)
        line["variants_f64"] = variant_sweep(b, a, xd, M_csr, flush, stream, bp)
        line["modified_cmrs"] = modified_cmrs(b, a, xd, rp, ci, va, flush, stream)
        line["heights_f64_row"] = height_sweep(b, a, xd, rp, ci, va, flush, stream)
        plain = line["heights_f64_row"]["h4"]["ms"]
        line["speedup_vs_plain_f64_cmrs"] = {
            "plain": "plain CMRS h=4 (the paper's best single FP64 height on its K20M, Section 6.2), FP64, ROW", "plain_ms": plain,
            "speedup": plain / per_ms,
            "by_form": {k: plain / v["ms"] for k, v in line["forms"].items()}}
        line["strip_sorted_vs_unsorted_f64"] = sorted_strips(b, a, xd, rp, ci, va, flush, stream)
        line["selector"] = selector_cost(b, a, rp, ci)
        line["conversion"] = conversion_times(b, a, rp, ci, va, M_csr, h,
                                              args.slots if args.variant == "padded" else None)
        # the other workloads, each with its own beta+ roofline
        import oracle
        pl = powerlaw_block(b, inputs, oracle, dev, flush, stream, 100, args.warmup)
        pl.pop("_keep")
        line["powerlaw"] = pl
        bt = batched_block(b, inputs, oracle, dev, flush, stream, 20, args.warmup, (1, 2, 4, 8, 16, 32), 256)
        line["batched"] = {"ms": bt["ms"], "gbs": bt["gbs"], "config": bt["config"], "roofline": bt["roofline"],
                           "e2e": bt["e2e"], **bt["extra"]}
        line["selector_sample"] = selector_sample(b, dev)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate(a, x, strips)
        line["cpu_baseline_all_cores"] = cpu_oracle_rate_all_cores(a, x, strips)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def storage_forms(b, a, x, rp, ci, va, h, flush, stream, f64_ms, slots=None, steps=200):
    """FP32 / BF16 / split-BF16 storage of the same matrix, in the headline's
    format (padded with `slots` per row per pass, else plain CMRS with ROW):
    speed, speed-up over the FP64 kernel and error against the FP64 oracle
    (max and median of |y - y*| / (|A||x|)_i)."""
    import oracle
    import torch
    yref, scale = oracle.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    out = {}
    x32 = torch.from_numpy(x.astype(np.float32)).to(va.device)
    strips = (a.rows + h - 1) // h
    for name, dt, sv in (("f32", b.CMRS_F32, 4), ("bf16", b.CMRS_BF16, 2), ("bf16x2", b.CMRS_BF16X2, 4)):
        M = b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=dt)
        v = b.CMRS_VARIANT_ROW
        if slots:
            M, v = b.cmrs_pad(M, slots), b.CMRS_VARIANT_PADDED
        y = torch.empty(a.rows, dtype=torch.float32, device=va.device)
        ws = M.spmv_workspace(v)
        for _ in range(3):
            b.cmrs_spmv(M, x32, y, v, ws)
        ts = time_steps(lambda: b.cmrs_spmv(M, x32, y, v, ws), steps, flush, stream)
        ms = statistics.mean(ts)
        rel = np.abs(y.cpu().numpy().astype(np.float64) - yref) / np.where(scale > 0, scale, 1)
        bp = beta_plus(a.nnz, a.rows, strips, sv if name != "bf16x2" else 4) if name != "bf16" else \
            6 * a.nnz + 4 * strips + 8 * a.rows
        if name == "bf16x2":
            bp = 8 * a.nnz + 4 * strips + 8 * a.rows
        out[name] = {"gbs": bp / (ms / 1e3) / 1e9, "ms": ms, "speedup_vs_f64": f64_ms / ms,
                     "gflops": 2 * a.nnz / (ms / 1e3) / 1e9,
                     "err_vs_f64_oracle": {"max": float(rel.max()), "median": float(np.median(rel))}}
        del M
    return out


def conversion_times(b, a, rp, ci, va, M, h, slots=None, reps=5):
    """CRS -> CMRS (plain and strip-sorted) and CMRS -> CRS on the same matrix:
    median wall time of `reps` calls (each call synchronises once), and GB/s
    over the arrays read and written (24 B per entry + the pointer arrays)."""
    import torch

    def tm(fn):
        ts = []
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts[1:]) * 1e3
    S = (a.rows + h - 1) // h
    moved = 24 * a.nnz + 4 * (a.rows + 1) + 4 * (S + 1)
    out = {}
    for name, flags in (("from_csr_f64", 0), ("from_csr_f64_sorted", b.CMRS_SORTED)):
        ms = tm(lambda: b.cmrs_from_csr(rp, ci, va, a.cols, h, flags=flags, dtype=b.CMRS_F64))
        out[name] = {"ms": ms, "gbs": moved / (ms / 1e3) / 1e9}
    ms = tm(lambda: b.cmrs_to_csr(M))
    out["to_csr_f64"] = {"ms": ms, "gbs": moved / (ms / 1e3) / 1e9}
    if slots:
        # Section 6.6 arrangement of the plain CMRS matrix (layout pass, one read-back, fill pass)
        ms = tm(lambda: b.cmrs_pad(M, slots))
        out["to_padded_f64_m%d" % slots] = {"ms": ms, "gbs": moved / (ms / 1e3) / 1e9}
    out["note"] = "includes the binding's output allocations and one status read-back per call"
    return out


def height_sweep(b, a, xd, rp, ci, va, flush, stream, steps=60):
    import torch
    out = {}
    y = torch.empty(a.rows, dtype=torch.float64, device=xd.device)
    for h in (1, 2, 4, 8, 16, 32):
        M = b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=b.CMRS_F64)
        ws = M.spmv_workspace(0)
        for _ in range(3):
            b.cmrs_spmv(M, xd, y, 0, ws)
        ms = statistics.mean(time_steps(lambda: b.cmrs_spmv(M, xd, y, 0, ws), steps, flush, stream))
        S = (a.rows + h - 1) // h
        out["h%d" % h] = {"ms": ms, "gbs": beta_plus(a.nnz, a.rows, S, 8) / (ms / 1e3) / 1e9}
        del M
    return out


def modified_cmrs(b, a, xd, rp, ci, va, flush, stream, steps=100):
    """Section 6.6: padded strips and the slot-buffer kernel, FP64, at the
    paper's height 16 and M = 8 and at other (height, M); GB/s on the unpadded
    beta+."""
    import torch
    out = {}
    y = torch.empty(a.rows, dtype=torch.float64, device=xd.device)
    for h, m in ((16, 8), (32, 8), (16, 2), (32, 2), (32, 1)):
        P = b.cmrs_pad(b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=b.CMRS_F64), m)
        ws = P.spmv_workspace(b.CMRS_VARIANT_PADDED)
        for _ in range(3):
            b.cmrs_spmv(P, xd, y, b.CMRS_VARIANT_PADDED, ws)
        ms = statistics.mean(time_steps(lambda: b.cmrs_spmv(P, xd, y, b.CMRS_VARIANT_PADDED, ws), steps, flush,
                                        stream))
        bp = beta_plus(a.nnz, a.rows, (a.rows + h - 1) // h, 8)
        out["h%d_m%d" % (h, m)] = {"ms": ms, "gbs": bp / (ms / 1e3) / 1e9, "padded_items_per_nnz": P.nnz / a.nnz}
        del P
    return out


def variant_sweep(b, a, xd, M64, flush, stream, bp, steps=100):
    import torch
    out = {}
    y = torch.empty(a.rows, dtype=torch.float64, device=xd.device)
    for name, v in b.VARIANTS.items():
        ws = M64.spmv_workspace(v)
        for _ in range(3):
            b.cmrs_spmv(M64, xd, y, v, ws)
        ms = statistics.mean(time_steps(lambda: b.cmrs_spmv(M64, xd, y, v, ws), steps, flush, stream))
        out[name] = {"ms": ms, "gbs": bp / (ms / 1e3) / 1e9}
    return out


def selector_cost(b, a, rp, ci, reps=5):
    """The strip selector on the headline matrix: the committed network
    (features pass + forward + argmin, one read-back) and its choice, median
    wall time of `reps` calls."""
    import torch
    from paper_1203_2946_gb300 import selector
    model = selector.load_model(os.path.join(ROOT, "paper_1203_2946_gb300", "data", "selector_model.npz"))
    ts, pick = [], None
    for _ in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pick = b.cmrs_select_strip(rp, ci, a.cols, model)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    h, v, m = pick
    name = ("h=%d/padded-m%d" % (h, m)) if v == b.CMRS_VARIANT_PADDED else "h=%d/%s" % (h, ("row", "strip", "merge")[v])
    return {"ms": statistics.median(ts[1:]) * 1e3, "choice": name}


def selector_sample(b, dev, count=24, seed=5):
    """The committed selector on `count` of its 500 held-out corpus matrices
    (seeded choice), each regenerated on the device and timed again by the
    exhaustive sweep here: regret t(network's choice) / t(best), against the
    fixed default h = 4, ROW."""
    from paper_1203_2946_gb300 import corpus, inputs, selector
    model = selector.load_model(os.path.join(ROOT, "paper_1203_2946_gb300", "data", "selector_model.npz"))
    specs = inputs.selector_family_specs(2000, seed=11)
    _, held = selector.split(len(specs), 500, seed=0)
    pick = np.random.default_rng(seed).choice(held, count, replace=False)
    timer = selector.Timer(dev)
    net, default, names, sizes = [], [], [], []
    for i in pick:
        rows, cols, rp, ci, va = corpus.device_matrix(specs[i], dev)
        _, t = selector.time_all_choices(rows, cols, rp, ci, va, timer)
        h, v, m = b.cmrs_select_strip(rp, ci, cols, model)
        c = 18 + b.SEL_PADDED.index((h, m)) if v == b.CMRS_VARIANT_PADDED else 3 * b.SEL_HEIGHTS.index(h) + v
        net.append(t[c] / t.min())
        default.append(t[3 * b.SEL_HEIGHTS.index(4)] / t.min())
        names.append(selector.choice_name(c))
        sizes.append(int(ci.numel()))
    geo = lambda r: float(np.exp(np.mean(np.log(r))))  # noqa: E731
    return {"matrices": count, "nnz_range": [min(sizes), max(sizes)], "network_regret_geomean": geo(net),
            "network_within_10pct": float(np.mean(np.array(net) <= 1.10)), "network_regret_max": float(max(net)),
            "fixed_default_h4_row_geomean": geo(default),
            "note": "held-out corpus matrices regenerated and timed again in this run (21 choices, L2 flushed)"}


def sorted_strips(b, a, xd, rp, ci, va, flush, stream, steps=60):
    """Section 4's fourth optimisation: the STRIP kernel (Algorithm 1) on
    unsorted strips and on strips stably sorted by column, at heights 4 and 16
    (FP64, beta+ of each height)."""
    import torch
    out = {}
    y = torch.empty(a.rows, dtype=torch.float64, device=xd.device)
    for h in (4, 16):
        S = (a.rows + h - 1) // h
        bp = 12 * a.nnz + 4 * S + 16 * a.rows
        for tag, flags in (("unsorted", 0), ("sorted", b.CMRS_SORTED)):
            M = b.cmrs_from_csr(rp, ci, va, a.cols, h, flags=flags, dtype=b.CMRS_F64)
            ws = M.spmv_workspace(b.CMRS_VARIANT_STRIP)
            for _ in range(3):
                b.cmrs_spmv(M, xd, y, b.CMRS_VARIANT_STRIP, ws)
            ms = statistics.mean(time_steps(lambda: b.cmrs_spmv(M, xd, y, b.CMRS_VARIANT_STRIP, ws), steps, flush,
                                            stream))
            out["h%d_%s" % (h, tag)] = {"ms": ms, "gbs": bp / (ms / 1e3) / 1e9}
            del M
    return out


def main():
    args = args_parse()
    if args.variant is None:
        args.variant = {"stencil27": "padded", "powerlaw": "merge", "p7": "padded", "dense4": "padded"}.get(
            args.workload, "row")
    args.height_given = args.height is not None
    if args.height is None:
        args.height = 8 if args.workload == "dense4" else (
            32 if args.workload in ("powerlaw", "p7") or args.variant == "padded" else 4)
    if args.slots is None:
        args.slots = {"irregular": 2, "dense4": 4}.get(args.workload, 1)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "stencil27":
        run_ours(args)
    elif args.workload == "irregular":
        run_irregular(args)
    elif args.workload == "powerlaw":
        run_powerlaw(args)
    else:
        run_secondary(args)



# --------------------------------------------------------------------------- secondary workloads
def _line(args, metric_value, unit, per_ms, dtype, config, roofline, e2e, launches, clocks, extra=None):
    line = {"metric": METRIC, "value": metric_value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config, "roofline": roofline,
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    if extra:
        line.update(extra)
    return line


def run_secondary(args):
    import torch
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding as b, inputs
    import oracle
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    flush = L2Flush(dev)
    peak, peak_kind = measured_peaks()
    sampler = ClockSampler(None)
    steps = args.steps
    if args.workload in ("laplacian", "p7", "dense4"):
        if args.workload == "p7":
            a = inputs.permutation_matrix()
            x = inputs.uniform_vector(a.cols, 0)
            dt, sv, name = b.CMRS_F64, 8, "f64"
            wl = "p7: 10^7 x 10^7 random permutation (one entry per row), FP64"
        elif args.workload == "dense4":
            a = inputs.dense_as_sparse()
            x = inputs.uniform_vector(a.cols, 0)
            dt, sv, name = b.CMRS_F64, 8, "f64"
            wl = "dense4: 10^4 x 10^4 dense matrix stored as sparse (nnz = 10^8), FP64"
        else:
            a, x = inputs.workload_laplacian_64()
            dt, sv, name = b.CMRS_F64, 8, "f64"
            wl = "5-point Laplacian 64x64 (n=4096, nnz=20224), FP64"
        h, v = args.height, dict(b.VARIANTS, auto=b.CMRS_VARIANT_AUTO, padded=b.CMRS_VARIANT_PADDED)[args.variant]
        rp, ci = torch.from_numpy(a.row_ptr).to(dev), torch.from_numpy(a.col_ind).to(dev)
        va = torch.from_numpy(np.ascontiguousarray(a.val)).to(dev)
        M = M_plain = b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=dt)
        if args.variant == "padded":
            M = b.cmrs_pad(M, args.slots)
        ran = b.cmrs_spmv_variant(M, v)
        xd = torch.from_numpy(x).to(dev)
        yd = torch.empty(a.rows, dtype=xd.dtype, device=dev)
        ws = M.spmv_workspace(v)
        fn = lambda: b.cmrs_spmv(M, xd, yd, v, ws)  # noqa: E731
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        with sampler:
            times = time_steps(fn, steps, flush, stream, warm_steps=max(3, args.warmup), warm_s=0.25)
        per_ms = statistics.mean(times)
        S = (a.rows + h - 1) // h
        bp = beta_plus(a.nnz, a.rows, S, sv)
        gbs = bp / (per_ms / 1e3) / 1e9
        yref, scale = oracle.csr_spmv(a.row_ptr, a.col_ind, a.val.astype(np.float64), x.astype(np.float64))
        rel = np.abs(yd.cpu().numpy().astype(np.float64) - yref) / np.where(scale > 0, scale, 1)
        extra = {"gflops": 2 * a.nnz / (per_ms / 1e3) / 1e9,
                 "eta": eta(a.nnz, a.rows, S, sv, per_ms, peak),
                 "err_vs_f64_oracle": {"max": float(rel.max()), "median": float(np.median(rel))}}
        if not args.no_cpu:
            extra["cpu_baseline"] = cpu_oracle_rate(inputs.CSR(a.rows, a.cols, a.row_ptr, a.col_ind,
                                                               a.val.astype(np.float64)), x.astype(np.float64), S)
        extra["stored_items_per_nnz"] = M.nnz / max(a.nnz, 1)
        if args.workload == "p7":
            extra["gather_floor"] = gather_floor(b, ci, None, xd.float(), flush, stream, per_ms)
        if args.workload in ("p7", "dense4"):
            var = {}
            for vn, vv in b.VARIANTS.items():  # plain CMRS at the same height
                vws = M_plain.spmv_workspace(vv)
                g = lambda: b.cmrs_spmv(M_plain, xd, yd, vv, vws)  # noqa: E731
                for _ in range(2):
                    g()
                vms = statistics.mean(time_steps(g, 20, flush, stream))
                var[vn] = {"ms": vms, "gbs": bp / (vms / 1e3) / 1e9}
            extra["variants_f64"] = var
            if args.workload == "dense4" and args.variant == "padded":
                pads = {}  # the other padded forms (few long strips: each strip split over several warps)
                for ph, pm in ((4, 8), (8, 4), (16, 2), (32, 1)):
                    Q = b.cmrs_pad(b.cmrs_from_csr(rp, ci, va, a.cols, ph, dtype=b.CMRS_F64), pm)
                    qws = Q.spmv_workspace(b.CMRS_VARIANT_PADDED)
                    g = lambda: b.cmrs_spmv(Q, xd, yd, b.CMRS_VARIANT_PADDED, qws)  # noqa: E731
                    for _ in range(2):
                        g()
                    qms = statistics.mean(time_steps(g, 20, flush, stream))
                    pads["h%d_m%d" % (ph, pm)] = {"ms": qms, "gbs": bp / (qms / 1e3) / 1e9}
                    del Q
                extra["padded_forms_f64"] = pads
            fn()
        xh = torch.from_numpy(x).pin_memory()
        yhs = [torch.empty(a.rows, dtype=xd.dtype).pin_memory() for _ in range(2)]
        e_ms = e2e_pipelined(lambda xv, yv: b.cmrs_spmv(M, xv, yv, v, ws), xh, [xd, torch.empty_like(xd)],
                             [yd, torch.empty_like(yd)], yhs, max(20, min(steps, 200)))
        kname = {0: row_kernel(M), 1: "k_spmv_strip", 2: "k_spmv_merge", 3: "k_spmv_padded"}[ran]
        split = ran == 3 and ws.numel() > 256  # a padded workspace past the status word: strips split over warps
        if split:
            kname = "k_spmv_padded_split"  # + k_pad_combine
        line = _line(args, gbs, "GB/s", per_ms, name,
                     {"workload": wl, "height": h, "variant": args.variant,
                      "kernel_variant": ("row", "strip", "merge", "padded")[ran], "bytes_per_step": bp,
                      "l2": L2_NOTE},
                     {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                      "peak_kind": peak_kind + " (hbm_gbs)", "kernel": kname,
                      "traffic": traffic_record(kname, "%s_%s_h%d" % (args.workload, name, h) + (
                          "_m%d" % args.slots if args.variant == "padded" else ""))},
                     {"value": bp / (e_ms / 1e3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(x.nbytes),
                      "d2h_bytes_per_step": int(a.rows * x.itemsize), "ms_per_step": e_ms},
                     steps * (3 if ran == 2 else 2 if split else 1), sampler.summary(), extra)
        print(json.dumps(line), flush=True)
        return

    # ---- batched: 256 banded-random matrices, k right-hand sides each
    r = batched_block(b, inputs, oracle, dev, flush, stream, steps, args.warmup,
                      (args.height,) if args.height_given else (1, 2, 4, 8, 16, 32), args.batch_count, sampler)
    line = _line(args, r["gbs"], "GB/s", r["ms"], "f32", r["config"], r["roofline"], r["e2e"], r["gpu_launches"],
                 sampler.summary(), r["extra"])
    print(json.dumps(line), flush=True)


def spmm_traffic(bp):
    """DRAM bytes per batch: the ncu capture of the first 16 matrices scaled by
    their algorithmic bytes to the whole batch (its traffic equals its
    algorithmic bytes to 1%), while the kernel's source is unchanged."""
    t = traffic_record("k_spmm_queue", "batched16")
    if t is None:
        return None
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        alg = json.load(f)["k_spmm_queue"]["batched16"]["algorithmic_bytes"]
    return int(t / alg * bp)


def batched_block(b, inputs, oracle, dev, flush, stream, steps, warmup, heights, count, sampler=None):
    """The batched workload: `count` banded-random matrices with k right-hand
    sides each, one persistent graph-replayed launch per step, its schedule
    autotuned (each matrix's strip height among `heights`, then the work-unit
    size), against per-matrix launches and per-column plain FP64 SpMV; a
    parity sample against the oracle; e2e with X in and Y out every step."""
    from paper_1203_2946_gb300 import batch
    import contextlib
    import torch
    specs = inputs.batched_banded_specs()[:count]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        mats_host = pool.map(_gen_batched, specs, chunksize=4)
    peak, peak_kind = measured_peaks()
    csrs, Xs, Ys, bp, nnz_total, rows_total = [], [], [], 0, 0, 0
    for (rp_, ci_, val_, X_), sp_ in zip(mats_host, specs):
        n = rp_.size - 1
        csrs.append((torch.from_numpy(rp_).to(dev), torch.from_numpy(ci_).to(dev), torch.from_numpy(val_).to(dev)))
        Xs.append(torch.from_numpy(X_).to(dev))
        Ys.append(torch.empty((n, X_.shape[1]), dtype=torch.float32, device=dev))
    t0 = time.perf_counter()
    mats, hs, best, _, _ = batch.tune(csrs, Xs, Ys, heights=heights)
    tune_s = time.perf_counter() - t0
    del csrs
    for (rp_, ci_, val_, X_), h in zip(mats_host, hs):
        n, nnz = rp_.size - 1, int(ci_.size)
        bp += beta_plus(nnz, n, (n + h - 1) // h, 4) + 8 * (X_.shape[1] - 1) * n
        nnz_total += nnz * X_.shape[1]
        rows_total += n
    plan = b.SpmmPlan(mats, Xs, Ys, work_target=best, use_graph=True)
    fn = lambda: b.cmrs_spmm_batched(plan)  # noqa: E731
    for _ in range(max(3, warmup)):
        fn()
    torch.cuda.synchronize()
    with (sampler if sampler is not None else contextlib.nullcontext()):
        times = time_steps(fn, steps, flush, stream, warm_steps=max(3, warmup), warm_s=0.25)
    per_ms = statistics.mean(times)
    gbs = bp / (per_ms / 1e3) / 1e9
    # per-matrix plain launches of the same kernel, no graph
    plain = lambda: [b.cmrs_spmm(M, X, Y) for M, X, Y in zip(mats, Xs, Ys)]  # noqa: E731
    plain()
    plain_ms = statistics.mean(time_steps(plain, 5, flush, stream))
    # sampled parity against the oracle: 8 matrices, every column
    worst = 0.0
    for i in range(0, len(specs), max(1, len(specs) // 8)):
        rp_, ci_, val_, X_ = mats_host[i]
        Y = Ys[i].cpu().numpy()
        L = np.diff(rp_)
        for c in range(X_.shape[1]):
            yref, sc = oracle.csr_spmv(rp_, ci_, val_.astype(np.float64), X_[:, c].astype(np.float64))
            err = np.abs(Y[:, c] - yref)
            worst = max(worst, float(np.max(err / np.maximum((L + 2) * 2.0**-24 * sc, 1e-300))))
    # plain FP64 CMRS SpMV, one launch per matrix and right-hand side (the baseline kernel)
    f64_ms = None
    sub = list(range(0, len(specs), 4))
    mats64, cols64 = [], []
    for i in sub:
        rp_, ci_, val_, X_ = mats_host[i]
        n = rp_.size - 1
        M64 = b.cmrs_from_csr(torch.from_numpy(rp_).to(dev), torch.from_numpy(ci_).to(dev),
                              torch.from_numpy(val_.astype(np.float64)).to(dev), n, hs[i], dtype=b.CMRS_F64)
        xs = [torch.from_numpy(np.ascontiguousarray(X_[:, c], dtype=np.float64)).to(dev) for c in range(X_.shape[1])]
        mats64.append((M64, xs, torch.empty(n, dtype=torch.float64, device=dev), M64.spmv_workspace(0)))
    f64 = lambda: [b.cmrs_spmv(M64, xc, y64, 0, w64) for M64, xs, y64, w64 in mats64 for xc in xs]  # noqa: E731
    f64()
    f64_sub_ms = statistics.mean(time_steps(f64, 3, flush, stream))
    plain_sub = lambda: [b.cmrs_spmm(mats[i], Xs[i], Ys[i]) for i in sub]  # noqa: E731
    plain_sub()
    plain_sub_ms = statistics.mean(time_steps(plain_sub, 3, flush, stream))
    # e2e: every step copies all X in and all Y out.  Each buffer set is one
    # allocation with every matrix's X (or Y) at a 256-byte boundary inside it,
    # so a step moves X in one host->device copy and Y in one device->host
    # copy; two sets and two plans let the copies of neighbouring steps
    # overlap a replay.
    def contiguous(mats_like, device, pin=False):
        offs, total = [], 0
        for T in mats_like:
            offs.append(total)
            total += (T.numel() + 63) // 64 * 64
        buf = torch.empty(total, dtype=torch.float32, device=device, pin_memory=pin)
        return buf, [buf[o:o + T.numel()].view(T.shape) for o, T in zip(offs, mats_like)]
    Xh, Xh_views = contiguous(Xs, "cpu", pin=True)
    for H, X in zip(Xh_views, Xs):
        H.copy_(X.cpu())
    dsets = [(contiguous(Xs, dev), contiguous(Ys, dev)) for _ in range(2)]
    plans = [b.SpmmPlan(mats, xv, yv, work_target=best, use_graph=True) for (_, xv), (_, yv) in dsets]
    Yh = [contiguous(Ys, "cpu", pin=True)[0] for _ in range(2)]

    def copy_in(s):
        dsets[s][0][0].copy_(Xh, non_blocking=True)

    def copy_out(s):
        Yh[s].copy_(dsets[s][1][0], non_blocking=True)
    e_ms = e2e_pipelined_sets(lambda s: b.cmrs_spmm_batched(plans[s]), copy_in, copy_out, 10, warm=2)
    info = plan.info()
    return {"ms": per_ms, "gbs": gbs,
            "config": {"workload": "%d banded-random matrices (n~U[1000,200000], bandwidth~U[64,2048], 10-60 nnz/row, "
                                   "k in {1,4,8,32}), FP32, CMRS with each matrix's strip height autotuned; one "
                                   "persistent graph-replayed launch" % len(specs),
                       "matrices": len(specs), "rows_total": rows_total, "entry_columns": nnz_total,
                       "bytes_per_step": bp,
                       "schedule": {"work_target": best, **info,
                                    "heights": {str(h): hs.count(h) for h in sorted(set(hs))},
                                    "height_candidates": list(heights), "tuning_s": tune_s},
                       "l2": L2_NOTE},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "peak_kind": peak_kind + " (hbm_gbs)", "traffic": spmm_traffic(bp),
                         "kernel": "k_spmm_queue"},
            "e2e": {"value": bp / (e_ms / 1e3) / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": int(Xh.numel() * 4), "d2h_bytes_per_step": int(Yh[0].numel() * 4),
                    "ms_per_step": e_ms, "note": "X in and Y out in one copy each per step (every matrix's block "
                    "at a 256-byte boundary of one buffer), two buffer sets, copies of neighbouring steps overlap"},
            "gpu_launches": steps,
            "extra": {"gflops": 2 * nnz_total / (per_ms / 1e3) / 1e9,
                      "per_matrix_launches": {"ms": plain_ms, "speedup_of_batched": plain_ms / per_ms},
                      "plain_f64_spmv_per_column": {"matrices": len(sub), "ms": f64_sub_ms,
                                                    "batched_f32_ms_same_subset": plain_sub_ms,
                                                    "speedup_of_f32_spmm": f64_sub_ms / plain_sub_ms},
                      "parity_sample": {"matrices": 8, "max_err_over_tolerance": worst}}}


def row_kernel(M):
    """The kernel the library's ROW variant runs for matrix M: one, two or
    four lanes per row (k_spmv_lane) for mean rows of at most 28, 56, 112
    entries at heights dividing 32, 16, 8; else k_spmv_row."""
    mu = M.nnz / max(M.rows, 1)
    for lanes, bound in ((1, 28), (2, 56), (4, 112)):
        if mu <= bound:
            return "k_spmv_lane" if (32 // lanes) % M.height == 0 else "k_spmv_row"
    return "k_spmv_row"


def gather_floor(b, ci, va, x32, flush, stream, kernel_ms, steps=50):
    """k_gather_dot on the matrix's own column array (and FP32 values, if
    given): the time any SpMV kernel pays for the streams and the x gathers
    alone, with the row structure taken away; and the kernel's distance to it."""
    import torch
    out = torch.empty(1, dtype=torch.float32, device=x32.device)
    fn = lambda: b.cmrs_gather_probe(ci, va, x32, out)  # noqa: E731
    ms = statistics.mean(time_steps(fn, steps, flush, stream))
    return {"ms": ms, "kernel": "k_gather_dot", "streams": "columns" + (" and FP32 values" if va is not None else ""),
            "kernel_frac_of_floor": ms / kernel_ms,
            "note": "floor = one pass over the streams with every x gather, no row bounds, sums or y"}


def powerlaw_block(b, inputs, oracle, dev, flush, stream, steps, warmup, h=32, sampler=None, forms=True):
    """Power-law rows, n = 4,194,304 (Zipf(2.1) clipped to [1, 100000]), FP32
    values and x, MERGE at height h: time, beta+ GB/s, error against the FP64
    oracle, the gather floor, and the BF16 form."""
    import contextlib
    import torch
    peak, peak_kind = measured_peaks()
    a, x = inputs.workload_powerlaw_4m()
    rp, ci = torch.from_numpy(a.row_ptr).to(dev), torch.from_numpy(a.col_ind).to(dev)
    va = torch.from_numpy(np.ascontiguousarray(a.val)).to(dev)
    M = b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=b.CMRS_F32)
    v = b.CMRS_VARIANT_MERGE
    xd = torch.from_numpy(x).to(dev)
    yd = torch.empty(a.rows, dtype=torch.float32, device=dev)
    ws = M.spmv_workspace(v)
    fn = lambda: b.cmrs_spmv(M, xd, yd, v, ws)  # noqa: E731
    for _ in range(max(3, warmup)):
        fn()
    torch.cuda.synchronize()
    with (sampler if sampler is not None else contextlib.nullcontext()):
        times = time_steps(fn, steps, flush, stream, warm_steps=max(3, warmup), warm_s=0.25)
    ms = statistics.mean(times)
    S = (a.rows + h - 1) // h
    bp = beta_plus(a.nnz, a.rows, S, 4)
    gbs = bp / (ms / 1e3) / 1e9
    yref, scale = oracle.csr_spmv(a.row_ptr, a.col_ind, a.val.astype(np.float64), x.astype(np.float64))
    rel = np.abs(yd.cpu().numpy().astype(np.float64) - yref) / np.where(scale > 0, scale, 1)
    out = {"workload": "power-law rows, Zipf(2.1) clipped to [1,100000], n=%d, nnz=%d (mean %.2f), FP32 values and "
                       "x, CMRS h=%d, MERGE" % (a.rows, a.nnz, a.nnz / a.rows, h),
           "ms": ms, "gbs": gbs, "bytes_per_step": bp, "gflops": 2 * a.nnz / (ms / 1e3) / 1e9,
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                        "peak_kind": peak_kind + " (hbm_gbs)", "kernel": "k_spmv_merge",
                        "traffic": traffic_record("k_spmv_merge", "powerlaw_f32_h%d" % h)},
           "eta": eta(a.nnz, a.rows, S, 4, ms, peak),
           "err_vs_f64_oracle": {"max": float(rel.max()), "median": float(np.median(rel))},
           "gather_floor": gather_floor(b, ci, va, xd, flush, stream, ms)}
    if forms:
        F = b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=b.CMRS_BF16)
        fws = F.spmv_workspace(v)
        ff = lambda: b.cmrs_spmv(F, xd, yd, v, fws)  # noqa: E731
        fms = statistics.mean(time_steps(ff, min(steps, 200), flush, stream))
        frel = np.abs(yd.cpu().numpy().astype(np.float64) - yref) / np.where(scale > 0, scale, 1)
        fbp = 6 * a.nnz + 4 * S + 8 * a.rows
        out["forms"] = {"bf16": {"gbs": fbp / (fms / 1e3) / 1e9, "ms": fms, "speedup_vs_f32": ms / fms,
                                 "bytes_per_step": fbp,
                                 "err_vs_f64_oracle": {"max": float(frel.max()), "median": float(np.median(frel))}}}
    out["_keep"] = (a, x, M, xd, yd, ws, S)
    return out


def run_powerlaw(args):
    import torch
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding as b, inputs
    import oracle
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    flush = L2Flush(dev)
    sampler = ClockSampler(None)
    r = powerlaw_block(b, inputs, oracle, dev, flush, stream, args.steps, args.warmup, args.height, sampler)
    a, x, M, xd, yd, ws, S = r.pop("_keep")
    v = b.CMRS_VARIANT_MERGE
    var = {}
    for vn, vv in b.VARIANTS.items():
        vws = M.spmv_workspace(vv)
        g = lambda: b.cmrs_spmv(M, xd, yd, vv, vws)  # noqa: E731
        vms = statistics.mean(time_steps(g, 20, flush, stream))
        var[vn] = {"ms": vms, "gbs": r["bytes_per_step"] / (vms / 1e3) / 1e9}
    xh = torch.from_numpy(x).pin_memory()
    yhs = [torch.empty(a.rows, dtype=torch.float32).pin_memory() for _ in range(2)]
    e_ms = e2e_pipelined(lambda xv, yv: b.cmrs_spmv(M, xv, yv, v, ws), xh, [xd, torch.empty_like(xd)],
                         [yd, torch.empty_like(yd)], yhs, max(20, min(args.steps, 200)))
    extra = {k: r[k] for k in ("gflops", "eta", "err_vs_f64_oracle", "gather_floor", "forms")}
    extra["variants_f32"] = var
    if not args.no_cpu:
        extra["cpu_baseline"] = cpu_oracle_rate(inputs.CSR(a.rows, a.cols, a.row_ptr, a.col_ind,
                                                           a.val.astype(np.float64)), x.astype(np.float64), S)
    line = _line(args, r["gbs"], "GB/s", r["ms"], "f32",
                 {"workload": r["workload"], "height": args.height, "variant": "merge", "kernel_variant": "merge",
                  "bytes_per_step": r["bytes_per_step"], "l2": L2_NOTE},
                 r["roofline"],
                 {"value": r["bytes_per_step"] / (e_ms / 1e3) / 1e9, "unit": "GB/s",
                  "h2d_bytes_per_step": int(x.nbytes), "d2h_bytes_per_step": int(a.rows * 4), "ms_per_step": e_ms},
                 args.steps * 3, sampler.summary(), extra)
    print(json.dumps(line), flush=True)


def _gen_batched(spec):
    from paper_1203_2946_gb300 import inputs
    a, X = inputs.batched_banded(spec)
    return a.row_ptr, a.col_ind, a.val, X




# --------------------------------------------------------------------------- row reordering
def run_irregular(args):
    """Banded-random rows of 4..60 entries (n = 2^21, FP64): modified CMRS at
    h = 32, M = 1 after row reordering (windows of --window rows), the product
    written back in the original order through the row map; against the same
    form without reordering, M = 8, and plain CMRS with ROW and MERGE."""
    import torch
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding as b, inputs
    import oracle
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    flush = L2Flush(dev)
    peak, peak_kind = measured_peaks()
    sampler = ClockSampler(None)
    a, x = inputs.workload_irregular()
    h, steps = 32, args.steps
    rp, ci, va = (torch.from_numpy(t).to(dev) for t in (a.row_ptr, a.col_ind, a.val))
    xd = torch.from_numpy(x).to(dev)
    yd = torch.empty(a.rows, dtype=torch.float64, device=dev)
    S = (a.rows + h - 1) // h
    bp = beta_plus(a.nnz, a.rows, S, 8)

    def reorder(window):
        perm = b.cmrs_row_order(rp, window)
        rp2, ci2, va2 = b.cmrs_permute_csr(rp, ci, va, perm)
        return perm, b.cmrs_from_csr(rp2, ci2, va2, a.cols, h, dtype=b.CMRS_F64)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.window:
        perm, M = reorder(args.window)
    else:
        perm, M = None, b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=b.CMRS_F64)
    P = b.cmrs_pad(M, args.slots)
    torch.cuda.synchronize()
    prep_ms = (time.perf_counter() - t0) * 1e3
    ws = P.spmv_workspace(b.CMRS_VARIANT_PADDED)
    if perm is None:
        fn = lambda: b.cmrs_spmv(P, xd, yd, b.CMRS_VARIANT_PADDED, ws)  # noqa: E731
    else:
        fn = lambda: b.cmrs_spmv_rows(P, xd, perm, yd, b.CMRS_VARIANT_PADDED, ws)  # noqa: E731
    for _ in range(max(3, args.warmup)):
        fn()
    torch.cuda.synchronize()
    with sampler:
        times = time_steps(fn, steps, flush, stream, warm_steps=max(3, args.warmup), warm_s=0.25)
    per_ms = statistics.mean(times)
    gbs = bp / (per_ms / 1e3) / 1e9
    yref, scale = oracle.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    rel = np.abs(yd.cpu().numpy() - yref) / np.where(scale > 0, scale, 1)

    def timed(f, n=100):
        for _ in range(3):
            f()
        return statistics.mean(time_steps(f, n, flush, stream))

    others = {}
    M0 = b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=b.CMRS_F64)
    p256, M256 = reorder(256)
    p4096, M4096 = reorder(4096)
    for name, mat, v, rows_map in (
            ("padded_m1", b.cmrs_pad(M0, 1), b.CMRS_VARIANT_PADDED, None),
            ("padded_m8", b.cmrs_pad(M0, 8), b.CMRS_VARIANT_PADDED, None),
            ("reordered_w256_padded_m1", b.cmrs_pad(M256, 1), b.CMRS_VARIANT_PADDED, p256),
            ("reordered_w4096_padded_m1", b.cmrs_pad(M4096, 1), b.CMRS_VARIANT_PADDED, p4096),
            ("reordered_w4096_padded_m2", b.cmrs_pad(M4096, 2), b.CMRS_VARIANT_PADDED, p4096),
            ("row_h32", M0, b.CMRS_VARIANT_ROW, None),
            ("row_h16_two_lanes_per_row", b.cmrs_from_csr(rp, ci, va, a.cols, 16, dtype=b.CMRS_F64), b.CMRS_VARIANT_ROW,
             None),
            ("merge_h32", M0, b.CMRS_VARIANT_MERGE, None),
            ("reordered_w4096_row_h32", M4096, b.CMRS_VARIANT_ROW, p4096)):
        w2 = mat.spmv_workspace(v)
        if rows_map is None:
            f = lambda mat=mat, v=v, w2=w2: b.cmrs_spmv(mat, xd, yd, v, w2)  # noqa: E731
        else:
            f = lambda mat=mat, v=v, w2=w2, pm=rows_map: b.cmrs_spmv_rows(mat, xd, pm, yd, v, w2)  # noqa: E731
        ms = timed(f)
        others[name] = {"ms": ms, "gbs": bp / (ms / 1e3) / 1e9, "stored_items_per_nnz": mat.nnz / a.nnz}
    xh = torch.from_numpy(x).pin_memory()
    yhs = [torch.empty(a.rows, dtype=torch.float64).pin_memory() for _ in range(2)]
    if perm is None:
        run = lambda xv, yv: b.cmrs_spmv(P, xv, yv, b.CMRS_VARIANT_PADDED, ws)  # noqa: E731
    else:
        run = lambda xv, yv: b.cmrs_spmv_rows(P, xv, perm, yv, b.CMRS_VARIANT_PADDED, ws)  # noqa: E731
    e_ms = e2e_pipelined(run, xh, [xd, torch.empty_like(xd)], [yd, torch.empty_like(yd)], yhs,
                         max(20, min(steps, 200)))
    extra = {"gflops": 2 * a.nnz / (per_ms / 1e3) / 1e9, "eta": eta(a.nnz, a.rows, S, 8, per_ms, peak),
             "err_vs_f64_oracle": {"max": float(rel.max()), "median": float(np.median(rel))},
             "reorder_pad_prep_ms": prep_ms, "others": others}
    if not args.no_cpu:
        extra["cpu_baseline"] = cpu_oracle_rate(a, x, S)
    line = _line(args, gbs, "GB/s", per_ms, "f64",
                 {"workload": "banded random n=%d, window 2048, rows of 4..60 entries (nnz=%d), FP64; %smodified "
                              "CMRS h=32, M=%d" % (a.rows, a.nnz, "rows reordered by length in windows of %d, y through "
                                                   "the row map; " % args.window if args.window else "", args.slots),
                  "height": h, "variant": "padded", "slots": args.slots, "window": args.window,
                  "stored_items_per_nnz": P.nnz / a.nnz, "bytes_per_step": bp,
                  "l2": L2_NOTE},
                 {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                  "peak_kind": peak_kind + " (hbm_gbs)", "traffic": None, "kernel": "k_spmv_padded"},
                 {"value": bp / (e_ms / 1e3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(x.nbytes),
                  "d2h_bytes_per_step": int(a.rows * 8), "ms_per_step": e_ms},
                 steps, sampler.summary(), extra)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
