#!/usr/bin/env python3
"""CMRS SpMV benchmark on GB300.

Workload (default): 27-point stencil on a 128^3 grid, non-periodic
(n = 2,097,152 rows, nnz = 55,742,968), FP64 values, x ~ U[-1, 1], CMRS with
strip height h, SpMV kernel variant ROW.  One step = one y = A x through
cmrs_spmv.  Inputs are resident in HBM before the timed region; the L2 is
flushed (256 MiB write) between steps and every step is timed by its own pair
of CUDA events on the launching stream.

Metric: GB/s = beta_plus / t with beta_plus = (s_v + s_i) nnz + s_i strips +
2 s_v rows (Eq. 6.1: matrix, x and y moved once), also GFLOP/s = 2 nnz / t and
the paper's (2 nnz - rows) / t.  e2e: the same metric through the C ABI with x
copied from pinned host memory and y copied back inside the timed region.

  python bench.py [--steps K] [--warmup W] [--height H] [--variant row|strip|merge]
  python bench.py --impl reference      # the CPU oracle on the same workload
  torchrun --nproc-per-node N bench.py --gpus N   # N independent replicas
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
    p.add_argument("--height", type=int, default=4)
    p.add_argument("--variant", default="row", choices=["row", "strip", "merge"])
    p.add_argument("--no-extras", action="store_true", help="skip the secondary storage-form measurements")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return p.parse_args()


def beta_plus(nnz, rows, strips, s_v, s_i=4):
    return (s_v + s_i) * nnz + s_i * strips + 2 * s_v * rows


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


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1203_2946_gb300 import inputs
    a, x = inputs.workload_stencil27_128()
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
            "config": {"workload": "27-point stencil 128^3 (n=2097152, nnz=55742968), FP64, CRS order; "
                                   "each step a slice of %d rows" % nrow},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "%d consecutive rows per step (%.3f of the matrix), %d steps" % (
                                 nrow, nrow / a.rows, len(ts))},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU leg
def traffic_record(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, valid only while
    the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)[kernel][workload]
        src = os.path.join(ROOT, "paper_1203_2946_gb300", "csrc", "spmv.cu")
        h = hashlib.sha1(open(src, "rb").read()).hexdigest()
        return rec["bytes_per_launch"] if rec.get("spmv_cu_sha1") == h else None
    except Exception:
        return None


def time_steps(fn, steps, flush, stream):
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xFF)
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def run_ours(args):
    import torch
    rank, world, dist = dist_setup(args.gpus)
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding as b, inputs
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    variant = binding_variant = b.VARIANTS[args.variant]
    a, x = inputs.workload_stencil27_128()
    h = args.height
    strips = (a.rows + h - 1) // h
    rp = torch.from_numpy(a.row_ptr).to(dev)
    ci = torch.from_numpy(a.col_ind).to(dev)
    va = torch.from_numpy(a.val).to(dev)
    M = b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=b.CMRS_F64)
    xd = torch.from_numpy(x).to(dev)
    yd = torch.empty(a.rows, dtype=torch.float64, device=dev)
    ws = M.spmv_workspace(variant)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        b.cmrs_spmv(M, xd, yd, binding_variant, ws)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    bp = beta_plus(a.nnz, a.rows, strips, 8)
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
        times = time_steps(step, args.steps, flush, stream)
    barrier(dist)
    wall = time.perf_counter() - wall0
    total_ms = max_over_ranks(dist, sum(times))
    per_ms = total_ms / args.steps
    value = world * bp * args.steps / (total_ms / 1e3) / 1e9
    b.cmrs_spmv_check(M, variant)

    # e2e through the C ABI with host buffers
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty(a.rows, dtype=torch.float64).pin_memory()

    def e2e_step():
        xd.copy_(xh, non_blocking=True)
        b.cmrs_spmv(M, xd, yd, binding_variant, ws)
        yh.copy_(yd, non_blocking=True)

    e2e_steps = max(20, min(args.steps, 200))
    for _ in range(3):
        e2e_step()
    e2e_times = time_steps(e2e_step, e2e_steps, flush, stream)
    e2e_ms = max_over_ranks(dist, statistics.mean(e2e_times))

    kname = {0: "k_spmv_row", 1: "k_spmv_strip", 2: "k_spmv_merge"}[variant]
    trimmed = sorted(times)[:-1] if len(times) > 1 else times
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "27-point stencil 128^3 (n=2097152, nnz=55742968), FP64 values and x, "
                               "CMRS h=%d, variant %s" % (h, args.variant),
                   "height": h, "variant": args.variant, "bytes_per_step": bp,
                   "l2": "flushed between steps (256 MiB write), each step timed by its own CUDA events",
                   "parallelism": "replicas x%d" % world if world > 1 else "single GPU"},
        "gflops": 2 * a.nnz / (per_ms / 1e3) / 1e9,
        "gflops_paper": (2 * a.nnz - a.rows) / (per_ms / 1e3) / 1e9,
        "pct_of_hbm_peak": 100.0 * (value / world) / peak,
        "pct_of_nominal_8tbs": 100.0 * (value / world) / 8000.0,
        "paper_protocol": {"mean_ms": statistics.mean(trimmed), "std_ms": statistics.pstdev(trimmed),
                           "min_ms": min(times)},
        "roofline": {"bound": "hbm", "achieved": bp / (per_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": bp / (per_ms / 1e3) / 1e9 / peak, "peak_kind": peak_kind + " (hbm_gbs)",
                     "traffic": traffic_record(kname, "stencil27_128_f64_h%d" % h), "kernel": kname},
        "e2e": {"value": world * bp / (e2e_ms / 1e3) / 1e9, "unit": "GB/s",
                "h2d_bytes_per_step": int(x.nbytes), "d2h_bytes_per_step": int(a.rows * 8),
                "ms_per_step": e2e_ms, "note": "x host->device, cmrs_spmv, y device->host; matrix resident"},
        "gpu_launches": args.steps * (3 if variant == 2 else 1),
        "clocks": sampler.summary(),
        "wall_s_timed_region": wall,
    }
    if rank == 0 and not args.no_extras and world == 1:
        line["forms"] = storage_forms(b, a, x, rp, ci, va, h, flush, stream, per_ms)
        line["variants_f64"] = variant_sweep(b, a, xd, M, flush, stream, bp)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate(a, x, strips)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def storage_forms(b, a, x, rp, ci, va, h, flush, stream, f64_ms, steps=200):
    """FP32 / BF16 / split-BF16 storage of the same matrix: speed, speed-up over
    the FP64 kernel and error against the FP64 oracle (max and median of
    |y - y*| / (|A||x|)_i)."""
    import oracle
    import torch
    yref, scale = oracle.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    out = {}
    x32 = torch.from_numpy(x.astype(np.float32)).to(va.device)
    strips = (a.rows + h - 1) // h
    for name, dt, sv in (("f32", b.CMRS_F32, 4), ("bf16", b.CMRS_BF16, 2), ("bf16x2", b.CMRS_BF16X2, 4)):
        M = b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=dt)
        y = torch.empty(a.rows, dtype=torch.float32, device=va.device)
        ws = M.spmv_workspace(0)
        for _ in range(3):
            b.cmrs_spmv(M, x32, y, 0, ws)
        ts = time_steps(lambda: b.cmrs_spmv(M, x32, y, 0, ws), steps, flush, stream)
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


def main():
    args = args_parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
