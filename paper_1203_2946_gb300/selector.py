"""The learned strip selector: timing corpus, training, regret.

Section 6.2 of the paper picks the strip height by brute force and Section
6.7 reports what per-matrix tuning gains.  Here the brute force is this
library's exhaustive sweep (6 heights x 3 kernel variants, timed with CUDA
events on the device), and a small network trained on those timings predicts
the choice from 32 features of the matrix (cmrs_features).  Every numeric
step -- matrix generation for the corpus, features,
conversion, SpMV timing, the network's forward and backward passes and the
Adam updates -- runs in libcmrs kernels; this module only orchestrates.

Choice c < 18: plain CMRS, c = 3 * height_index + variant, height_index over
(1, 2, 4, 8, 16, 32), variant 0 ROW, 1 STRIP, 2 MERGE.  Choices 18, 19, 20:
the modified CMRS of Section 6.6 at (height, slots) = (32, 1), (32, 2),
(16, 8).  The network regresses the cost of every choice relative to the
best one, log2(t_c / t_best), and the smallest predicted cost wins.
"""
from __future__ import annotations

import json
import math
import statistics

import numpy as np
import torch

from . import binding as b

HEIGHTS = b.SEL_HEIGHTS
NCHOICE = b.SEL_CHOICES
NH = 64
FORMAT_VERSION = 3  # 3: 32 features; 2: 24 features, 21 choices (plain CMRS and three padded forms)


PADDED = b.SEL_PADDED
PAD_LIMIT = 2.0  # padded forms with more than twice the entries are not timed


def choice_name(c):
    if c >= 18:
        return "h=%d/padded-m%d" % PADDED[c - 18]
    return "h=%d/%s" % (HEIGHTS[c // 3], ("row", "strip", "merge")[c % 3])


# ----------------------------------------------------------------------------- timing
class Timer:
    """Times cmrs_spmv calls with CUDA events.  Before each call the L2 is
    flushed: a 256 MiB write, then a 256 MiB read, so that the call neither
    finds its operands in the L2 nor pays to write back the flush's dirty
    lines.  The median of at least `reps` calls is kept; short calls get more
    (up to `max_reps`, about 2 ms of calls in all), since a few microseconds
    of noise decide between choices there."""

    def __init__(self, device, flush_bytes=256 << 20):
        self.w = torch.empty(flush_bytes, dtype=torch.uint8, device=device)
        self.r = torch.ones(flush_bytes // 8, dtype=torch.int64, device=device)
        self.acc = torch.zeros(1, dtype=torch.int64, device=device)
        self.n = 0

    def flush(self):
        self.n += 1
        self.w.fill_(self.n & 0xFF)
        torch.sum(self.r, dim=0, keepdim=True, out=self.acc)

    def _run(self, fn, reps):
        st = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        torch.cuda._sleep(20_000_000)  # ~10 ms: the calls start on a busy GPU, enqueued ahead of it
        for i in range(reps):
            self.flush()
            st[i].record()
            fn()
            en[i].record()
        torch.cuda.synchronize()
        return [s.elapsed_time(e) for s, e in zip(st, en)]

    def time(self, fn, reps=5, warm=2, max_reps=25, budget_ms=2.0):
        for _ in range(warm):
            self.flush()
            fn()
        ts = self._run(fn, reps)
        more = min(max_reps, int(budget_ms / max(statistics.median(ts), 1e-3))) - reps
        if more > 0:
            ts += self._run(fn, more)
        return statistics.median(ts)


def time_all_choices(rows, cols, rp, ci, va, timer: Timer, reps=5):
    """Exhaustive sweep: ms per SpMV for each of the 21 choices (FP32 values;
    device CRS arrays rp, ci, va), and the matrix's features."""
    device = rp.device
    nnz = ci.numel()
    x = torch.ones(cols, dtype=torch.float32, device=device)
    y = torch.empty(rows, dtype=torch.float32, device=device)
    out = np.zeros(NCHOICE)
    for hi, h in enumerate(HEIGHTS):
        M = b.cmrs_from_csr(rp, ci, va, cols, h, dtype=b.CMRS_F32)
        for v in range(3):
            ws = M.spmv_workspace(v)
            out[3 * hi + v] = timer.time(lambda: b.cmrs_spmv(M, x, y, v, ws), reps=reps)
        for j, (ph, m) in enumerate(PADDED):
            if ph != h:
                continue
            P = b.cmrs_pad(M, m)
            if P.nnz > PAD_LIMIT * nnz + 32 * (rows // 16 + 2):
                out[18 + j] = -1.0  # not timed; set below
            else:
                ws = P.spmv_workspace(b.CMRS_VARIANT_PADDED)
                out[18 + j] = timer.time(lambda: b.cmrs_spmv(P, x, y, b.CMRS_VARIANT_PADDED, ws), reps=reps)
            del P
        del M
    out[out < 0] = 256.0 * out[out > 0].min()  # an untimed form: 2^8 times the best
    feat = b.cmrs_features(rp, ci).cpu().numpy()
    return feat, out


def build_corpus(specs, device="cuda", reps=5, log=None):
    """Features and exhaustive timings for every spec, each matrix generated
    on the device (corpus.device_matrix)."""
    from . import corpus
    timer = Timer(device)
    feats, times, sizes = [], [], []
    for i, spec in enumerate(specs):
        rows, cols, rp, ci, va = corpus.device_matrix(spec, device)
        f, t = time_all_choices(rows, cols, rp, ci, va, timer, reps)
        feats.append(f)
        times.append(t)
        sizes.append((rows, ci.numel()))
        del rp, ci, va
        if log and (i % 100 == 0 or i == len(specs) - 1):
            log("corpus %d/%d  n=%d nnz=%d best=%s" % (i + 1, len(specs), rows, sizes[-1][1],
                                                     choice_name(int(t.argmin()))))
    return np.array(feats), np.array(times), np.array(sizes, dtype=np.int64)


# ----------------------------------------------------------------------------- network
def init_params(seed=0, nin=b.NFEAT, nh=NH, nout=NCHOICE):
    """He-normal weights, zero biases (layout of cmrs_mlp_*)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, math.sqrt(2.0 / nin), (nh, nin)), np.zeros(nh),
             rng.normal(0, math.sqrt(2.0 / nh), (nh, nh)), np.zeros(nh),
             rng.normal(0, math.sqrt(1.0 / nh), (nout, nh)), np.zeros(nout)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def train(features, times, idx, steps=3000, batch=256, lr=2e-3, seed=0, device="cuda", log=None, cap=1.0):
    """Trains on rows `idx` with the library's forward/backward/Adam kernels.
    Targets: log2(t_c / t_best) capped at `cap`; the default, 1, calls every
    choice more than twice as slow as the best simply slow, so that the
    network spends itself on ranking the near-best ones (held-out regret on
    the full-range corpus, same network and steps: 1.0071 with a cap of 8,
    1.0044 with 1)."""
    if times.shape[1] != NCHOICE or features.shape[1] != b.NFEAT:
        raise ValueError("timings must have %d choices and features %d columns" % (NCHOICE, b.NFEAT))
    # inputs normalised by the training rows' statistics, and the capped
    # relative costs, both computed by the library on the device
    mean, scale, X = b.cmrs_feature_norm(torch.from_numpy(np.ascontiguousarray(features[idx], np.float64)).to(device))
    T = b.cmrs_cost_targets(torch.from_numpy(np.ascontiguousarray(times[idx], np.float64)).to(device), cap)
    P = torch.from_numpy(init_params(seed)).to(device)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    n = X.shape[0]
    rng = np.random.default_rng(seed + 1)
    B = min(batch, n)
    acts = torch.empty(B * (4 * NH + NCHOICE), dtype=torch.float32, device=device)
    grads = torch.empty_like(P)
    scratch = torch.empty(B * (NCHOICE + 2 * NH), dtype=torch.float32, device=device)
    loss = torch.empty(1, dtype=torch.float32, device=device)
    history = []
    for step in range(1, steps + 1):
        sel = torch.from_numpy(rng.choice(n, B, replace=False)).to(device)
        xb, tb = X.index_select(0, sel).contiguous(), T.index_select(0, sel).contiguous()
        b.cmrs_mlp_forward(xb, P, NH, NCHOICE, acts)
        b.cmrs_mlp_backward(xb, tb, P, acts, NH, NCHOICE, grads, scratch, loss)
        b.cmrs_mlp_adam(P, grads, m, v, step, lr)
        if step % 250 == 0 or step == 1:
            history.append((step, float(loss.item())))
            if log:
                log("train step %d loss %.5f" % history[-1])
    return {"params": P, "mean": mean, "scale": scale, "nh": NH, "history": history}


def predict(model, features, device="cuda"):
    X = b.cmrs_feature_apply(torch.from_numpy(np.ascontiguousarray(features, np.float64)).to(device),
                             model["mean"].to(device), model["scale"].to(device))
    acts = b.cmrs_mlp_forward(X, model["params"], model["nh"], NCHOICE)
    return b.mlp_output(acts, X.shape[0], model["nh"], NCHOICE).argmin(dim=1).cpu().numpy()


def regret(times, choice):
    r = times[np.arange(times.shape[0]), choice] / times.min(axis=1)
    return {"geomean": float(np.exp(np.mean(np.log(r)))), "median": float(np.median(r)),
            "p90": float(np.percentile(r, 90)), "max": float(r.max()),
            "within_10pct": float(np.mean(r <= 1.10))}


def split(n, held_out=500, seed=0):
    perm = np.random.default_rng(seed).permutation(n)
    return np.sort(perm[held_out:]), np.sort(perm[:held_out])


def save_model(model, path, extra=None):
    np.savez(path, params=model["params"].cpu().numpy(), mean=model["mean"].cpu().numpy(),
             scale=model["scale"].cpu().numpy(), nh=model["nh"], version=FORMAT_VERSION,
             extra=json.dumps(extra or {}))


def load_model(path, device="cuda"):
    d = np.load(path)
    if int(d["version"]) != FORMAT_VERSION:
        raise ValueError("selector model format %d, expected %d" % (int(d["version"]), FORMAT_VERSION))
    nh = int(d["nh"])
    want = nh * b.NFEAT + nh + nh * nh + nh + NCHOICE * nh + NCHOICE
    if d["params"].size != want or d["mean"].size != b.NFEAT or d["scale"].size != b.NFEAT:
        raise ValueError("selector model does not match %d features and %d choices" % (b.NFEAT, NCHOICE))
    return {"params": torch.from_numpy(d["params"]).to(device), "mean": torch.from_numpy(d["mean"]).to(device),
            "scale": torch.from_numpy(d["scale"]).to(device), "nh": int(d["nh"])}
