"""Builds the strip selector on the current GPU.

1. Corpus: `count` seeded synthetic matrices (families stencil 2D/3D, banded
   random, block diagonal, power-law rows, uniform random; n log-uniform in
   [1e4, 2e6]; target nnz/row log-uniform in [2, 200]; no size cap unless
   --max-nnz is given), each generated on the device and timed by the
   exhaustive sweep of the 21 choices (6 heights x 3 variants on plain CMRS,
   3 padded forms; FP32 values, L2 flushed, median of at least --reps calls).
2. Training: the network of selector.py on all but the --held-out matrices,
   with the library's forward / backward / Adam kernels.
3. Report: regret on the held-out matrices -- t(choice) / t(best of sweep),
   geometric mean, median, p90, max -- for the network, for the fixed default
   (h = 4, ROW) and for the best single fixed choice picked on the training
   set, with the realised ranges of rows and entries.

  python -m paper_1203_2946_gb300.build_selector --out paper_1203_2946_gb300/data
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=2000)
    ap.add_argument("--held-out", type=int, default=500)
    ap.add_argument("--max-nnz", type=int, default=None)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--cap", type=float, default=1.0, help="cap of the log2 cost targets")
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "data"))
    ap.add_argument("--corpus", default=None, help="reuse an existing corpus .npz instead of timing")
    a = ap.parse_args(argv)

    from . import inputs, selector
    import torch

    os.makedirs(a.out, exist_ok=True)
    log = lambda s: print("[%7.1fs] %s" % (time.time() - t0, s), flush=True)  # noqa: E731
    t0 = time.time()
    specs = inputs.selector_family_specs(a.count, seed=a.seed, max_nnz=a.max_nnz)
    corpus_path = os.path.join(a.out, "selector_corpus.npz")
    if a.corpus:
        d = np.load(a.corpus)
        feats, times, sizes = d["features"], d["times"], d["sizes"]
    else:
        feats, times, sizes = selector.build_corpus(specs, reps=a.reps, log=log)
        np.savez_compressed(corpus_path, features=feats, times=times, sizes=sizes, specs=json.dumps(specs),
                            device=torch.cuda.get_device_name(0), reps=a.reps)
        log("corpus written: %s" % corpus_path)
    train_idx, test_idx = selector.split(len(times), a.held_out, seed=0)
    model = selector.train(feats, times, train_idx, steps=a.steps, lr=a.lr, log=log, cap=a.cap)
    pred = selector.predict(model, feats[test_idx])
    default = 3 * selector.HEIGHTS.index(4) + 0
    fixed_best = int(np.argmin(np.exp(np.mean(np.log(times[train_idx] / times[train_idx].min(1, keepdims=True)),
                                              axis=0))))
    fam = np.array([s["family"] for s in specs])[test_idx]
    report = {
        "device": torch.cuda.get_device_name(0),
        "count": int(len(times)), "held_out": int(len(test_idx)), "reps": a.reps, "max_nnz": a.max_nnz,
        "realised": {"rows": [int(sizes[:, 0].min()), int(sizes[:, 0].max())],
                     "nnz": [int(sizes[:, 1].min()), int(sizes[:, 1].max())],
                     "nnz_per_row": [float((sizes[:, 1] / sizes[:, 0]).min()),
                                     float((sizes[:, 1] / sizes[:, 0]).max())],
                     "total_nnz": int(sizes[:, 1].sum())},
        "training": {"steps": a.steps, "lr": a.lr, "cap": a.cap},
        "train_loss": model["history"],
        "network": selector.regret(times[test_idx], pred),
        "fixed_default_h4_row": selector.regret(times[test_idx], np.full(len(test_idx), default)),
        "fixed_best_single": {"choice": selector.choice_name(fixed_best),
                              **selector.regret(times[test_idx], np.full(len(test_idx), fixed_best))},
        "best_choice_histogram": {selector.choice_name(c): int(n) for c, n in
                                  zip(*np.unique(times.argmin(1), return_counts=True))},
        "network_by_family": {f: selector.regret(times[test_idx][fam == f], pred[fam == f])
                              for f in sorted(set(fam))},
    }
    big = sizes[test_idx, 1] >= 2_000_000
    if big.any():
        report["network_nnz_2M_and_more"] = selector.regret(times[test_idx][big], pred[big])
        report["network_nnz_under_2M"] = selector.regret(times[test_idx][~big], pred[~big])
    selector.save_model(model, os.path.join(a.out, "selector_model.npz"), extra={"report": "selector_report.json"})
    with open(os.path.join(a.out, "selector_report.json"), "w") as f:
        json.dump(report, f, indent=1)
    log(json.dumps({k: report[k] for k in ("network", "fixed_default_h4_row", "fixed_best_single", "realised")}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
