"""The committed selector corpus and model, checked on the CPU: shapes, and
the held-out regret of the committed network recomputed with the oracle's
FP64 forward pass (tests/test_gpu_selector_regret.py retrains it on the GPU)."""
import json
import os

import numpy as np
import pytest

import oracle

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1203_2946_gb300", "data")


def _split(n, held_out=500, seed=0):
    perm = np.random.default_rng(seed).permutation(n)
    return np.sort(perm[held_out:]), np.sort(perm[:held_out])


def test_corpus_shapes_and_report():
    d = np.load(os.path.join(DATA, "selector_corpus.npz"))
    f, t = d["features"], d["times"]
    assert f.shape == (2000, 32) and t.shape == (2000, 21)
    assert np.isfinite(f).all() and (t > 0).all()
    specs = json.loads(str(d["specs"]))
    assert len(specs) == 2000 and {s["family"] for s in specs} >= {"stencil2d", "stencil3d", "banded", "blockdiag",
                                                                   "powerlaw", "uniform"}
    rep = json.load(open(os.path.join(DATA, "selector_report.json")))
    assert rep["count"] == 2000 and rep["held_out"] == 500
    assert rep["network"]["geomean"] <= 1.10 < rep["fixed_default_h4_row"]["geomean"]
    # the whole stated range: n from 1e4 to 2e6, 2 to 200 entries per row, no size cap
    sizes = d["sizes"]
    assert sizes.shape == (2000, 2) and rep["max_nnz"] is None
    assert sizes[:, 0].min() < 12_000 and sizes[:, 0].max() > 1_900_000
    mu = sizes[:, 1] / sizes[:, 0]
    assert mu.min() < 2.5 and mu.max() > 190 and sizes[:, 1].max() > 300_000_000
    assert rep["realised"]["nnz"] == [int(sizes[:, 1].min()), int(sizes[:, 1].max())]


def test_committed_model_regret_with_oracle_forward():
    d = np.load(os.path.join(DATA, "selector_corpus.npz"))
    m = np.load(os.path.join(DATA, "selector_model.npz"))
    nin, nh, nout = 32, int(m["nh"]), 21
    p = m["params"].astype(np.float64)
    sizes = [nh * nin, nh, nh * nh, nh, nout * nh, nout]
    parts = np.split(p, np.cumsum(sizes)[:-1])
    W1, b1, W2, b2, W3, b3 = (parts[0].reshape(nh, nin), parts[1], parts[2].reshape(nh, nh), parts[3],
                              parts[4].reshape(nout, nh), parts[5])
    X = (d["features"] - m["mean"].astype(np.float64)) * m["scale"].astype(np.float64)
    O = oracle.mlp_forward(X, W1, b1, W2, b2, W3, b3)["O"]
    times = d["times"]
    _, te = _split(len(times))
    choice = O[te].argmin(axis=1)
    r = times[te, choice] / times[te].min(axis=1)
    assert np.exp(np.mean(np.log(r))) <= 1.10


def test_model_file_checks(tmp_path):
    """load_model refuses an older format or a network of another width."""
    from paper_1203_2946_gb300 import selector
    m = dict(np.load(os.path.join(DATA, "selector_model.npz")))
    ok = selector.load_model(os.path.join(DATA, "selector_model.npz"), device="cpu")
    assert ok["params"].numel() == m["params"].size
    bad = dict(m, params=m["params"][:-3 * 65])  # 18 outputs
    np.savez(tmp_path / "narrow.npz", **bad)
    with pytest.raises(ValueError):
        selector.load_model(str(tmp_path / "narrow.npz"), device="cpu")
    old = dict(m, version=np.array(1))
    np.savez(tmp_path / "old.npz", **old)
    with pytest.raises(ValueError):
        selector.load_model(str(tmp_path / "old.npz"), device="cpu")
