"""GPU parity for the batched SpMM and the strip selector.

SpMM: every column of Y against the oracle's FP64 CRS SpMV of the FP32
values and that column of X, within (len_i + 2) * 2^-24 * (|A||x_col|)_i.
Selector: device features against the oracle's features (same integer sums,
rel. 1e-12); FP32 network forward, gradients and Adam step against the FP64
oracle network (whose gradients are pinned by finite differences)."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1203_2946_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding
    return binding


def to_dev(a):
    return (torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col_ind).cuda(),
            torch.from_numpy(np.ascontiguousarray(a.val, dtype=np.float32)).cuda())


def check_spmm(a, X, Y, rows=None):
    Y = Y.cpu().numpy() if torch.is_tensor(Y) else Y
    X = X.cpu().numpy() if torch.is_tensor(X) else X
    v = a.val.astype(np.float32).astype(np.float64)
    L = np.diff(a.row_ptr)
    for c in range(X.shape[1]):
        y, s = orc.csr_spmv(a.row_ptr, a.col_ind, v, X[:, c].astype(np.float64))
        err = np.abs(Y[:, c].astype(np.float64) - y)
        tol = (L + 2) * 2.0**-24 * s
        assert (err <= tol).all(), (c, np.nonzero(err > tol)[0][:5])


@pytest.mark.parametrize("k", [1, 3, 4, 8, 32, 40])
@pytest.mark.parametrize("h", [1, 4, 32])
def test_spmm_single(b, k, h):
    a = inputs.banded_random(3001, 300, 10, 60, seed=k + h)
    rp, ci, va = to_dev(a)
    M = b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=b.CMRS_F32)
    X = torch.from_numpy(np.random.default_rng(k).standard_normal((a.cols, k)).astype(np.float32)).cuda()
    check_spmm(a, X, b.cmrs_spmm(M, X))


def small_batch(b, count=24, seed=3):
    rng = np.random.default_rng(seed)
    mats, Xs, Ys, host = [], [], [], []
    for i in range(count):
        n = int(rng.integers(500, 20000))
        a = inputs.banded_random(n, int(rng.integers(64, 2049)), 10, 60, seed=int(rng.integers(1 << 30)))
        k = int(rng.choice([1, 4, 8, 32, 5]))
        h = int(rng.choice([1, 4, 16]))
        rp, ci, va = to_dev(a)
        mats.append(b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=b.CMRS_F32))
        X = np.random.default_rng(i).standard_normal((a.cols, k)).astype(np.float32)
        Xs.append(torch.from_numpy(X).cuda())
        Ys.append(torch.full((a.rows, k), float("nan"), dtype=torch.float32, device="cuda"))
        host.append((a, X))
    return mats, Xs, Ys, host


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("target", [512, 8192, 1 << 20])
def test_spmm_batched(b, use_graph, target):
    mats, Xs, Ys, host = small_batch(b)
    plan = b.SpmmPlan(mats, Xs, Ys, work_target=target, use_graph=use_graph)
    b.cmrs_spmm_batched(plan)
    first = [Y.clone() for Y in Ys]
    for (a, X), Y in zip(host, Ys):
        check_spmm(a, X, Y)
    for Y in Ys:
        Y.fill_(float("nan"))
    b.cmrs_spmm_batched(plan)
    for Y, F in zip(Ys, first):
        assert torch.equal(Y, F)  # replays are bit-identical
    assert plan.info()["units"] >= len(mats)
    plan.close()


def _batched_member(spec):
    """One matrix of the 256-matrix banded batch, and the oracle's FP64 values
    (with |A||x|) of a sample of its rows for every column of its X: the first
    and last rows, rows on both sides of a strip edge, and random rows.  Runs
    in a spawned worker."""
    a, X = inputs.batched_banded(spec)
    n = a.rows
    rng = np.random.default_rng(spec["seed"] + 2)
    rows = np.unique(np.concatenate([[0, 1, 3, 4, n - 2, n - 1], rng.integers(0, n, 58)]))
    lens = np.diff(a.row_ptr)[rows]
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    idx = np.concatenate([np.arange(a.row_ptr[r], a.row_ptr[r + 1]) for r in rows])
    ci, v = a.col_ind[idx], a.val[idx].astype(np.float32).astype(np.float64)
    ref = np.empty((rows.size, X.shape[1]))
    scale = np.empty_like(ref)
    for c in range(X.shape[1]):
        ref[:, c], scale[:, c] = orc.csr_spmv(rp, ci, v, X[:, c].astype(np.float64))
    return a.row_ptr, a.col_ind, a.val, X, rows, ref, scale, lens


def test_spmm_batched_full_size(b):
    """The batched workload at full size: 256 banded-random matrices (n
    1,000..200,000, bandwidth 64..2,048, 10..60 entries per row, k in
    {1, 4, 8, 32}), in the configuration the benchmark times: each matrix's
    strip height and the work-unit size autotuned, one graph-captured
    persistent launch.  Sampled rows of every matrix (64 each: the first, the
    last, both sides of a strip edge, random ones), every right-hand side,
    against the FP64 oracle; every row written; a second replay
    bit-identical."""
    from paper_1203_2946_gb300 import batch
    import multiprocessing as mp
    import os
    orc.lib()  # built before the workers load it
    specs = inputs.batched_banded_specs()
    assert len(specs) == 256
    with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        parts = pool.map(_batched_member, specs, chunksize=4)
    csrs, Xs, Ys = [], [], []
    for rp, ci, val, X, *_ in parts:
        n = rp.size - 1
        csrs.append((torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(val).cuda()))
        Xs.append(torch.from_numpy(X).cuda())
        Ys.append(torch.empty((n, X.shape[1]), dtype=torch.float32, device="cuda"))
    mats, heights, best, _, table = batch.tune(csrs, Xs, Ys)
    del csrs
    assert sum(M.nnz for M in mats) > 500_000_000
    assert all(M.height == h and t[batch.HEIGHTS.index(h)] == min(t) for M, h, t in zip(mats, heights, table))
    plan = b.SpmmPlan(mats, Xs, Ys, work_target=best, use_graph=True)
    for Y in Ys:
        Y.fill_(float("nan"))
    b.cmrs_spmm_batched(plan)
    got = []
    for Y, p in zip(Ys, parts):
        assert not torch.isnan(Y).any()
        got.append(Y[torch.from_numpy(p[4]).cuda()].cpu().numpy())
    for Y in Ys:
        Y.fill_(float("nan"))
    b.cmrs_spmm_batched(plan)
    for i, (Y, p, g) in enumerate(zip(Ys, parts, got)):
        rows, ref, scale, lens = p[4], p[5], p[6], p[7]
        assert np.array_equal(Y[torch.from_numpy(rows).cuda()].cpu().numpy(), g)
        tol = (lens[:, None] + 2) * 2.0**-24 * scale
        err = np.abs(g.astype(np.float64) - ref)
        assert (err <= tol).all(), (i, np.argwhere(err > tol)[:5])
    plan.close()


def test_schedule_autotuner_small_batch(b):
    """batch.tune: every matrix converted at the height whose single launch
    timed fastest, a work target from the candidates, and the plan built on
    that schedule gives the right product for every matrix."""
    from paper_1203_2946_gb300 import batch
    _, Xs, Ys, host = small_batch(b, 10, seed=9)
    csrs = [to_dev(a) for a, _ in host]
    mats, heights, best, ms, table = batch.tune(csrs, Xs, Ys, heights=(1, 4, 16), work_targets=(1024, 16384))
    assert best in (1024, 16384) and ms > 0 and len(table) == len(mats) == 10
    for M, h, t in zip(mats, heights, table):
        assert h in (1, 4, 16) and M.height == h and t[(1, 4, 16).index(h)] == min(t)
    plan = b.SpmmPlan(mats, Xs, Ys, work_target=best)
    for Y in Ys:
        Y.fill_(float("nan"))
    b.cmrs_spmm_batched(plan)
    for (a, X), Y in zip(host, Ys):
        check_spmm(a, X, Y)
    plan.close()


def test_spmm_autotune(b):
    mats, Xs, Ys, host = small_batch(b, 12, seed=5)
    best, ms = b.cmrs_spmm_autotune(mats, Xs, Ys, candidates=(1024, 16384), reps=3)
    assert best in (1024, 16384) and ms > 0
    plan = b.SpmmPlan(mats, Xs, Ys, work_target=best)
    b.cmrs_spmm_batched(plan)
    for (a, X), Y in zip(host, Ys):
        check_spmm(a, X, Y)


def test_spmm_rejects_f64_and_sorted(b):
    a = inputs.banded_random(1000, 100, seed=1)
    rp, ci, va = to_dev(a)
    M = b.cmrs_from_csr(rp, ci, va.double(), a.cols, 4, dtype=b.CMRS_F64)
    X = torch.zeros((a.cols, 4), device="cuda")
    with pytest.raises(b.CmrsError) as e:
        b.cmrs_spmm(M, X)
    assert e.value.code == 6
    S = b.cmrs_from_csr(rp, ci, va, a.cols, 4, flags=b.CMRS_SORTED, dtype=b.CMRS_F32)
    with pytest.raises(b.CmrsError):
        b.cmrs_spmm(S, X)


# ----------------------------------------------------------------------------- selector
@pytest.mark.parametrize("maker", [
    lambda: inputs.workload_laplacian_64()[0],
    lambda: inputs.random_csr(3000, 2000, 0.003, seed=2, empty_row_frac=0.2),
    lambda: inputs.powerlaw_rows(40000, 2.1, 5000, seed=1),
    lambda: inputs.block_diagonal(5000, 7, seed=1),
    lambda: inputs.stencil_3d_27pt(20, 20, 20, seed=1),
])
def test_features_match_oracle(b, maker):
    a = maker()
    rp, ci, _ = to_dev(a)
    f = b.cmrs_features(rp, ci).cpu().numpy()
    ref = orc.features(a.row_ptr, a.col_ind)
    assert np.allclose(f, ref, rtol=1e-12, atol=1e-12), np.abs(f - ref).max()


def _net(rng, nin=24, nh=64, nout=18):
    return [rng.normal(0, 0.3, (nh, nin)), rng.normal(0, 0.1, nh), rng.normal(0, 0.15, (nh, nh)),
            rng.normal(0, 0.1, nh), rng.normal(0, 0.15, (nout, nh)), rng.normal(0, 0.1, nout)]


def test_mlp_forward_backward_adam_vs_oracle(b):
    rng = np.random.default_rng(0)
    W1, b1, W2, b2, W3, b3 = _net(rng)
    B = 37
    X = rng.normal(0, 1, (B, 24))
    T = rng.normal(0, 1, (B, 18))
    flat = np.concatenate([p.ravel() for p in (W1, b1, W2, b2, W3, b3)]).astype(np.float32)
    assert b.mlp_param_count(24, 64, 18) == flat.size
    P = torch.from_numpy(flat).cuda()
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    acts = b.cmrs_mlp_forward(Xd, P, 64, 18)
    O = b.mlp_output(acts, B, 64, 18).cpu().numpy()
    # the oracle on the FP32-rounded parameters and inputs
    p32 = [p.astype(np.float32).astype(np.float64) for p in (W1, b1, W2, b2, W3, b3)]
    loss, g, fw = orc.mlp_loss_grad(X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64),
                                    *p32)
    assert np.allclose(O, fw["O"], rtol=1e-4, atol=1e-4)
    grads, dl = b.cmrs_mlp_backward(Xd, Td, P, acts, 64, 18)
    assert abs(float(dl.item()) - loss) <= 1e-4 * abs(loss)
    ref = np.concatenate([g[n].ravel() for n in ("W1", "b1", "W2", "b2", "W3", "b3")])
    got = grads.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-3 * scale
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 1e-4
    # one Adam step against the oracle's
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    b.cmrs_mlp_adam(P, grads, m, v, 1, 1e-3)
    p64 = flat.astype(np.float64)
    m64, v64 = np.zeros_like(p64), np.zeros_like(p64)
    orc.adam_step(p64, got, m64, v64, 1, 1e-3)
    assert np.allclose(P.cpu().numpy(), p64, rtol=0, atol=2e-6)


def test_feature_norm_and_cost_targets(b):
    """The training data the library prepares on the device: per-feature
    mean and 1/std over the rows (0 for a constant feature), the normalised
    FP32 inputs, and the capped log2 costs relative to each row's best."""
    rng = np.random.default_rng(3)
    F = rng.normal(5.0, 3.0, (300, b.NFEAT))
    F[:, 7] = 2.5  # constant: leaves the input
    mean, scale, X = b.cmrs_feature_norm(torch.from_numpy(F).cuda())
    m_ref, s_ref = F.mean(0), F.std(0)
    assert np.allclose(mean.cpu().numpy(), m_ref.astype(np.float32), rtol=1e-6, atol=1e-6)
    sc = scale.cpu().numpy()
    assert sc[7] == 0.0
    keep = np.arange(b.NFEAT) != 7
    assert np.allclose(sc[keep], (1.0 / s_ref[keep]).astype(np.float32), rtol=1e-6)
    ref = (F.astype(np.float32) - mean.cpu().numpy()) * sc
    assert np.allclose(X.cpu().numpy(), ref, rtol=1e-6, atol=1e-6)
    assert torch.equal(b.cmrs_feature_apply(torch.from_numpy(F).cuda(), mean, scale), X)
    t = rng.uniform(0.01, 5.0, (200, 21))
    T = b.cmrs_cost_targets(torch.from_numpy(t).cuda(), 1.0).cpu().numpy()
    want = np.minimum(np.log2(t / t.min(1, keepdims=True)), 1.0)
    assert np.allclose(T, want.astype(np.float32), rtol=1e-6, atol=1e-7)
    assert (T.min(1) == 0.0).all() and T.max() <= 1.0


def test_training_reduces_loss(b):
    from paper_1203_2946_gb300 import selector
    rng = np.random.default_rng(1)
    feats = rng.normal(0, 1, (300, b.NFEAT))
    # synthetic costs with a learnable structure: the best choice depends on the features
    w = rng.normal(0, 1, (b.NFEAT, selector.NCHOICE))
    times = np.exp(0.3 * np.tanh(feats @ w))
    idx = np.arange(300)
    model = selector.train(feats, times, idx, steps=600, batch=128, lr=3e-3)
    hist = model["history"]
    assert hist[-1][1] < 0.5 * hist[0][1]
    pred = selector.predict(model, feats)
    assert selector.regret(times, pred)["geomean"] < selector.regret(times, np.full(300, 6))["geomean"]


def test_select_strip_exhaustive_and_model(b):
    from paper_1203_2946_gb300 import selector
    a = inputs.banded_random(20000, 500, 10, 60, seed=4)
    rp, ci, _ = to_dev(a)
    h, v, m = b.cmrs_select_strip(rp, ci, a.cols, None)
    assert h in b.SEL_HEIGHTS and (v in (0, 1, 2) and m == 0 or (h, m) in b.SEL_PADDED and v == b.CMRS_VARIANT_PADDED)
    model = {"params": torch.from_numpy(selector.init_params(3)).cuda(), "mean": torch.zeros(b.NFEAT).cuda(),
             "scale": torch.full((b.NFEAT,), 0.1).cuda(), "nh": 64}
    h2, v2, m2 = b.cmrs_select_strip(rp, ci, a.cols, model)
    # the device argmin agrees with the host-side prediction of the same network
    f = b.cmrs_features(rp, ci).cpu().numpy()[None, :]
    c = int(selector.predict(model, f)[0])
    want = ((b.SEL_PADDED[c - 18][0], b.CMRS_VARIANT_PADDED, b.SEL_PADDED[c - 18][1]) if c >= 18
            else (b.SEL_HEIGHTS[c // 3], c % 3, 0))
    assert (h2, v2, m2) == want
