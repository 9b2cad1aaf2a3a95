"""The learned strip selector against the exhaustive sweep it replaces.

The committed corpus (paper_1203_2946_gb300/data/selector_corpus.npz) holds
the exhaustive timings (21 choices: 6 heights x 3 variants on plain CMRS and
3 padded forms) of 2,000 seeded matrices on a GB300 -- n from 1e4 to 2e6, 2
to 200 entries per row, up to 3.4e8 entries -- produced by
build_selector.py.  Here the network is retrained from scratch with the
library's own forward/backward/Adam kernels and judged on the 500 held-out
matrices: its regret t(choice)/t(best) must stay within 10% (geometric mean)
on all of them and on the large ones alone, and beat the method without it
-- the fixed default h = 4, ROW, and the best single fixed choice picked on
the training matrices.  On the 27-point 128^3 matrix (outside the corpus:
2.1M rows) the committed network's choice is timed against the fastest
padded form there."""
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1203_2946_gb300", "data")


@pytest.fixture(scope="module")
def corpus():
    from paper_1203_2946_gb300 import build
    build.build()
    d = np.load(os.path.join(DATA, "selector_corpus.npz"))
    return d["features"], d["times"], d["sizes"]


def choice_tuple(b, c):
    if c >= 18:
        return b.SEL_PADDED[c - 18][0], b.CMRS_VARIANT_PADDED, b.SEL_PADDED[c - 18][1]
    return b.SEL_HEIGHTS[c // 3], c % 3, 0


def test_retrained_network_regret_on_held_out(corpus):
    from paper_1203_2946_gb300 import selector
    feats, times, sizes = corpus
    assert feats.shape == (2000, 32) and times.shape == (2000, 21)
    tr, te = selector.split(len(times), 500, seed=0)
    model = selector.train(feats, times, tr, steps=4000)
    pred = selector.predict(model, feats[te])
    net = selector.regret(times[te], pred)
    big = sizes[te, 1] >= 2_000_000  # past the largest matrix of the earlier, capped corpus
    assert big.sum() >= 150
    assert selector.regret(times[te][big], pred[big])["geomean"] <= 1.10
    default = selector.regret(times[te], np.full(len(te), 3 * selector.HEIGHTS.index(4)))
    fixed = int(np.argmin(np.exp(np.mean(np.log(times[tr] / times[tr].min(1, keepdims=True)), axis=0))))
    single = selector.regret(times[te], np.full(len(te), fixed))
    assert net["geomean"] <= 1.10, net
    assert net["geomean"] < default["geomean"] and net["geomean"] < single["geomean"]
    assert net["median"] <= 1.01


def test_committed_model_through_select_strip(corpus):
    from paper_1203_2946_gb300 import binding as b, inputs, selector
    model = selector.load_model(os.path.join(DATA, "selector_model.npz"))
    feats, times, _ = corpus
    tr, te = selector.split(len(times), 500, seed=0)
    assert selector.regret(times[te], selector.predict(model, feats[te]))["geomean"] <= 1.10
    # the device path (features, normalisation, network, argmin in libcmrs)
    # picks a valid choice and agrees with the host-side prediction
    a = inputs.banded_random(50000, 700, 10, 60, seed=12)
    rp, ci = torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col_ind).cuda()
    h, v, m = b.cmrs_select_strip(rp, ci, a.cols, model)
    f = b.cmrs_features(rp, ci).cpu().numpy()[None, :]
    c = int(selector.predict(model, f)[0])
    assert (h, v, m) == choice_tuple(b, c)


def test_committed_model_on_the_27_point_128_cube(corpus):
    """The headline matrix lies outside the corpus (n = 2,097,152 > 2e6); the
    committed network's pick, timed in FP32 like the corpus, stays within 10%
    of the modified CMRS at (32, 1), the fastest form there."""
    from paper_1203_2946_gb300 import binding as b, inputs, selector
    model = selector.load_model(os.path.join(DATA, "selector_model.npz"))
    a = inputs.stencil_3d_27pt(128, 128, 128, seed=1, dtype=np.float32)
    rp, ci = torch.from_numpy(a.row_ptr).cuda(), torch.from_numpy(a.col_ind).cuda()
    va = torch.from_numpy(a.val).cuda()
    h, v, m = b.cmrs_select_strip(rp, ci, a.cols, model)
    timer = selector.Timer("cuda")
    x = torch.ones(a.cols, dtype=torch.float32, device="cuda")
    y = torch.empty(a.rows, dtype=torch.float32, device="cuda")

    def t_of(h, v, m):
        M = b.cmrs_from_csr(rp, ci, va, a.cols, h, dtype=b.CMRS_F32)
        if v == b.CMRS_VARIANT_PADDED:
            M = b.cmrs_pad(M, m)
        ws = M.spmv_workspace(v)
        return timer.time(lambda: b.cmrs_spmv(M, x, y, v, ws), reps=9)
    t_pick, t_ref = t_of(h, v, m), t_of(32, b.CMRS_VARIANT_PADDED, 1)
    assert t_pick <= 1.10 * t_ref, ((h, v, m), t_pick, t_ref)
