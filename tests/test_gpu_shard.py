"""Strip sharding on one GPU: every rank's share of the product built and
multiplied in turn (ShardedSpmv, its own CMRS conversion of its strips, x
given whole, as after the exchange), the rows put together and compared with
the oracle's product of the whole matrix element by element."""
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


def sharded_product(b, a, x, world, height, dtype, slots=None):
    from paper_1203_2946_gb300 import shard
    ys = []
    for rank in range(world):
        s = shard.ShardedSpmv(a, rank, world, height, dtype=dtype, slots=slots)
        s.x_full.copy_(torch.from_numpy(x))
        ys.append(s.product().cpu().numpy())
        assert ys[-1].shape == (s.r1 - s.r0,)
    return np.concatenate(ys)


@pytest.mark.parametrize("world", [2, 3, 8])
@pytest.mark.parametrize("case", ["stencil27", "powerlaw", "stencil27_padded"])
def test_sharded_product_matches_oracle(b, world, case):
    if case.startswith("stencil27"):
        a = inputs.stencil_3d_27pt(40, 40, 40, seed=1)
        height, slots = (32, 1) if case.endswith("padded") else (4, None)
    else:
        a = inputs.powerlaw_rows(200_000, 2.1, 30_000, seed=4)
        a = inputs.CSR(a.rows, a.cols, a.row_ptr, a.col_ind, a.val.astype(np.float64))
        height, slots = 32, None
    x = np.random.default_rng(world).uniform(-1, 1, a.cols)
    y = sharded_product(b, a, x, world, height, b.CMRS_F64, slots)
    yref, scale = orc.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    err = np.abs(y - yref)
    assert np.all(err <= 1e-12 * scale), float((err / np.maximum(scale, 1e-300)).max())


def test_sharded_product_more_parts_than_strips(b):
    a = inputs.random_csr(40, 40, 0.2, seed=3)
    x = np.random.default_rng(1).uniform(-1, 1, a.cols)
    y = sharded_product(b, a, x, 8, 16, b.CMRS_F64)  # 3 strips, 8 parts: 5 ranks hold no rows
    yref, scale = orc.csr_spmv(a.row_ptr, a.col_ind, a.val, x)
    assert np.all(np.abs(y - yref) <= 1e-12 * scale)


def test_bench_sharded_path_runs_and_checks(b):
    """bench.py's strip-sharded path (the one torchrun runs for N > 1), on one
    GPU with --shard: a JSON line with its row bounds, strong scaling, and
    the rank's product equal to the oracle's."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--shard", "--grid", "40", "--steps", "3",
                          "--warmup", "3", "--no-cpu"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["scaling"] == "strong" and line["n_gpus"] == 1
    assert line["config"]["row_bounds"] == [0, 40 ** 3]
    assert line["value"] > 0 and line["e2e"]["value"] > 0
    assert line["err_vs_f64_oracle_max_over_ranks"] <= 1e-12
