"""Strip sharding over several GPUs, its host logic on the CPU: the row
ranges of cmrs_shard_rows (whole strips, covering every row once, balanced),
and two or three gloo ranks that split a matrix, exchange their pieces of x
by broadcasts and multiply their rows (with the oracle standing in for the
device product), whose results put together equal the product of the whole
matrix bit for bit."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

from paper_1203_2946_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def b():
    from paper_1203_2946_gb300 import build
    build.build()
    from paper_1203_2946_gb300 import binding
    return binding


def weight(rp, r0, r1):
    return int(rp[r1] - rp[r0]) + (r1 - r0)


@pytest.mark.parametrize("maker", [
    lambda: inputs.powerlaw_rows(20000, 2.1, 5000, seed=3),
    lambda: inputs.stencil_3d_27pt(12, 12, 12, seed=1),
    lambda: inputs.random_csr(300, 300, 0.05, seed=2, empty_row_frac=0.5),
])
@pytest.mark.parametrize("height", [1, 4, 32])
@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_shard_rows_are_whole_strips_and_balanced(b, maker, height, parts):
    a = maker()
    bd = b.cmrs_shard_rows(a.row_ptr, height, parts)
    assert bd[0] == 0 and bd[-1] == a.rows and np.all(np.diff(bd) >= 0)
    assert all(int(x) % height == 0 for x in bd[1:-1] if x < a.rows)
    total = weight(a.row_ptr, 0, a.rows)
    strip_w = max(weight(a.row_ptr, s, min(s + height, a.rows)) for s in range(0, a.rows, height))
    for p in range(parts):
        # a part overshoots its share by at most the strip that crosses it
        assert weight(a.row_ptr, int(bd[p]), int(bd[p + 1])) <= -(-total // parts) + strip_w


def test_shard_rows_edge_cases(b):
    rp = np.array([0, 3, 3, 7], np.int32)
    assert list(b.cmrs_shard_rows(rp, 4, 3)) == [0, 3, 3, 3]  # one strip: the other parts are empty
    assert list(b.cmrs_shard_rows(np.array([0], np.int32), 4, 2)) == [0, 0, 0]
    with pytest.raises(b.CmrsError):
        b.cmrs_shard_rows(rp, 33, 2)
    with pytest.raises(b.CmrsError):
        b.cmrs_shard_rows(rp, 4, 0)
    with pytest.raises(b.CmrsError):
        b.cmrs_shard_rows(np.array([1, 3], np.int32), 4, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1203_2946_gb300 import binding as b, shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a = inputs.powerlaw_rows(30000, 2.1, 4000, seed=11)
    a = inputs.CSR(a.rows, a.cols, a.row_ptr, a.col_ind, a.val.astype(np.float64))
    x = inputs.uniform_vector(a.cols, 3)
    bounds = b.cmrs_shard_rows(a.row_ptr, 4, world)
    r0, r1 = int(bounds[rank]), int(bounds[rank + 1])
    x_full = torch.full((a.cols,), float("nan"), dtype=torch.float64)
    x_full[r0:r1] = torch.from_numpy(x[r0:r1])  # this rank's piece only
    shard.exchange_x(x_full, bounds)
    assert np.array_equal(x_full.numpy(), x)
    rp, ci, va = shard.local_rows(a.row_ptr, a.col_ind, a.val, r0, r1)
    y_local = oracle.csr_spmv(rp, ci, va, x_full.numpy())[0] if r1 > r0 else np.zeros(0)
    pieces = [None] * world
    dist.all_gather_object(pieces, (rank, y_local))
    if rank == 0:
        y = np.concatenate([p[1] for p in sorted(pieces, key=lambda t: t[0])])
        q.put(bool(np.array_equal(y, oracle.csr_spmv(a.row_ptr, a.col_ind, a.val, x)[0])))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_x_and_multiply_their_strips(b, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    same = q.get(timeout=180)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert same
