"""The N > 1 host logic of bench.py on CPU: two gloo ranks, rendezvous on
127.0.0.1, barrier, max-over-ranks of the timing value, and the reference arm
doing no work on ranks other than 0."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    r, w, dist = bench.dist_setup(world)
    bench.barrier(dist)
    m = bench.max_over_ranks(dist, 1.5 * (rank + 1))
    bench.barrier(dist)
    if rank == 1:
        class A:
            steps, warmup, height, gpus = 3, 1, 4, 2
        bench.run_reference(A())  # returns at once: only rank 0 runs the reference arm
    q.put((r, w, m))
    dist.destroy_process_group()


def test_two_ranks_barrier_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 3.0), (1, 2, 3.0)]


def test_beta_plus_matches_eq_6_1():
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    for nnz, rows, strips, sv in [(55_742_968, 2_097_152, 524_288, 8), (20_224, 4_096, 1_024, 8)]:
        assert bench.beta_plus(nnz, rows, strips, sv) == oracle.beta(nnz, rows, strips, sv)[1]


def test_beta_minus_and_eta_match_eq_6_1():
    """The bench's beta- (input vector not cached) and eta+- follow Eq. 6.1 as the oracle states it."""
    import bench
    import oracle
    for nnz, rows, strips, sv in ((55742968, 2097152, 65536, 8), (21503218, 4194304, 131072, 4), (20224, 4096, 1024, 8)):
        bm, bp = oracle.beta(nnz, rows, strips, sv)
        assert bench.beta_minus(nnz, rows, strips, sv) == bm
        e = bench.eta(nnz, rows, strips, sv, 0.1, 1000.0)  # 0.1 ms, B = 1000 GB/s
        assert abs(e["eta_plus"] - bp / 1e-4 / 1e9 / 1000.0) < 1e-12
        assert abs(e["eta_minus"] - bm / 1e-4 / 1e9 / 1000.0) < 1e-12
        assert abs(e["beta_minus_gbs"] - bm / 1e-4 / 1e9) < 1e-9


def test_reference_arm_line_contract():
    """bench.py --impl reference: one JSON line timing the oracle on the host
    cores, with the keys of the benchmark line, its own cpu_baseline and an
    e2e block with no host-device copies (the 64x64 Laplacian: whole-matrix
    steps of microseconds)."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "laplacian", "--height", "4", "--steps", "3", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == "GB/s" and line["steps"] == 3 and line["warmup"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True and line["vs_baseline"] is None
    cb, e2e = line["cpu_baseline"], line["e2e"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
