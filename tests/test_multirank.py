"""The N > 1 path of bench.py on the CPU: two gloo ranks.  Queries are independent,
so every rank answers its own batch against its own replica of the index
(no collective on the data path); the only collective is the max over ranks of
the timed region, and the whole-job rate counts every rank's queries."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, X, Qs = bench.workload(rank, n_override=500, q_override=40)
        t = bench.max_over_ranks(1.0 + 0.5 * rank, dist)  # rank 1 is the slower one
        out.put((rank, X[:4].tolist(), Qs[:4].tolist(), t, bench.whole_job_rate(40, world, 3, t)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_own_batches_and_the_slowest_rank_times_the_job():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, x0, q0, t0, v0), (r1, x1, q1, t1, v1) = res
    assert (r0, r1) == (0, 1)
    assert x0 == x1  # the same points (each rank builds the same index)
    assert q0 != q1  # its own queries
    assert t0 == t1 == 1.5  # max over ranks
    assert v0 == v1 == 40 * 2 * 3 / 1.5


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.whole_job_rate(10, 1, 4, 2.0) == 20.0


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--points", "3000", "--queries", "60",
           "--budget", str(16 << 20)]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["value"] == d["value"]


def test_traffic_summary_only_for_the_profiled_workload():
    sys.path.insert(0, ROOT)
    import bench

    base = dict(points=None, queries=None, budget=None, mode="learned", train_queries=100_000, epochs=20, recall=0.9)
    import argparse

    for key, other in (("points", 5000), ("queries", 100), ("budget", 1 << 30), ("mode", "bf16"),
                       ("train_queries", 20_000), ("epochs", 5), ("recall", 0.95)):
        a = argparse.Namespace(**dict(base, **{key: other}))
        assert bench.search_kernel_traffic(a) is None, key
    # the default workload gets the committed figure while the source is unchanged
    # (or None once the kernel differs from the profiled one)
    v = bench.search_kernel_traffic(argparse.Namespace(**base))
    assert v is None or v > 1e10


def test_synthetic_workload_host_side():
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np

    w, X, Qs = bench.workload(0, n_override=25_000, q_override=8, name="paper-synthetic-n1m-d300")
    assert X.shape == (25_000, 300) and Qs.shape == (8, 300) and w["k"] == 10 and w["recall"] == 0.99
    # another rank: other queries of the same construction (same v)
    _, _, Q1 = bench.workload(1, n_override=25_000, q_override=8, name="paper-synthetic-n1m-d300")
    assert np.array_equal(Q1[:, :100], Qs[:, :100]) and not np.array_equal(Q1, Qs)
    assert bench.METRICS["paper-synthetic-n1m-d300"].startswith("k-NN queries/s")


def test_cpu_baseline_reports_all_cores_and_one_thread():
    sys.path.insert(0, ROOT)
    import bench

    w, X, Qs = bench.workload(0, n_override=4000, q_override=40)
    cpu = bench.cpu_baseline(w, X, Qs, 12, 10, 0.9, q_target_s=0.5, single_target_s=0.3)
    assert cpu["kind"] == "oracle" and cpu["value"] > 0 and cpu["cores"] >= 1
    assert "all 4,000 points" in cpu["sample"] and cpu["build_s"] > 0
    st = cpu["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and "one after another" in st["sample"]
