"""Host logic of bench.py that needs no GPU: the max-over-ranks reduction used for
N replicas (gloo, world size 2, on CPU) and the reference arm's sample setup."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.reduce_max(10.0 + rank * 5.0, dist)
    out.put((rank, v))
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    import multiprocessing as mp
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == {0: 15.0, 1: 15.0}


def test_reduce_max_without_group_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, None) == 3.5


def test_reference_arm_runs_on_the_small_workload():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "wave_dirichlet_4x4_p12_N21", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_plan_levels_match_the_library_plan():
    """bench.py's level sizes (for the algorithmic flops and bytes of the
    rooflines) against the library's own tree plan, seen through the operator
    memory it reports: per pole, ZU and S blocks of every merge level."""
    sys.path.insert(0, ROOT)
    import bench
    lv = bench.plan_levels(16, 16, 14)
    assert [l["nbox"] for l in lv] == [128, 64, 32, 16, 8, 4, 2, 1]
    assert [l["n3"] for l in lv] == [14, 28, 28, 56, 56, 112, 112, 224]
    assert [l["nbd"] for l in lv] == [84, 112, 168, 224, 336, 448, 672, 896]
    # rectangular grid: merges along x until one column remains, then along y
    lv = bench.plan_levels(4, 1, 6)
    assert [l["nbox"] for l in lv] == [2, 1]
    assert [l["n3"] for l in lv] == [6, 6]
    assert lv[-1]["nbd"] == 2 * (4 + 1) * 6


def test_class_work_counts_for_the_shallow_water_workload():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W

    class Op:
        alpha = 4.5 + 1j * __import__("numpy").arange(-2878, 2879)     # one line, 2879 with Im >= 0
    w = W.SW_16X16_P16
    work = bench.class_work(Op(), w, 1, "df32", fd=True)
    P, q = 2879, 14
    # fast-diagonal leaves: (4K + 32) q^2 flops per (pole, leaf, rhs), K = 3
    assert work["up_leaf"][0] == (4 * 3 + 32) * q * q * P * 256
    # root wall solve: one complex multiply-add per entry of the 896 x 896 block
    assert work["root"][0] == 8.0 * P * 896 * 896
    assert work["root"][1] == P * 896 * 896 * 16 + P * 2 * 896 * 16
    # the four Fourier blocks of the square domain: a quarter of the entries
    w4 = bench.class_work(Op(), w, 1, "df32", fd=True, root_c4=True)
    assert w4["root"][0] == 8.0 * P * 4 * 224 * 224
    assert w4["root"][1] == P * 4 * 224 * 224 * 16 + P * 2 * 896 * 16
    # top up merge: ZU has n3 + nbd rows and n3 columns
    assert work["up_merge"][0] > 8.0 * P * (224 + 896) * 224


def test_all_core_oracle_baseline_runs_one_process_per_core():
    # the all-core CPU baseline: spawned processes, single-threaded BLAS, one distinct
    # pole each, throughput scaled to applies/s (small wave workload, short budget)
    import types
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    from oracle import sem
    w = W.WAVE_4X4_P12
    op = types.SimpleNamespace(alpha=4.5 + 1j * np.arange(-3, 4), b=np.ones(7, complex), tau=0.01)
    og = sem.Grid(w.nlx, w.nly, w.p)
    u0 = np.zeros((2, og.n_nodes))
    u0[1] = 1.0
    r = bench.cpu_baseline_all_cores(w, op, u0, budget_s=0.3, max_workers=2)
    assert r["kind"] == "oracle" and r["cores"] == min(2, os.cpu_count()) and r["value"] > 0
    assert "4 distinct poles" in r["sample"]
    assert os.environ["OPENBLAS_NUM_THREADS"] == "1"
