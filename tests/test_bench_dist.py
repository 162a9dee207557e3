"""The multi-process host logic of bench.py on CPU (gloo, world size 2): one
replica per rank with no data-path exchange; the timing is the maximum over
ranks and the work the sum over ranks; only rank 0 prints."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=2)
    try:
        mx = bench.max_over_ranks(1.5 + rank, dist)
        sm = bench.sum_over_ranks(1.0 + rank, dist)
        out.put((rank, mx, sm))
    finally:
        dist.destroy_process_group()


def test_max_and_sum_over_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2.5, 3.0), (1, 2.5, 3.0)]


def test_reference_arm_under_torchrun_prints_once():
    pytest.importorskip("torch")
    port = _free_port()
    env = dict(os.environ, BSQ_BENCH_BACKEND="gloo", MASTER_ADDR="127.0.0.1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3", "--grid", "48"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_bench_workload_grids():
    # the timed workloads and their grids: barred beach n x n, planar beach
    # n x n/4, rip-channel beach n x 3n/2 (1000 x 1500: the 0.02 m cells of Eq. 48's basin)
    sys.path.insert(0, ROOT)
    import bench

    assert bench.case_dims("barred_beach", 2048) == (2048, 2048)
    assert bench.case_dims("planar_beach", 1024) == (1024, 256)
    assert bench.case_dims("hamm_rip", 1000) == (1000, 1500)
    c = bench.make_case("hamm_rip", 100)
    p = c["params"]
    assert (p["nx"], p["ny"]) == (100, 150)
    assert abs(p["dx"] - 0.2) < 1e-12 and abs(p["dy"] - 0.2) < 1e-12
    assert c["comps"].shape == (68, 4) and p["friction"] == 0.0025
