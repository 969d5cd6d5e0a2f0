"""Multi-rank host logic on the CPU with gloo, world size 2: the benchmark's
max / sum reductions and barrier, the weak-scaling split of a workload into
disjoint per-rank batches of the same size, and the reference arm under
torchrun (rank 0 alone prints its line, every rank exits 0)."""
import json
import multiprocessing
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    try:
        out = {"max": bench.dist_max(float(rank + 1), 2), "sum": bench.dist_sum(float(rank + 1), 2)}
        bench.barrier(2)
        w = bench.make_workload("uneven10k", rank, quick=True)
        out["B"] = int(w.B)
        out["L"] = [int(x) for x in w.L]
        out["noise0"] = [float(x) for x in w.noise[0][:4]]
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_gloo_reductions_and_weak_scaling_split():
    pytest.importorskip("torch")
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=240) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0]["max"] == res[1]["max"] == 2.0
    assert res[0]["sum"] == res[1]["sum"] == 3.0
    # every rank fits its own batch of the same size: together the first 2B
    # saccades of the generator, disjoint
    assert res[0]["B"] == res[1]["B"] == 256
    full = W.uneven10k(B=512)
    assert res[0]["L"] == [int(x) for x in full.L[:256]]
    assert res[1]["L"] == [int(x) for x in full.L[256:]]
    np.testing.assert_array_equal(res[1]["noise0"], full.noise[256][:4])
    assert res[0]["noise0"] != res[1]["noise0"]


def test_reference_arm_under_torchrun_prints_one_line():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--quick", "--workload", "single10"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
