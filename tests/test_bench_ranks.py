"""Multi-rank logic of bench.py on CPU (gloo, world size 2): barrier, the
slowest rank's time, the whole-job rate under weak scaling, and the reference
arm doing nothing on ranks other than 0. The GPU path of the bench runs one
replica per rank with no data-path collective, so this is all that N > 1 adds."""
import json
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.rank_barrier(dist, torch, cuda=False)
    t = bench.rank_max(dist, torch, 1.0 + rank, "cpu")            # rank r "took" 1 + r seconds
    rate = bench.whole_job_rate(32, world, t)
    class A:  # the reference arm's arguments
        gpus, steps, warmup = world, 1, 0
    rc = bench.run_reference(A(), rank) if rank != 0 else None  # rank 0 would time the oracle
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max": t, "rate": rate, "ref_rc": rc}, f)
    dist.destroy_process_group()


def test_two_ranks_gloo(tmp_path):
    port = free_port()
    mp.start_processes(worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    r0 = json.load(open(tmp_path / "r0.json"))
    r1 = json.load(open(tmp_path / "r1.json"))
    assert r0["max"] == r1["max"] == 2.0                # every rank sees the slowest rank's time
    assert r0["rate"] == r1["rate"] == 32 * 2 / 2.0     # total units over that time
    assert r1["ref_rc"] == 0                            # non-zero ranks exit 0 without work


def test_single_rank_helpers():
    assert bench.rank_max(None, torch, 3.5, "cpu") == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0


def test_bench_sets_hardware_queues_before_cuda():
    """Importing bench.py sets CUDA_DEVICE_MAX_CONNECTIONS (32 queues for the
    32-stream batch graph) without importing torch, so the value is in place
    before any CUDA context exists; a value set by the caller is kept."""
    import subprocess
    code = ("import os, sys; sys.path.insert(0, sys.argv[1]); import bench; "
            "print(os.environ['CUDA_DEVICE_MAX_CONNECTIONS'], 'torch' in sys.modules)")
    env = {k: v for k, v in os.environ.items() if k != "CUDA_DEVICE_MAX_CONNECTIONS"}
    out = subprocess.run([sys.executable, "-c", code, ROOT], env=env, capture_output=True, text=True, check=True)
    assert out.stdout.split() == ["32", "False"]
    env["CUDA_DEVICE_MAX_CONNECTIONS"] = "16"
    out = subprocess.run([sys.executable, "-c", code, ROOT], env=env, capture_output=True, text=True, check=True)
    assert out.stdout.split() == ["16", "False"]
