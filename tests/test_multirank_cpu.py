"""The N > 1 launch path on CPU: two gloo ranks.

bench.py runs one replica of the workload per GPU (no data-path
collective: the path does not shard without an exchange step); across ranks
it only synchronises (barrier) and takes the slowest rank's time. These tests
run that logic with world size 2 on the gloo backend, and the reference arm
under torchrun, where rank 0 alone works and prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    bench.barrier(world)
    t = bench.max_over_ranks(1.0 + rank, world)  # rank 1 is the slow one
    out[rank] = t
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier_with_two_gloo_ranks():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a threaded test process
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        assert dict(out) == {0: 2.0, 1: 2.0}


def test_reference_arm_under_torchrun_prints_once():
    # The reference arm is CPU work: rank 0 runs a bounded oracle sample and
    # prints the JSON line; rank 1 exits 0 without work or output.
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    # the arm reports what it timed: one sample step, converted to RK2 steps/s
    # of the whole workload (32 term samples per RK2 step), on the same config
    # dict as the GPU arm
    assert rec["steps"] == 1
    assert abs(rec["value"] * 32 * rec["ms_per_step"] / 1e3 - 1) < 1e-9
    sys.path.insert(0, ROOT)
    import bench
    assert rec["config"] == bench.bench_config(2)
