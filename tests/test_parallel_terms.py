"""The term-parallel split of one system (paper_1905_09071_gb300/parallel.py).

Host logic on the CPU: the partition covers every CP rank term once and is
balanced; the partial right-hand sides of the parts (by the oracle) sum to the
full one; and two gloo ranks running the split RK2 step (partial right-hand
side, all-reduce, stage update) reproduce the oracle's trajectory of the whole
system. On the GPU: two processes sharing cuda:0, each evaluating its terms
with the library and summing over gloo, against the oracle. The two processes'
kernels never wait on each other; the exchange is on the host.
"""
import os
import socket
import sys
import tempfile

import numpy as np
import pytest

import oracle
from paper_1905_09071_gb300 import parallel, workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("D,N,ranks,world", [(4, 65536, [16, 16, 16], 2), (4, 65536, [16, 16, 16], 3),
                                             (3, 500, [2, 5], 4), (4, 100, [3, 0, 2], 5),
                                             (2, 10, [3], 3)])
def test_partition_covers_every_term_once_and_balances(D, N, ranks, world):
    parts = parallel.partition_terms(D, N, ranks, world)
    assert len(parts) == world
    seen = sorted((d, r) for p in parts for d, rs in p.items() for r in rs)
    assert seen == sorted((d, r) for d in range(2, D + 1) for r in range(ranks[d - 2]))
    assert all(sum(len(v) for v in p.values()) >= 1 for p in parts)
    loads = [sum(parallel.term_cost(d, N) * len(rs) for d, rs in p.items()) for p in parts]
    costs = sorted((parallel.term_cost(d, N) for d in range(2, D + 1) for _ in range(ranks[d - 2])),
                   reverse=True)
    # no assignment beats this: the mean load, the largest term, and (with more
    # terms than processes) two of the world + 1 largest terms on one process
    lower = max(sum(costs) / world, costs[0], costs[world - 1] + costs[world] if len(costs) > world else 0)
    assert max(loads) <= 4.0 / 3.0 * lower + 1e-9 * lower  # Graham's bound for largest-first


def test_partition_needs_a_term_per_process():
    with pytest.raises(ValueError):
        parallel.partition_terms(3, 10, [1, 1], 3)


@pytest.mark.parametrize("world", [2, 3])
def test_parts_sum_to_the_full_right_hand_side(world):
    s = wl.random_cp(4, 40, [3, 2, 4], seed=31)
    p_full, q_full = oracle.rhs(s.n0, s.D, s.ranks, s.factors)
    p_sum, q_sum = np.zeros(s.N), np.zeros(s.N)
    for part in parallel.partition_terms(s.D, s.N, s.ranks, world):
        r, f = parallel.sub_system(s.D, s.N, s.ranks, s.factors, part)
        p, q = oracle.rhs(s.n0, s.D, r, f)
        p_sum += p
        q_sum += q
    scale = np.abs(p_full).max() + np.abs(q_full).max()
    assert np.abs(p_sum - p_full).max() / scale < 1e-14
    assert np.abs(q_sum - q_full).max() / scale < 1e-14


def _heun_stage(stage, n, nstar, k1, k, dt):
    # the Heun rule, restated on host arrays for this CPU test
    if stage == 0:
        k1[:] = k
        nstar[:] = n + dt * k
    else:
        n[:] = n + 0.5 * dt * (k1 + k)


def _gloo_worker(rank, world, port, path):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = wl.random_cp(3, 60, [3, 4], seed=32)
    part = parallel.partition_terms(s.D, s.N, s.ranks, world)[rank]
    r, f = parallel.sub_system(s.D, s.N, s.ranks, s.factors, part)

    def evaluate(x, out):
        p, q = oracle.rhs(x.numpy(), s.D, r, f)
        out.copy_(torch.from_numpy(p + q))

    def allreduce(x):
        dist.all_reduce(x, op=dist.ReduceOp.SUM)

    def stage(st, n, nstar, k1, k, dt):
        _heun_stage(st, n.numpy(), nstar.numpy(), k1.numpy(), k.numpy(), dt)

    n = torch.tensor(s.n0)
    k, nstar, k1 = torch.empty_like(n), torch.empty_like(n), torch.empty_like(n)
    for _ in range(3):
        parallel.rk2_step_split(evaluate, allreduce, stage, n, k, nstar, k1, 0.05)
    np.save(os.path.join(path, f"n{rank}.npy"), n.numpy())
    dist.destroy_process_group()


def test_split_rk2_with_two_gloo_ranks_matches_the_whole_system():
    import torch.multiprocessing as mp
    s = wl.random_cp(3, 60, [3, 4], seed=32)
    n_ref, _ = oracle.integrate(s.n0, s.D, s.ranks, s.factors, 0.05, 3, diag=False)
    with tempfile.TemporaryDirectory() as tmp:
        mp.spawn(_gloo_worker, args=(2, _free_port(), tmp), nprocs=2, join=True)
        n0 = np.load(os.path.join(tmp, "n0.npy"))
        n1 = np.load(os.path.join(tmp, "n1.npy"))
    assert np.array_equal(n0, n1)  # every rank holds the same state
    assert np.abs(n0 - n_ref).max() / np.abs(n_ref).max() < 1e-13


def _gpu_worker(rank, world, port, path, prec):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = wl.random_cp(4, 3000, [3, 2, 3], seed=33)
    with parallel.TermParallelPlan(s.N, s.D, s.ranks, s.factors, prec=prec) as tp:
        n = torch.tensor(s.n0, device="cuda")
        out = torch.empty_like(n)
        tp.rhs(n, out)
        tp.integrate(n, 1e-3, 2)
        torch.cuda.synchronize()
        assert tp.sync_status() == 0
        np.save(os.path.join(path, f"rhs{rank}.npy"), out.cpu().numpy())
        np.save(os.path.join(path, f"n{rank}.npy"), n.cpu().numpy())
    dist.destroy_process_group()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])  # SAG_FP64, SAG_FP32_SPLIT
def test_term_parallel_plan_two_processes_match_oracle(prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    s = wl.random_cp(4, 3000, [3, 2, 3], seed=33)
    p_ref, q_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors)
    n_ref, _ = oracle.integrate(s.n0, s.D, s.ranks, s.factors, 1e-3, 2, diag=False)
    tol = 1e-12 if prec == 0 else 1e-10
    with tempfile.TemporaryDirectory() as tmp:
        mp.spawn(_gpu_worker, args=(2, _free_port(), tmp, prec), nprocs=2, join=True)
        r = [np.load(os.path.join(tmp, f"rhs{i}.npy")) for i in range(2)]
        n = [np.load(os.path.join(tmp, f"n{i}.npy")) for i in range(2)]
    assert np.array_equal(r[0], r[1]) and np.array_equal(n[0], n[1])
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    assert np.abs(r[0] - (p_ref + q_ref)).max() / scale < tol
    assert np.abs(n[0] - n_ref).max() <= tol * 2 * 1e-3 * scale + 32 * np.finfo(float).eps * np.abs(s.n0).max()
