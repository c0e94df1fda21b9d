"""One system split across processes by its CP rank terms (the rank-parallel
alternative the paper weighs in Sec. 3).

The paper distributes one system along the size axis N over MPI ranks and
leaves the FFTs to a distributed library; it mentions splitting the work over
the kernel's rank terms instead and rejects that on its CPU cluster. On GPUs
the term split needs one exchange per right-hand side and no distributed FFT:
both operators of Sec. 1 are sums over the CP terms (d, r),

    p_k^(d) = 1/d! sum_r (a^(1)_r * ... * a^(d)_r)_k,   a^(m)_r = U^(m)_r o n,
    q_k^(d) = -n_k/(d-1)! sum_r sum_m w_m U^(m)_r(k) prod_{m' != m} <U^(m')_r, n>,

so a process that owns a subset of the terms evaluates its partial
right-hand side with an ordinary plan of those terms (a CP rank of 0 leaves an
order out), and one all-reduce (sum) of the N-vector gives the full right-hand
side. The RK2 stages then run on every process with sag_rk2_stage, so all
processes hold the same state.

Terms are assigned by longest-processing-time first on an FFT cost model: a
term of order d transforms d vectors of length L_d >= d N, about
d L_d log2 L_d each. The exchange uses ``torch.distributed`` (NCCL on GPUs,
gloo for CPU tests); the arithmetic stays in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as _wl


def term_cost(d: int, N: int) -> float:
    """Relative cost of one CP rank term of order d: d forward transforms of
    length about d N (the FFT stage dominates the right-hand side)."""
    L = d * N
    return d * L * math.log2(max(L, 2))


def partition_terms(D: int, N: int, ranks, world: int) -> list:
    """Assigns every CP rank term (d, r) to one of `world` processes,
    heaviest first to the least loaded (ties to the lowest rank). Returns, per
    process, a dict {d: [r, ...]} with the ranks r in increasing order.
    Raises ValueError when a process would get no term."""
    terms = [(d, r) for d in range(2, D + 1) for r in range(int(ranks[d - 2]))]
    if world < 1 or len(terms) < world:
        raise ValueError(f"{len(terms)} CP rank terms cannot be split over {world} processes")
    terms.sort(key=lambda t: (-term_cost(t[0], N), t[0], t[1]))
    load = [0.0] * world
    out = [dict() for _ in range(world)]
    for d, r in terms:
        p = min(range(world), key=lambda i: (load[i], i))
        load[p] += term_cost(d, N)
        out[p].setdefault(d, []).append(r)
    for part in out:
        for d in part:
            part[d].sort()
    return out


def sub_system(D: int, N: int, ranks, factors, part: dict):
    """The CP factors of the terms in `part` ({d: [r, ...]}), in the layout of
    include/sag.h: returns (ranks, factors) with rank 0 for orders it lacks."""
    factors = np.asarray(factors, dtype=np.float64)
    offs = _wl.cp_layout(D, N, ranks)
    per = {}
    for d in range(2, D + 1):
        U = factors[offs[d - 2]:offs[d - 1]].reshape(d, int(ranks[d - 2]), N)
        per[d] = U[:, part.get(d, []), :]
    return _wl.cp_from_vectors(D, N, per)


def rk2_step_split(evaluate, allreduce, stage, n, k, nstar, k1, dt):
    """One RK2 step of a system whose right-hand side is summed across
    processes: k = allreduce(evaluate(n)); stage 0 (k1 = k, nstar = n + h1 k);
    k = allreduce(evaluate(nstar)); stage 1 (n advanced). The callables are the
    process's partial right-hand side (into k), the sum over processes (in
    place on k) and the plan's stage update."""
    evaluate(n, k)
    allreduce(k)
    stage(0, n, nstar, k1, k, dt)
    evaluate(nstar, k)
    allreduce(k)
    stage(1, n, nstar, k1, k, dt)
    return n


class TermParallelPlan:
    """A CP system split over the processes of a ``torch.distributed`` group
    by rank terms; every process passes the full state and gets the full
    right-hand side and the same RK2 steps. Extra keyword arguments go to
    ``sag.Plan`` (precision, RK rule, ...)."""

    def __init__(self, N: int, D: int, ranks, factors, group=None, **plan_kw):
        import torch.distributed as dist
        from . import sag
        self._dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.N, self.D = int(N), int(D)
        self.parts = partition_terms(D, N, ranks, self.world)
        self.terms = self.parts[self.rank]
        r_sub, f_sub = sub_system(D, N, ranks, factors, self.terms)
        self.plan = sag.Plan(N, D, r_sub, f_sub, **plan_kw)
        self._buf = None

    def _bufs(self, like):
        import torch
        if self._buf is None or self._buf[0].device != like.device:
            self._buf = tuple(torch.empty(self.N, dtype=torch.float64, device=like.device) for _ in range(3))
        return self._buf

    def _allreduce(self, x):
        self._dist.all_reduce(x, op=self._dist.ReduceOp.SUM, group=self.group)

    def rhs(self, n, dndt):
        """dndt = the full right-hand side at n (partial terms + all-reduce)."""
        self.plan.rhs(n, dndt)
        self._allreduce(dndt)
        return dndt

    def rk2_step(self, n, dt: float):
        k, nstar, k1 = self._bufs(n)
        return rk2_step_split(self.plan.rhs, self._allreduce, self.plan.rk2_stage, n, k, nstar, k1, dt)

    def integrate(self, n, dt: float, steps: int):
        for _ in range(int(steps)):
            self.rk2_step(n, dt)
        return n

    def sync_status(self) -> int:
        return self.plan.sync_status()

    def close(self):
        self.plan.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
