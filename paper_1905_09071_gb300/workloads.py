"""Seeded synthetic inputs for the multi-particle Smoluchowski right-hand side.

This module only draws numbers and lays them out; it holds none of the
method's arithmetic, so both the GPU library's tests and the CPU oracle's tests
can take their inputs from it. Seeds use ``numpy.random.default_rng`` (PCG64)
with the draws in the order written below.

Layouts follow the library convention: size k is stored at index k-1; CP
factors per order d are [d][R_d][N] (mode, rank, size) and orders d = 2..D are
concatenated; TT cores per order d are, for lambda = 1..d, [R_{l-1}][R_l][N].

Workloads (the paper's model from Sec. 1; shapes of its Sec. 3 experiment and
of the derived configurations):
  * ``constant_monodisperse`` - D=3, N=64, C^(2)=C^(3)=1 (CP rank 1, all-ones
    factors), n = e_1, Heun dt=0.01, 100 steps.
  * ``brownian_cp`` - D=3, N=4096, C^(d) = (sum_m i_m^{1/3})(sum_m i_m^{-1/3})
    as an exact CP of rank d^2, n_k = exp(-k)/sum exp(-k), dt=1e-3.
  * ``random_power_cp`` - D=4, N=65536, R=16 per order, U^(m)_r(i) =
    u_{m,r} i^{a_{m,r}} with u ~ U[0.5,1.5], a ~ U[-0.3,0.3], n_k = exp(-k/10)
    normalised to M0 = 1, dt=1e-4 (the throughput workload).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1905


@dataclass
class System:
    """One Smoluchowski system: orders 2..D, N size classes, a kernel per order."""
    D: int
    N: int
    fmt: str                      # "cp" or "tt"
    ranks: list                   # CP: [R_2..R_D]; TT: per order d its d+1 ranks, flattened
    factors: np.ndarray           # float64, layout above
    n0: np.ndarray                # float64 [N]
    dt: float = 1e-3
    steps: int = 1
    name: str = ""
    meta: dict = field(default_factory=dict)


def sizes(N: int) -> np.ndarray:
    """Sizes 1..N as float64 (exact integers)."""
    return np.arange(1, N + 1, dtype=np.float64)


def cp_layout(D: int, N: int, ranks) -> list:
    """Offsets (in doubles) of each order's block [d][R_d][N]; last entry = total."""
    offs = [0]
    for d in range(2, D + 1):
        offs.append(offs[-1] + d * int(ranks[d - 2]) * N)
    return offs


def cp_from_vectors(D: int, N: int, per_order: dict) -> tuple[list, np.ndarray]:
    """per_order[d] is an array [d][R_d][N]; returns (ranks, flat factors)."""
    ranks = [int(per_order[d].shape[1]) for d in range(2, D + 1)]
    flat = np.concatenate([np.asarray(per_order[d], dtype=np.float64).reshape(-1)
                           for d in range(2, D + 1)])
    return ranks, flat


def normalised(v: np.ndarray) -> np.ndarray:
    return v / v.sum()


def constant_monodisperse(D: int = 3, N: int = 64) -> System:
    per = {d: np.ones((d, 1, N)) for d in range(2, D + 1)}
    ranks, f = cp_from_vectors(D, N, per)
    n0 = np.zeros(N)
    n0[0] = 1.0
    return System(D, N, "cp", ranks, f, n0, dt=0.01, steps=100, name="constant_monodisperse")


def brownian_cp(D: int = 3, N: int = 4096) -> System:
    """(sum_m i_m^{1/3})(sum_m i_m^{-1/3}): term (a, b) has i^{1/3} in mode a,
    i^{-1/3} in mode b (their product, 1, when a = b) and ones elsewhere."""
    i = sizes(N)
    up, dn = np.cbrt(i), 1.0 / np.cbrt(i)
    per = {}
    for d in range(2, D + 1):
        U = np.ones((d, d * d, N))
        for a in range(d):
            for b in range(d):
                r = a * d + b
                if a != b:
                    U[a, r] = up
                    U[b, r] = dn
        per[d] = U
    ranks, f = cp_from_vectors(D, N, per)
    e = np.exp(-i)
    return System(D, N, "cp", ranks, f, normalised(e), dt=1e-3, steps=1000, name="brownian_cp")


def random_power_cp(D: int = 4, N: int = 65536, R: int = 16, seed: int = BASE_SEED,
                    u_range=(0.5, 1.5), a_range=(-0.3, 0.3), decay: float = 10.0) -> System:
    """For d = 2..D in order: u = U[u_range] (d, R), then a = U[a_range] (d, R);
    U^(m)_{d,r}(i) = u[m, r] * i^{a[m, r]} evaluated in FP64 from integer i."""
    rng = np.random.default_rng(seed)
    i = sizes(N)
    logi = np.log(i)
    per, power = {}, {}
    for d in range(2, D + 1):
        u = rng.uniform(u_range[0], u_range[1], (d, R))
        a = rng.uniform(a_range[0], a_range[1], (d, R))
        per[d] = u[:, :, None] * np.exp(a[:, :, None] * logi[None, None, :])
        power[d] = np.stack([u, a], axis=-1)  # [d][R][2]
    ranks, f = cp_from_vectors(D, N, per)
    n0 = normalised(np.exp(-i / decay))
    return System(D, N, "cp", ranks, f, n0, dt=1e-4, steps=100, name="random_power_cp",
                  meta={"seed": seed, "R": R, "power": power})


def power_params(D: int, power: dict) -> np.ndarray:
    """The (u, a) pairs of a kernel whose CP factors are U^(m)_r(i) = u i^a,
    per order d the array [d][R_d][2] flattened, orders concatenated (the
    parametric-factor layout of the library's plan)."""
    return np.concatenate([np.asarray(power[d], dtype=np.float64).reshape(-1) for d in range(2, D + 1)])


def expand_power(D: int, N: int, power: dict) -> tuple[list, np.ndarray]:
    """The same kernel's CP factors u i^a in FP64 (u * i**a), orders d = 2..D:
    returns (ranks, flat factors)."""
    i = sizes(N)
    per = {d: np.asarray(power[d])[:, :, 0:1] * i[None, None, :] ** np.asarray(power[d])[:, :, 1:2]
           for d in range(2, D + 1)}
    return cp_from_vectors(D, N, per)


def random_cp(D: int, N: int, ranks, seed: int, lo: float = 0.5, hi: float = 1.5) -> System:
    """Unstructured positive CP factors, for small parity cases."""
    rng = np.random.default_rng(seed)
    per = {d: rng.uniform(lo, hi, (d, int(ranks[d - 2]), N)) for d in range(2, D + 1)}
    rk, f = cp_from_vectors(D, N, per)
    n0 = rng.uniform(0.0, 1.0, N)
    n0 = normalised(n0)
    return System(D, N, "cp", rk, f, n0, name=f"random_cp_D{D}_N{N}", meta={"seed": seed})


def cp_to_tt_diagonal(sys: System) -> System:
    """The same kernel in TT form by the diagonal embedding: H^(1) = row of
    U^(1), H^(l)_{r,i,r'} = delta_{rr'} U^(l)_r(i), H^(d) = column of U^(d)."""
    assert sys.fmt == "cp"
    D, N = sys.D, sys.N
    offs = cp_layout(D, N, sys.ranks)
    ranks_tt, blocks = [], []
    for d in range(2, D + 1):
        R = sys.ranks[d - 2]
        U = sys.factors[offs[d - 2]:offs[d - 1]].reshape(d, R, N)
        rk = [1] + [R] * (d - 1) + [1]
        ranks_tt += rk
        for l in range(1, d + 1):
            H = np.zeros((rk[l - 1], rk[l], N))
            if l == 1:
                H[0, :, :] = U[0]
            elif l == d:
                H[:, 0, :] = U[d - 1]
            else:
                for r in range(R):
                    H[r, r, :] = U[l - 1, r]
            blocks.append(H.reshape(-1))
    return System(D, N, "tt", ranks_tt, np.concatenate(blocks), sys.n0.copy(), sys.dt, sys.steps,
                  name=sys.name + "_tt", meta=dict(sys.meta))


def brownian_tt_cores(mu, N: int):
    """TT cores of the generalized Brownian kernel (Eq. ch3.eq17) in the form the
    proof of Theorem 1 builds them: ranks binom(D, l); core l maps a rank index
    (an l-1 element subset of {1..D}) and a size i to the l-element subsets that
    add one element j, with entry i^{mu_j}. Subsets are numbered by their bit
    masks in increasing order. Returns (ranks[D+1], flat cores)."""
    D = len(mu)
    i = sizes(N)
    subsets = [[m for m in range(1 << D) if bin(m).count("1") == l] for l in range(D + 1)]
    ranks = [len(s) for s in subsets]
    blocks = []
    for l in range(1, D + 1):
        H = np.zeros((ranks[l - 1], ranks[l], N))
        for a, sa in enumerate(subsets[l - 1]):
            for b, sb in enumerate(subsets[l]):
                diff = sb & ~sa
                if (sa & ~sb) == 0 and bin(diff).count("1") == 1:
                    j = diff.bit_length() - 1
                    H[a, b] = i ** mu[j]
        blocks.append(H.reshape(-1))
    return ranks, np.concatenate(blocks)


def brownian_tt(D: int, N: int, mu, n0=None, decay: float = 10.0) -> System:
    """Orders d = 2..D, order d's kernel the Eq. ch3.eq17 kernel with the first
    d exponents mu[:d], each in its Theorem-1 TT form."""
    ranks_all, blocks = [], []
    for d in range(2, D + 1):
        r, c = brownian_tt_cores(list(mu[:d]), N)
        ranks_all += r
        blocks.append(c)
    if n0 is None:
        n0 = normalised(np.exp(-sizes(N) / decay))
    return System(D, N, "tt", ranks_all, np.concatenate(blocks), n0, name=f"brownian_tt_D{D}_N{N}",
                  meta={"mu": list(mu)})


def paper_ternary(N: int = 1 << 19, fmt: str = "tt", mu=(1 / 3, -1 / 3, 0.0), decay: float = 10.0,
                  dt: float = 1e-3) -> System:
    """The shape of the paper's own experiment (Sec. 3): pure ternary
    aggregation (only the d = 3 term) with the 3-D generalized Brownian kernel
    of Eq. ch3.eq17, C(i, j, l) = sum over permutations s of (i^mu_s1 j^mu_s2
    l^mu_s3). The paper does not state mu, the start or the step; these
    defaults are ours. fmt "tt": the Theorem-1 cores (ranks 1, 3, 3, 1) and an
    all-zero d = 2 order (ranks 1, 1, 1); fmt "cp": rank 0 for d = 2 and one
    rank-one term per permutation (rank 6) for d = 3."""
    i = sizes(N)
    n0 = normalised(np.exp(-i / decay))
    if fmt == "tt":
        r3, c3 = brownian_tt_cores(list(mu), N)
        return System(3, N, "tt", [1, 1, 1] + r3, np.concatenate([np.zeros(2 * N), c3]), n0, dt=dt,
                      name=f"paper_ternary_tt_N{N}", meta={"mu": list(mu)})
    import itertools
    perms = list(itertools.permutations(range(3)))
    U = np.stack([np.stack([i ** mu[p[m]] for p in perms]) for m in range(3)])  # [3][6][N]
    ranks, f = cp_from_vectors(3, N, {2: np.zeros((2, 0, N)), 3: U})
    return System(3, N, "cp", [0, 6], f, n0, dt=dt, name=f"paper_ternary_cp_N{N}", meta={"mu": list(mu)})


def random_tt(D: int, N: int, ranks_per_order: dict, seed: int, lo: float = 0.2,
              hi: float = 1.0) -> System:
    """Dense positive TT cores: ranks_per_order[d] = [1, R_1, ..., R_{d-1}, 1]."""
    rng = np.random.default_rng(seed)
    ranks_all, blocks = [], []
    for d in range(2, D + 1):
        rk = list(ranks_per_order[d])
        ranks_all += rk
        for l in range(1, d + 1):
            blocks.append(rng.uniform(lo, hi, rk[l - 1] * rk[l] * N))
    n0 = normalised(rng.uniform(0.0, 1.0, N))
    return System(D, N, "tt", ranks_all, np.concatenate(blocks), n0, name=f"random_tt_D{D}_N{N}",
                  meta={"seed": seed})


def batched_power_cp(B: int = 256, seed: int = BASE_SEED + 1, n_range=(1024, 32768),
                     rank_range=(4, 32), u_range=(0.5, 1.5), a_range=(-0.5, 0.5),
                     decay: float = 10.0) -> list:
    """B independent systems: for each in turn N = round(exp(U[ln n_lo, ln n_hi])),
    D uniform in {3, 4}, then for d = 2..D: R uniform in rank_range, u ~ U[u_range]
    (d, R), a ~ U[a_range] (d, R); U^(m)_r(i) = u i^a; n_k = exp(-k/10)
    normalised to M0 = 1."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(B):
        N = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        D = int(rng.integers(3, 5))
        logi = np.log(sizes(N))
        per = {}
        for d in range(2, D + 1):
            R = int(rng.integers(rank_range[0], rank_range[1] + 1))
            u = rng.uniform(u_range[0], u_range[1], (d, R))
            a = rng.uniform(a_range[0], a_range[1], (d, R))
            per[d] = u[:, :, None] * np.exp(a[:, :, None] * logi[None, None, :])
        ranks, f = cp_from_vectors(D, N, per)
        out.append(System(D, N, "cp", ranks, f, normalised(np.exp(-sizes(N) / decay)), dt=1e-4,
                          name=f"batched_{b}", meta={"seed": seed, "index": b}))
    return out


def adjoint_fit_problem(N: int = 8192, R: int = 9, seed: int = BASE_SEED + 2, extra_scale: float = 1e-3,
                        rel_perturb: float = 0.05) -> dict:
    """Kernel fitting: D = 3 with CP rank R for both orders. The first terms of
    each order are the Brownian CP of ``brownian_cp`` (4 for d = 2, 9 for
    d = 3); the remaining terms of order 2 are u i^a with u = extra_scale^{1/d}
    per mode and a ~ U[-0.3, 0.3] (drawn in order). The initial factors are
    rounded to FP32 (trainable FP32 parameters). The target kernel scales each
    factor vector by (1 + rel_perturb N(0, 1)) (drawn in vector order after the
    exponents). Start n_k proportional to exp(-k), Heun dt = 1e-3, 200 steps,
    checkpoints every 20."""
    rng = np.random.default_rng(seed)
    D = 3
    base = brownian_cp(D, N)
    offs = cp_layout(D, N, base.ranks)
    i = sizes(N)
    per = {}
    for d in range(2, D + 1):
        Rb = base.ranks[d - 2]
        Ub = base.factors[offs[d - 2]:offs[d - 1]].reshape(d, Rb, N)
        U = np.empty((d, R, N))
        U[:, :Rb] = Ub[:, :min(Rb, R)]
        for r in range(Rb, R):
            a = rng.uniform(-0.3, 0.3, d)
            for m in range(d):
                U[m, r] = extra_scale ** (1.0 / d) * i ** a[m]
        per[d] = U
    ranks, f = cp_from_vectors(D, N, per)
    f0 = f.astype(np.float32).astype(np.float64)
    nvec = f.size // N
    scale = 1.0 + rel_perturb * rng.normal(size=nvec)
    target = (f0.reshape(nvec, N) * scale[:, None]).reshape(-1)
    return {"D": D, "N": N, "ranks": ranks, "factors0": f0, "target_factors": target,
            "n0": base.n0.copy(), "dt": 1e-3, "steps": 200, "ckpt": 20}
