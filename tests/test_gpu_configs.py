"""The workload configurations end to end against the CPU oracle, through the C ABI.

Each test runs one configuration at its own size (or the stated slice of it)
on the GPU and compares every output element with the oracle's FP64 direct
low-rank evaluation (sequential truncated convolutions and inner products, no
FFT). Tolerances (normwise, as in the other parity tests):
  right-hand sides and RK2 increments: FP64 1e-12, FP32-split 1e-10,
  FP32-split exact 1e-12, relative to steps * dt * (max|P| + max|Q|) at n0,
  plus the state's own rounding (a few ulp of max|n| per stage);
  long trajectories (1000 steps): FP64 and FP32-split exact 1e-11, FP32-split
  1e-9, relative to max|n|;
  adjoints: 10x the cotangent tolerances of the adjoint tests.
The oracle runs here on the host cores (OpenMP); the largest case (two Heun
steps at N = 65536, four right-hand sides of 96 length-65536 convolutions)
takes about a minute on 16 cores.
"""
import numpy as np
import pytest

import oracle
from paper_1905_09071_gb300 import sag, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [sag.SAG_FP64, sag.SAG_FP32_SPLIT, sag.SAG_FP32_SPLIT_EXACT]
TOL = {sag.SAG_FP64: 1e-12, sag.SAG_FP32_SPLIT: 1e-10, sag.SAG_FP32_SPLIT_EXACT: 1e-12}
TRAJ_TOL = {sag.SAG_FP64: 1e-11, sag.SAG_FP32_SPLIT: 1e-9, sag.SAG_FP32_SPLIT_EXACT: 1e-11}
ADJ_TOL = {sag.SAG_FP64: 1e-10, sag.SAG_FP32_SPLIT: 1e-8, sag.SAG_FP32_SPLIT_EXACT: 1e-10}
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def increment_error(n_gpu, n_ref, n0, steps, dt, rhs_scale):
    """max |(n_gpu - n0) - (n_ref - n0)| against the bound the right-hand side's
    tolerance implies: steps * dt * rhs_scale, and per stage a few ulp of the
    state (n + dt k is rounded in FP64 on both sides)."""
    err = float(np.max(np.abs(np.asarray(n_gpu) - n_ref)))
    return err, steps * dt * rhs_scale, 8 * 2 * steps * EPS * float(np.max(np.abs(n0)))


def _prefix_gain(s, K):
    """The oracle's gain term at sizes k <= K: the kernel restricted to sizes
    1..K has the same gain there (no tuple of sizes summing to k <= K uses a
    size above K)."""
    offs = wl.cp_layout(s.D, s.N, s.ranks)
    per = {d: s.factors[offs[d - 2]:offs[d - 1]].reshape(d, s.ranks[d - 2], s.N)[:, :, :K]
           for d in range(2, s.D + 1)}
    rk, f = wl.cp_from_vectors(s.D, K, per)
    p, _ = oracle.rhs(s.n0[:K], s.D, rk, f, mode=oracle.DIRECT)
    return p


# ------------------------------------------------- throughput workload: two Heun steps
@pytest.fixture(scope="module")
def throughput_two_steps():
    s = wl.random_power_cp()  # D=4, N=65536, R=16 per order, dt=1e-4
    steps = 2
    n_ref, _ = oracle.integrate(s.n0, s.D, s.ranks, s.factors, s.dt, steps, mode=oracle.DIRECT, diag=False)
    scale = np.abs(_prefix_gain(s, 2048)).max() + np.abs(oracle.loss(s.n0, s.D, s.ranks, s.factors)).max()
    return s, steps, n_ref, scale


@pytest.mark.parametrize("prec", PRECS)
def test_throughput_workload_two_heun_steps_match_oracle(throughput_two_steps, prec):
    # N = 65536, D = 4, R = 16: the full state after two Heun steps (four
    # right-hand sides) against the oracle's direct CP mode, every element.
    s, steps, n_ref, scale = throughput_two_steps
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec) as pl:
        n = dev(s.n0)
        pl.integrate(n, s.dt, steps)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
        n = n.cpu().numpy()
    err, bound, rounding = increment_error(n, n_ref, s.n0, steps, s.dt, scale)
    assert err <= TOL[prec] * bound + rounding, (err / bound, rounding / bound)
    assert np.max(np.abs(n - n_ref)) / np.max(np.abs(n_ref)) < TOL[prec]


# ------------------------------------------------- Brownian kernel: 1000 steps
@pytest.fixture(scope="module")
def brownian_trajectory():
    s = wl.brownian_cp(3, 4096)  # exact CP of rank d^2, n_k ~ exp(-k), dt = 1e-3
    n_ref, d_ref = oracle.integrate(s.n0, s.D, s.ranks, s.factors, s.dt, s.steps, mode=oracle.DIRECT)
    return s, n_ref, d_ref


@pytest.mark.parametrize("prec", PRECS)
def test_brownian_thousand_steps_match_oracle(brownian_trajectory, prec):
    # D = 3, N = 4096, 1000 Heun steps of dt = 1e-3 to t = 1: the final state
    # and every diagnostics row (M0, M1, cumulative outflow) against the oracle.
    s, n_ref, d_ref = brownian_trajectory
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec) as pl:
        n = dev(s.n0)
        diag = torch.zeros((s.steps + 1, 3), dtype=torch.float64, device="cuda")
        pl.integrate(n, s.dt, s.steps, diag)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
        n, diag = n.cpu().numpy(), diag.cpu().numpy()
    assert np.max(np.abs(n - n_ref)) / np.max(np.abs(n_ref)) < TRAJ_TOL[prec]
    # M0 and M1 relative to their initial values; the outflow relative to M1
    assert np.max(np.abs(diag[:, 0] - d_ref[:, 0])) / d_ref[0, 0] < TRAJ_TOL[prec]
    m1_tol = 1e-9 if prec == sag.SAG_FP32_SPLIT else 1e-11
    assert np.max(np.abs(diag[:, 1] - d_ref[:, 1])) / d_ref[0, 1] < m1_tol
    assert np.max(np.abs(diag[:, 2] - d_ref[:, 2])) / d_ref[0, 1] < m1_tol
    assert d_ref[-1, 2] > 0  # mass does leave the truncated system


# ------------------------------------------------- 256-system batch
@pytest.fixture(scope="module")
def batch_case():
    systems = wl.batched_power_cp()  # B = 256, N in [1024, 32768], D in {3, 4}, R in [4, 32]
    Ns = np.array([s.N for s in systems])
    order = np.argsort(Ns, kind="stable")
    picked = [int(b) for b in order[:8]] + [int(order[-1])]  # the 8 smallest and the largest
    steps = 2
    ref = {}
    for b in picked:
        s = systems[b]
        p, q = oracle.rhs(s.n0, s.D, s.ranks, s.factors, mode=oracle.DIRECT)
        n2, _ = oracle.integrate(s.n0, s.D, s.ranks, s.factors, s.dt, steps, mode=oracle.DIRECT, diag=False)
        ref[b] = (p, q, n2)
    return systems, picked, steps, ref


@pytest.mark.parametrize("prec", [sag.SAG_FP32_SPLIT, sag.SAG_FP64])
def test_batched_workload_per_system_matches_oracle(batch_case, prec):
    # One plan over all 256 systems (every kernel launched once over the batch);
    # the gain, the loss and two Heun steps of the 8 smallest systems and the
    # largest against the oracle, each system on its own.
    systems, picked, steps, ref = batch_case
    with sag.Plan.batch([(s.N, s.D, s.ranks, s.factors, sag.SAG_CP) for s in systems], prec=prec) as pl:
        off = pl.layout()
        n = dev(np.concatenate([s.n0 for s in systems]))
        p, q = torch.empty_like(n), torch.empty_like(n)
        pl.rhs_parts(n, p, q)
        pl.integrate(n, systems[0].dt, steps)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
        p, q, n = p.cpu().numpy(), q.cpu().numpy(), n.cpu().numpy()
    for b in picked:
        s = systems[b]
        p_ref, q_ref, n_ref = ref[b]
        sl = slice(off[b], off[b + 1])
        scale = np.abs(p_ref).max() + np.abs(q_ref).max()
        assert np.max(np.abs(p[sl] - p_ref)) / scale < TOL[prec], b
        assert np.max(np.abs(q[sl] - q_ref)) / scale < TOL[prec], b
        err, bound, rounding = increment_error(n[sl], n_ref, s.n0, steps, s.dt, scale)
        assert err <= TOL[prec] * bound + rounding, (b, err / bound)


# ------------------------------------------------- kernel-fitting adjoint
@pytest.fixture(scope="module")
def fit_adjoint():
    p = wl.adjoint_fit_problem()  # D = 3, N = 8192, CP rank 9, FP32-rounded factors
    D, N, ranks, dt = p["D"], p["N"], p["ranks"], p["dt"]
    steps, ckpt = 20, 5
    nT, _ = oracle.integrate(p["n0"], D, ranks, p["factors0"], dt, steps, diag=False)
    nt, _ = oracle.integrate(p["n0"], D, ranks, p["target_factors"], dt, steps, diag=False)
    g = 2.0 * (nT - nt)  # cotangent of the loss ||n(T) - n_target||^2
    gn_ref, gU_ref = oracle.integrate_vjp(p["n0"], D, ranks, p["factors0"], dt, steps, g)
    return p, steps, ckpt, nt, g, gn_ref, gU_ref


@pytest.mark.parametrize("prec", PRECS)
def test_fit_adjoint_matches_oracle_adjoint(fit_adjoint, prec):
    # N = 8192, 20 Heun steps with checkpoints every 5: the library's discrete
    # adjoint (recomputation from checkpoints, cached segment graphs) against
    # the oracle's (every state kept), for the initial state and every factor.
    p, steps, ckpt, _, g, gn_ref, gU_ref = fit_adjoint
    with sag.Plan(p["N"], p["D"], p["ranks"], p["factors0"], prec=prec) as pl:
        gn = torch.empty(p["N"], dtype=torch.float64, device="cuda")
        gU = torch.empty(p["factors0"].size, dtype=torch.float64, device="cuda")
        pl.integrate_vjp(dev(p["n0"]), p["dt"], steps, dev(g), gn, gU, ckpt=ckpt)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
    gn, gU = gn.cpu().numpy(), gU.cpu().numpy()
    assert np.max(np.abs(gn - gn_ref)) / np.max(np.abs(gn_ref)) < ADJ_TOL[prec]
    assert np.max(np.abs(gU - gU_ref)) / np.max(np.abs(gU_ref)) < ADJ_TOL[prec]


def test_fit_gradient_matches_oracle_central_differences(fit_adjoint):
    # The loss gradient of the FP64 library adjoint against central differences
    # (h = 1e-6) of the oracle's own FP64 forward, along random unit directions
    # of the factors and of the initial state.
    p, steps, ckpt, nt, g, _, _ = fit_adjoint
    D, N, ranks, dt = p["D"], p["N"], p["ranks"], p["dt"]
    with sag.Plan(N, D, ranks, p["factors0"], prec=sag.SAG_FP64) as pl:
        gn = torch.empty(N, dtype=torch.float64, device="cuda")
        gU = torch.empty(p["factors0"].size, dtype=torch.float64, device="cuda")
        pl.integrate_vjp(dev(p["n0"]), dt, steps, dev(g), gn, gU, ckpt=ckpt)
        torch.cuda.synchronize()
    gn, gU = gn.cpu().numpy(), gU.cpu().numpy()

    def loss(n0, f):
        n, _ = oracle.integrate(n0, D, ranks, f, dt, steps, diag=False)
        return float(((n - nt) ** 2).sum())

    rng = np.random.default_rng(1907)
    h = 1e-6
    for which in ("factors", "factors", "n0"):
        if which == "factors":
            u = rng.normal(size=p["factors0"].size)
            u /= np.linalg.norm(u)
            fd = (loss(p["n0"], p["factors0"] + h * u) - loss(p["n0"], p["factors0"] - h * u)) / (2 * h)
            an = float(gU @ u)
            gnorm = np.linalg.norm(gU)
        else:
            u = rng.normal(size=N) * p["n0"]  # relative perturbation of the start
            u /= np.linalg.norm(u)
            fd = (loss(p["n0"] + h * u, p["factors0"]) - loss(p["n0"] - h * u, p["factors0"])) / (2 * h)
            an = float(gn @ u)
            gnorm = np.linalg.norm(gn)
        # the oracle's own FP64 adjoint meets this check at about 1.2e-6
        assert abs(fd - an) <= 1e-5 * (abs(fd) + 1e-3 * gnorm), (which, fd, an)
