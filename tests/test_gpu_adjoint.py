"""The adjoint: vector-Jacobian products of the right-hand side and the
checkpointed discrete adjoint of RK2, against the CPU oracle's adjoint and
central finite differences; the PyTorch autograd wrapper on the kernel-fitting
workload (D=3, N=8192, CP rank 9, 200 Heun steps, checkpoints every 20)."""
import numpy as np
import pytest

import oracle
from paper_1905_09071_gb300 import sag, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [sag.SAG_FP64, sag.SAG_FP32_SPLIT, sag.SAG_FP32_SPLIT_EXACT]
# relative max-norm tolerances of cotangents
TOL = {sag.SAG_FP64: 1e-11, sag.SAG_FP32_SPLIT: 1e-9, sag.SAG_FP32_SPLIT_EXACT: 1e-11}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def rel(x, ref):
    return float(np.max(np.abs(np.asarray(x) - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("sym", [1, 0])
@pytest.mark.parametrize("D,N,ranks", [(2, 7, [3]), (3, 100, [2, 3]), (4, 333, [2, 1, 2]),
                                       (3, 1537, [3, 2])])
def test_rhs_vjp_matches_oracle(D, N, ranks, sym, prec):
    s = wl.random_cp(D, N, ranks, seed=80 + N)
    g = np.random.default_rng(81).normal(size=N)
    gn_ref, gU_ref = oracle.rhs_vjp(s.n0, g, D, s.ranks, s.factors, sym=sym)
    with sag.Plan(N, D, s.ranks, s.factors, prec=prec, symmetrize_q=sym) as pl:
        assert pl.factor_count() == s.factors.size
        gn = torch.empty(N, dtype=torch.float64, device="cuda")
        gU = torch.empty(s.factors.size, dtype=torch.float64, device="cuda")
        pl.rhs_vjp(dev(s.n0), dev(g), gn, gU)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
    assert rel(gn.cpu().numpy(), gn_ref) < TOL[prec]
    assert rel(gU.cpu().numpy(), gU_ref) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_integrate_vjp_graphs_match_direct_launches(prec):
    # The adjoint's segment phases replay cached CUDA graphs; with per-kernel
    # profiling on, the same kernels launch one by one. Both orders of work are
    # identical, so the gradients agree bitwise, also on a cached second call,
    # and for segment lengths 4, 4, 4, 1 and then 5, 5, 3 with new buffers.
    s = wl.random_cp(3, 300, [2, 3], seed=93)
    g = dev(np.random.default_rng(94).normal(size=s.N))
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec) as pl:
        n0 = dev(s.n0)
        outs = []
        for prof, steps, ckpt in ((False, 13, 4), (False, 13, 4), (True, 13, 4), (False, 13, 5), (True, 13, 5)):
            pl.profile(prof)
            gn = torch.empty_like(n0)
            gU = torch.empty(s.factors.size, dtype=torch.float64, device="cuda")
            pl.integrate_vjp(n0, 0.05, steps, g, gn, gU, ckpt=ckpt)
            torch.cuda.synchronize()
            if prof:
                pl.profile_read()
            outs.append((gn.cpu().numpy(), gU.cpu().numpy()))
        pl.profile(False)
        assert pl.sync_status() == sag.SAG_OK
    for a, b in ((0, 1), (0, 2), (3, 4)):
        assert np.array_equal(outs[a][0], outs[b][0]) and np.array_equal(outs[a][1], outs[b][1]), (a, b)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rk", [sag.SAG_HEUN, sag.SAG_MIDPOINT])
def test_integrate_vjp_matches_oracle_adjoint(prec, rk):
    s = wl.random_cp(3, 256, [3, 4], seed=90)
    steps, dt, ckpt = 13, 0.05, 4  # segments of 4, 4, 4, 1 steps
    g = np.random.default_rng(91).normal(size=s.N)
    method = oracle.HEUN if rk == sag.SAG_HEUN else oracle.MIDPOINT
    gn_ref, gU_ref = oracle.integrate_vjp(s.n0, s.D, s.ranks, s.factors, dt, steps, g, method=method)
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec, rk=rk) as pl:
        n0 = dev(s.n0)
        gn = torch.empty_like(n0)
        gU = torch.empty(s.factors.size, dtype=torch.float64, device="cuda")
        pl.integrate_vjp(n0, dt, steps, dev(g), gn, gU, ckpt=ckpt)
        torch.cuda.synchronize()
        assert torch.equal(n0, dev(s.n0))  # the initial state is not modified
    assert rel(gn.cpu().numpy(), gn_ref) < 10 * TOL[prec]
    assert rel(gU.cpu().numpy(), gU_ref) < 10 * TOL[prec]


def test_vjp_dot_product_identity():
    # <v, J u> = <J^T v, u> with J u from central differences of the FP64 path.
    s = wl.random_cp(4, 700, [2, 3, 2], seed=92)
    rng = np.random.default_rng(93)
    u = rng.normal(size=s.N)
    v = rng.normal(size=s.N)
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=sag.SAG_FP64) as pl:
        def F(x):
            out = torch.empty(s.N, dtype=torch.float64, device="cuda")
            pl.rhs(dev(x), out)
            torch.cuda.synchronize()
            return out.cpu().numpy()
        h = 1e-6
        Ju = (F(s.n0 + h * u) - F(s.n0 - h * u)) / (2 * h)
        gn = torch.empty(s.N, dtype=torch.float64, device="cuda")
        pl.rhs_vjp(dev(s.n0), dev(v), gn, None)
        torch.cuda.synchronize()
    lhs, r = v @ Ju, gn.cpu().numpy() @ u
    assert abs(lhs - r) < 1e-7 * (np.abs(v) @ np.abs(Ju))


@pytest.fixture(scope="module")
def fit_problem():
    return wl.adjoint_fit_problem()


def _final_state(plan, factors64, n0, dt, steps):
    plan.update_factors(factors64)
    n = dev(n0)
    plan.integrate(n, dt, steps)
    torch.cuda.synchronize()
    return n.cpu().numpy()


def test_autograd_gradient_matches_central_differences(fit_problem):
    from paper_1905_09071_gb300 import autograd as sag_autograd
    p = fit_problem
    D, N, ranks, dt, steps, ckpt = p["D"], p["N"], p["ranks"], p["dt"], p["steps"], p["ckpt"]
    with sag.Plan(N, D, ranks, p["target_factors"], prec=sag.SAG_FP64) as ref_plan:
        n_target = _final_state(ref_plan, p["target_factors"], p["n0"], dt, steps)
        with sag.Plan(N, D, ranks, p["factors0"], prec=sag.SAG_FP32_SPLIT) as plan:
            factors = torch.tensor(p["factors0"], dtype=torch.float32, device="cuda", requires_grad=True)
            n0 = dev(p["n0"])
            nT = sag_autograd.integrate(factors, n0, plan, dt, steps, ckpt)
            loss = ((nT - dev(n_target)) ** 2).sum()
            loss.backward()
            grad = factors.grad.double().cpu().numpy()
        assert np.isfinite(grad).all() and np.abs(grad).max() > 0
        # central differences of the FP64 forward along 16 random unit directions
        rng = np.random.default_rng(94)
        f0 = p["factors0"]

        def L(f):
            n = _final_state(ref_plan, f, p["n0"], dt, steps)
            return float(((n - n_target) ** 2).sum())

        h = 1e-6
        for _ in range(16):
            u = rng.normal(size=f0.size)
            u /= np.linalg.norm(u)
            fd = (L(f0 + h * u) - L(f0 - h * u)) / (2 * h)
            an = float(grad @ u)
            assert abs(fd - an) <= 1e-5 * (abs(fd) + 1e-3 * np.linalg.norm(grad)), (fd, an)


def test_gpu_adjoint_matches_oracle_adjoint_on_fit_problem_prefix():
    # The fitting workload's kernel on its first 384 sizes, 20 steps: the
    # library's FP64 adjoint against the oracle's.
    p = wl.adjoint_fit_problem(N=384)
    D, N, ranks, dt = p["D"], p["N"], p["ranks"], p["dt"]
    steps = 20
    g = np.random.default_rng(95).normal(size=N)
    gn_ref, gU_ref = oracle.integrate_vjp(p["n0"], D, ranks, p["factors0"], dt, steps, g)
    with sag.Plan(N, D, ranks, p["factors0"], prec=sag.SAG_FP64) as pl:
        gn = torch.empty(N, dtype=torch.float64, device="cuda")
        gU = torch.empty(p["factors0"].size, dtype=torch.float64, device="cuda")
        pl.integrate_vjp(dev(p["n0"]), dt, steps, dev(g), gn, gU, ckpt=5)
        torch.cuda.synchronize()
    assert rel(gn.cpu().numpy(), gn_ref) < 1e-10
    assert rel(gU.cpu().numpy(), gU_ref) < 1e-10


# ---------------------------------------------------------------- TT adjoint
TT_CASES = [
    ("random_D3_N100", lambda: wl.random_tt(3, 100, {2: [1, 2, 1], 3: [1, 2, 3, 1]}, seed=101)),
    ("random_D4_N333", lambda: wl.random_tt(4, 333, {2: [1, 3, 1], 3: [1, 2, 2, 1], 4: [1, 2, 3, 2, 1]},
                                            seed=102)),
    ("theorem1_D3_N300", lambda: wl.brownian_tt(3, 300, [0.4, -0.2, 0.1])),   # zero core entries
    ("paper_ternary_N300", lambda: wl.paper_ternary(300, "tt")),             # an all-zero order
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("sym", [1, 0])
@pytest.mark.parametrize("name,make", TT_CASES)
def test_tt_rhs_vjp_matches_oracle(name, make, sym, prec):
    # Cotangents of n and of every TT core entry (the caller's core layout,
    # also entries whose vector is zero) against the oracle's chain rule.
    t = make()
    g = np.random.default_rng(103).normal(size=t.N)
    gn_ref, gH_ref = oracle.rhs_vjp(t.n0, g, t.D, t.ranks, t.factors, sym=sym, fmt=oracle.TT)
    with sag.Plan(t.N, t.D, t.ranks, t.factors, fmt=sag.SAG_TT, prec=prec, symmetrize_q=sym) as pl:
        assert pl.factor_count() == t.factors.size
        gn = torch.empty(t.N, dtype=torch.float64, device="cuda")
        gH = torch.empty(t.factors.size, dtype=torch.float64, device="cuda")
        pl.rhs_vjp(dev(t.n0), dev(g), gn, gH)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
    assert rel(gn.cpu().numpy(), gn_ref) < TOL[prec]
    assert rel(gH.cpu().numpy(), gH_ref) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rk", [sag.SAG_HEUN, sag.SAG_MIDPOINT])
def test_tt_integrate_vjp_matches_oracle_adjoint(prec, rk):
    t = wl.random_tt(3, 256, {2: [1, 2, 1], 3: [1, 3, 2, 1]}, seed=104)
    steps, dt, ckpt = 9, 0.05, 4  # segments of 4, 4, 1 steps
    g = np.random.default_rng(105).normal(size=t.N)
    method = oracle.HEUN if rk == sag.SAG_HEUN else oracle.MIDPOINT
    gn_ref, gH_ref = oracle.integrate_vjp(t.n0, t.D, t.ranks, t.factors, dt, steps, g, method=method,
                                          fmt=oracle.TT)
    with sag.Plan(t.N, t.D, t.ranks, t.factors, fmt=sag.SAG_TT, prec=prec, rk=rk) as pl:
        gn = torch.empty(t.N, dtype=torch.float64, device="cuda")
        gH = torch.empty(t.factors.size, dtype=torch.float64, device="cuda")
        pl.integrate_vjp(dev(t.n0), dt, steps, dev(g), gn, gH, ckpt=ckpt)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
    assert rel(gn.cpu().numpy(), gn_ref) < 10 * TOL[prec]
    assert rel(gH.cpu().numpy(), gH_ref) < 10 * TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_tt_rhs_vjp_large_blocks_matches_oracle(prec):
    # N = 4096 with 15 distinct core vectors: the column blocks and the TT row
    # blocks of the adjoint both need more than 48 KB of shared memory.
    t = wl.random_tt(3, 4096, {2: [1, 4, 1], 3: [1, 3, 3, 1]}, seed=109)
    g = np.random.default_rng(110).normal(size=t.N)
    gn_ref, gH_ref = oracle.rhs_vjp(t.n0, g, t.D, t.ranks, t.factors, fmt=oracle.TT)
    with sag.Plan(t.N, t.D, t.ranks, t.factors, fmt=sag.SAG_TT, prec=prec) as pl:
        gn = torch.empty(t.N, dtype=torch.float64, device="cuda")
        gH = torch.empty(t.factors.size, dtype=torch.float64, device="cuda")
        pl.rhs_vjp(dev(t.n0), dev(g), gn, gH)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
    assert rel(gn.cpu().numpy(), gn_ref) < TOL[prec]
    assert rel(gH.cpu().numpy(), gH_ref) < TOL[prec]


def test_tt_vjp_of_diagonal_embedding_equals_cp_vjp():
    # The library's TT adjoint of the diagonal embedding of a CP kernel gives
    # the CP adjoint's n-cotangent (FP64).
    s = wl.random_cp(4, 500, [3, 2, 2], seed=106)
    t = wl.cp_to_tt_diagonal(s)
    g = dev(np.random.default_rng(107).normal(size=s.N))
    outs = []
    for sysm, fmt in ((s, sag.SAG_CP), (t, sag.SAG_TT)):
        with sag.Plan(sysm.N, sysm.D, sysm.ranks, sysm.factors, fmt=fmt, prec=sag.SAG_FP64) as pl:
            gn = torch.empty(s.N, dtype=torch.float64, device="cuda")
            pl.rhs_vjp(dev(sysm.n0), g, gn, None)
            torch.cuda.synchronize()
            outs.append(gn.cpu().numpy())
    assert rel(outs[1], outs[0]) < 1e-12


@pytest.mark.parametrize("prec", [sag.SAG_FP64, sag.SAG_FP32_SPLIT])
def test_tt_integrate_vjp_paper_shape_matches_oracle(prec):
    # The paper's Sec. 3 kernel family (pure ternary generalized Brownian
    # kernel, Theorem-1 cores with ranks 1, 3, 3, 1 and structural zeros, an
    # all-zero d = 2 order) at N = 4096: 4 Heun steps, checkpoints every 2.
    t = wl.paper_ternary(4096, "tt")
    g = np.random.default_rng(108).normal(size=t.N) * t.n0  # a cotangent shaped like the state
    steps, dt = 4, 1e-3
    gn_ref, gH_ref = oracle.integrate_vjp(t.n0, t.D, t.ranks, t.factors, dt, steps, g, fmt=oracle.TT)
    with sag.Plan(t.N, t.D, t.ranks, t.factors, fmt=sag.SAG_TT, prec=prec) as pl:
        gn = torch.empty(t.N, dtype=torch.float64, device="cuda")
        gH = torch.empty(t.factors.size, dtype=torch.float64, device="cuda")
        pl.integrate_vjp(dev(t.n0), dt, steps, dev(g), gn, gH, ckpt=2)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
    assert rel(gn.cpu().numpy(), gn_ref) < 10 * TOL[prec]
    assert rel(gH.cpu().numpy(), gH_ref) < 10 * TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_autograd_forward_after_training_apart_repeated_vectors(prec):
    # The fitting workload starts from the Brownian factors, whose vectors
    # repeat; a training step makes them differ. A plan made with
    # keep_repeats = 1 from the starting factors follows the new factors (its
    # forward against the oracle's); a default plan refuses them.
    from paper_1905_09071_gb300 import autograd as sag_autograd
    p = wl.adjoint_fit_problem(N=384)
    D, N, ranks, dt = p["D"], p["N"], p["ranks"], p["dt"]
    steps = 20
    f1 = p["factors0"] * (1.0 + 1e-3 * np.random.default_rng(96).normal(size=p["factors0"].size))
    n_ref, _ = oracle.integrate(p["n0"], D, ranks, f1, dt, steps, diag=False)
    with sag.Plan(N, D, ranks, p["factors0"], prec=prec, keep_repeats=1) as pl:
        nT = sag_autograd.integrate(torch.tensor(f1, device="cuda"), dev(p["n0"]), pl, dt, steps, 5)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
    assert rel(nT.cpu().numpy(), n_ref) < TOL[prec]
    with sag.Plan(N, D, ranks, p["factors0"], prec=prec) as pl:
        with pytest.raises(sag.SagError, match="keep_repeats"):
            sag_autograd.integrate(torch.tensor(f1, device="cuda"), dev(p["n0"]), pl, dt, steps, 5)
