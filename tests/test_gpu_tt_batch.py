"""Parity of the TT path and of batched plans with the CPU oracle.

TT (Eq. ch3.eq4): kernels given by their cores; the GPU forms each order's
spectral sum by a per-frequency matrix chain. Batched: one plan holding
systems of different N, D and ranks, every kernel launched once for all of
them. Same error metric and tolerances as test_gpu_parity.py.
"""
import numpy as np
import pytest

import oracle
from paper_1905_09071_gb300 import sag, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {sag.SAG_FP64: 1e-12, sag.SAG_FP32_SPLIT: 1e-10, sag.SAG_FP32_SPLIT_EXACT: 1e-12}
PRECS = [sag.SAG_FP64, sag.SAG_FP32_SPLIT, sag.SAG_FP32_SPLIT_EXACT]
FMT = {"cp": sag.SAG_CP, "tt": sag.SAG_TT}
OFMT = {"cp": oracle.CP, "tt": oracle.TT}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def nerr(x, ref, scale):
    return float(np.max(np.abs(np.asarray(x) - ref)) / scale)


def run_parts(pl, n0):
    n = dev(n0)
    p, q = torch.empty_like(n), torch.empty_like(n)
    o = torch.zeros(pl.B, dtype=torch.float64, device="cuda")
    pl.rhs_parts(n, p, q, o)
    torch.cuda.synchronize()
    assert pl.sync_status() == sag.SAG_OK
    return p.cpu().numpy(), q.cpu().numpy(), o.cpu().numpy()


def plan_of(s, prec, sym=1):
    return sag.Plan(s.N, s.D, s.ranks, s.factors, fmt=FMT[s.fmt], prec=prec, symmetrize_q=sym)


# ------------------------------------------------------------------ TT path
TT_CASES = [
    ("diag_D4_N333", lambda: wl.cp_to_tt_diagonal(wl.random_cp(4, 333, [3, 2, 4], seed=31))),
    ("brownian_D3_N500", lambda: wl.brownian_tt(3, 500, [0.4, -0.2, 0.1])),
    ("brownian_D4_N1200", lambda: wl.brownian_tt(4, 1200, [1 / 3, -1 / 3, 0.2, -0.1])),
    ("dense_D3_N257", lambda: wl.random_tt(3, 257, {2: [1, 3, 1], 3: [1, 2, 4, 1]}, seed=33)),
    ("dense_D4_N4100", lambda: wl.random_tt(4, 4100, {2: [1, 5, 1], 3: [1, 3, 2, 1],
                                                      4: [1, 2, 16, 3, 1]}, seed=34)),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("sym", [1, 0])
@pytest.mark.parametrize("name,make", TT_CASES)
def test_tt_rhs_matches_oracle(name, make, sym, prec):
    s = make()
    p_ref, q_ref, o_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors, fmt=oracle.TT,
                                     mode=oracle.DIRECT, sym=sym, outflow=True)
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    with plan_of(s, prec, sym) as pl:
        p, q, o = run_parts(pl, s.n0)
    assert nerr(p, p_ref, scale) < TOL[prec]
    assert nerr(q, q_ref, scale) < TOL[prec]
    flux = np.sum(np.arange(1, s.N + 1) * np.abs(p_ref)) + abs(o_ref) + 1e-300
    assert abs(o[0] - o_ref) <= 1e3 * TOL[prec] * flux


def _distinct_nonzero_core_vectors(s):
    """Per order, the bitwise-distinct nonzero vectors over all of its cores."""
    out, off, rk = [], 0, 0
    for d in range(2, s.D + 1):
        r = s.ranks[rk:rk + d + 1]
        seen = set()
        for l in range(1, d + 1):
            for _ in range(r[l - 1] * r[l]):
                x = s.factors[off:off + s.N]
                off += s.N
                if np.any(x != 0):
                    seen.add(x.tobytes())
        out.append(len(seen))
        rk += d + 1
    return out


@pytest.mark.parametrize("prec", PRECS)
def test_tt_cores_share_vectors_across_cores(prec):
    # Theorem-1 cores repeat the powers i^mu_j in every core: an order's
    # identical vectors are transformed once whatever core holds them. N =
    # 12000 puts the d = 3 rows at 128 points (compile-time TT row kernels in
    # the double-word paths).
    s = wl.brownian_tt(3, 12000, [0.4, -0.2, 0.1])
    want = _distinct_nonzero_core_vectors(s)
    p_ref, q_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors, fmt=oracle.TT, mode=oracle.DIRECT)
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    with plan_of(s, prec) as pl:
        orders = pl.describe()["orders"]
        assert [o["transformed"] for o in orders] == want
        assert want[-1] < sum(s.ranks[3 + l] * s.ranks[4 + l] for l in range(3))  # fewer than the entries
        if prec != sag.SAG_FP64:
            assert orders[-1]["M2"] == 128 and orders[-1]["compile_time"][1] == 1
        p, q, _ = run_parts(pl, s.n0)
    assert nerr(p, p_ref, scale) < TOL[prec]
    assert nerr(q, q_ref, scale) < TOL[prec]


def _tt_prefix(s, K):
    """The same TT kernel restricted to sizes 1..K (every core vector cut to its
    first K entries): its gain term equals the full system's at every k <= K."""
    return s.factors.reshape(-1, s.N)[:, :K].reshape(-1).copy()


@pytest.mark.parametrize("prec", PRECS)
def test_tt_rows_at_256_points_sampled_parity(prec):
    # N = 50000 puts both orders' rows at 256 points. The gain outputs
    # k <= 2048 against the oracle on the size prefix, every loss output
    # against the oracle's inner-product route; a slowly decaying start keeps
    # every size in play.
    b = wl.brownian_tt(3, 50000, [0.4, -0.2, 0.1])
    n0 = wl.normalised(np.exp(-wl.sizes(b.N) / (b.N / 8)))
    K = 2048
    p_pre, _ = oracle.rhs(n0[:K], b.D, b.ranks, _tt_prefix(b, K), fmt=oracle.TT, mode=oracle.DIRECT)
    q_ref = oracle.loss(n0, b.D, b.ranks, b.factors, fmt=oracle.TT)
    with plan_of(b, prec) as pl:
        orders = pl.describe()["orders"]
        if prec != sag.SAG_FP64:
            assert [o["M2"] for o in orders] == [256, 256]
            assert all(o["compile_time"][1] == 1 for o in orders)
        p, q, _ = run_parts(pl, n0)
    scale = np.abs(p).max() + np.abs(q_ref).max()
    assert nerr(p[:K], p_pre, scale) < TOL[prec]
    assert nerr(q, q_ref, scale) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_tt_all_zero_cores_are_rejected(prec):
    # An order whose cores are all zero is idle (no FFT blocks; the paper
    # shape's d = 2 order is one); a system whose every order is zero has no
    # right-hand side to speak of and is refused when the plan is made.
    N, D, ranks = 3000, 3, [1, 2, 1, 1, 2, 3, 1]
    f = np.zeros(N * (2 + 2 + 2 + 6 + 3))
    with pytest.raises(sag.SagError, match="identically zero"):
        sag.Plan(N, D, ranks, f, fmt=sag.SAG_TT, prec=prec)


@pytest.mark.parametrize("prec", PRECS)
def test_tt_tiny_matches_brute_force(prec):
    s = wl.brownian_tt(4, 6, [0.3, -0.2, 0.15, 0.05])
    p_ref, q_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors, fmt=oracle.TT, mode=oracle.BRUTE)
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    with plan_of(s, prec) as pl:
        p, q, _ = run_parts(pl, s.n0)
    assert nerr(p, p_ref, scale) < TOL[prec] and nerr(q, q_ref, scale) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_tt_diagonal_embedding_equals_cp_at_full_size(prec):
    # The throughput workload (D=4, N=65536, R=16) in both formats.
    s = wl.random_power_cp()
    t = wl.cp_to_tt_diagonal(s)
    with plan_of(s, prec) as pl:
        p1, q1, _ = run_parts(pl, s.n0)
    with plan_of(t, prec) as pl:
        p2, q2, _ = run_parts(pl, t.n0)
    scale = np.abs(p1).max() + np.abs(q1).max()
    assert nerr(p2, p1, scale) < 2 * TOL[prec]
    assert nerr(q2, q1, scale) < 2 * TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_tt_trajectory_matches_oracle(prec):
    s = wl.brownian_tt(3, 300, [0.4, -0.2, 0.1])
    n_ref, d_ref = oracle.integrate(s.n0, s.D, s.ranks, s.factors, 1e-3, 5, fmt=oracle.TT)
    with plan_of(s, prec) as pl:
        n = dev(s.n0)
        diag = torch.zeros((6, 1, 3), dtype=torch.float64, device="cuda")
        pl.integrate(n, 1e-3, 5, diag)
        torch.cuda.synchronize()
        n = n.cpu().numpy()
        diag = diag.cpu().numpy()[:, 0, :]
    assert nerr(n, n_ref, np.abs(n_ref).max()) < TOL[prec]
    assert np.max(np.abs(diag[:, :2] - d_ref[:, :2]) / np.abs(d_ref[:, :2]).max(axis=0)) < TOL[prec]


# ------------------------------------------------------------------ batched plans
def mixed_batch():
    return [
        wl.random_cp(2, 1, [2], seed=41),
        wl.random_cp(3, 7, [2, 3], seed=42),
        wl.random_cp(4, 100, [3, 1, 2], seed=43),
        wl.random_cp(3, 1000, [5, 4], seed=44),
        wl.brownian_cp(3, 4097),
        wl.random_cp(4, 5000, [6, 5, 4], seed=45),
    ]


def packed(systems, attr="n0"):
    return np.concatenate([getattr(s, attr) for s in systems])


@pytest.mark.parametrize("prec", PRECS)
def test_batched_rhs_matches_oracle_per_system(prec):
    systems = mixed_batch()
    with sag.Plan.batch([(s.N, s.D, s.ranks, s.factors, FMT[s.fmt]) for s in systems],
                        prec=prec) as pl:
        off = pl.layout()
        assert off[-1] == sum(s.N for s in systems)
        p, q, o = run_parts(pl, packed(systems))
    for b, s in enumerate(systems):
        p_ref, q_ref, o_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors, mode=oracle.DIRECT,
                                         outflow=True)
        scale = np.abs(p_ref).max() + np.abs(q_ref).max()
        assert nerr(p[off[b]:off[b + 1]], p_ref, scale) < TOL[prec], b
        assert nerr(q[off[b]:off[b + 1]], q_ref, scale) < TOL[prec], b
        flux = np.sum(np.arange(1, s.N + 1) * np.abs(p_ref)) + abs(o_ref) + 1e-300
        assert abs(o[b] - o_ref) <= 1e3 * TOL[prec] * flux, b


def test_batched_equals_one_plan_per_system():
    systems = mixed_batch()
    with sag.Plan.batch([(s.N, s.D, s.ranks, s.factors, FMT[s.fmt]) for s in systems]) as pl:
        off = pl.layout()
        n = dev(packed(systems))
        out = torch.empty_like(n)
        pl.rhs(n, out)
        torch.cuda.synchronize()
        out = out.cpu().numpy()
    for b, s in enumerate(systems):
        with plan_of(s, sag.SAG_FP32_SPLIT) as one:
            x = dev(s.n0)
            y = torch.empty_like(x)
            one.rhs(x, y)
            torch.cuda.synchronize()
            assert np.array_equal(out[off[b]:off[b + 1]], y.cpu().numpy()), b


def test_autotuned_batch_gives_the_same_results():
    systems = mixed_batch()
    res = []
    for autotune in (0, 1):
        with sag.Plan.batch([(s.N, s.D, s.ranks, s.factors, FMT[s.fmt]) for s in systems],
                            autotune=autotune) as pl:
            assert 1 <= pl.describe()["blocks"]["fft_groups"] <= 4
            n = dev(packed(systems))
            out = torch.empty_like(n)
            pl.rhs(n, out)
            pl.integrate(n, 1e-3, 2)
            torch.cuda.synchronize()
            res.append((out.cpu().numpy(), n.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])


@pytest.mark.parametrize("prec", PRECS)
def test_batched_integrate_diagnostics_layout(prec):
    systems = [wl.constant_monodisperse(3, 64), wl.random_cp(3, 50, [2, 2], seed=46),
               wl.random_cp(4, 40, [1, 2, 1], seed=47)]
    steps, dt = 20, 0.01
    with sag.Plan.batch([(s.N, s.D, s.ranks, s.factors, FMT[s.fmt]) for s in systems],
                        prec=prec) as pl:
        off = pl.layout()
        n = dev(packed(systems))
        diag = torch.zeros((steps + 1, len(systems), 3), dtype=torch.float64, device="cuda")
        pl.integrate(n, dt, steps, diag)
        torch.cuda.synchronize()
        n = n.cpu().numpy()
        diag = diag.cpu().numpy()
    for b, s in enumerate(systems):
        n_ref, d_ref = oracle.integrate(s.n0, s.D, s.ranks, s.factors, dt, steps)
        assert nerr(n[off[b]:off[b + 1]], n_ref, np.abs(n_ref).max()) < TOL[prec], b
        assert np.max(np.abs(diag[:, b, :2] - d_ref[:, :2])) < 1e3 * TOL[prec] * np.abs(d_ref).max(), b
        tot = diag[:, b, 1] + diag[:, b, 2]
        assert np.max(np.abs(tot - tot[0])) < 1e3 * TOL[prec] * tot[0], b


def test_batched_tt_plan():
    systems = [wl.brownian_tt(3, 300, [0.4, -0.2, 0.1]),
               wl.random_tt(4, 150, {2: [1, 2, 1], 3: [1, 3, 2, 1], 4: [1, 2, 2, 2, 1]}, seed=48)]
    with sag.Plan.batch([(s.N, s.D, s.ranks, s.factors, FMT[s.fmt]) for s in systems],
                        prec=sag.SAG_FP64) as pl:
        off = pl.layout()
        p, q, _ = run_parts(pl, packed(systems))
    for b, s in enumerate(systems):
        p_ref, q_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors, fmt=oracle.TT, mode=oracle.DIRECT)
        scale = np.abs(p_ref).max() + np.abs(q_ref).max()
        assert nerr(p[off[b]:off[b + 1]], p_ref, scale) < 1e-12, b
        assert nerr(q[off[b]:off[b + 1]], q_ref, scale) < 1e-12, b
