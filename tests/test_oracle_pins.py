"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle (``oracle/``) against something other than itself:
brute force against the low-rank route, closed forms derived from the
definitions of Sec. 1, invariants, textbook special cases, the explicit TT
cores printed in Sec. 2 and the rank bound of Theorem 1. No test here needs a
GPU or the CUDA library.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1905_09071_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(x, ref, scale=None):
    s = np.max(np.abs(ref)) if scale is None else scale
    return float(np.max(np.abs(np.asarray(x) - np.asarray(ref))) / s)


# ---------------------------------------------------------------- P1 brute vs low rank
@pytest.mark.parametrize("D,N,ranks", [(2, 9, [3]), (3, 7, [2, 3]), (4, 5, [2, 2, 3])])
@pytest.mark.parametrize("sym", [0, 1])
def test_brute_equals_direct_cp(D, N, ranks, sym):
    s = wl.random_cp(D, N, ranks, seed=11 + D)
    pb, qb, ob = oracle.rhs(s.n0, D, s.ranks, s.factors, mode=oracle.BRUTE, sym=sym, outflow=True)
    pd, qd, od = oracle.rhs(s.n0, D, s.ranks, s.factors, mode=oracle.DIRECT, sym=sym, outflow=True)
    scale = np.abs(pb).max() + np.abs(qb).max()
    assert _rel(pd, pb, scale) < 1e-14
    assert _rel(qd, qb, scale) < 1e-14
    assert abs(od - ob) <= 1e-14 * abs(ob)


@pytest.mark.parametrize("mode", [oracle.BRUTE, oracle.DIRECT])
def test_tt_diagonal_embedding_equals_cp(mode):
    s = wl.random_cp(4, 6, [3, 2, 2], seed=5)
    t = wl.cp_to_tt_diagonal(s)
    p1, q1, o1 = oracle.rhs(s.n0, 4, s.ranks, s.factors, mode=mode, outflow=True)
    p2, q2, o2 = oracle.rhs(t.n0, 4, t.ranks, t.factors, fmt=oracle.TT, mode=mode, outflow=True)
    scale = np.abs(p1).max() + np.abs(q1).max()
    assert _rel(p2, p1, scale) < 1e-14 and _rel(q2, q1, scale) < 1e-14
    assert abs(o2 - o1) <= 1e-13 * abs(o1)


def test_symmetrised_q_differs_from_literal_for_asymmetric_kernel():
    # Guards against the sym flag being ignored: a random CP kernel is not symmetric.
    s = wl.random_cp(3, 6, [2, 2], seed=3)
    _, q1 = oracle.rhs(s.n0, 3, s.ranks, s.factors, sym=1)
    _, q0 = oracle.rhs(s.n0, 3, s.ranks, s.factors, sym=0)
    assert _rel(q1, q0) > 1e-3


# ---------------------------------------------------------------- P2 monodisperse start
@pytest.mark.parametrize("mode", [oracle.BRUTE, oracle.DIRECT])
def test_constant_kernel_monodisperse_rhs(mode):
    D, N = 4, 8
    s = wl.constant_monodisperse(D, N)
    p, q = oracle.rhs(s.n0, D, s.ranks, s.factors, mode=mode)
    rhs = p + q
    want = np.zeros(N)
    want[0] = -sum(1.0 / math.factorial(d - 1) for d in range(2, D + 1))
    for d in range(2, D + 1):
        want[d - 1] += 1.0 / math.factorial(d)
    assert np.max(np.abs(rhs - want)) < 1e-15


# ---------------------------------------------------------------- P3 geometric closed forms
def _geometric(N, A=0.3, qr=0.8):
    k = np.arange(1, N + 1, dtype=np.float64)
    return A * qr ** (k - 1), A, qr


def _binom(n, k):
    return math.comb(int(n), int(k))


@pytest.mark.parametrize("mode", [oracle.BRUTE, oracle.DIRECT])
def test_geometric_constant_kernel(mode):
    D, N = 4, (12 if mode == oracle.BRUTE else 40)
    n, A, qr = _geometric(N)
    s = wl.constant_monodisperse(D, N)
    p, q = oracle.rhs(n, D, s.ranks, s.factors, mode=mode)
    M0 = n.sum()
    pw, qw = np.zeros(N), np.zeros(N)
    for d in range(2, D + 1):
        for k in range(d, N + 1):
            # compositions of k into d positive parts: binom(k-1, d-1)
            pw[k - 1] += A ** d * qr ** (k - d) * _binom(k - 1, d - 1) / math.factorial(d)
        qw += -n * M0 ** (d - 1) / math.factorial(d - 1)
    assert _rel(p, pw) < 1e-14
    assert _rel(q, qw) < 1e-14


@pytest.mark.parametrize("mode", [oracle.BRUTE, oracle.DIRECT])
def test_geometric_product_kernel(mode):
    # Rank-one kernel C = prod_m i_m: sum over compositions of prod i_m = binom(k+d-1, 2d-1).
    D, N = 4, (10 if mode == oracle.BRUTE else 40)
    n, A, qr = _geometric(N)
    i = wl.sizes(N)
    per = {d: np.broadcast_to(i, (d, 1, N)).copy() for d in range(2, D + 1)}
    ranks, f = wl.cp_from_vectors(D, N, per)
    p, q = oracle.rhs(n, D, ranks, f, mode=mode)
    M1 = (i * n).sum()
    pw, qw = np.zeros(N), np.zeros(N)
    for d in range(2, D + 1):
        for k in range(d, N + 1):
            pw[k - 1] += A ** d * qr ** (k - d) * _binom(k + d - 1, 2 * d - 1) / math.factorial(d)
        qw += -n * i * M1 ** (d - 1) / math.factorial(d - 1)
    assert _rel(p, pw) < 1e-14
    assert _rel(q, qw) < 1e-14


# ---------------------------------------------------------------- P4 total concentration
def test_m0_identity_constant_kernel_no_tail():
    # n supported on sizes <= N/D: no tuple leaves the system, so
    # sum_k rhs_k = -sum_d (d-1)/d! M0^d exactly.
    D, N = 4, 24
    rng = np.random.default_rng(7)
    n = np.zeros(N)
    n[: N // D] = rng.uniform(0.1, 1.0, N // D)
    s = wl.constant_monodisperse(D, N)
    p, q = oracle.rhs(n, D, s.ranks, s.factors)
    M0 = n.sum()
    want = -sum((d - 1) / math.factorial(d) * M0 ** d for d in range(2, D + 1))
    assert abs((p + q).sum() - want) < 1e-14 * abs(want)


def _scalar_rk2(f, M, dt, steps, method):
    """The two explicit second-order Runge-Kutta rules on a scalar ODE, written
    out from their textbook definitions (Sec. 3 states two evaluations per step)."""
    for _ in range(steps):
        k1 = f(M)
        if method == oracle.HEUN:      # explicit trapezoid
            M = M + 0.5 * dt * (k1 + f(M + dt * k1))
        else:                          # explicit midpoint
            M = M + dt * f(M + 0.5 * dt * k1)
    return M


@pytest.mark.parametrize("method", [oracle.HEUN, oracle.MIDPOINT])
def test_m0_discrete_rk2_matches_scalar_rk2(method):
    # For C = 1 the sizes sum to the scalar ODE dM0/dt = -M0^2/2 - M0^3/3 (D = 3,
    # no tail at these sizes), and the full system's RK2 step summed over k is the
    # same RK2 rule applied to that scalar ODE.
    s = wl.constant_monodisperse()  # D=3, N=64, n=e_1, dt=0.01, 100 steps
    n, diag = oracle.integrate(s.n0, s.D, s.ranks, s.factors, s.dt, s.steps, method=method)
    f = lambda M: -M * M / 2.0 - M ** 3 / 3.0
    Ms = _scalar_rk2(f, 1.0, s.dt, s.steps, method)
    assert abs(diag[-1, 0] - Ms) < 1e-14
    assert abs(n.sum() - Ms) < 1e-14
    # the other rule's scalar recursion is far away: the method flag is honoured
    other = _scalar_rk2(f, 1.0, s.dt, s.steps, oracle.MIDPOINT if method == oracle.HEUN else oracle.HEUN)
    assert abs(Ms - other) > 1e-8


def _m0_exact(t, a=0.5, b=1.0 / 3.0):
    # dM/dt = -M^2 (a + b M): F(M) = -1/(aM) + (b/a^2) ln((a+bM)/M), F(M(t)) - F(1) = -t.
    F = lambda M: -1.0 / (a * M) + b / a ** 2 * math.log((a + b * M) / M)
    target = F(1.0) - t
    lo, hi = 1e-6, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if F(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("method", [oracle.HEUN, oracle.MIDPOINT])
def test_m0_exact_solution_second_order(method):
    exact = _m0_exact(1.0)
    assert abs(exact - 0.5724637494) < 1e-9
    errs = []
    for steps in (50, 100, 200):
        s = wl.constant_monodisperse()
        _, diag = oracle.integrate(s.n0, s.D, s.ranks, s.factors, 1.0 / steps, steps, method=method)
        errs.append(abs(diag[-1, 0] - exact))
    assert errs[1] < 1e-5
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.5 < e0 / e1 < 4.5  # second order


# ---------------------------------------------------------------- P5 mass invariant
@pytest.mark.parametrize("D,N,ranks", [(3, 7, [2, 2]), (4, 5, [2, 2, 2])])
def test_m1_identity_equals_outflow(D, N, ranks):
    s = wl.random_cp(D, N, ranks, seed=21)
    p, q, o = oracle.rhs(s.n0, D, s.ranks, s.factors, mode=oracle.BRUTE, outflow=True)
    k = wl.sizes(N)
    assert abs((k * (p + q)).sum() + o) < 1e-13 * abs(o)


@pytest.mark.parametrize("method", [oracle.HEUN, oracle.MIDPOINT])
def test_m1_plus_cumulative_outflow_is_conserved(method):
    # Per step M1 falls by the RK2 rule's quadrature of the outflow: Heun
    # dt/2 (O(n) + O(n*)), midpoint dt O(n*).
    s = wl.random_cp(3, 16, [2, 3], seed=4)
    _, diag = oracle.integrate(s.n0, 3, s.ranks, s.factors, 0.05, 20, method=method)
    total = diag[:, 1] + diag[:, 2]
    assert np.max(np.abs(total - total[0])) < 1e-14 * total[0]
    assert diag[-1, 2] > 0


# ---------------------------------------------------------------- P6 binary textbook case
@pytest.mark.parametrize("method", [oracle.HEUN, oracle.MIDPOINT])
def test_binary_constant_kernel_closed_form(method):
    # D=2, C=1, n(0)=e_1: n_k(t) = tau^{k-1}/(1+tau)^{k+1}, tau = t/2; every
    # component is pinned and the error falls 4x when dt halves (second order).
    N, T = 200, 0.6
    s = wl.constant_monodisperse(2, N)
    k = wl.sizes(N)
    tau = T / 2
    exact = tau ** (k - 1) / (1 + tau) ** (k + 1)
    errs = []
    for steps in (30, 60):
        n, _ = oracle.integrate(s.n0, 2, s.ranks, s.factors, T / steps, steps, method=method, diag=False)
        errs.append(np.max(np.abs(n - exact)))
    assert errs[1] < 2e-5
    assert 3.5 < errs[0] / errs[1] < 4.5
    # The closed form satisfies the truncated right-hand side up to its tail.
    p, q = oracle.rhs(exact, 2, s.ranks, s.factors)
    dndt = (tau ** (k - 2) * (k - 1 - 2 * tau)) / (2 * (1 + tau) ** (k + 2))
    assert np.max(np.abs(p + q - dndt)) < 1e-15


# ---------------------------------------------------------------- P7 kernel identities
def test_brownian_cp_is_eq17_combination():
    # (sum i^{1/3})(sum i^{-1/3}) = C^(d)[1/3,-1/3,0..]/(d-2)! + C^(d)[0..0]/(d-1)!
    s = wl.brownian_cp(3, 6)
    rng = np.random.default_rng(1)
    for d in (2, 3):
        mu1 = [1 / 3, -1 / 3] + [0.0] * (d - 2)
        mu0 = [0.0] * d
        for _ in range(20):
            idx = rng.integers(1, 7, d)
            got = oracle.kernel_entry(oracle.CP, 3, 6, s.ranks, s.factors, idx)
            want = (oracle.brownian_entry(mu1, idx) / math.factorial(d - 2)
                    + oracle.brownian_entry(mu0, idx) / math.factorial(d - 1))
            assert abs(got - want) < 1e-13 * abs(want)


def _tt_contract(ranks, cores, N, idx):
    off, v = 0, np.ones(1)
    for l in range(1, len(ranks)):
        H = cores[off: off + ranks[l - 1] * ranks[l] * N].reshape(ranks[l - 1], ranks[l], N)
        v = v @ H[:, :, idx[l - 1] - 1]
        off += ranks[l - 1] * ranks[l] * N
    return float(v[0])


@pytest.mark.parametrize("D", [2, 3, 4, 5])
def test_theorem1_cores_reproduce_eq17(D):
    N = 5
    rng = np.random.default_rng(D)
    mu = rng.uniform(-0.5, 0.5, D)
    ranks, cores = oracle.brownian_tt(mu, N)
    assert list(ranks) == [math.comb(D, l) for l in range(D + 1)]
    for _ in range(30):
        idx = rng.integers(1, N + 1, D)
        want = oracle.brownian_entry(mu, idx)
        assert abs(_tt_contract(ranks, cores, N, idx) - want) < 1e-13 * abs(want)


@pytest.mark.parametrize("D", [3, 4])
def test_tt_ranks_bounded_by_theorem1(D):
    # Ranks of the unfoldings of the full tensor never exceed binom(D, lambda).
    N = 7
    mu = np.random.default_rng(9).uniform(-0.6, 0.6, D)
    full = np.zeros((N,) * D)
    for idx in np.ndindex(*full.shape):
        full[idx] = oracle.brownian_entry(mu, np.array(idx) + 1)
    for l in range(1, D):
        mat = full.reshape(N ** l, -1)
        sv = np.linalg.svd(mat, compute_uv=False)
        rank = int((sv > 1e-11 * sv[0]).sum())
        assert rank <= math.comb(D, l)


def _read_golden_patterns():
    pats = {}
    with open(os.path.join(GOLDEN, "brownian_tt_d2_d3_cores.txt")) as fh:
        lines = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        _, D, lam, rows, cols = lines[i]
        D, lam, rows, cols = int(D), int(lam), int(rows), int(cols)
        pats[(D, lam)] = np.array([[int(x) for x in lines[i + 1 + r]] for r in range(rows)])
        assert pats[(D, lam)].shape == (rows, cols)
        i += 1 + rows
    return pats


@pytest.mark.parametrize("D", [2, 3])
def test_printed_cores_reproduce_eq17(D):
    pats = _read_golden_patterns()
    N = 6
    rng = np.random.default_rng(30 + D)
    mu = rng.uniform(-0.5, 0.5, D)
    ranks = [1] + [pats[(D, l)].shape[1] for l in range(1, D + 1)]
    i = wl.sizes(N)
    blocks = []
    for l in range(1, D + 1):
        pat = pats[(D, l)]
        H = np.zeros(pat.shape + (N,))
        for a in range(pat.shape[0]):
            for b in range(pat.shape[1]):
                if pat[a, b]:
                    H[a, b] = i ** mu[pat[a, b] - 1]
        blocks.append(H.reshape(-1))
    cores = np.concatenate(blocks)
    for idx in np.ndindex(*(N,) * D):
        idx = np.array(idx) + 1
        want = oracle.brownian_entry(mu, idx)
        assert abs(_tt_contract(ranks, cores, N, idx) - want) < 1e-13 * abs(want)


def test_theorem1_tt_rhs_matches_brute_force():
    D, N = 3, 6
    mu = [0.4, -0.2, 0.1]
    ranks3, cores3 = oracle.brownian_tt(mu, N)
    ranks2, cores2 = oracle.brownian_tt(mu[:2], N)
    ranks = list(ranks2) + list(ranks3)
    f = np.concatenate([cores2, cores3])
    n = np.random.default_rng(2).uniform(0, 1, N)
    pb, qb, ob = oracle.rhs(n, D, ranks, f, fmt=oracle.TT, mode=oracle.BRUTE, outflow=True)
    pd, qd, od = oracle.rhs(n, D, ranks, f, fmt=oracle.TT, mode=oracle.DIRECT, outflow=True)
    scale = np.abs(pb).max() + np.abs(qb).max()
    assert _rel(pd, pb, scale) < 1e-14 and _rel(qd, qb, scale) < 1e-14
    assert abs(od - ob) < 1e-13 * abs(ob)


@pytest.mark.parametrize("D", [2, 3, 4])
def test_workload_theorem1_cores_reproduce_eq17(D):
    # The input generator's TT cores (used as GPU inputs) against the oracle's
    # permutation-sum definition of Eq. ch3.eq17.
    N = 5
    mu = np.random.default_rng(40 + D).uniform(-0.5, 0.5, D)
    ranks, cores = wl.brownian_tt_cores(list(mu), N)
    assert ranks == [math.comb(D, l) for l in range(D + 1)]
    rng = np.random.default_rng(D)
    for _ in range(30):
        idx = rng.integers(1, N + 1, D)
        want = oracle.brownian_entry(mu, idx)
        assert abs(_tt_contract(ranks, cores, N, idx) - want) < 1e-13 * abs(want)


# ---------------------------------------------------------------- P9 adjoint
def _F(n, D, ranks, f, sym):
    p, q = oracle.rhs(n, D, ranks, f, sym=sym)
    return p + q


@pytest.mark.parametrize("sym", [1, 0])
@pytest.mark.parametrize("D,N,ranks", [(2, 11, [3]), (3, 9, [2, 3]), (4, 7, [2, 1, 2])])
def test_rhs_vjp_matches_central_differences(D, N, ranks, sym):
    s = wl.random_cp(D, N, ranks, seed=60 + D)
    rng = np.random.default_rng(61)
    g = rng.normal(size=N)
    un = rng.normal(size=N)
    uf = rng.normal(size=s.factors.size)
    gn, gU = oracle.rhs_vjp(s.n0, g, D, s.ranks, s.factors, sym=sym)
    h = 1e-6
    dn = (_F(s.n0 + h * un, D, s.ranks, s.factors, sym) - _F(s.n0 - h * un, D, s.ranks, s.factors, sym)) / (2 * h)
    df = (_F(s.n0, D, s.ranks, s.factors + h * uf, sym) - _F(s.n0, D, s.ranks, s.factors - h * uf, sym)) / (2 * h)
    assert abs(g @ dn - gn @ un) < 1e-8 * (abs(g) @ abs(dn) + 1e-30)
    assert abs(g @ df - gU @ uf) < 1e-8 * (abs(g) @ abs(df) + 1e-30)


@pytest.mark.parametrize("method", [oracle.HEUN, oracle.MIDPOINT])
def test_integrate_vjp_matches_central_differences(method):
    D, N = 3, 12
    s = wl.random_cp(D, N, [2, 2], seed=70)
    rng = np.random.default_rng(71)
    g = rng.normal(size=N)
    un = rng.normal(size=N)
    uf = rng.normal(size=s.factors.size)
    dt, steps = 0.05, 6
    gn0, gU = oracle.integrate_vjp(s.n0, D, s.ranks, s.factors, dt, steps, g, method=method)

    def L(n0, f):
        n, _ = oracle.integrate(n0, D, s.ranks, f, dt, steps, method=method, diag=False)
        return g @ n

    h = 1e-6
    d_n = (L(s.n0 + h * un, s.factors) - L(s.n0 - h * un, s.factors)) / (2 * h)
    d_f = (L(s.n0, s.factors + h * uf) - L(s.n0, s.factors - h * uf)) / (2 * h)
    assert abs(d_n - gn0 @ un) < 1e-7 * abs(d_n)
    assert abs(d_f - gU @ uf) < 1e-7 * abs(d_f)


def test_paper_ternary_forms_agree():
    # Pure ternary Brownian kernel (only the d = 3 term; the d = 2 order is
    # absent: CP rank 0, or an all-zero TT order): brute force over the kernel
    # entries of both forms, and the direct modes, agree.
    s = wl.paper_ternary(40, "cp")
    t = wl.paper_ternary(40, "tt")
    pb, qb = oracle.rhs(s.n0, s.D, s.ranks, s.factors, mode=oracle.BRUTE)
    scale = np.abs(pb).max() + np.abs(qb).max()
    for sysm, fmt in ((s, oracle.CP), (t, oracle.TT)):
        for mode in (oracle.BRUTE, oracle.DIRECT):
            p, q = oracle.rhs(sysm.n0, sysm.D, sysm.ranks, sysm.factors, mode=mode, fmt=fmt)
            assert np.abs(p - pb).max() / scale < 1e-14
            assert np.abs(q - qb).max() / scale < 1e-14
    # the d = 2 order contributes nothing: a D = 3 system whose d = 2 factors
    # are zero gives the same right-hand side
    z = wl.cp_from_vectors(3, 40, {2: np.zeros((2, 1, 40)),
                                  3: s.factors.reshape(3, 6, 40)})
    p, q = oracle.rhs(s.n0, 3, z[0], z[1], mode=oracle.DIRECT)
    assert np.abs(p - pb).max() / scale < 1e-14 and np.abs(q - qb).max() / scale < 1e-14


# ---------------------------------------------------------------- TT adjoint
def _F_tt(n, D, ranks, f, sym):
    p, q = oracle.rhs(n, D, ranks, f, fmt=oracle.TT, sym=sym)
    return p + q


@pytest.mark.parametrize("sym", [1, 0])
@pytest.mark.parametrize("D,N,ranks", [(2, 10, {2: [1, 3, 1]}), (3, 9, {2: [1, 2, 1], 3: [1, 2, 3, 1]}),
                                       (4, 7, {2: [1, 1, 1], 3: [1, 2, 2, 1], 4: [1, 2, 3, 2, 1]})])
def test_tt_rhs_vjp_matches_central_differences(D, N, ranks, sym):
    t = wl.random_tt(D, N, ranks, seed=90 + D)
    rng = np.random.default_rng(91)
    g, un, uf = rng.normal(size=N), rng.normal(size=N), rng.normal(size=t.factors.size)
    gn, gH = oracle.rhs_vjp(t.n0, g, D, t.ranks, t.factors, sym=sym, fmt=oracle.TT)
    h = 1e-6
    dn = (_F_tt(t.n0 + h * un, D, t.ranks, t.factors, sym) - _F_tt(t.n0 - h * un, D, t.ranks, t.factors, sym)) / (2 * h)
    df = (_F_tt(t.n0, D, t.ranks, t.factors + h * uf, sym) - _F_tt(t.n0, D, t.ranks, t.factors - h * uf, sym)) / (2 * h)
    assert abs(g @ dn - gn @ un) < 1e-8 * (abs(g) @ abs(dn) + 1e-30)
    assert abs(g @ df - gH @ uf) < 1e-8 * (abs(g) @ abs(df) + 1e-30)


@pytest.mark.parametrize("sym", [1, 0])
def test_tt_vjp_of_diagonal_embedding_equals_cp_vjp(sym):
    # The CP kernel and its TT diagonal embedding are the same function of n,
    # and each CP factor value sits at one core entry: the n-cotangents agree,
    # and so do the factor cotangents at the embedded entries.
    s = wl.random_cp(4, 8, [2, 3, 2], seed=5)
    t = wl.cp_to_tt_diagonal(s)
    g = np.random.default_rng(6).normal(size=s.N)
    gn1, gU = oracle.rhs_vjp(s.n0, g, 4, s.ranks, s.factors, sym=sym)
    gn2, gH = oracle.rhs_vjp(t.n0, g, 4, t.ranks, t.factors, sym=sym, fmt=oracle.TT)
    assert np.abs(gn1 - gn2).max() < 1e-14 * np.abs(gn1).max()
    offs = wl.cp_layout(4, s.N, s.ranks)
    toff = 0
    for d in range(2, 5):
        R = s.ranks[d - 2]
        gUd = gU[offs[d - 2]:offs[d - 1]].reshape(d, R, s.N)
        rk = [1] + [R] * (d - 1) + [1]
        for l in range(1, d + 1):
            blk = gH[toff:toff + rk[l - 1] * rk[l] * s.N].reshape(rk[l - 1], rk[l], s.N)
            toff += rk[l - 1] * rk[l] * s.N
            for r in range(R):
                emb = blk[0, r] if l == 1 else blk[r, 0] if l == d else blk[r, r]
                assert np.abs(emb - gUd[l - 1, r]).max() < 1e-14 * np.abs(gU).max()


def test_tt_integrate_vjp_matches_central_differences():
    D, N = 3, 10
    t = wl.random_tt(D, N, {2: [1, 2, 1], 3: [1, 2, 2, 1]}, seed=95)
    rng = np.random.default_rng(96)
    g, un, uf = rng.normal(size=N), rng.normal(size=N), rng.normal(size=t.factors.size)
    dt, steps = 0.05, 5
    gn0, gH = oracle.integrate_vjp(t.n0, D, t.ranks, t.factors, dt, steps, g, fmt=oracle.TT)

    def L(n0, f):
        n, _ = oracle.integrate(n0, D, t.ranks, f, dt, steps, fmt=oracle.TT, diag=False)
        return g @ n

    h = 1e-6
    d_n = (L(t.n0 + h * un, t.factors) - L(t.n0 - h * un, t.factors)) / (2 * h)
    d_f = (L(t.n0, t.factors + h * uf) - L(t.n0, t.factors - h * uf)) / (2 * h)
    assert abs(d_n - gn0 @ un) < 1e-7 * abs(d_n)
    assert abs(d_f - gH @ uf) < 1e-7 * abs(d_f)
