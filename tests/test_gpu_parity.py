"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Error metric (normwise, as the gain and loss parts can cancel):
    err = max_k |x_k - x_ref_k| / (max |P_ref| + max |Q_ref|).
Tolerances: FP64 path 1e-12; double-word FP32 paths 1e-10 with grid-aligned
butterflies (SAG_FP32_SPLIT) and 1e-12 with plain double-word butterflies
(SAG_FP32_SPLIT_EXACT). Trajectories are compared relative to max |n_ref|.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1905_09071_gb300 import sag, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {sag.SAG_FP64: 1e-12, sag.SAG_FP32_SPLIT: 1e-10, sag.SAG_FP32_SPLIT_EXACT: 1e-12}
PRECS = [sag.SAG_FP64, sag.SAG_FP32_SPLIT, sag.SAG_FP32_SPLIT_EXACT]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def gpu_parts(s, n0, prec, sym=1, rk=sag.SAG_HEUN, check=None, **kw):
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec, symmetrize_q=sym, rk=rk, **kw) as pl:
        if check:
            check(pl.describe())
        n = dev(n0)
        p, q = torch.empty_like(n), torch.empty_like(n)
        o = torch.zeros(1, dtype=torch.float64, device="cuda")
        pl.rhs_parts(n, p, q, o)
        out = torch.empty_like(n)
        pl.rhs(n, out)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
        return p.cpu().numpy(), q.cpu().numpy(), float(o.item()), out.cpu().numpy()


def nerr(x, ref, scale):
    return float(np.max(np.abs(np.asarray(x) - ref)) / scale)


# ------------------------------------------------------------------ RHS parity
SMALL = [
    ("D2_N1", lambda: wl.random_cp(2, 1, [2], seed=1)),
    ("D3_N2", lambda: wl.random_cp(3, 2, [1, 2], seed=2)),
    ("D4_N3", lambda: wl.random_cp(4, 3, [2, 1, 2], seed=3)),
    ("D2_N9", lambda: wl.random_cp(2, 9, [3], seed=4)),
    ("D3_N7", lambda: wl.random_cp(3, 7, [2, 3], seed=5)),
    ("D4_N5", lambda: wl.random_cp(4, 5, [2, 2, 3], seed=6)),
    ("D6_N3", lambda: wl.random_cp(6, 3, [1, 2, 1, 1, 2], seed=7)),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("sym", [0, 1])
@pytest.mark.parametrize("name,make", SMALL)
def test_rhs_matches_brute_force(name, make, sym, prec):
    s = make()
    p_ref, q_ref, o_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors, mode=oracle.BRUTE, sym=sym,
                                     outflow=True)
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    p, q, o, r = gpu_parts(s, s.n0, prec, sym)
    assert nerr(p, p_ref, scale) < TOL[prec]
    assert nerr(q, q_ref, scale) < TOL[prec]
    assert nerr(r, p_ref + q_ref, scale) < TOL[prec]
    # outflow is a difference of two first-moment fluxes of size ~ sum k |P_k|
    flux = np.sum(np.arange(1, s.N + 1) * np.abs(p_ref)) + abs(o_ref) + 1e-300
    assert abs(o - o_ref) <= 1e3 * TOL[prec] * flux


MEDIUM = [
    ("D3_N100_ragged", lambda: wl.random_cp(3, 100, [3, 4], seed=8)),
    ("D4_N333_ragged", lambda: wl.random_cp(4, 333, [2, 3, 2], seed=9)),
    ("D2_N1000_R40", lambda: wl.random_cp(2, 1000, [40], seed=10)),
    ("D4_N1537_ragged", lambda: wl.random_cp(4, 1537, [3, 2, 2], seed=11)),
    ("brownian_D3_N4096", lambda: wl.brownian_cp(3, 4096)),
    ("D8_N40", lambda: wl.random_cp(8, 40, [2, 1, 1, 2, 1, 1, 2], seed=17)),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,make", MEDIUM)
def test_rhs_matches_direct_oracle(name, make, prec):
    s = make()
    p_ref, q_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors, mode=oracle.DIRECT)
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    p, q, _, r = gpu_parts(s, s.n0, prec)
    assert nerr(p, p_ref, scale) < TOL[prec]
    assert nerr(q, q_ref, scale) < TOL[prec]
    assert nerr(r, p_ref + q_ref, scale) < TOL[prec]


def _prefix(s, K):
    """The same kernel restricted to sizes 1..K: its gain term equals the full
    system's gain term at every size k <= K."""
    offs = wl.cp_layout(s.D, s.N, s.ranks)
    per = {}
    for d in range(2, s.D + 1):
        R = s.ranks[d - 2]
        per[d] = s.factors[offs[d - 2]:offs[d - 1]].reshape(d, R, s.N)[:, :, :K]
    ranks, f = wl.cp_from_vectors(s.D, K, per)
    return ranks, f


@pytest.fixture(scope="module")
def throughput_case():
    s = wl.random_power_cp()  # D=4, N=65536, R=16: the throughput workload
    K = 2048
    ranks_k, f_k = _prefix(s, K)
    p_pre, _ = oracle.rhs(s.n0[:K], s.D, ranks_k, f_k, mode=oracle.DIRECT)
    q_ref = oracle.loss(s.n0, s.D, s.ranks, s.factors)
    return s, K, p_pre, q_ref


def test_fp32_split_loss_sizewise(throughput_case):
    # The FP32-split path keeps the inner products s_v = <U_v, n> and
    # q = n sum_v coef_v U_v in FP64 beside its double-word FFTs: every loss
    # output at N = 65536 against the oracle, sizewise relative error.
    s, _, _, q_ref = throughput_case
    _, q, _, _ = gpu_parts(s, s.n0, sag.SAG_FP32_SPLIT)
    # The state decays to subnormal and zero values at the largest sizes; q
    # follows it there, and a sizewise relative error means nothing for
    # subnormal values.
    nz = s.n0 > 1e-290
    assert nz.sum() > 1000 and np.all(q_ref[nz] < 0)
    assert np.all(q[s.n0 == 0] == 0.0)
    assert float(np.max(np.abs(q[nz] - q_ref[nz]) / np.abs(q_ref[nz]))) < 1e-13


@pytest.mark.parametrize("prec", [sag.SAG_FP32_SPLIT, sag.SAG_FP32_SPLIT_EXACT])
@pytest.mark.parametrize("scale", [1e-40, 1e40])
def test_loss_at_extreme_factor_scales(prec, scale):
    # Factors near 1e+-40 (beyond FP32's range, so the double-word copies
    # rely on their per-vector powers of two), loss weights near 1e+-80, and
    # a state of mixed sign: the loss against the oracle.
    t = wl.random_cp(3, 3000, [3, 2], seed=111)
    f = t.factors * scale
    n0 = t.n0 * np.where(np.arange(t.N) % 7 == 3, -1.0, 1.0)
    q_ref = oracle.loss(n0, t.D, t.ranks, f)
    _, q, _, _ = gpu_parts(wl.System(t.D, t.N, "cp", t.ranks, f, n0), n0, prec)
    assert nerr(q, q_ref, np.abs(q_ref).max()) < 1e-13


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_sampled_parity(throughput_case, prec):
    # N = 65536: every gain output k <= 2048 against the oracle on the prefix
    # system, every loss output against the oracle's inner-product route.
    s, K, p_pre, q_ref = throughput_case
    p, q, _, r = gpu_parts(s, s.n0, prec)
    scale = np.abs(p).max() + np.abs(q_ref).max()
    assert np.abs(p).max() <= 1.0001 * np.abs(p_pre).max() + 1e-300  # the maximum is in the prefix
    assert nerr(p[:K], p_pre, scale) < TOL[prec]
    assert nerr(q, q_ref, scale) < TOL[prec]
    assert nerr(r[:K], p_pre + q_ref[:K], scale) < TOL[prec]


# Four-step splits M = M1 M2 with M2 capped: pair-form columns of 512, 768 and
# 1024 points (max_m2 = 128); 1024-point pair columns, a compile-time
# 1536-point column of single vectors and a 2048-point run-time column
# (max_m2 = 64).
CAPPED_SPLITS = {128: [[512, 128, 1], [768, 128, 1], [1024, 128, 1]],
                 64: [[1024, 64, 1], [1536, 64, 0], [2048, 64, 0]]}


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("max_m2", sorted(CAPPED_SPLITS))
def test_capped_row_length_parity(throughput_case, prec, max_m2):
    s, K, p_pre, q_ref = throughput_case

    def check(desc):
        got = [[o["M1"], o["M2"], o["pairs"]] for o in desc["orders"]]
        want = [[m1, m2, pr if prec != sag.SAG_FP64 else 0] for m1, m2, pr in CAPPED_SPLITS[max_m2]]
        assert got == want

    p, q, _, r = gpu_parts(s, s.n0, prec, max_m2=max_m2, check=check)
    scale = np.abs(p).max() + np.abs(q_ref).max()
    assert nerr(p[:K], p_pre, scale) < TOL[prec]
    assert nerr(q, q_ref, scale) < TOL[prec]
    assert nerr(r[:K], p_pre + q_ref[:K], scale) < TOL[prec]


@pytest.mark.parametrize("prec", [sag.SAG_FP32_SPLIT, sag.SAG_FP32_SPLIT_EXACT])
def test_geometry_autotuner(throughput_case, prec):
    # The rule's splits are timed first, then d = 2, 3 and 4 in turn with M2
    # halved (d = 4: 1024-point pair columns); the plan keeps the last
    # candidate marked kept, and its results match the oracle.
    s, K, p_pre, q_ref = throughput_case
    seen = {}

    def check(desc):
        seen.update(desc)

    p, q, _, r = gpu_parts(s, s.n0, prec, autotune=1, check=check)
    log = seen["geometry_autotune"]
    assert len(log) == 4
    assert log[0]["splits"] == [[256, 256], [384, 256], [512, 256]] and log[0]["kept"]
    assert log[1]["splits"] == [[512, 128], [384, 256], [512, 256]]
    assert log[2]["splits"][1] == [768, 128] and log[2]["splits"][2] == [512, 256]
    assert log[3]["splits"][2] == [1024, 128]
    assert all(e["ms_per_step"] > 0 for e in log)
    chosen = [[o["M1"], o["M2"]] for o in seen["orders"]]
    assert chosen == [e for e in log if e["kept"]][-1]["splits"]
    assert all(o["pairs"] == 1 for o in seen["orders"])
    scale = np.abs(p).max() + np.abs(q_ref).max()
    assert nerr(p[:K], p_pre, scale) < TOL[prec]
    assert nerr(q, q_ref, scale) < TOL[prec]
    assert nerr(r[:K], p_pre + q_ref[:K], scale) < TOL[prec]


def test_m2_reproduces_tuned_splits(throughput_case):
    # Passing back the splits an autotuned plan reports builds the same
    # geometry without tuning, with bitwise the same right-hand side.
    s, K, p_pre, q_ref = throughput_case
    outs, splits = [], None
    for kw in (dict(autotune=1), "m2"):
        if kw == "m2":
            kw = dict(m2=splits)
        with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=sag.SAG_FP32_SPLIT, **kw) as pl:
            desc = pl.describe()
            got = [o["M2"] for o in desc["orders"]]
            if splits is None:
                splits = got
            else:
                assert got == splits and desc["geometry_autotune"] == []
            n = dev(s.n0)
            out = torch.empty_like(n)
            pl.rhs(n, out)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    with pytest.raises(sag.SagError):  # one entry per order
        sag.Plan(s.N, s.D, s.ranks, s.factors, m2=splits[:2])
    with pytest.raises(sag.SagError):  # M2 must divide M = L/2 = 65536 (d = 2) with M1 <= 4096
        sag.Plan(s.N, s.D, s.ranks, s.factors, m2=[8, 0, 0])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("fmt", ["cp", "tt"])
def test_paper_shape_sampled_parity(fmt, prec):
    # The paper's Sec. 3 shape at full size (pure ternary Brownian kernel,
    # N = 2^19, FFT length 3 2^19): every gain output k <= 2048 against the
    # oracle on the size prefix (CP form), every loss output against the
    # oracle's inner-product route; the TT form computes the same kernel.
    s = wl.paper_ternary(1 << 19, "cp")
    K = 2048
    ranks_k, f_k = _prefix(s, K)
    p_pre, _ = oracle.rhs(s.n0[:K], s.D, ranks_k, f_k, mode=oracle.DIRECT)
    q_ref = oracle.loss(s.n0, s.D, s.ranks, s.factors)
    g = s if fmt == "cp" else wl.paper_ternary(1 << 19, "tt")
    with sag.Plan(g.N, g.D, g.ranks, g.factors, fmt=sag.SAG_TT if fmt == "tt" else sag.SAG_CP,
                  prec=prec) as pl:
        n = dev(g.n0)
        p, q = torch.empty_like(n), torch.empty_like(n)
        pl.rhs_parts(n, p, q)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
        p, q = p.cpu().numpy(), q.cpu().numpy()
    scale = np.abs(p).max() + np.abs(q_ref).max()
    assert np.abs(p).max() <= 1.0001 * np.abs(p_pre).max() + 1e-300  # the maximum is in the prefix
    assert nerr(p[:K], p_pre, scale) < TOL[prec]
    assert nerr(q, q_ref, scale) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_factor_update_that_separates_repeated_vectors(prec):
    # The Brownian CP kernel repeats vectors (the ones vector in many terms).
    # A plan that shares their transforms refuses new factors that make them
    # differ and keeps its old ones; a plan made with keep_repeats = 1
    # transforms every vector and takes the update.
    s = wl.brownian_cp(3, 500)
    f2 = s.factors.copy()
    f2[:s.N] *= 1.0 + 1e-3 * wl.sizes(s.N) / s.N  # order 2, mode 0, term 0: a ones vector
    p_old, q_old = oracle.rhs(s.n0, s.D, s.ranks, s.factors, mode=oracle.DIRECT)
    p_new, q_new = oracle.rhs(s.n0, s.D, s.ranks, f2, mode=oracle.DIRECT)
    for keep, f_ref in ((0, (p_old, q_old)), (1, (p_new, q_new))):
        with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec, keep_repeats=keep) as pl:
            o = pl.describe()["orders"]
            assert all((x["transformed"] == x["vectors"]) == bool(keep) for x in o)
            if keep:
                pl.update_factors(f2)
            else:
                with pytest.raises(sag.SagError, match="keep_repeats"):
                    pl.update_factors(f2)
            n = dev(s.n0)
            p, q = torch.empty_like(n), torch.empty_like(n)
            pl.rhs_parts(n, p, q)
            torch.cuda.synchronize()
            assert pl.sync_status() == sag.SAG_OK
        scale = np.abs(f_ref[0]).max() + np.abs(f_ref[1]).max()
        assert nerr(p.cpu().numpy(), f_ref[0], scale) < TOL[prec]
        assert nerr(q.cpu().numpy(), f_ref[1], scale) < TOL[prec]
    with pytest.raises(sag.SagError):
        sag.Plan(s.N, s.D, s.ranks, s.factors, keep_repeats=2)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,m2", [(12000, 128), (50000, 256)])
def test_repeated_vector_rows_sampled_parity(N, m2, prec):
    # The Brownian CP kernel repeats its factor vectors (27 vectors, 3
    # distinct, for d = 3): the row pass transforms each distinct spectrum
    # once and forms the rank terms from those rows. N = 12000 and 50000 put
    # the d = 3 rows at 128 and 256 points (the Brownian configuration and the
    # paper shape cover 64 and 512). A slowly decaying start keeps every size
    # in play; gain outputs k <= 2048 against the oracle on the size prefix,
    # every loss output against its inner-product route.
    b = wl.brownian_cp(3, N)
    n0 = wl.normalised(np.exp(-wl.sizes(N) / (N / 8)))
    s = wl.System(3, N, "cp", b.ranks, b.factors, n0)
    K = 2048
    ranks_k, f_k = _prefix(s, K)
    p_pre, _ = oracle.rhs(n0[:K], s.D, ranks_k, f_k, mode=oracle.DIRECT)
    q_ref = oracle.loss(n0, s.D, s.ranks, s.factors)
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec) as pl:
        o3 = pl.describe()["orders"][-1]
        assert o3["transformed"] == 3 and o3["vectors"] == 27
        if prec != sag.SAG_FP64:
            assert o3["M2"] == m2 and o3["compile_time"][1] == 1
        n = dev(n0)
        p, q = torch.empty_like(n), torch.empty_like(n)
        pl.rhs_parts(n, p, q)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
        p, q = p.cpu().numpy(), q.cpu().numpy()
    scale = np.abs(p).max() + np.abs(q_ref).max()
    assert nerr(p[:K], p_pre, scale) < TOL[prec]
    assert nerr(q, q_ref, scale) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kernel", ["constant", "product"])
def test_full_length_fft_geometric_closed_form(kernel, prec):
    # n_k = A r^(k-1) at N = 65536, D = 4 (FFT lengths 2^17, 3 2^16, 2^18):
    # constant kernel p_k^(d) = A^d r^(k-d) binom(k-1, d-1)/d!,
    # product kernel C = prod i_m: p_k^(d) = A^d r^(k-d) binom(k+d-1, 2d-1)/d!.
    N, D, A, rr = 65536, 4, 1e-4, 0.9999
    k = np.arange(1, N + 1, dtype=np.float64)
    n0 = A * rr ** (k - 1)
    vec = np.ones(N) if kernel == "constant" else k.copy()
    per = {d: np.broadcast_to(vec, (d, 1, N)).copy() for d in range(2, D + 1)}
    ranks, f = wl.cp_from_vectors(D, N, per)
    s = wl.System(D, N, "cp", ranks, f, n0)
    p, q, _, _ = gpu_parts(s, n0, prec)
    def binom(a, b):  # exact products for the small b used here
        out = np.ones_like(a)
        for i in range(b):
            out = out * (a - i) / (i + 1)
        return out

    p_ref = np.zeros(N)
    for d in range(2, D + 1):
        kk = k[d - 1:]
        b = binom(kk - 1, d - 1) if kernel == "constant" else binom(kk + d - 1, 2 * d - 1)
        p_ref[d - 1:] += A ** d * rr ** (kk - d) * b / math.factorial(d)
    if kernel == "constant":
        M = n0.sum()
        q_ref = sum(-n0 * M ** (d - 1) / math.factorial(d - 1) for d in range(2, D + 1))
    else:
        M1 = (k * n0).sum()
        q_ref = sum(-n0 * k * M1 ** (d - 1) / math.factorial(d - 1) for d in range(2, D + 1))
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    assert nerr(p, p_ref, scale) < max(TOL[prec], 1e-11)
    assert nerr(q, q_ref, scale) < max(TOL[prec], 1e-11)


# ------------------------------------------------------------------ buffers and status
def test_host_buffers_equal_device_buffers():
    s = wl.random_cp(3, 500, [3, 3], seed=12)
    with sag.Plan(s.N, s.D, s.ranks, s.factors) as pl:
        out_h = np.zeros(s.N)
        pl.rhs(s.n0.copy(), out_h)
        n = dev(s.n0)
        out_d = torch.empty_like(n)
        pl.rhs(n, out_d)
        torch.cuda.synchronize()
        assert np.array_equal(out_h, out_d.cpu().numpy())
        nh = s.n0.copy()
        pl.rk2_step(nh, 1e-2)
        pl.rk2_step(n, 1e-2)
        torch.cuda.synchronize()
        assert np.array_equal(nh, n.cpu().numpy())


@pytest.mark.parametrize("prec", PRECS)
def test_launches_per_step(prec):
    # One RK2 step's graph: per stage the side branch (k_dot, k_coef, k_qterm)
    # and the epilogue; per FFT group one forward-column, one row and one
    # inverse-column launch (here each group holds one order of one kernel
    # kind); the double-word first stage adds k_nmax and k_nsplit.
    s = wl.random_cp(3, 500, [2, 2], seed=17)
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec) as pl:
        desc = pl.describe()
        G = desc["blocks"]["fft_groups"]
        if prec == sag.SAG_FP64:
            assert G == 1 and desc["launches_per_step"] == 14
        else:
            assert G == 2 and desc["launches_per_step"] == 2 * (4 + 3 * G) + 2


def test_rhs_in_place_alias():
    s = wl.random_cp(3, 300, [2, 2], seed=13)
    with sag.Plan(s.N, s.D, s.ranks, s.factors) as pl:
        n = dev(s.n0)
        ref = torch.empty_like(n)
        pl.rhs(n, ref)
        pl.rhs(n, n)
        torch.cuda.synchronize()
        assert torch.equal(n, ref)


def test_nonfinite_input_is_latched_and_cleared():
    s = wl.random_cp(3, 64, [2, 2], seed=14)
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=sag.SAG_FP64) as pl:
        bad = s.n0.copy()
        bad[5] = np.nan
        n = dev(bad)
        out = torch.empty_like(n)
        pl.rhs(n, out)
        assert pl.sync_status() == sag.SAG_ENONFINITE
        assert pl.sync_status() == sag.SAG_OK
        pl.rhs(dev(s.n0), out)
        assert pl.sync_status() == sag.SAG_OK


def test_scale_invariance_of_double_word_path():
    # n and the factors far outside FP32's range: the power-of-two scaling of
    # the double-word path keeps the relative error unchanged.
    s = wl.random_cp(3, 200, [2, 3], seed=15)
    n_small = s.n0 * 1e-60
    f_big = s.factors * 1e50
    p_ref, q_ref = oracle.rhs(n_small, s.D, s.ranks, f_big, mode=oracle.DIRECT)
    s2 = wl.System(s.D, s.N, "cp", s.ranks, f_big, n_small)
    p, q, _, _ = gpu_parts(s2, n_small, sag.SAG_FP32_SPLIT)
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    assert np.isfinite(scale) and scale > 0
    assert nerr(p, p_ref, scale) < 1e-10
    assert nerr(q, q_ref, scale) < 1e-10


# ------------------------------------------------------------------ time integration
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rk", [sag.SAG_HEUN, sag.SAG_MIDPOINT])
def test_constant_kernel_trajectory(prec, rk):
    s = wl.constant_monodisperse()  # D=3, N=64, n=e_1, dt=0.01, 100 steps
    method = oracle.HEUN if rk == sag.SAG_HEUN else oracle.MIDPOINT
    n_ref, d_ref = oracle.integrate(s.n0, s.D, s.ranks, s.factors, s.dt, s.steps, method=method)
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec, rk=rk) as pl:
        n = dev(s.n0)
        diag = torch.zeros((s.steps + 1, 3), dtype=torch.float64, device="cuda")
        pl.integrate(n, s.dt, s.steps, diag)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
        n, diag = n.cpu().numpy(), diag.cpu().numpy()
    assert nerr(n, n_ref, np.abs(n_ref).max()) < TOL[prec]
    # Diagnostics (M0 <= 1, M1 = 1): FP64 and plain double-word to rounding
    # level; the grid-aligned FFTs carry about 1e-13 relative error per
    # right-hand side, i.e. about 1e-11 in the size-weighted M1 over the run.
    lim = (TOL[prec],) * 3 if prec == sag.SAG_FP32_SPLIT else (1e-13, 1e-14, 1e-12)
    e_diag = np.max(np.abs(diag[:, :2] - d_ref[:, :2]))
    assert e_diag < lim[0], e_diag
    # total concentration follows the scalar RK2 recursion of the closed-form
    # M0 equation exactly (Heun), and M1 + outflow is conserved
    if rk == sag.SAG_HEUN:
        f = lambda M: -M * M / 2 - M ** 3 / 3
        M = 1.0
        for _ in range(s.steps):
            k1 = f(M)
            M = M + 0.5 * s.dt * (k1 + f(M + s.dt * k1))
        assert abs(diag[-1, 0] - M) < lim[1], abs(diag[-1, 0] - M)
    tot = diag[:, 1] + diag[:, 2]
    assert np.max(np.abs(tot - tot[0])) < lim[2], np.max(np.abs(tot - tot[0]))


@pytest.mark.parametrize("prec", PRECS)
def test_brownian_trajectory_matches_oracle(prec):
    s = wl.brownian_cp(3, 4096)
    steps = 4
    n_ref, d_ref = oracle.integrate(s.n0, s.D, s.ranks, s.factors, s.dt, steps)
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec) as pl:
        n = dev(s.n0)
        diag = torch.zeros((steps + 1, 3), dtype=torch.float64, device="cuda")
        pl.integrate(n, s.dt, steps, diag)
        torch.cuda.synchronize()
        n = n.cpu().numpy()
        diag = diag.cpu().numpy()
    assert nerr(n, n_ref, np.abs(n_ref).max()) < TOL[prec]
    assert np.max(np.abs(diag[:, :2] - d_ref[:, :2]) / np.abs(d_ref[:, :2]).max(axis=0)) < TOL[prec]


def test_graph_recaptured_when_dt_or_buffer_changes():
    s = wl.random_cp(3, 128, [2, 2], seed=16)
    refs = {dt: oracle.integrate(s.n0, s.D, s.ranks, s.factors, dt, 3, diag=False)[0]
            for dt in (0.01, 0.02)}
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=sag.SAG_FP64) as pl:
        for dt in (0.01, 0.02, 0.01):
            for _ in range(2):
                n = dev(s.n0)
                pl.integrate(n, dt, 3)
                torch.cuda.synchronize()
                assert nerr(n.cpu().numpy(), refs[dt], np.abs(refs[dt]).max()) < 1e-12


def test_fp32_split_tracks_fp64_over_long_trajectory():
    # Brownian kernel, N = 4096, 1000 steps of dt = 1e-3: the double-word path
    # stays within 1e-9 of the FP64 path, and both conserve M1 + outflow.
    s = wl.brownian_cp(3, 4096)
    res = {}
    for prec in PRECS:
        with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec) as pl:
            n = dev(s.n0)
            diag = torch.zeros((s.steps + 1, 3), dtype=torch.float64, device="cuda")
            pl.integrate(n, s.dt, s.steps, diag)
            torch.cuda.synchronize()
            res[prec] = (n.cpu().numpy(), diag.cpu().numpy())
    n64, d64 = res[sag.SAG_FP64]
    ndw, ddw = res[sag.SAG_FP32_SPLIT]
    nx, dx = res[sag.SAG_FP32_SPLIT_EXACT]
    assert nerr(ndw, n64, np.abs(n64).max()) < 1e-9
    # plain double-word butterflies: FP64-level state and size-weighted M1
    assert nerr(nx, n64, np.abs(n64).max()) < 1e-12
    assert abs(dx[-1, 1] - d64[-1, 1]) < 1e-11 * d64[0, 1], abs(dx[-1, 1] - d64[-1, 1]) / d64[0, 1]
    for dg in (d64, ddw, dx):
        tot = dg[:, 1] + dg[:, 2]
        assert np.max(np.abs(tot - tot[0])) < 1e-9 * tot[0]


def test_plans_with_different_footprints_coexist():
    # A later plan with smaller shared-memory blocks must not break an earlier one.
    big = wl.random_cp(4, 20000, [2, 2, 2], seed=18)
    small = wl.random_cp(2, 16, [1], seed=19)
    for prec in PRECS:
        with sag.Plan(big.N, big.D, big.ranks, big.factors, prec=prec) as p1, \
                sag.Plan(small.N, small.D, small.ranks, small.factors, prec=prec) as p2:
            for pl, s in ((p2, small), (p1, big), (p2, small)):
                n = dev(s.n0)
                out = torch.empty_like(n)
                pl.rhs(n, out)
                torch.cuda.synchronize()
                assert pl.sync_status() == sag.SAG_OK


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECS)
def test_autotuned_plan_gives_the_same_results(prec):
    # The stream-group autotuner only changes how the FFT stage is split into
    # launches and streams: right-hand side and trajectory are bitwise the
    # same. (These lengths have no compile-time pair kernels, so the split
    # autotuner has no candidates.)
    import torch
    s = wl.random_cp(4, 5000, [4, 3, 2], seed=61)
    outs = []
    for autotune in (0, 1):
        with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec, autotune=autotune) as pl:
            assert 1 <= pl.describe()["blocks"]["fft_groups"] <= 3
            assert pl.describe()["geometry_autotune"] == []
            n = dev(s.n0)
            out = torch.empty_like(n)
            pl.rhs(n, out)
            pl.integrate(n, 1e-3, 3)
            torch.cuda.synchronize()
            outs.append((out.cpu().numpy(), n.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("make", [
    lambda: wl.paper_ternary(300, "cp"),
    lambda: wl.paper_ternary(300, "tt"),
    lambda: wl.random_cp(4, 257, [2, 0, 1], seed=62),
], ids=["ternary_cp", "ternary_tt", "D4_no_d3"])
def test_absent_orders(make, prec):
    # Orders left out (CP rank 0, or an all-zero TT order) contribute nothing.
    import torch
    s = make()
    fmt = sag.SAG_TT if s.fmt == "tt" else sag.SAG_CP
    ofmt = oracle.TT if s.fmt == "tt" else oracle.CP
    p_ref, q_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors, mode=oracle.DIRECT, fmt=ofmt)
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    with sag.Plan(s.N, s.D, s.ranks, s.factors, fmt=fmt, prec=prec) as pl:
        n = dev(s.n0)
        p, q = torch.empty_like(n), torch.empty_like(n)
        pl.rhs_parts(n, p, q)
        torch.cuda.synchronize()
    assert nerr(p.cpu().numpy(), p_ref, scale) < TOL[prec]
    assert nerr(q.cpu().numpy(), q_ref, scale) < TOL[prec]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECS)
def test_duplicate_vectors_are_transformed_once(prec):
    # The Brownian kernel's CP form repeats three functions (1, i^{1/3},
    # i^{-1/3}) over its rank terms: the forward pass transforms each once per
    # order, and the right-hand side still matches the oracle.
    import torch
    s = wl.brownian_cp(3, 1500)
    p_ref, q_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors, mode=oracle.DIRECT)
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec) as pl:
        orders = pl.describe()["orders"]
        assert [o["transformed"] for o in orders] == [3, 3]
        assert [o["vectors"] for o in orders] == [8, 27]
        n = dev(s.n0)
        p, q = torch.empty_like(n), torch.empty_like(n)
        pl.rhs_parts(n, p, q)
        torch.cuda.synchronize()
    assert nerr(p.cpu().numpy(), p_ref, scale) < TOL[prec]
    assert nerr(q.cpu().numpy(), q_ref, scale) < TOL[prec]
