"""CPU oracle for the multi-particle Smoluchowski right-hand side.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()``, the
CPU-baseline leg of ``bench.py`` (which also yields the reference outputs of
its one-RHS error report) and its reference arm may import this package. The GPU library never
does, and this package imports nothing from it: the two share no code.

The arithmetic lives in ``sag_oracle.c`` (plain C, FP64, compensated sums);
this module only compiles it on first use and marshals numpy arrays.

Model (paper Sec. 1): dn/dt = sum_{d=2..D} (P^(d)[n] + Q^(d)[n]).
Conventions: size k at index k-1; CP factors per order d laid out [d][R_d][N];
TT cores per order d laid out, for lambda = 1..d, [R_{lambda-1}][R_lambda][N]
(Eq. ch3.eq4); orders d = 2..D concatenated.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sag_oracle.c")
_HDR = os.path.join(_HERE, "sag_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

BRUTE, DIRECT = 0, 1
CP, TT = 0, 1
HEUN, MIDPOINT = 0, 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle to a shared library (gcc, OpenMP). Returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.orc_set_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_factor_count.restype = ctypes.c_long
        lib.orc_factor_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p]
        lib.orc_kernel_entry.restype = ctypes.c_double
        lib.orc_kernel_entry.argtypes = [ctypes.c_int] * 3 + [i32p, f64p, ctypes.c_int, i32p]
        lib.orc_rhs.restype = ctypes.c_int
        lib.orc_rhs.argtypes = [ctypes.c_int] * 4 + [i32p, f64p, f64p, ctypes.c_int, f64p, f64p, f64p]
        lib.orc_loss.restype = ctypes.c_int
        lib.orc_loss.argtypes = [ctypes.c_int] * 3 + [i32p, f64p, f64p, ctypes.c_int, f64p]
        lib.orc_integrate.restype = ctypes.c_int
        lib.orc_integrate.argtypes = ([ctypes.c_int] * 4 + [i32p, f64p, f64p, ctypes.c_double,
                                      ctypes.c_long, ctypes.c_int, ctypes.c_int, f64p])
        lib.orc_rhs_vjp.restype = ctypes.c_int
        lib.orc_rhs_vjp.argtypes = [ctypes.c_int, ctypes.c_int, i32p, f64p, f64p, f64p, ctypes.c_int,
                                    f64p, f64p]
        lib.orc_integrate_vjp.restype = ctypes.c_int
        lib.orc_integrate_vjp.argtypes = [ctypes.c_int, ctypes.c_int, i32p, f64p, f64p, ctypes.c_double,
                                          ctypes.c_long, ctypes.c_int, ctypes.c_int, f64p, f64p, f64p]
        lib.orc_rhs_vjp_fmt.restype = ctypes.c_int
        lib.orc_rhs_vjp_fmt.argtypes = [ctypes.c_int] * 3 + [i32p, f64p, f64p, f64p, ctypes.c_int, f64p, f64p]
        lib.orc_integrate_vjp_fmt.restype = ctypes.c_int
        lib.orc_integrate_vjp_fmt.argtypes = ([ctypes.c_int] * 3 + [i32p, f64p, f64p, ctypes.c_double,
                                              ctypes.c_long, ctypes.c_int, ctypes.c_int, f64p, f64p, f64p])
        lib.orc_brownian_entry.restype = ctypes.c_double
        lib.orc_brownian_entry.argtypes = [ctypes.c_int, f64p, i32p]
        lib.orc_brownian_tt_count.restype = ctypes.c_long
        lib.orc_brownian_tt_count.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.orc_brownian_tt.restype = ctypes.c_int
        lib.orc_brownian_tt.argtypes = [ctypes.c_int, ctypes.c_int, f64p, i32p, f64p]
        _lib = lib
        return lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def set_threads(n: int = 0) -> int:
    """Host threads of the oracle's OpenMP loops for later calls from this
    thread (n > 0 sets the count); returns the current count."""
    return int(_load().orc_set_threads(int(n)))


def factor_count(fmt: int, D: int, N: int, ranks) -> int:
    r, rp = _i32(ranks)
    c = _load().orc_factor_count(fmt, D, N, rp)
    if c < 0:
        raise ValueError("invalid format/ranks")
    return int(c)


def kernel_entry(fmt: int, D: int, N: int, ranks, factors, idx) -> float:
    """C^(d)_{idx} with d = len(idx) and 1-based sizes in idx."""
    r, rp = _i32(ranks)
    f, fp = _f64(factors)
    i, ip = _i32(idx)
    return float(_load().orc_kernel_entry(fmt, D, N, rp, fp, len(i), ip))


def rhs(n, D: int, ranks, factors, *, fmt: int = CP, mode: int = DIRECT, sym: int = 1,
        outflow: bool = False):
    """Returns (P, Q[, outflow]) with P = sum_d P^(d)[n], Q = sum_d Q^(d)[n]."""
    n, np_ = _f64(n)
    N = n.shape[0]
    r, rp = _i32(ranks)
    f, fp = _f64(factors)
    if f.size != factor_count(fmt, D, N, r):
        raise ValueError("factor array has the wrong length")
    p = np.zeros(N)
    q = np.zeros(N)
    o = np.zeros(1)
    rc = _load().orc_rhs(mode, fmt, D, N, rp, fp, np_, sym,
                         p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         o.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if outflow else None)
    if rc != 0:
        raise ValueError(f"orc_rhs failed ({rc})")
    return (p, q, float(o[0])) if outflow else (p, q)


def loss(n, D: int, ranks, factors, *, fmt: int = CP, sym: int = 1):
    """Q = sum_d Q^(d)[n] alone (inner products only; cheap at any N)."""
    n, np_ = _f64(n)
    N = n.shape[0]
    r, rp = _i32(ranks)
    f, fp = _f64(factors)
    if f.size != factor_count(fmt, D, N, r):
        raise ValueError("factor array has the wrong length")
    q = np.zeros(N)
    rc = _load().orc_loss(fmt, D, N, rp, fp, np_, sym,
                          q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError(f"orc_loss failed ({rc})")
    return q


def integrate(n0, D: int, ranks, factors, dt: float, steps: int, *, fmt: int = CP,
              mode: int = DIRECT, sym: int = 1, method: int = HEUN, diag: bool = True):
    """Explicit RK2 (Sec. 3). Returns (n_final, diag[steps+1, 3] or None)."""
    n = np.array(n0, dtype=np.float64, copy=True)
    N = n.shape[0]
    r, rp = _i32(ranks)
    f, fp = _f64(factors)
    if f.size != factor_count(fmt, D, N, r):
        raise ValueError("factor array has the wrong length")
    dg = np.zeros((steps + 1, 3)) if diag else None
    rc = _load().orc_integrate(mode, fmt, D, N, rp, fp,
                               n.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(dt),
                               int(steps), sym, method,
                               dg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if diag else None)
    if rc != 0:
        raise ValueError(f"orc_integrate failed ({rc})")
    return n, dg


def rhs_vjp(n, g, D: int, ranks, factors, *, sym: int = 1, fmt: int = CP):
    """(dF/dn)^T g and (dF/dU)^T g (factor or core layout; direct mode)."""
    n, np_ = _f64(n)
    g, gp = _f64(g)
    N = n.shape[0]
    r, rp = _i32(ranks)
    f, fp = _f64(factors)
    if f.size != factor_count(fmt, D, N, r):
        raise ValueError("factor array has the wrong length")
    gn = np.zeros(N)
    gU = np.zeros(f.size)
    rc = _load().orc_rhs_vjp_fmt(fmt, D, N, rp, fp, np_, gp, sym,
                                 gn.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 gU.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError(f"orc_rhs_vjp failed ({rc})")
    return gn, gU


def integrate_vjp(n0, D: int, ranks, factors, dt: float, steps: int, g_final, *, sym: int = 1,
                  method: int = HEUN, fmt: int = CP):
    """Discrete adjoint of `steps` RK2 steps: returns (g_n0, g_U)."""
    n0, np_ = _f64(n0)
    g, gp = _f64(g_final)
    N = n0.shape[0]
    r, rp = _i32(ranks)
    f, fp = _f64(factors)
    if f.size != factor_count(fmt, D, N, r):
        raise ValueError("factor array has the wrong length")
    gn0 = np.zeros(N)
    gU = np.zeros(f.size)
    rc = _load().orc_integrate_vjp_fmt(fmt, D, N, rp, fp, np_, float(dt), int(steps), sym, method, gp,
                                       gn0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       gU.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError(f"orc_integrate_vjp failed ({rc})")
    return gn0, gU


def brownian_entry(mu, idx) -> float:
    """Eq. ch3.eq17 element for the 1-based index tuple idx (D = len(mu))."""
    m, mp = _f64(mu)
    i, ip = _i32(idx)
    return float(_load().orc_brownian_entry(len(m), mp, ip))


def brownian_tt(mu, N: int):
    """Theorem 1 TT cores of the Eq. ch3.eq17 kernel. Returns (ranks[D+1], cores)."""
    m, mp = _f64(mu)
    D = len(m)
    lib = _load()
    cnt = lib.orc_brownian_tt_count(D, N)
    if cnt < 0:
        raise ValueError("bad D or N")
    ranks = np.zeros(D + 1, dtype=np.int32)
    cores = np.zeros(cnt)
    rc = lib.orc_brownian_tt(D, N, mp, ranks.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                             cores.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("orc_brownian_tt failed")
    return ranks, cores
