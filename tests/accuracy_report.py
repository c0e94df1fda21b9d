"""Accuracy report: the library against the oracle on the five configurations.

Run on a machine with a GPU, from the repository root:

    python tests/accuracy_report.py [--fast]

It prints one line per (configuration, path) with the errors the GPU tests
bound. The errors are max-norm errors relative to the oracle's scale: for a
right-hand side, max|P| + max|Q|; for a state, max|n|. This is a report, not a
test: the bounds live in tests/test_gpu_*.py. --fast shortens the two long
trajectories (configuration 2: 200 steps instead of 1000).
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1905_09071_gb300 import sag, workloads as wl  # noqa: E402

PRECS = (("fp64", sag.SAG_FP64), ("fp32_split", sag.SAG_FP32_SPLIT),
         ("fp32_split_exact", sag.SAG_FP32_SPLIT_EXACT))


def dev(x):
    import torch
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def rel(x, ref, scale=None):
    scale = np.max(np.abs(ref)) if scale is None else scale
    return float(np.max(np.abs(np.asarray(x) - ref)) / scale)


def trajectory(s, steps, dt, prec):
    """Final state and diagnostics of `steps` Heun steps on the GPU."""
    import torch
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec) as pl:
        n = dev(s.n0)
        diag = torch.zeros((steps + 1, 1, 3), dtype=torch.float64, device="cuda")
        pl.integrate(n, dt, steps, diag)
        torch.cuda.synchronize()
        return n.cpu().numpy(), diag.cpu().numpy()[:, 0, :]


def config1(out):
    # D=3, N=64, C = 1, monodisperse, dt 0.01, 100 steps (t = 1)
    s = wl.constant_monodisperse(3, 64)
    steps, dt = 100, 0.01
    n_ref, d_ref = oracle.integrate(s.n0, s.D, s.ranks, s.factors, dt, steps)
    m0_exact = 0.5724637494  # implicit exact solution of dM0/dt = -M0^2/2 - M0^3/3
    for name, prec in PRECS:
        n, d = trajectory(s, steps, dt, prec)
        tot = d[:, 1] + d[:, 2]
        out.append(dict(config="1: D=3 N=64 C=1", path=name, steps=steps,
                        state_err=rel(n, n_ref), m0_gpu=float(d[-1, 0]),
                        m0_minus_exact=float(d[-1, 0] - m0_exact),
                        m0_minus_oracle=float(d[-1, 0] - d_ref[-1, 0]),
                        m1_plus_outflow_drift=float(np.max(np.abs(tot - tot[0])))))


def config2(out, steps):
    # D=3, N=4096, Brownian kernel as an exact CP of rank d^2, dt 1e-3
    s = wl.brownian_cp(3, 4096)
    dt = 1e-3
    t0 = time.perf_counter()
    n_ref, d_ref = oracle.integrate(s.n0, s.D, s.ranks, s.factors, dt, steps)
    t_or = time.perf_counter() - t0
    for name, prec in PRECS:
        n, d = trajectory(s, steps, dt, prec)
        out.append(dict(config="2: D=3 N=4096 Brownian CP", path=name, steps=steps,
                        state_err=rel(n, n_ref),
                        m1_err=float(abs(d[-1, 1] - d_ref[-1, 1]) / d_ref[0, 1]),
                        oracle_seconds=round(t_or, 1)))


def config4(out, count):
    # batched systems: one plan for all, each system's RHS against the oracle
    # for the `count` smallest systems, and the batched RHS against one plan
    # per system for every system
    import torch
    systems = wl.batched_power_cp(B=256)
    with sag.Plan.batch([(x.N, x.D, x.ranks, x.factors, sag.SAG_CP) for x in systems]) as pl:
        off = pl.layout()
        n = dev(np.concatenate([x.n0 for x in systems]))
        y = torch.empty_like(n)
        pl.rhs(n, y)
        torch.cuda.synchronize()
        y = y.cpu().numpy()
    order = np.argsort([x.N for x in systems])[:count]
    errs = []
    for b in order:
        x = systems[b]
        p_ref, q_ref = oracle.rhs(x.n0, x.D, x.ranks, x.factors, mode=oracle.DIRECT)
        scale = np.abs(p_ref).max() + np.abs(q_ref).max()
        errs.append(rel(y[off[b]:off[b + 1]], p_ref + q_ref, scale))
    diff = 0.0
    for b, x in enumerate(systems):
        with sag.Plan(x.N, x.D, x.ranks, x.factors) as one:
            xi = dev(x.n0)
            yi = torch.empty_like(xi)
            one.rhs(xi, yi)
            torch.cuda.synchronize()
            diff = max(diff, float(np.max(np.abs(yi.cpu().numpy() - y[off[b]:off[b + 1]]))))
    out.append(dict(config="4: 256 systems, one plan", path="fp32_split",
                    rhs_err_max=max(errs), systems_checked=len(errs),
                    max_abs_diff_batched_vs_one_plan_each=diff))


def config5(out):
    # adjoint: the fitting problem's kernel on its first 384 sizes, 20 steps,
    # the library's adjoint against the oracle's
    import torch
    p = wl.adjoint_fit_problem(N=384)
    D, N, ranks, dt, steps = p["D"], p["N"], p["ranks"], p["dt"], 20
    g = np.random.default_rng(95).normal(size=N)
    gn_ref, gU_ref = oracle.integrate_vjp(p["n0"], D, ranks, p["factors0"], dt, steps, g)
    for name, prec in PRECS:
        with sag.Plan(N, D, ranks, p["factors0"], prec=prec) as pl:
            gn = torch.empty(N, dtype=torch.float64, device="cuda")
            gU = torch.empty(p["factors0"].size, dtype=torch.float64, device="cuda")
            pl.integrate_vjp(dev(p["n0"]), dt, steps, dev(g), gn, gU, ckpt=5)
            torch.cuda.synchronize()
        out.append(dict(config="5: adjoint, D=3 N=384 R=9, 20 steps", path=name,
                        grad_n_err=rel(gn.cpu().numpy(), gn_ref), grad_U_err=rel(gU.cpu().numpy(), gU_ref)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--fast", action="store_true")
    args = ap.parse_args()
    out = []
    config1(out)
    config2(out, 200 if args.fast else 1000)
    config4(out, 8)
    config5(out)
    for r in out:
        print(json.dumps(r))


if __name__ == "__main__":
    main()
