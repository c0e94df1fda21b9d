"""PyTorch autograd over the library's RK2 integrator, for fitting kernel factors.

``integrate(factors, n0, plan, dt, steps, ckpt)`` returns n(T) after `steps`
RK2 steps from n0 with the CP factors ``factors`` (a trainable tensor, any
float dtype, in the plan's vector layout). The backward pass calls the
library's checkpointed discrete adjoint (sag_integrate_vjp); nothing is
differentiated by PyTorch itself. Gradients come back in the factors' dtype.
The plan takes each call's factors by sag_plan_update_factors: build it with
``keep_repeats=1`` when factor vectors that start out identical (the Brownian
kernel's) will be trained apart.
"""
from __future__ import annotations

import torch

from . import sag


class _SagIntegrate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, factors, n0, plan, dt, steps, ckpt):
        f64 = factors.detach().to(device="cuda", dtype=torch.float64).contiguous()
        plan.update_factors(f64)
        n = n0.detach().to(device="cuda", dtype=torch.float64).clone()
        plan.integrate(n, dt, steps)
        ctx.plan, ctx.dt, ctx.steps, ctx.ckpt = plan, dt, steps, ckpt
        ctx.save_for_backward(f64, n0.detach().to(device="cuda", dtype=torch.float64).clone())
        ctx.factor_dtype, ctx.n0_dtype = factors.dtype, n0.dtype
        return n.to(n0.dtype)

    @staticmethod
    def backward(ctx, g_out):
        f64, n0 = ctx.saved_tensors
        plan = ctx.plan
        plan.update_factors(f64)
        g = g_out.detach().to(device="cuda", dtype=torch.float64).contiguous()
        g_n0 = torch.empty_like(n0)
        g_U = torch.empty_like(f64)
        plan.integrate_vjp(n0, ctx.dt, ctx.steps, g, g_n0, g_U, ckpt=ctx.ckpt)
        return g_U.to(ctx.factor_dtype), g_n0.to(ctx.n0_dtype), None, None, None, None


def integrate(factors: torch.Tensor, n0: torch.Tensor, plan: "sag.Plan", dt: float, steps: int,
              ckpt: int = 0) -> torch.Tensor:
    """n(T) for the given factors; differentiable in factors and n0."""
    return _SagIntegrate.apply(factors, n0, plan, dt, steps, ckpt)
