"""torch.autograd.Function over the compressed M2L.

forward  = kifmm_m2l_apply          (p = A q)
backward = kifmm_m2l_apply_adjoint  (q_bar = A^T p_bar, the core K~_o^T on
           the reversed offset), so adjoint and sensitivity solves of a BEM
           can run the same translation.
"""
from __future__ import annotations

import torch


class M2LFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q_up, plan, level, instance):
        ctx.plan, ctx.level, ctx.instance = plan, level, instance
        return plan.apply(q_up.contiguous(), level, instance)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.plan.apply_adjoint(grad_out.contiguous(), ctx.level, ctx.instance)
        return g, None, None, None


def m2l(q_up: torch.Tensor, plan, level: int, instance: int = 0) -> torch.Tensor:
    """Differentiable compressed M2L of one registered level."""
    return M2LFunction.apply(q_up, plan, level, instance)


class M2LLevelsFunction(torch.autograd.Function):
    """Levels level_lo..level_hi in one batch (kifmm_m2l_apply_levels and its
    adjoint); inputs and outputs hold the levels' arrays back to back."""

    @staticmethod
    def forward(ctx, q_all, plan, level_lo, level_hi, instance):
        ctx.plan, ctx.lo, ctx.hi, ctx.instance = plan, level_lo, level_hi, instance
        return plan.apply_levels(q_all.contiguous(), level_lo, level_hi, instance)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.plan.apply_levels(grad_out.contiguous(), ctx.lo, ctx.hi, ctx.instance, adjoint=True)
        return g, None, None, None, None


def m2l_levels(q_all: torch.Tensor, plan, level_lo: int, level_hi: int, instance: int = 0) -> torch.Tensor:
    """Differentiable compressed M2L of the registered levels level_lo..level_hi."""
    return M2LLevelsFunction.apply(q_all, plan, level_lo, level_hi, instance)
