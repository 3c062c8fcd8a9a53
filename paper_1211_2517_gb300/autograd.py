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
