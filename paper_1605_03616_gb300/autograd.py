"""torch.autograd.Function for u = K g with the IBF plan.

Backward is the hand-written adjoint (include/ibf.h: ibf_apply_adjoint, the
conjugate-transposed factors of Sec. 3 in reverse order).  For the C-linear
map u = K g, PyTorch's complex convention gives the vector-Jacobian product
grad_g = K^* grad_u.
"""
from __future__ import annotations

import torch


class IBFApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g: torch.Tensor, plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.apply(g.contiguous())

    @staticmethod
    def backward(ctx, grad_u: torch.Tensor):
        if grad_u is None:
            return None, None
        return ctx.plan.adjoint(grad_u.contiguous()), None


class IBFAdjoint(torch.autograd.Function):
    """g = K^* y, differentiable (its backward is the forward apply)."""

    @staticmethod
    def forward(ctx, y: torch.Tensor, plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.adjoint(y.contiguous())

    @staticmethod
    def backward(ctx, grad_g: torch.Tensor):
        if grad_g is None:
            return None, None
        return ctx.plan.apply(grad_g.contiguous()), None


def ibf_apply(plan, g: torch.Tensor) -> torch.Tensor:
    """Differentiable u = K g."""
    return IBFApply.apply(g, plan)


def ibf_adjoint(plan, y: torch.Tensor) -> torch.Tensor:
    """Differentiable g = K^* y."""
    return IBFAdjoint.apply(y, plan)
