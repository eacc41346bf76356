"""torch.autograd.Function wrappers: forward runs lc_execute, backward runs
the hand-written transposed pass lc_adjoint (A^T C^-1 for L2C, (A^-1 C)^T
for C2L) -- the map is linear, so the vector-Jacobian product is the
adjoint applied to the incoming gradient."""
from __future__ import annotations

import torch

from .api import get_plan


class _Transform(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, direction, dtype, options):
        batch = 1 if x.dim() == 1 else x.shape[0]
        plan = get_plan(x.shape[-1], direction, batch, dtype, x.device, **options)
        ctx.plan = plan
        return plan(x.contiguous())

    @staticmethod
    def backward(ctx, grad):
        return ctx.plan(grad.contiguous(), adjoint=True), None, None, None


def _dtype_for(x, dtype):
    if dtype is not None:
        return dtype
    return "f32" if x.dtype == torch.float32 else "f64"


def leg2cheb(x: torch.Tensor, dtype: str | None = None, **options) -> torch.Tensor:
    """Differentiable f_cheb = C^-1 A f_leg along the last dimension (1-D or 2-D input)."""
    return _Transform.apply(x, "l2c", _dtype_for(x, dtype), options)


def cheb2leg(x: torch.Tensor, dtype: str | None = None, **options) -> torch.Tensor:
    """Differentiable f_leg = A^-1 C f_cheb along the last dimension (1-D or 2-D input)."""
    return _Transform.apply(x, "c2l", _dtype_for(x, dtype), options)
