"""The Katsevich operator as a differentiable layer (the paper's "domain
transfer layer", Sec. III): forward = steps 1-7, backward = their exact
transpose (``katsevich_adjoint``).

The operator is linear, f = A g, so dL/dg = A^T dL/df needs no activations:
the backward pass keeps only the plan.  Pitch-by-pitch training (one
sinogram window per step, as the paper trains) therefore checkpoints nothing
beyond the window itself.

With a reduced-precision forward (BF16 / FP16 storage of the intermediate
data) the backward is still the FP32 transpose: it is the exact adjoint of the
operator the reduced form approximates, within the reduced form's tolerance.
"""
from __future__ import annotations

import torch

from . import KATS_PREC_FP32, Plan


class KatsevichFunction(torch.autograd.Function):
    """f = A g for sinograms g [..., n_views, n_rows, n_cols] -> volumes [..., nz, ny, nx]."""

    @staticmethod
    def forward(ctx, sino: torch.Tensor, plan: Plan, precision: int = KATS_PREC_FP32):
        ctx.plan = plan
        ctx.precision = precision
        return plan.recon(sino.contiguous(), precision=precision)

    @staticmethod
    def backward(ctx, grad_vol: torch.Tensor):
        grad = ctx.plan.adjoint(grad_vol.contiguous()) if ctx.needs_input_grad[0] else None
        return grad, None, None


class KatsevichLayer(torch.nn.Module):
    """nn.Module holding one geometry's plan; ``layer(sino)`` reconstructs with autograd support."""

    def __init__(self, geom: dict, precision: int = KATS_PREC_FP32):
        super().__init__()
        self.plan = Plan(geom)
        self.precision = precision

    def forward(self, sino: torch.Tensor) -> torch.Tensor:
        return KatsevichFunction.apply(sino, self.plan, self.precision)
