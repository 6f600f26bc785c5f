"""The forward transform as a torch.autograd.Function.

forward:  U = W f            (os3d_forward, Eq. construction1Discrete)
backward: grad_f = Re W^* G  (os3d_adjoint; the adjoint of Sec. 4.1 / App. A)

PyTorch hands backward the conjugate-Wirtinger gradient G = dL/dconj(U) of a
real loss, for which the gradient with respect to a real image is Re W^* G.
"""
from __future__ import annotations

import torch

from .os3d import Bank, os3d_adjoint, os3d_forward


class OrientationScore(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f: torch.Tensor, bank: Bank):
        ctx.bank = bank
        ctx.in_shape = f.shape
        fc = f.contiguous()
        U = os3d_forward(bank, fc)
        return U if f.dim() > 3 else U[0]

    @staticmethod
    def backward(ctx, gU: torch.Tensor):
        g = gU.contiguous()
        if g.dim() == 4:
            g = g.unsqueeze(0)
        grad = os3d_adjoint(ctx.bank, g)
        return grad.reshape(ctx.in_shape), None


def orientation_score(f: torch.Tensor, bank: Bank) -> torch.Tensor:
    """Differentiable U = W f for float32 CUDA volumes f of shape
    (nz, ny, nx) or (batch, nz, ny, nx)."""
    return OrientationScore.apply(f, bank)
