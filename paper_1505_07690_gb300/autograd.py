"""The forward transform and a score energy as torch.autograd.Functions.

forward:  U = W f            (os3d_forward, Eq. construction1Discrete)
backward: grad_f = Re W^* G  (os3d_adjoint; the adjoint of Sec. 4.1 / App. A)

PyTorch hands backward the conjugate-Wirtinger gradient G = dL/dconj(U) of a
real loss, for which the gradient with respect to a real image is Re W^* G.

weighted_energy(U, w) = sum w |U|^2, the (weighted) squared L_2(R^3 x S^2)
norm of a score (Sec. 2, the norm-preservation identity), in one streaming
kernel, with the gradient 2 g w U in another.

score_energy(f, bank, w) = sum w |W f|^2 in one Function. On the planes of the
plane pass its forward is one sweep (os3d_score_energy_grad) that yields the
loss and the gradient for g = 1 without storing the score, and its backward
scales that gradient by g. With sweep=False the forward stores U and the
backward is the weighted adjoint Re W^*(2 g w U), which weights U inside the
transform's load and never stores the score-sized gradient; on planes the
plane pass does not hold (pencil passes) the backward stores G = 2 g w U and
takes os3d_adjoint.
"""
from __future__ import annotations

import torch

from .os3d import (OS3D_EUNSUPPORTED, Bank, OS3DError, os3d_adjoint, os3d_adjoint_weighted,
                   os3d_forward, os3d_scale_by, os3d_score_energy_grad, os3d_weighted_energy,
                   os3d_weighted_energy_grad)


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


class WeightedEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U: torch.Tensor, w):
        Uc = U.contiguous()
        wc = None if w is None else w.contiguous()
        ctx.save_for_backward(Uc, wc)
        return os3d_weighted_energy(Uc, wc)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        U, w = ctx.saved_tensors
        return os3d_weighted_energy_grad(U, w, g.reshape(()).float().contiguous()), None


def weighted_energy(U: torch.Tensor, w: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable L = sum w |U|^2 of a complex64 CUDA score U with
    constant float32 weights w of U's shape (w = 1 when None): a 0-dim float32
    tensor, summed in FP32 over 16 terms and FP64 above, bit-identical from
    call to call."""
    if w is not None and w.requires_grad:
        raise ValueError("weighted_energy differentiates U only; w must not require grad")
    return WeightedEnergy.apply(U, w)


class ScoreEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f: torch.Tensor, bank: Bank, w: torch.Tensor, sweep: bool = True):
        ctx.bank = bank
        ctx.in_shape = f.shape
        fc = f.contiguous()
        wc = w.contiguous()
        if not ctx.needs_input_grad[0]:
            # the loss alone: the forward transform and the energy kernel
            ctx.sweep = False
            return os3d_weighted_energy(os3d_forward(bank, fc), wc)
        if sweep:
            try:
                loss, grad = os3d_score_energy_grad(bank, fc, wc)
                ctx.sweep = True
                ctx.save_for_backward(grad)
                return loss
            except OS3DError as e:
                if e.status != OS3D_EUNSUPPORTED:
                    raise
        ctx.sweep = False
        U = os3d_forward(bank, fc)
        ctx.save_for_backward(U, wc)
        return os3d_weighted_energy(U, wc)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        gs = g.reshape(()).float().contiguous()
        if ctx.sweep:
            (grad,) = ctx.saved_tensors
            return os3d_scale_by(grad, gs).reshape(ctx.in_shape), None, None, None
        U, w = ctx.saved_tensors
        try:
            grad = os3d_adjoint_weighted(ctx.bank, U, w, gs)
        except OS3DError as e:
            if e.status != OS3D_EUNSUPPORTED:
                raise
            # planes outside the plane pass: the gradient G = 2 g w U stored
            grad = os3d_adjoint(ctx.bank, os3d_weighted_energy_grad(U, w, gs))
        return grad.reshape(ctx.in_shape), None, None, None


def score_energy(f: torch.Tensor, bank: Bank, w: torch.Tensor, sweep: bool = True) -> torch.Tensor:
    """Differentiable L = sum w |W f|^2 for float32 CUDA volumes f of shape
    (nz, ny, nx) or (batch, nz, ny, nx) and constant float32 weights w of the
    score's shape ((batch,) N_o, nz, ny, nx); equal to
    weighted_energy(orientation_score(f, bank), w). sweep=True computes the
    gradient with the loss in one sweep that stores no score (the planes of the
    plane pass: square 16^2 to 128^2, 256^2, 128 x 160); sweep=False, or other
    planes, store U for the weighted adjoint."""
    if w.requires_grad:
        raise ValueError("score_energy differentiates f only; w must not require grad")
    return ScoreEnergy.apply(f, bank, w, sweep)
