"""torch.autograd front end of libtt: the forward model, the squared loss and
the regularisers as differentiable functions whose backward passes are
libtt's hand-written kernels (the exact adjoint of the Joseph projector and
the analytic regulariser gradients), so that a loss such as

    squared_loss(h, c, I, W) + mu_l2 * l2_norm(h, c) + mu_tv * tv_huber(h, c, delta)

composes with ordinary autograd (Section "Optimization": LossFunction =
residual norm + Regularizers).  Marshalling only: no arithmetic of the path
runs here.
"""
from __future__ import annotations

import torch

from .tt import Handle


class _Project(torch.autograd.Function):
    """I = A c (Eq. forward_model); backward: A^T grad_I (exact adjoint)."""

    @staticmethod
    def forward(ctx, c, handle):
        ctx.handle = handle
        return handle.project(c.contiguous())

    @staticmethod
    def backward(ctx, grad_I):
        return ctx.handle.adjoint(grad_I.contiguous()), None


class _SquaredLoss(torch.autograd.Function):
    """sum W (A c - I)^2 with the fused gradient 2 A^T (W (A c - I))."""

    @staticmethod
    def forward(ctx, c, handle, I, W):
        loss, g = handle.gradient_residual(c.contiguous(), I, W, want_grad=c.requires_grad)
        ctx.save_for_backward(g if g is not None else torch.empty(0, device=c.device))
        return torch.tensor(loss, dtype=c.dtype, device=c.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None


class _L2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, handle):
        v, g = handle.l2_norm(c.contiguous(), want_grad=c.requires_grad)
        ctx.save_for_backward(g if g is not None else torch.empty(0, device=c.device))
        return torch.tensor(v, dtype=c.dtype, device=c.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None


class _TV(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, handle, delta):
        v, g = handle.tv_huber(c.contiguous(), delta, want_grad=c.requires_grad)
        ctx.save_for_backward(g if g is not None else torch.empty(0, device=c.device))
        return torch.tensor(v, dtype=c.dtype, device=c.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None


def project(handle: Handle, c: torch.Tensor) -> torch.Tensor:
    return _Project.apply(c, handle)


def squared_loss(handle: Handle, c: torch.Tensor, I: torch.Tensor, W: torch.Tensor | None = None) -> torch.Tensor:
    return _SquaredLoss.apply(c, handle, I, W)


def l2_norm(handle: Handle, c: torch.Tensor) -> torch.Tensor:
    return _L2.apply(c, handle)


def tv_huber(handle: Handle, c: torch.Tensor, delta: float = 1e-2) -> torch.Tensor:
    return _TV.apply(c, handle, float(delta))
