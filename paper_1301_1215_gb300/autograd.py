"""F of Eq. 2 and the whole Gauss-Newton reconstruction (Eq. 3) as differentiable PyTorch operations.

NlinvForward: the forward pass is the library's nlinv_forward; the backward pass applies the library's adjoint
chain nlinv_adjoint (DF^H) to the incoming gradient.  F is complex-bilinear in x = (rho, chat), hence holomorphic,
so in PyTorch's conjugate-Wirtinger convention the gradient with respect to x is DF_x^H applied to the gradient
with respect to F(x).

NlinvReconstruct: the forward pass is nlinv_reconstruct_checkpoints (every Gauss-Newton iterate kept); the
backward pass is nlinv_reconstruct_vjp, which differentiates each Newton step implicitly (its CG solve taken as
exact) from the last checkpoint back to the first.

Every pass runs in the CUDA kernels; this module only wires them into autograd.
"""
from __future__ import annotations

import torch

from .nlinv import Nlinv

__all__ = ["NlinvForward", "forward", "NlinvReconstruct", "reconstruct"]


class NlinvForward(torch.autograd.Function):
    """y = F(x) with dL/dx = DF_x^H (dL/dy).  Inputs: x (1+J, n, n) complex64, mask (n, n) uint8, a context."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, mask: torch.Tensor, op: Nlinv) -> torch.Tensor:
        x = x.detach().contiguous()
        y = op.forward(x, mask)
        ctx.save_for_backward(x, mask)
        ctx.op = op
        return y

    @staticmethod
    def backward(ctx, grad_y: torch.Tensor):
        x, mask = ctx.saved_tensors
        grad_x = None
        if ctx.needs_input_grad[0]:
            grad_x = ctx.op.adjoint(x, mask, grad_y.contiguous())
        return grad_x, None, None


def forward(op: Nlinv, x: torch.Tensor, mask: torch.Tensor) -> torch.Tensor:
    """Differentiable F(x) on the context ``op``."""
    return NlinvForward.apply(x, mask, op)


class NlinvReconstruct(torch.autograd.Function):
    """x_N = IRGNM(y; x_0, x_ref) with gradients with respect to y, x_0 and x_ref.  Inputs: y (J, n, n) complex64,
    mask (n, n) uint8, x0 (1+J, n, n) complex64, x_ref (1+J, n, n) complex64 or None (= x0), a context."""

    @staticmethod
    def forward(ctx, y: torch.Tensor, mask: torch.Tensor, x0: torch.Tensor, x_ref, op: Nlinv) -> torch.Tensor:
        y = y.detach().contiguous()
        xr = None if x_ref is None else x_ref.detach().contiguous()
        x, ck = op.reconstruct_checkpoints(y, mask, x0.detach().contiguous(), xr)
        ctx.save_for_backward(y, mask, ck)
        ctx.op = op
        ctx.tied = x_ref is None
        return x

    @staticmethod
    def backward(ctx, grad_x: torch.Tensor):
        y, mask, ck = ctx.saved_tensors
        want_ref = (not ctx.tied) and ctx.needs_input_grad[3]
        gy, g0, gr = ctx.op.reconstruct_vjp(y, mask, ck, grad_x.contiguous(), want_xref=want_ref, tied=ctx.tied)
        return gy, None, g0, gr, None


def reconstruct(op: Nlinv, y: torch.Tensor, mask: torch.Tensor, x0: torch.Tensor, x_ref=None) -> torch.Tensor:
    """Differentiable Gauss-Newton reconstruction on the context ``op`` (x_ref None: regularise toward x0)."""
    return NlinvReconstruct.apply(y, mask, x0, x_ref, op)
