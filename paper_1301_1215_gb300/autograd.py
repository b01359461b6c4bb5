"""F of Eq. 2 as a differentiable PyTorch operation.

The forward pass is the library's nlinv_forward; the backward pass applies the library's adjoint chain
nlinv_adjoint (DF^H) to the incoming gradient.  F is complex-bilinear in x = (rho, chat), hence holomorphic, so in
PyTorch's conjugate-Wirtinger convention the gradient with respect to x is DF_x^H applied to the gradient with
respect to F(x).  Both passes run in the CUDA kernels; this module only wires them into autograd.
"""
from __future__ import annotations

import torch

from .nlinv import Nlinv

__all__ = ["NlinvForward", "forward"]


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
