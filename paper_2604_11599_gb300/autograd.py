"""torch.autograd binding of the adjoint-gradient kernel.

``energy(params, grad_handle)`` returns <H>(theta) for every row of a
[P, n_params] float64 CUDA tensor; backward multiplies the incoming gradient
by dE/dtheta, which the same kernel launch computed (adjoint method), so a VQE
optimisation loop runs one compiled program with new parameters each step
(the paper's compile-once, run-many use of OpenQASM ``input``, Sec. III-D and
IV-D).
"""
from __future__ import annotations

import torch

from .sv import Grad


class _ExpvalFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, handle: Grad) -> torch.Tensor:
        val, grad = handle.run(params)
        ctx.save_for_backward(grad)
        return val

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return grad_out.to(grad.dtype)[:, None] * grad, None


def energy(params: torch.Tensor, handle: Grad) -> torch.Tensor:
    """<H> per parameter set, differentiable with respect to ``params``."""
    squeeze = params.dim() == 1
    p = params[None, :] if squeeze else params
    e = _ExpvalFunction.apply(p, handle)
    return e[0] if squeeze else e
