"""The cost of Eq. (12) as a differentiable function of the parameters.

`cost(handle, Q, W, H, g)` sets the context's state to the given device
tensors, evaluates Eq. (12) and its gradient with the library's kernels
(dfmnmf_cost_gradient) and returns the cost as a 0-d float64 tensor whose
backward hands those gradients to autograd.  For the complex Q the gradient
is dL/dRe Q + i dL/dIm Q, PyTorch's convention for a real loss of complex
inputs.  Only the cost at the given state is differentiated: no MM iteration
is taken inside.
"""
from __future__ import annotations

import torch

from . import dfmnmf as D


class _Cost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, handle, Q, W, H, g):
        Q, W, H, g = (a.detach().contiguous() for a in (Q, W, H, g))
        D.dfmnmf_set_params(handle, Q, W, H, g)
        dQ, dW, dH, dg = (torch.empty_like(a) for a in (Q, W, H, g))
        nll = D.dfmnmf_cost_gradient(handle, dQ, dW, dH, dg)
        ctx.save_for_backward(dQ, dW, dH, dg)
        return torch.tensor(nll, dtype=torch.float64, device=W.device)

    @staticmethod
    def backward(ctx, gout):
        dQ, dW, dH, dg = ctx.saved_tensors
        return (None, dQ * gout.to(torch.float64), dW * gout.to(dW.dtype), dH * gout.to(dH.dtype),
                dg * gout.to(dg.dtype))


def cost(handle: "D.Context", Q: torch.Tensor, W: torch.Tensor, H: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
    """Eq. (12) at (Q, W, H, g) for the observation held by `handle` (layouts of dfmnmf_init)."""
    return _Cost.apply(handle, Q, W, H, g)
