"""The cost of Eq. (12) as a differentiable function of the parameters.

`cost(handle, Q, W, H, g)` sets the context's state to the given device
tensors, evaluates Eq. (12) and its gradient with the library's kernels
(dfmnmf_cost_gradient) and returns the cost as a 0-d float64 tensor whose
backward hands those gradients to autograd.  For the complex Q the gradient
is dL/dRe Q + i dL/dIm Q, PyTorch's convention for a real loss of complex
inputs.  Only the cost at the given state is differentiated: no MM iteration
is taken inside.

`unrolled(adj, Q0, W0, H0, g0, loss, c_true)` differentiates through
iterations: it sets the context of `adj` (a dfmnmf_adjoint_create workspace)
to the given initial state, runs the workspace's n_iter iterations, and
returns the loss of the final state (Eq. 12, or the Wiener filter's mean
squared error against c_true) as a 0-d float64 tensor whose backward hands
the library's reverse-pass gradients (dfmnmf_adjoint_run) to autograd.
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


class _Unrolled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, adj, loss, c_true, Q0, W0, H0, g0):
        Q0, W0, H0, g0 = (a.detach().contiguous() for a in (Q0, W0, H0, g0))
        D.dfmnmf_set_params(adj.ctx, Q0, W0.float(), H0.float(), g0.float())
        dQ = torch.empty_like(Q0)
        dW, dH, dg = (torch.empty(a.shape, dtype=torch.float64, device=a.device) for a in (W0, H0, g0))
        val = D.dfmnmf_adjoint_run(adj, loss, c_true, dQ, dW, dH, dg)
        ctx.save_for_backward(dQ, dW, dH, dg)
        ctx.dtypes = (W0.dtype, H0.dtype, g0.dtype)
        return torch.tensor(val, dtype=torch.float64, device=W0.device)

    @staticmethod
    def backward(ctx, gout):
        dQ, dW, dH, dg = ctx.saved_tensors
        gw, gh, gg = ctx.dtypes
        go = gout.to(torch.float64)
        return None, None, None, dQ * go, (dW * go).to(gw), (dH * go).to(gh), (dg * go).to(gg)


def unrolled(adj: "D.Adjoint", Q0: torch.Tensor, W0: torch.Tensor, H0: torch.Tensor, g0: torch.Tensor,
             loss: str = "nll", c_true: torch.Tensor = None) -> torch.Tensor:
    """Loss of the state reached after adj.n_iter iterations from (Q0, W0, H0, g0), differentiable
    with respect to all four (layouts of dfmnmf_init; Q0 complex128, c_true complex64 [N][F][T][M])."""
    code = {"nll": D.DFMNMF_LOSS_NLL, "wiener_mse": D.DFMNMF_LOSS_WIENER_MSE}[loss]
    return _Unrolled.apply(adj, code, c_true, Q0, W0, H0, g0)
