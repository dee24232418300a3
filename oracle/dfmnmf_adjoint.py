"""FP64 CPU reference gradient of unrolled distributed-FastMNMF iterations.

TEST INFRASTRUCTURE ONLY (like ``dfmnmf_oracle``): nothing in the library
imports it; it shares no code with the CUDA path.

The MM iteration of Sec. III-B (Eqs. 2, 8-10, 13-15) is restated here with
plain PyTorch CPU operations in float64, so that ``torch.autograd`` can
differentiate a loss of the state reached after ``n_iter`` iterations with
respect to the initial state (Q0, W0, H0, g0).  The forward is the same
sequence of steps as ``dfmnmf_oracle.mm_iteration`` (pinned equal to it in
the tests); the one difference is the IP solve, a library solve
(``torch.linalg.solve``) with no pseudo-inverse branch: the gradient is only
defined where every system A = Q V_mu is nonsingular.

Losses of the final state:
* ``"nll"``         Eq. (12) exactly as printed (no F T M ln(pi) constant);
* ``"wiener_mse"``  mean over (n, f, t, m) of |c_hat - c_true|^2, with c_hat
                    the multichannel Wiener filter output of the final state
                    (c_n = Q^{-1} diag(lambda_n g_n / yhat) Q x per subarray)
                    and source n matched to ground-truth image n.

Complex gradients follow PyTorch's convention for a real loss: the gradient
with respect to Q is dL/dRe Q + i dL/dIm Q, so that a perturbation dQ
changes the loss by Re(sum conj(grad) dQ).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np
import torch

EPS = 1e-6


def _offsets(mics: Sequence[int]):
    o = [0]
    for m in mics:
        o.append(o[-1] + int(m))
    return o


def model_variance(W, H, g, eps=EPS):
    """Eq. (2) and the model: yhat[f,t,m] = max(sum_n (W H)[n,f,t] g[f,n,m], eps)."""
    lam = W @ H                                              # [N][F][T]
    y = torch.einsum("nft,fnm->ftm", lam, g)
    return lam, torch.clamp(y, min=eps)


def ip_update(Qk, Vk, eps=EPS):
    """Eqs. (14)-(15) for every row mu of the blocks Q_fk, in ascending order."""
    F, mk, _ = Qk.shape
    rows = [Qk[:, i, :] for i in range(mk)]
    for mu in range(mk):
        Q = torch.stack(rows, dim=1)
        A = Q @ Vk[:, mu]
        e = torch.zeros((F, mk, 1), dtype=Qk.dtype)
        e[:, mu, 0] = 1.0
        q = torch.linalg.solve(A, e)[..., 0]                 # A^{-1} e_mu
        s = torch.real(torch.einsum("fa,fab,fb->f", q.conj(), Vk[:, mu], q))
        q = q / torch.sqrt(torch.clamp(s, min=eps))[:, None]
        rows[mu] = q.conj()                                   # row mu <- q^H
    return torch.stack(rows, dim=1)


def iteration(x, mics, Q: List[torch.Tensor], W, H, g, eps=EPS):
    """One MM iteration: IP of every block (Eq. 13 covariances), then Eqs. 8, 9, 10."""
    F, T, M = x.shape
    off = _offsets(mics)
    _, y = model_variance(W, H, g, eps)
    Qn, P = [], []
    for k, mk in enumerate(mics):
        xk = x[:, :, off[k]:off[k] + mk]
        w = 1.0 / y[:, :, off[k]:off[k] + mk]
        V = torch.einsum("ftu,fta,ftb->fuab", w.to(x.dtype), xk, xk.conj()) / T
        Qk = ip_update(Q[k], V, eps)
        Qn.append(Qk)
        P.append(torch.abs(torch.einsum("fuv,ftv->ftu", Qk, xk)) ** 2)
    P = torch.cat(P, dim=2)

    def stats(W_, H_):
        _, y_ = model_variance(W_, H_, g, eps)
        A = torch.einsum("fnm,ftm->nft", g, P / y_ ** 2)
        D = torch.einsum("fnm,ftm->nft", g, 1.0 / y_)
        return A, D

    A, D = stats(W, H)
    W1 = W * torch.sqrt((A @ H.transpose(1, 2)) / torch.clamp(D @ H.transpose(1, 2), min=eps))
    A, D = stats(W1, H)
    H1 = H * torch.sqrt((W1.transpose(1, 2) @ A) / torch.clamp(W1.transpose(1, 2) @ D, min=eps))
    lam, y = model_variance(W1, H1, g, eps)
    num = torch.einsum("nft,ftm->fnm", lam, P / y ** 2)
    den = torch.einsum("nft,ftm->fnm", lam, 1.0 / y)
    g1 = g * torch.sqrt(num / torch.clamp(den, min=eps))
    return Qn, W1, H1, g1


def neg_loglik(x, mics, Q, W, H, g, eps=EPS):
    """Eq. (12) of a state."""
    T = x.shape[1]
    off = _offsets(mics)
    _, y = model_variance(W, H, g, eps)
    out = 0.0
    for k, mk in enumerate(mics):
        z = torch.einsum("fuv,ftv->ftu", Q[k], x[:, :, off[k]:off[k] + mk])
        yk = y[:, :, off[k]:off[k] + mk]
        out = out + torch.sum(torch.abs(z) ** 2 / yk + torch.log(yk))
        out = out - T * torch.sum(torch.log(torch.abs(torch.linalg.det(Q[k])) ** 2))
    return out


def wiener_mse(x, mics, Q, W, H, g, c_true, eps=EPS):
    """Mean |c_hat - c_true|^2 of the Wiener filter output of a state."""
    off = _offsets(mics)
    lam, y = model_variance(W, H, g, eps)
    N = W.shape[0]
    err = 0.0
    for k, mk in enumerate(mics):
        sl = slice(off[k], off[k] + mk)
        z = torch.einsum("fuv,ftv->ftu", Q[k], x[:, :, sl])
        Qi = torch.linalg.inv(Q[k])
        for n in range(N):
            gain = lam[n][:, :, None] * g[:, n, None, sl] / y[:, :, sl]
            c = torch.einsum("fuv,ftv->ftu", Qi, gain.to(z.dtype) * z)
            err = err + torch.sum(torch.abs(c - c_true[n][:, :, sl]) ** 2)
    return err / c_true.numel()


def unrolled_loss(x, mics, Q0, W0, H0, g0, n_iter, loss="nll", c_true=None, eps=EPS):
    """Loss of the state reached after n_iter iterations from (Q0, W0, H0, g0) (torch tensors)."""
    Q, W, H, g = list(Q0), W0, H0, g0
    for _ in range(n_iter):
        Q, W, H, g = iteration(x, mics, Q, W, H, g, eps)
    if loss == "nll":
        return neg_loglik(x, mics, Q, W, H, g, eps)
    if loss == "wiener_mse":
        return wiener_mse(x, mics, Q, W, H, g, c_true, eps)
    raise ValueError(loss)


def unrolled_gradient(x, mics, Q0, W0, H0, g0, n_iter, loss="nll", c_true=None, eps=EPS):
    """(loss, dQ0 list of [F][M_k][M_k] complex128, dW0, dH0, dg0) as numpy arrays.

    x [F][T][M] complex, Q0 list of K [F][M_k][M_k], W0 [N][F][B], H0 [N][B][T],
    g0 [F][N][M]; c_true [N][F][T][M] for the Wiener loss."""
    xt = torch.as_tensor(np.asarray(x, dtype=np.complex128))
    Qt = [torch.tensor(np.asarray(q, dtype=np.complex128), requires_grad=True) for q in Q0]
    Wt = torch.tensor(np.asarray(W0, dtype=np.float64), requires_grad=True)
    Ht = torch.tensor(np.asarray(H0, dtype=np.float64), requires_grad=True)
    gt = torch.tensor(np.asarray(g0, dtype=np.float64), requires_grad=True)
    ct = None if c_true is None else torch.as_tensor(np.asarray(c_true, dtype=np.complex128))
    L = unrolled_loss(xt, mics, Qt, Wt, Ht, gt, n_iter, loss, ct, eps)
    grads = torch.autograd.grad(L, Qt + [Wt, Ht, gt])
    K = len(Qt)
    return (float(L.detach()), [gr.numpy() for gr in grads[:K]], grads[K].numpy(), grads[K + 1].numpy(),
            grads[K + 2].numpy())
