"""Gradient of Eq. (12) on the GPU against the FP64 oracle's analytic gradient
and against FP64 central differences of the oracle's cost along random
directions (1e-4 relative), and through torch.autograd."""
import numpy as np
import pytest

import oracle as O
from paper_2605_19388_gb300 import synth
from tests._helpers import rel_err, elem_err_med

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_19388_gb300 import dfmnmf as D  # noqa: E402
from paper_2605_19388_gb300 import autograd as AG  # noqa: E402


def setup(mics, F=11, T=90, N=3, B=4, seed=80, precision=D.DFMNMF_FP32, iters=2):
    p = synth.make_problem(F, T, mics, N, B, seed=seed)
    Q0 = synth.random_blocks(F, mics, seed=seed + 1, scale=0.2)
    ctx = D.dfmnmf_init(F, T, mics, N, B, p.x, p.W0, p.H0, p.g0, Q0, precision=precision)
    D.dfmnmf_iterate(ctx, iters)  # a generic state (not a stationary point)
    return p, ctx


def gpu_grad(ctx):
    Q, W, H, g = D.params_numpy(ctx)
    dQ, dW, dH, dg = np.empty_like(Q), np.empty_like(W), np.empty_like(H), np.empty_like(g)
    nll = D.dfmnmf_cost_gradient(ctx, dQ, dW, dH, dg)
    return nll, (Q, W, H, g), (dQ, dW, dH, dg)


@pytest.mark.parametrize("mics", [(4, 4), (4, 4, 4, 4), (2, 2, 2), (16,)])
def test_gradient_matches_oracle(mics):
    p, ctx = setup(mics)
    nll, (Q, W, H, g), (dQ, dW, dH, dg) = gpu_grad(ctx)
    st = O.state_from_arrays(Q, W, H, g, p.mics)
    x = p.x.astype(np.complex128)
    rQ, rW, rH, rg = O.cost_gradient(x, p.mics, st)
    assert abs(nll - O.neg_loglik(x, p.mics, st)) <= 1e-5 * abs(O.neg_loglik(x, p.mics, st))
    assert rel_err(dW, rW) < 1e-4 and rel_err(dH, rH) < 1e-4 and rel_err(dg, rg) < 1e-4
    assert rel_err(O.unpack_Q(dQ, p.mics)[0], rQ[0]) < 1e-4
    for k in range(len(p.mics)):
        assert rel_err(O.unpack_Q(dQ, p.mics)[k], rQ[k]) < 1e-4
    # element by element against the median magnitude of each gradient (an entry is a difference of two
    # sums of positive terms -- den - num of the multiplicative rules -- and carries their absolute rounding)
    elem = {"W": elem_err_med(dW, rW), "H": elem_err_med(dH, rH), "g": elem_err_med(dg, rg),
            "Q": max(elem_err_med(O.unpack_Q(dQ, p.mics)[k], rQ[k]) for k in range(len(p.mics)))}
    print("cost gradient", mics, "element-wise", elem)
    assert max(elem.values()) < 1e-4, elem


def test_directional_derivatives_against_central_differences():
    """32 random directions, FP64 central differences of the oracle's cost (step 1e-6)."""
    p, ctx = setup((4, 4, 4, 4), F=9, T=80, N=5, B=4, seed=81)
    _, (Q, W, H, g), (dQ, dW, dH, dg) = gpu_grad(ctx)
    x = p.x.astype(np.complex128)
    rng = np.random.default_rng(82)
    h = 1e-6

    def cost(Qp, Wp, Hp, gp):
        return O.neg_loglik(x, p.mics, O.state_from_arrays(Qp, Wp, Hp, gp, p.mics))

    worst = 0.0
    for _ in range(32):
        sW = W * rng.standard_normal(W.shape)
        sH = H * rng.standard_normal(H.shape)
        sg = g * rng.standard_normal(g.shape)
        sQ = np.abs(Q).mean() * (rng.standard_normal(Q.shape) + 1j * rng.standard_normal(Q.shape))
        fd = (cost(Q + h * sQ, W + h * sW, H + h * sH, g + h * sg) -
              cost(Q - h * sQ, W - h * sW, H - h * sH, g - h * sg)) / (2 * h)
        an = (np.sum(dW.astype(np.float64) * sW) + np.sum(dH.astype(np.float64) * sH) +
              np.sum(dg.astype(np.float64) * sg) + np.real(np.sum(np.conj(dQ) * sQ)))
        worst = max(worst, abs(fd - an) / max(abs(fd), 1e-30))
    assert worst <= 1e-4, worst


def test_autograd_function_and_tensor_core_context():
    p, ctx = setup((4, 4, 4, 4), F=21, T=120, N=5, B=8, seed=83)
    _, (Q, W, H, g), (dQ, dW, dH, dg) = gpu_grad(ctx)
    dev = torch.device("cuda")
    tQ = torch.from_numpy(Q).to(dev).requires_grad_(True)
    tW, tH, tg = (torch.from_numpy(a).to(dev).requires_grad_(True) for a in (W, H, g))
    L = AG.cost(ctx, tQ, tW, tH, tg)
    (2.0 * L).backward()
    np.testing.assert_array_equal(tW.grad.cpu().numpy(), 2.0 * dW)
    np.testing.assert_array_equal(tQ.grad.cpu().numpy(), 2.0 * dQ)
    # the tensor-core context evaluates its gradient with the same float-float statistics
    ctx_tc = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, W, H, g, Q, precision=D.DFMNMF_BF16_TC)
    _, _, (eQ, eW, eH, eg) = gpu_grad(ctx_tc)
    for u, v in ((eQ, dQ), (eW, dW), (eH, dH), (eg, dg)):
        np.testing.assert_array_equal(u, v)
