"""Pins of the reference gradient of unrolled iterations (oracle/dfmnmf_adjoint.py).

The reference differentiates a PyTorch float64 restatement of the iteration
with torch.autograd.  It is pinned to things other than itself:
* its forward equals the NumPy oracle's mm_iteration (Sec. III-B schedule);
* its gradient equals central finite differences (FP64, step 1e-6) of the
  NumPy oracle's loss along random directions, for both losses;
* at zero iterations the cost gradient equals the analytic gradient of
  Eq. (12) (itself pinned by finite differences);
* invariances the model fixes.  After at least one iteration both losses
  are unchanged by a common scale c of W0 (or of H0, or of g0): lambda g and
  yhat scale by c, the IP normalisation (Eq. 15) scales Q by sqrt(c), the MU
  rules (Eqs. 8-10) are homogeneous of degree zero in that change, P / yhat
  and the Wiener gains do not move, and in Eq. (12) the F T M ln c of ln yhat
  cancels the -T ln|det Q|^2 change; so <dW, W> = <dH, H> = <dg, g> = 0.
  Both losses are unchanged by a unit phase on any row of Q0 (the IP update
  keeps each row's phase; P, |det Q| and the Wiener filter do not see it),
  so Im sum_j conj(dQ_muj) Q_muj = 0 for every row.
"""
import numpy as np
import pytest

import oracle as O
from paper_2605_19388_gb300 import synth

torch = pytest.importorskip("torch")
from oracle import dfmnmf_adjoint as OA  # noqa: E402


def problem(mics=(4, 4), F=7, T=30, N=5, seed=7):
    p = synth.make_problem(F, T, mics, N, 4, seed=seed, with_images=True)
    Q0 = synth.random_blocks(p.F, p.mics, seed=seed + 1, scale=0.2)
    return p, O.state_from_arrays(Q0, p.W0, p.H0, p.g0, p.mics)


def numpy_loss(p, st, n_iter, loss):
    x = p.x.astype(np.complex128)
    for _ in range(n_iter):
        st = O.mm_iteration(x, p.mics, st)
    if loss == "nll":
        return O.neg_loglik(x, p.mics, st)
    return float(np.mean(np.abs(O.wiener_filter(x, p.mics, st) - p.c) ** 2))


@pytest.mark.parametrize("mics", [(4, 4), (2, 2, 2), (3,)])
def test_forward_equals_numpy_oracle(mics):
    p, st = problem(mics, N=3)
    x = p.x.astype(np.complex128)
    ref = O.mm_iteration(x, p.mics, st)
    Q, W, H, g = OA.iteration(torch.as_tensor(x), p.mics, [torch.as_tensor(q) for q in st.Q],
                              torch.as_tensor(st.W), torch.as_tensor(st.H), torch.as_tensor(st.g))
    # N = 3 sources on 4-mic subarrays: determined, cond(V) ~ 1e7, so two exact
    # solvers (LAPACK here, elimination in the oracle) differ by ~1e-16 * cond
    for k in range(len(mics)):
        np.testing.assert_allclose(Q[k].numpy(), ref.Q[k], rtol=1e-8, atol=1e-8 * np.abs(ref.Q[k]).max())
    for a, b in ((W, ref.W), (H, ref.H), (g, ref.g)):  # through P, the same Q difference
        np.testing.assert_allclose(a.numpy(), b, rtol=1e-9)


@pytest.mark.parametrize("loss", ["nll", "wiener_mse"])
def test_gradient_matches_central_differences(loss):
    p, st = problem()
    n_iter = 3
    L, dQ, dW, dH, dg = OA.unrolled_gradient(p.x, p.mics, st.Q, st.W, st.H, st.g, n_iter, loss, p.c)
    assert abs(L - numpy_loss(p, st, n_iter, loss)) <= 1e-12 * abs(L)
    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(6):
        eQ = [rng.standard_normal(q.shape) + 1j * rng.standard_normal(q.shape) for q in st.Q]
        eW, eH, eg = (rng.standard_normal(a.shape) * a for a in (st.W, st.H, st.g))
        sp = O.State([q + h * e for q, e in zip(st.Q, eQ)], st.W + h * eW, st.H + h * eH, st.g + h * eg)
        sm = O.State([q - h * e for q, e in zip(st.Q, eQ)], st.W - h * eW, st.H - h * eH, st.g - h * eg)
        fd = (numpy_loss(p, sp, n_iter, loss) - numpy_loss(p, sm, n_iter, loss)) / (2 * h)
        an = (sum(np.real(np.sum(np.conj(a) * b)) for a, b in zip(dQ, eQ)) + np.sum(dW * eW)
              + np.sum(dH * eH) + np.sum(dg * eg))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * abs(L)), (fd, an)


def test_zero_iterations_equals_analytic_cost_gradient():
    p, st = problem()
    _, dQ, dW, dH, dg = OA.unrolled_gradient(p.x, p.mics, st.Q, st.W, st.H, st.g, 0, "nll")
    rQ, rW, rH, rg = O.cost_gradient(p.x, p.mics, st)
    for k in range(len(p.mics)):
        np.testing.assert_allclose(dQ[k], rQ[k], rtol=1e-10, atol=1e-10 * np.abs(rQ[k]).max())
    np.testing.assert_allclose(dW, rW, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dH, rH, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dg, rg, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("loss", ["nll", "wiener_mse"])
def test_gradient_respects_the_invariances(loss):
    p, st = problem()
    _, dQ, dW, dH, dg = OA.unrolled_gradient(p.x, p.mics, st.Q, st.W, st.H, st.g, 4, loss, p.c)
    for k in range(len(p.mics)):  # unit phase of each row of Q0
        im = np.imag(np.sum(np.conj(dQ[k]) * st.Q[k], axis=-1))
        assert np.abs(im).max() <= 1e-9 * np.abs(dQ[k] * st.Q[k]).sum()
    for d, v in ((dW, st.W), (dH, st.H), (dg, st.g)):  # common scale of W0, H0 or g0
        assert abs(np.sum(d * v)) <= 1e-9 * np.linalg.norm(d) * np.linalg.norm(v)
