"""Gradient through unrolled MM iterations (dfmnmf_adjoint_*) against the
reference gradient of the oracle (autograd of its float64 restatement, pinned
in tests/test_oracle_adjoint.py) and against FP64 central finite differences.

Tolerance: 1e-4 relative.  The GPU differentiates the FP32 form's own
trajectory (its reverse pass in FP64 around forward values recomputed from
the stored FP32-form states), the oracle the FP64 trajectory; the two
trajectories differ by the FP32 form's per-update error (<= 1e-5, measured
~1e-7), which bounds the gradient difference.  A directional derivative is
compared relative to sum_i |grad_i dir_i|, the scale its rounding and the
trajectory difference act on.
"""
import numpy as np
import pytest

import oracle as O
from paper_2605_19388_gb300 import synth
from tests._helpers import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import dfmnmf_adjoint as OA  # noqa: E402
from paper_2605_19388_gb300 import autograd as AG  # noqa: E402
from paper_2605_19388_gb300 import dfmnmf as D  # noqa: E402

TOL = 1e-4
DIR_FLOOR = 1e-2  # stated floor of the directional checks, as a fraction of sum_i |g_i d_i|
LOSSES = {"nll": D.DFMNMF_LOSS_NLL, "wiener_mse": D.DFMNMF_LOSS_WIENER_MSE}


def setup(F, T, mics, N, B, seed):
    p = synth.make_problem(F, T, mics, N, B, seed=seed, with_images=True)
    Q0 = synth.random_blocks(p.F, p.mics, seed=seed + 1, scale=0.2)
    ctx = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0, Q0)
    st = O.state_from_arrays(Q0, p.W0, p.H0, p.g0, p.mics)
    return p, Q0, ctx, st


def gpu_gradient(ctx, p, n_iter, every, loss):
    adj = D.dfmnmf_adjoint_create(ctx, n_iter, every)
    dQ = np.empty((p.F, sum(m * m for m in p.mics)), np.complex128)
    dW, dH, dg = np.empty((p.N, p.F, p.B)), np.empty((p.N, p.B, p.T)), np.empty((p.F, p.N, p.M))
    ct = torch.from_numpy(p.c).cuda() if loss == "wiener_mse" else None
    L = D.dfmnmf_adjoint_run(adj, LOSSES[loss], ct, dQ, dW, dH, dg)
    D.dfmnmf_adjoint_destroy(adj)
    return L, O.unpack_Q(dQ, p.mics), dW, dH, dg


def directions(st, count, seed):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        eQ = [(rng.standard_normal(q.shape) + 1j * rng.standard_normal(q.shape)) * np.abs(q).mean() for q in st.Q]
        yield eQ, rng.standard_normal(st.W.shape) * st.W, rng.standard_normal(st.H.shape) * st.H, \
            rng.standard_normal(st.g.shape) * st.g


def dot(grad, d):
    dQ, dW, dH, dg = grad
    eQ, eW, eH, eg = d
    terms = [np.real(np.conj(a) * b).ravel() for a, b in zip(dQ, eQ)] + [(dW * eW).ravel(), (dH * eH).ravel(),
                                                                           (dg * eg).ravel()]
    v = np.concatenate(terms)
    return float(v.sum()), float(np.abs(v).sum())


def torch_loss(p, st, n_iter, loss):
    with torch.no_grad():
        xt = torch.as_tensor(p.x.astype(np.complex128))
        return float(OA.unrolled_loss(xt, p.mics, [torch.as_tensor(q) for q in st.Q], torch.as_tensor(st.W),
                                      torch.as_tensor(st.H), torch.as_tensor(st.g), n_iter, loss,
                                      torch.as_tensor(p.c.astype(np.complex128))))


def check(p, st, n_iter, loss, got, n_dir, n_fd, seed):
    L, dQ, dW, dH, dg = got
    Lr, rQ, rW, rH, rg = OA.unrolled_gradient(p.x, p.mics, st.Q, st.W, st.H, st.g, n_iter, loss, p.c)
    errs = {"L": abs(L - Lr) / abs(Lr), "W": rel_err(dW, rW), "H": rel_err(dH, rH), "g": rel_err(dg, rg)}
    nrm = np.linalg.norm
    scale_q = sum(nrm(rQ[k]) * nrm(st.Q[k]) for k in range(len(p.mics)))
    scale_all = nrm(rW) * nrm(st.W) + nrm(rH) * nrm(st.H) + nrm(rg) * nrm(st.g)
    if scale_q > 1e-8 * scale_all:
        errs["Q"] = max(rel_err(dQ[k], rQ[k]) for k in range(len(p.mics)))
    else:  # one microphone per subarray: Q' = e^{i arg Q} / sqrt(V), no loss depends on Q0
        errs["Q"] = sum(nrm(dQ[k]) * nrm(st.Q[k]) for k in range(len(p.mics))) / scale_all
    # a directional derivative is compared relative to itself; where it cancels below DIR_FLOOR times
    # sum_i |g_i d_i| (the size of its terms), relative to that floor instead
    worst = 0.0
    for d in directions(st, n_dir, seed):
        a, scale = dot((dQ, dW, dH, dg), d)
        b, _ = dot((rQ, rW, rH, rg), d)
        worst = max(worst, abs(a - b) / max(abs(b), DIR_FLOOR * scale))
    errs["dir_vs_oracle"] = worst
    h, worst = 1e-6, 0.0
    for d in directions(st, n_fd, seed + 1):
        eQ, eW, eH, eg = d
        sp = O.State([q + h * e for q, e in zip(st.Q, eQ)], st.W + h * eW, st.H + h * eH, st.g + h * eg)
        sm = O.State([q - h * e for q, e in zip(st.Q, eQ)], st.W - h * eW, st.H - h * eH, st.g - h * eg)
        fd = (torch_loss(p, sp, n_iter, loss) - torch_loss(p, sm, n_iter, loss)) / (2 * h)
        a, scale = dot((dQ, dW, dH, dg), d)
        worst = max(worst, abs(a - fd) / max(abs(fd), DIR_FLOOR * scale))
    errs["dir_vs_fd"] = worst
    print(f"adjoint {loss}, {n_iter} iterations:", {k: float(f"{v:.2e}") for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= TOL, (k, v, errs)
    return errs


@pytest.mark.parametrize("loss", ["nll", "wiener_mse"])
def test_small_matches_oracle_and_finite_differences(loss):
    """6 iterations, checkpoints every 4 (a ragged last segment), 2 x 4 mics, N = 5."""
    p, Q0, ctx, st = setup(9, 40, (4, 4), 5, 4, seed=21)
    check(p, st, 6, loss, gpu_gradient(ctx, p, 6, 4, loss), 32, 32, seed=5)


@pytest.mark.parametrize("mics", [(2, 2, 2), (3, 3), (1, 1, 1, 1)])
def test_block_sizes(mics):
    p, Q0, ctx, st = setup(7, 33, mics, 3 if mics[0] > 1 else 2, 3, seed=22)
    check(p, st, 3, "nll", gpu_gradient(ctx, p, 3, 2, "nll"), 8, 4, seed=6)


def test_checkpoint_interval_does_not_change_the_result():
    """Recomputed segments replay the same deterministic iterations: bit-identical gradients
    (the loss value itself is summed across blocks with atomics, so only its last bits may
    move), and the context ends where dfmnmf_iterate would leave it."""
    p, Q0, ctx, st = setup(9, 40, (4, 4), 5, 4, seed=23)
    ref = None
    for every in (1, 3, 7, 10):
        D.dfmnmf_set_params(ctx, Q0, p.W0, p.H0, p.g0)
        got = gpu_gradient(ctx, p, 7, every, "nll")
        state = D.params_numpy(ctx)
        if ref is None:
            ref = got
            ctx2 = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0, Q0)
            D.dfmnmf_iterate(ctx2, 7)
            for a, b in zip(state, D.params_numpy(ctx2)):
                np.testing.assert_array_equal(a, b)
            continue
        assert abs(got[0] - ref[0]) <= 1e-14 * abs(ref[0])  # the loss sums blocks with atomics
        for a, b in zip(got[1] + list(got[2:]), ref[1] + list(ref[2:])):
            np.testing.assert_array_equal(a, b)


def test_zero_iterations_is_the_cost_gradient():
    p, Q0, ctx, st = setup(9, 40, (4, 4), 5, 4, seed=24)
    L, dQ, dW, dH, dg = gpu_gradient(ctx, p, 0, 5, "nll")
    rQ, rW, rH, rg = O.cost_gradient(p.x, p.mics, st)
    assert abs(L - O.neg_loglik(p.x.astype(np.complex128), p.mics, st)) <= 1e-12 * abs(L)
    for a, b in ((dW, rW), (dH, rH), (dg, rg)):
        assert rel_err(a, b) < 1e-10
    assert max(rel_err(dQ[k], rQ[k]) for k in range(2)) < 1e-10


def test_autograd_function():
    p, Q0, ctx, st = setup(9, 40, (4, 4), 5, 4, seed=25)
    adj = D.dfmnmf_adjoint_create(ctx, 4, 2)
    Qt = torch.tensor(Q0, device="cuda", requires_grad=True)
    Wt, Ht, gt = (torch.tensor(a, device="cuda", requires_grad=True) for a in (p.W0, p.H0, p.g0))
    ct = torch.from_numpy(p.c).cuda()
    L = AG.unrolled(adj, Qt, Wt, Ht, gt, "wiener_mse", ct)
    (3.0 * L).backward()
    _, rQ, rW, rH, rg = OA.unrolled_gradient(p.x, p.mics, st.Q, st.W, st.H, st.g, 4, "wiener_mse", p.c)
    assert rel_err(Wt.grad.cpu().numpy(), 3 * rW) < TOL
    assert rel_err(Ht.grad.cpu().numpy(), 3 * rH) < TOL
    assert rel_err(gt.grad.cpu().numpy(), 3 * rg) < TOL
    gQ = O.unpack_Q(Qt.grad.cpu().numpy(), p.mics)
    assert max(rel_err(gQ[k], 3 * rQ[k]) for k in range(2)) < TOL


def test_rejects_bad_arguments():
    p, Q0, ctx, st = setup(5, 20, (4, 4), 3, 2, seed=26)
    for n_iter, every in ((-1, 5), (3, 0)):
        with pytest.raises(D.DfmnmfError) as ei:
            D.dfmnmf_adjoint_create(ctx, n_iter, every)
        assert ei.value.code == D.DFMNMF_EINVAL
    tc = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0, precision=D.DFMNMF_BF16_TC)
    with pytest.raises(D.DfmnmfError) as ei:
        D.dfmnmf_adjoint_create(tc, 3, 1)
    assert ei.value.code == D.DFMNMF_EINVAL
    adj = D.dfmnmf_adjoint_create(ctx, 2, 1)
    for loss, ct in ((7, None), (D.DFMNMF_LOSS_WIENER_MSE, None)):
        with pytest.raises(D.DfmnmfError) as ei:
            D.dfmnmf_adjoint_run(adj, loss, ct)
        assert ei.value.code == D.DFMNMF_EINVAL


@pytest.mark.parametrize("loss,n_fd", [("nll", 32), ("wiener_mse", 32)])
def test_differentiation_workload_20_iterations(loss, n_fd):
    """4 x 4 mics, N = 5, B = 16, F = 257, T = 313; 20 iterations, checkpoints every 5;
    32 random directions against the oracle gradient, n_fd against FP64 central differences."""
    p, Q0, ctx, st = setup(257, 313, (4, 4, 4, 4), 5, 16, seed=27)
    errs = check(p, st, 20, loss, gpu_gradient(ctx, p, 20, 5, loss), 32, n_fd, seed=7)
    print("adjoint", loss, errs)
