"""Initialisation from given source images (Sec. IV-A, steps 3, 5, 6) on the
GPU against the FP64 oracle.

Each row of Q is a generalised eigenvector fixed only up to a unit phase
factor, so rows are compared after aligning their phase; g, h, the cost and
every update are phase-invariant.

Tolerances follow the arithmetic.  The GPU sums R from exact products in
float pairs (about 2^-44 relative per sum), the oracle in FP64, so the two R
differ by ~1e-14 relative; everything after that is FP64 up to the final
FP32 stores.  A generalised eigenvector moves by up to cond(R_b) times the
relative change of R, hence Q within max(1e-10, 1e-13 cond(R_b)) and g
within 1e-6 (FP32 storage, the same amplification on top).  h applies a
single-precision L^{-1} with single-precision sums: per frame,
|dz_i| <= e_i = ((i + 2) u + 1e-13 cond(R)) sum_k |X_ik| |c_k| (the dot-product
rounding bound with X = L^{-1} rounded to FP32, plus the covariance
perturbation), and |dh| <= sum_i (2 |z_i| e_i + e_i^2) / M + u h; the test
allows twice that bound, element by element.
"""
import numpy as np
import pytest

import oracle as O
from paper_2605_19388_gb300 import synth
from tests._helpers import rel_err, elem_err_Q, elem_err_med

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_19388_gb300 import dfmnmf as D  # noqa: E402


def images(F, T, mics, N, seed, noise_std=1e-3):
    """Soft-masked stand-in images c_n = (lambda_n / sum lambda) x with the generator's PSDs."""
    p = synth.make_problem(F, T, mics, N, 4, seed=seed, noise_std=noise_std)
    lam = O.source_psd(p.W0, p.H0) + 1e-3
    mask = lam / lam.sum(axis=0, keepdims=True)
    c = (mask[..., None] * p.x.astype(np.complex128)[None]).astype(np.complex64)
    return p, c


def phase_aligned(Qg, Qr):
    """Rotate every row of Qg ([F][mk][mk]) by the unit phase that best matches Qr."""
    d = np.sum(Qg * np.conj(Qr), axis=-1)
    ph = d / np.maximum(np.abs(d), 1e-300)
    return Qg * np.conj(ph)[..., None]


def run_init(p, c, with_h=True, precision=None):
    kw = {} if precision is None else {"precision": precision}
    ctx = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0, p.Q0, **kw)
    c_dev = torch.from_numpy(c).cuda()
    h = torch.full((p.N, p.F, p.T), -1.0, dtype=torch.float32, device="cuda") if with_h else None
    D.dfmnmf_init_from_images(ctx, c_dev, h)
    Q, W, H, g = D.params_numpy(ctx)
    st = O.state_from_arrays(Q, W, H, g, ctx.mics)
    return ctx, st, (h.cpu().numpy() if with_h else None)


CASES = [
    # F, T, mics, N, seed, noise_std
    (33, 150, (4, 4, 4, 4), 5, 301, 1e-3),   # the paper's 4 x 4-mic layout
    (7, 37, (3, 3), 2, 302, 1e-3),           # ragged frames (< one staged chunk), N = 2
    (5, 97, (2, 2, 2), 3, 303, 1e-3),        # partial last chunk
    (4, 64, (1, 1, 1, 1, 1, 1, 1, 1), 3, 304, 1e-3),  # one microphone per subarray
    (9, 120, (16,), 4, 305, 5e-2),           # all 16 microphones in one block
    (3, 80, (4,) * 8, 3, 306, 1e-2),         # M = 32, the largest supported
]


U32 = 2.0 ** -24


def q_tolerance(c, mics):
    """max(1e-10, 1e-13 cond(R_b)) over the blocks of the last source's covariance."""
    N, F, T, M = c.shape
    cd = c.astype(np.complex128)
    R = np.einsum("ftm,ftl->fml", cd[N - 1], np.conj(cd[N - 1])) / T
    off = O.mic_offsets(mics)
    kb = max(np.linalg.cond(R[f][off[k]:off[k] + mk, off[k]:off[k] + mk])
             for k, mk in enumerate(mics) for f in range(F))
    return max(1e-10, 1e-13 * kb)


def h_bound(c, h_ref):
    """Element-wise bound of the single-precision evaluation of h (module docstring)."""
    N, F, T, M = c.shape
    cd = c.astype(np.complex128)
    out = np.empty((N, F, T))
    for n in range(N):
        for f in range(F):
            R = cd[n, f].T @ np.conj(cd[n, f]) / T
            X = np.linalg.inv(np.linalg.cholesky(R))
            z = X @ cd[n, f].T                                     # [M][T]
            s = np.abs(X) @ np.abs(cd[n, f]).T
            e = ((np.arange(M) + 2)[:, None] * U32 + 1e-13 * np.linalg.cond(R)) * s
            out[n, f] = np.sum(2 * np.abs(z) * e + e * e, axis=0) / M + U32 * h_ref[n, f]
    return out


@pytest.mark.parametrize("F,T,mics,N,seed,noise", CASES)
def test_init_matches_oracle(F, T, mics, N, seed, noise):
    p, c = images(F, T, mics, N, seed, noise)
    ctx, st, h = run_init(p, c)
    h_ref, Q_ref, g_ref = O.init_from_images(c, p.mics)
    tq = q_tolerance(c, p.mics)
    errs = {f"Q{k}": rel_err(phase_aligned(st.Q[k], Q_ref[k]), Q_ref[k]) for k in range(len(p.mics))}
    errs["g"] = rel_err(st.g, g_ref)
    excess = np.abs(h - h_ref) / (2 * h_bound(c, h_ref))
    errs["h"] = rel_err(h, h_ref)
    for k in range(len(p.mics)):
        errs[f"Q{k}_elem"] = elem_err_Q(phase_aligned(st.Q[k], Q_ref[k]), Q_ref[k])
    errs["g_elem"] = elem_err_med(st.g, g_ref)
    print("initialisation from images", (F, T, mics, N), "tolerance", tq, errs)
    for k in range(len(p.mics)):
        assert errs[f"Q{k}"] <= tq, (errs, tq)
        # entries far below their row's largest carry that largest's absolute accuracy (row floor)
        assert errs[f"Q{k}_elem"] <= 10 * tq, (errs, tq)
    assert errs["g"] <= max(1e-6, tq), errs
    assert errs["g_elem"] <= 10 * max(1e-6, tq), errs
    assert excess.max() <= 1.0, (float(excess.max()), errs)
    # W and H are kept
    assert np.array_equal(st.W, p.W0.astype(np.float32))
    assert np.array_equal(st.H, p.H0.astype(np.float32))


def test_init_satisfies_the_generalised_eigenproblem():
    """Independently of the oracle: Q R_{N-1} Q^H = I, Q R_{N-2} Q^H diagonal with
    ascending entries, g of the last source = 1 and of the one before = those entries."""
    p, c = images(17, 200, (4, 4, 4, 4), 4, 311)
    _, st, _ = run_init(p, c, with_h=False)
    cd = c.astype(np.complex128)
    R = np.einsum("nftm,nftl->nfml", cd, np.conj(cd)) / p.T
    off = O.mic_offsets(p.mics)
    N = p.N
    tq = q_tolerance(c, p.mics)  # the identities hold for the GPU's own R, 1e-14 away from this one
    for k, mk in enumerate(p.mics):
        sl = slice(off[k], off[k] + mk)
        for f in range(p.F):
            Qf = st.Q[k][f]
            Bm = Qf @ R[N - 1, f][sl, sl] @ np.conj(Qf.T)
            A = Qf @ R[N - 2, f][sl, sl] @ np.conj(Qf.T)
            assert np.abs(Bm - np.eye(mk)).max() < tq
            assert np.abs(A - np.diag(np.diag(A))).max() < tq * np.abs(A).max()
            ev = np.real(np.diag(A))
            assert np.all(np.diff(ev) >= -tq * np.abs(ev).max())
            np.testing.assert_allclose(st.g[f, N - 1, sl], 1.0, rtol=1e-6)
            np.testing.assert_allclose(st.g[f, N - 2, sl], ev, rtol=1e-6)


def test_init_without_h_and_tensor_core_context():
    """h_out = NULL skips step 3's h; a BF16_TC context refreshes its single-precision Q."""
    p, c = images(12, 128, (4, 4, 4, 4), 5, 312)
    _, st_a, _ = run_init(p, c, with_h=False)
    ctx, st_b, h = run_init(p, c, with_h=True, precision=D.DFMNMF_BF16_TC)
    for k in range(4):
        np.testing.assert_array_equal(st_a.Q[k], st_b.Q[k])
    np.testing.assert_array_equal(st_a.g, st_b.g)
    # the iteration then starts from the new Q: Eq. (12) matches the oracle's from the same state
    x = p.x.astype(np.complex128)
    nll_gpu = D.dfmnmf_loglik(ctx)
    nll_ref = O.neg_loglik(x, p.mics, st_b)
    assert abs(nll_gpu - nll_ref) <= 1e-5 * abs(nll_ref)


def test_init_then_iterate_follows_the_oracle():
    """Initialise on both sides, then 10 MM iterations (FP32 form): Eq. (12) within 1e-3."""
    p, c = images(17, 160, (4, 4, 4, 4), 4, 313)
    ctx, _, _ = run_init(p, c, with_h=False)
    D.dfmnmf_iterate(ctx, 10)
    nll_gpu = D.dfmnmf_loglik(ctx)
    _, Q_ref, g_ref = O.init_from_images(c, p.mics)
    st = O.state_from_arrays(np.concatenate([q.reshape(p.F, -1) for q in Q_ref], axis=1),
                             p.W0, p.H0, g_ref, p.mics)
    x = p.x.astype(np.complex128)
    for _ in range(10):
        st = O.mm_iteration(x, p.mics, st)
    nll_ref = O.neg_loglik(x, p.mics, st)
    assert abs(nll_gpu - nll_ref) <= 1e-3 * abs(nll_ref), (nll_gpu, nll_ref)


def test_init_rejects_bad_arguments():
    p, c = images(3, 20, (2, 2), 2, 314)
    ctx = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0, p.Q0)
    with pytest.raises(D.DfmnmfError) as ei:  # host memory
        D.dfmnmf_init_from_images(ctx, c)
    assert ei.value.code == D.DFMNMF_EINVAL
    p1 = synth.make_problem(3, 20, (2, 2), 1, 2, seed=315)
    ctx1 = D.dfmnmf_init(p1.F, p1.T, p1.mics, p1.N, p1.B, p1.x, p1.W0, p1.H0, p1.g0, p1.Q0)
    c1 = torch.zeros((1, 3, 20, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(D.DfmnmfError) as ei:  # one source: no pair to diagonalise
        D.dfmnmf_init_from_images(ctx1, c1)
    assert ei.value.code == D.DFMNMF_EINVAL


def test_init_reports_a_singular_covariance():
    """The last source's image is zero in one bin: its block covariance is not positive definite."""
    p, c = images(4, 40, (2, 2), 3, 316)
    c[p.N - 1, 2] = 0
    ctx = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0, p.Q0)
    with pytest.raises(D.DfmnmfError) as ei:
        D.dfmnmf_init_from_images(ctx, torch.from_numpy(c).cuda())
    assert ei.value.code == D.DFMNMF_ENUMERIC
