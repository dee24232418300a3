"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: each checks it against a
library routine it does not call, a brute-force sum, a closed form, or an
invariant the paper states (MM / IP monotonicity, stationarity of the IP
update, the fixed point of the multiplicative updates, the block structure).
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2605_19388_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def tiny(seed=0, F=4, T=24, mics=(2, 3), N=2, B=3, noise=0.05):
    p = synth.make_problem(F, T, mics, N, B, seed=seed, noise_std=noise)
    st = O.state_from_arrays(p.Q0, p.W0, p.H0, p.g0, p.mics)
    x = p.x.astype(np.complex128)
    return p, st, x


# --------------------------------------------------------------------------- Eq. (13)
def test_weighted_covariance_brute_force():
    """Eq. (13) against a pure-Python triple loop on a tiny case."""
    p, st, x = tiny(F=2, T=5, mics=(2, 1, 3))
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    V = O.weighted_covariances(x, y, p.mics)
    off = O.mic_offsets(p.mics)
    for k, mk in enumerate(p.mics):
        for f in range(p.F):
            for mu in range(mk):
                ref = np.zeros((mk, mk), dtype=complex)
                for t in range(p.T):
                    for a in range(mk):
                        for b in range(mk):
                            ref[a, b] += x[f, t, off[k] + a] * np.conj(x[f, t, off[k] + b]) \
                                / y[f, t, off[k] + mu]
                ref /= p.T
                np.testing.assert_allclose(V[k][f, mu], ref, rtol=1e-12, atol=1e-14)


def test_weighted_covariance_unit_weights_is_sample_covariance():
    """With yhat == 1, Eq. (13) is the (zero-mean) sample covariance: numpy.cov."""
    rng = np.random.default_rng(3)
    F, T, mics = 3, 50, (3, 2)
    x = rng.standard_normal((F, T, 5)) + 1j * rng.standard_normal((F, T, 5))
    x -= x.mean(axis=1, keepdims=True)
    V = O.weighted_covariances(x, np.ones((F, T, 5)), mics)
    off = O.mic_offsets(mics)
    for k, mk in enumerate(mics):
        for f in range(F):
            c = np.cov(x[f, :, off[k]:off[k] + mk], rowvar=False, bias=True)
            for mu in range(mk):
                np.testing.assert_allclose(V[k][f, mu], c, rtol=1e-12, atol=1e-13)


# --------------------------------------------------------------------------- solves
def test_ge_solve_matches_numpy_solve():
    rng = np.random.default_rng(1)
    for n in (1, 2, 3, 4, 6):
        A = rng.standard_normal((20, n, n)) + 1j * rng.standard_normal((20, n, n))
        b = rng.standard_normal((20, n)) + 1j * rng.standard_normal((20, n))
        xs, minpiv, scale = O.ge_solve(A, b)
        ref = np.linalg.solve(A, b[..., None])[..., 0]
        np.testing.assert_allclose(xs, ref, rtol=1e-10, atol=1e-12)
        assert np.all(minpiv > 0)


def test_ge_detects_singular_and_pinv_matches_numpy():
    rng = np.random.default_rng(2)
    u = rng.standard_normal((4, 2)) + 1j * rng.standard_normal((4, 2))
    v = rng.standard_normal((2, 4)) + 1j * rng.standard_normal((2, 4))
    A = (u @ v)[None]                                   # rank 2
    e = np.zeros((1, 4), dtype=complex)
    e[0, 1] = 1
    q, singular = O.solve_or_pinv(A, e)
    assert singular[0]
    np.testing.assert_allclose(q[0], np.linalg.pinv(A[0], rcond=1e-12) @ e[0], rtol=1e-9, atol=1e-12)
    # zero matrix -> zero solution
    q0, s0 = O.solve_or_pinv(np.zeros((1, 3, 3), dtype=complex), np.eye(3, dtype=complex)[:1])
    assert s0[0] and np.all(q0 == 0)


def test_log_abs_det_matches_slogdet():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((7, 4, 4)) + 1j * rng.standard_normal((7, 4, 4))
    ref = 2 * np.linalg.slogdet(A)[1]
    np.testing.assert_allclose(O.log_abs_det_sq(A), ref, rtol=1e-12)


# --------------------------------------------------------------------------- Eqs. (14)-(15)
def test_ip_row_stationarity():
    """After row mu is updated: Q_new V_mu q = e_mu and q^H V_mu q = 1 (Eqs. 14-15)."""
    p, st, x = tiny(mics=(3, 4, 1), F=5, T=30)
    st.Q = O.unpack_Q(synth.random_blocks(p.F, p.mics, seed=9), p.mics)
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    V = O.weighted_covariances(x, y, p.mics)
    for k, mk in enumerate(p.mics):
        Qk = st.Q[k]
        for mu in range(mk):
            Qk = O.ip_update_row(Qk, V[k], mu)
            q = np.conj(Qk[:, mu, :])                          # column vector q
            lhs = np.einsum("fab,fbc,fc->fa", Qk, V[k][:, mu], q)
            e = np.zeros_like(lhs)
            e[:, mu] = 1
            np.testing.assert_allclose(lhs, e, atol=1e-10)
            quad = np.einsum("fa,fab,fb->f", np.conj(q), V[k][:, mu], q)
            np.testing.assert_allclose(quad, 1.0, atol=1e-10)


def test_ip_sweep_updates_rows_in_turn():
    """A whole sweep (Eq. 13 then Eqs. 14-15 for mu = 0, 1, ... in turn): the last row updated
    satisfies Q V_mu q = e_mu with the final block, which holds only if every row was solved
    from the block with the rows before it already replaced."""
    p, st, x = tiny(mics=(3, 4, 2), F=5, T=30)
    st.Q = O.unpack_Q(synth.random_blocks(p.F, p.mics, seed=19), p.mics)
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    V = O.weighted_covariances(x, y, p.mics)
    Qn = O.ip_update(st.Q, V)
    for k, mk in enumerate(p.mics):
        mu = mk - 1
        q = np.conj(Qn[k][:, mu, :])
        lhs = np.einsum("fab,fbc,fc->fa", Qn[k], V[k][:, mu], q)
        e = np.zeros_like(lhs)
        e[:, mu] = 1
        np.testing.assert_allclose(lhs, e, atol=1e-10)
        np.testing.assert_allclose(np.einsum("fa,fab,fb->f", np.conj(q), V[k][:, mu], q), 1.0, atol=1e-10)


def test_ip_single_mic_closed_form():
    """M_k = 1: the block becomes exp(i arg Q) / sqrt(V) (scalar case of Eqs. 14-15)."""
    p, st, x = tiny(mics=(1, 1, 1), F=3, T=17)
    rng = np.random.default_rng(5)
    st.Q = [q * (0.5 + rng.random(q.shape)) * np.exp(1j * rng.uniform(0, 6, q.shape)) for q in st.Q]
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    V = O.weighted_covariances(x, y, p.mics)
    Qn = O.ip_update(st.Q, V)
    for k in range(3):
        ref = np.exp(1j * np.angle(st.Q[k][:, 0, 0])) / np.sqrt(V[k][:, 0, 0, 0].real)
        np.testing.assert_allclose(Qn[k][:, 0, 0], ref, rtol=1e-12)


def test_ip_keeps_block_structure_and_dense_cost():
    """Q_f stays block diagonal; Eq. (12) equals the dense Eq. (4) with W_i^H = blkdiag."""
    p, st, x = tiny(mics=(2, 3), F=3, T=20)
    st = O.mm_iteration(x, p.mics, st)
    D = O.dense_Q(st.Q)
    M = p.M
    mask = np.zeros((M, M), dtype=bool)
    off = O.mic_offsets(p.mics)
    for k, mk in enumerate(p.mics):
        mask[off[k]:off[k] + mk, off[k]:off[k] + mk] = True
    assert np.all(D[:, ~mask] == 0)
    # dense Eq. (4)
    yv = np.einsum("fab,ftb->fta", D, x)
    eta = O.model_variance(O.source_psd(st.W, st.H), st.g)
    dense = np.sum(np.abs(yv) ** 2 / eta + np.log(eta)) - p.T * np.sum(2 * np.linalg.slogdet(D)[1])
    np.testing.assert_allclose(O.neg_loglik(x, p.mics, st), dense, rtol=1e-12)


# --------------------------------------------------------------------------- MM guarantee
def test_cost_non_increasing_after_every_substep():
    """IP rows and each MU rule never increase Eq. (12) (Sec. II-A / III-B MM guarantee)."""
    p, st, x = tiny(seed=11, F=6, T=40, mics=(3, 2, 4), N=3, B=4)
    st.Q = O.unpack_Q(synth.random_blocks(p.F, p.mics, seed=1), p.mics)
    cost = lambda s: O.neg_loglik(x, p.mics, s)
    prev = cost(st)
    for it in range(6):
        y = O.model_variance(O.source_psd(st.W, st.H), st.g)
        assert y.min() > O.EPS            # no floor binds in this fixture
        V = O.weighted_covariances(x, y, p.mics)
        for k, mk in enumerate(p.mics):
            for mu in range(mk):
                st.Q[k] = O.ip_update_row(st.Q[k], V[k], mu)
                c = cost(st)
                assert c <= prev + 1e-10 * abs(prev), (it, k, mu, c - prev)
                prev = c
        P = O.projected_power(x, st.Q, p.mics)
        for name in ("W", "H", "g"):
            fn = {"W": O.update_W, "H": O.update_H, "g": O.update_g}[name]
            setattr(st, name, fn(st.W, st.H, st.g, P))
            c = cost(st)
            assert c <= prev + 1e-10 * abs(prev), (it, name, c - prev)
            prev = c


def test_mu_fixed_point_when_power_equals_model():
    """Feeding P := yhat makes every ratio in Eqs. (8)-(10) equal to 1."""
    p, st, x = tiny(F=5, T=21, mics=(2, 2), N=3, B=2)
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    np.testing.assert_allclose(O.update_W(st.W, st.H, st.g, y), st.W, rtol=1e-13)
    np.testing.assert_allclose(O.update_H(st.W, st.H, st.g, y), st.H, rtol=1e-13)
    np.testing.assert_allclose(O.update_g(st.W, st.H, st.g, y), st.g, rtol=1e-13)


def test_mu_updates_match_direct_sums():
    """Eqs. (8)-(10) written as their literal double sums (no factorisation)."""
    p, st, x = tiny(F=3, T=7, mics=(2, 1), N=2, B=2)
    P = O.projected_power(x, st.Q, p.mics)
    W, H, g = st.W, st.H, st.g
    N, F, B = W.shape
    T, M = p.T, p.M
    eta = np.zeros((F, T, M))
    for f, t, m in itertools.product(range(F), range(T), range(M)):
        eta[f, t, m] = max(sum(W[n, f, b] * H[n, b, t] * g[f, n, m]
                               for n in range(N) for b in range(B)), O.EPS)
    Wr = W.copy()
    for n, f, b in itertools.product(range(N), range(F), range(B)):
        num = sum(H[n, b, t] * g[f, n, m] * P[f, t, m] / eta[f, t, m] ** 2 for t in range(T) for m in range(M))
        den = sum(H[n, b, t] * g[f, n, m] / eta[f, t, m] for t in range(T) for m in range(M))
        Wr[n, f, b] = W[n, f, b] * np.sqrt(num / max(den, O.EPS))
    np.testing.assert_allclose(O.update_W(W, H, g, P), Wr, rtol=1e-12)
    Hr = H.copy()
    for n, b, t in itertools.product(range(N), range(B), range(T)):
        num = sum(W[n, f, b] * g[f, n, m] * P[f, t, m] / eta[f, t, m] ** 2 for f in range(F) for m in range(M))
        den = sum(W[n, f, b] * g[f, n, m] / eta[f, t, m] for f in range(F) for m in range(M))
        Hr[n, b, t] = H[n, b, t] * np.sqrt(num / max(den, O.EPS))
    np.testing.assert_allclose(O.update_H(W, H, g, P), Hr, rtol=1e-12)
    gr = g.copy()
    for f, n, m in itertools.product(range(F), range(N), range(M)):
        lam = [sum(W[n, f, b] * H[n, b, t] for b in range(B)) for t in range(T)]
        num = sum(lam[t] * P[f, t, m] / eta[f, t, m] ** 2 for t in range(T))
        den = sum(lam[t] / eta[f, t, m] for t in range(T))
        gr[f, n, m] = g[f, n, m] * np.sqrt(num / max(den, O.EPS))
    np.testing.assert_allclose(O.update_g(W, H, g, P), gr, rtol=1e-12)


# --------------------------------------------------------------------------- reductions
def _conventional_fastmnmf_iteration(x, Wi, t, v, lam, eps=O.EPS):
    """Conventional FastMNMF (Eqs. 5-10) in the paper's own notation, dense M x M.

    Wi: [I][M][M] (columns w_im), t: [I][K][N], v: [K][J][N], lam: [I][N][M]."""
    I, J, M = x.shape

    def eta():
        h = np.einsum("ikn,kjn->ijn", t, v)
        return np.maximum(np.einsum("ijn,inm->ijm", h, lam), eps)

    e = eta()
    for i in range(I):
        for m in range(M):
            Qim = np.einsum("j,ja,jb->ab", 1 / e[i, :, m], x[i], np.conj(x[i])) / J
            w = np.linalg.solve(np.conj(Wi[i]).T @ Qim, np.eye(M)[m])
            w = w / np.sqrt(max(np.real(np.conj(w) @ Qim @ w), eps))
            Wi[i][:, m] = w
    y2 = np.abs(np.einsum("iam,ija->ijm", np.conj(Wi), x)) ** 2
    e = eta()
    t = t * np.sqrt(np.einsum("kjn,inm,ijm->ikn", v, lam, y2 / e ** 2)
                    / np.maximum(np.einsum("kjn,inm,ijm->ikn", v, lam, 1 / e), eps))
    e = eta()
    v = v * np.sqrt(np.einsum("ikn,inm,ijm->kjn", t, lam, y2 / e ** 2)
                    / np.maximum(np.einsum("ikn,inm,ijm->kjn", t, lam, 1 / e), eps))
    h = np.einsum("ikn,kjn->ijn", t, v)
    e = eta()
    lam = lam * np.sqrt(np.einsum("ijn,ijm->inm", h, y2 / e ** 2)
                        / np.maximum(np.einsum("ijn,ijm->inm", h, 1 / e), eps))
    return Wi, t, v, lam


def test_single_block_reduces_to_conventional_fastmnmf():
    """K = 1 (L = 1 in the paper) is conventional FastMNMF (Sec. III-B, last paragraph)."""
    p, st, x = tiny(F=3, T=25, mics=(4,), N=2, B=3)
    st.Q = O.unpack_Q(synth.random_blocks(p.F, p.mics, seed=2), p.mics)
    Wi = np.conj(np.transpose(st.Q[0], (0, 2, 1))).copy()
    t = np.transpose(st.W, (1, 2, 0)).copy()
    v = np.transpose(st.H, (1, 2, 0)).copy()
    lam = np.transpose(st.g, (0, 1, 2)).copy()
    for _ in range(3):
        st = O.mm_iteration(x, p.mics, st)
        Wi, t, v, lam = _conventional_fastmnmf_iteration(x, Wi, t, v, lam)
    np.testing.assert_allclose(st.Q[0], np.conj(np.transpose(Wi, (0, 2, 1))), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(st.W, np.transpose(t, (2, 0, 1)), rtol=1e-9)
    np.testing.assert_allclose(st.H, np.transpose(v, (2, 0, 1)), rtol=1e-9)
    np.testing.assert_allclose(st.g, lam, rtol=1e-9)


def test_unshared_nmf_equals_separate_subarray_runs():
    """Per-subarray NMF matches one-subarray FastMNMF to machine precision (Sec. IV-B).

    The unshared variant is the distributed model with N*K sources where source
    (n, k) has g = 0 outside subarray k; multiplicative updates keep those zeros."""
    p, st, x = tiny(seed=5, F=4, T=30, mics=(2, 3), N=2, B=3)
    K, N = p.K, p.N
    off = O.mic_offsets(p.mics)
    rng = np.random.default_rng(8)
    Wk = [rng.uniform(0.1, 1, (N, p.F, p.B)) for _ in range(K)]
    Hk = [rng.uniform(0.1, 1, (N, p.B, p.T)) for _ in range(K)]
    gk = [rng.uniform(0.1, 1, (p.F, N, mk)) for mk in p.mics]
    # joint (unshared) run
    g_joint = np.zeros((p.F, N * K, p.M))
    for k, mk in enumerate(p.mics):
        g_joint[:, k * N:(k + 1) * N, off[k]:off[k] + mk] = gk[k]
    joint = O.State([q.copy() for q in st.Q], np.concatenate(Wk), np.concatenate(Hk), g_joint)
    seps = [O.State([st.Q[k].copy()], Wk[k].copy(), Hk[k].copy(), gk[k].copy()) for k in range(K)]
    for _ in range(4):
        joint = O.mm_iteration(x, p.mics, joint)
        seps = [O.mm_iteration(x[:, :, off[k]:off[k] + mk], (mk,), seps[k])
                for k, mk in enumerate(p.mics)]
    for k, mk in enumerate(p.mics):
        np.testing.assert_allclose(joint.Q[k], seps[k].Q[0], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(joint.W[k * N:(k + 1) * N], seps[k].W, rtol=1e-12)
        np.testing.assert_allclose(joint.H[k * N:(k + 1) * N], seps[k].H, rtol=1e-12)
        np.testing.assert_allclose(joint.g[:, k * N:(k + 1) * N, off[k]:off[k] + mk], seps[k].g,
                                   rtol=1e-12)


# --------------------------------------------------------------------------- Wiener filter
def test_wiener_sums_to_mixture_and_matches_dense_posterior_mean():
    p, st, x = tiny(F=3, T=9, mics=(2, 3), N=3, B=2)
    st.Q = O.unpack_Q(synth.random_blocks(p.F, p.mics, seed=4), p.mics)
    c = O.wiener_filter(x, p.mics, st)
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    assert y.min() > O.EPS
    np.testing.assert_allclose(c.sum(axis=0), x, rtol=1e-11, atol=1e-12)
    # dense posterior mean lambda_n R_n Sigma^{-1} x, R_n = Q^{-1} diag(g_n) Q^{-H} (Eqs. 1, 3)
    D = O.dense_Q(st.Q)
    lam = O.source_psd(st.W, st.H)
    for f in range(p.F):
        Di = np.linalg.inv(D[f])
        R = [Di @ np.diag(st.g[f, n]) @ np.conj(Di).T for n in range(p.N)]
        for t in range(p.T):
            S = sum(lam[n, f, t] * R[n] for n in range(p.N))
            for n in range(p.N):
                ref = lam[n, f, t] * R[n] @ np.linalg.solve(S, x[f, t])
                np.testing.assert_allclose(c[n, f, t], ref, rtol=1e-9, atol=1e-11)


def test_wiener_invariant_to_row_scaling_of_Q():
    """c_n = Q^{-1} diag(lambda_n g_n / yhat) Q x: the gain is diagonal and does not involve P,
    so scaling the rows of every block by nonzero complex factors (Q -> D Q) leaves c unchanged."""
    p, st, x = tiny(F=3, T=11, mics=(2, 3, 1), N=2, B=2, seed=12)
    st.Q = O.unpack_Q(synth.random_blocks(p.F, p.mics, seed=13), p.mics)
    c = O.wiener_filter(x, p.mics, st)
    rng = np.random.default_rng(14)
    scaled = []
    for Qk in st.Q:
        d = rng.uniform(0.3, 3.0, Qk.shape[:2]) * np.exp(1j * rng.uniform(0, 2 * np.pi, Qk.shape[:2]))
        scaled.append(d[:, :, None] * Qk)
    c2 = O.wiener_filter(x, p.mics, O.State(scaled, st.W, st.H, st.g))
    np.testing.assert_allclose(c2, c, rtol=1e-10, atol=1e-12 * np.abs(c).max())


# --------------------------------------------------------------------------- Appendix theorem
def test_block_joint_diagonalisability_theorem():
    """Appendix: block-diagonal R_n are jointly diagonalisable iff every block family is.

    Checked with the commutator criterion on normalised matrices S^{-1/2} R_n S^{-1/2}."""
    rng = np.random.default_rng(6)
    mics, N = (2, 3), 3

    def commutators(Rs):
        S = sum(Rs)
        w, U = np.linalg.eigh(S)
        Sm = U @ np.diag(w ** -0.5) @ np.conj(U).T
        Rt = [Sm @ R @ Sm for R in Rs]
        return max(np.abs(a @ b - b @ a).max() for a in Rt for b in Rt)

    def blkdiag(blocks):
        M = sum(b.shape[0] for b in blocks)
        out = np.zeros((M, M), dtype=complex)
        o = 0
        for b in blocks:
            out[o:o + b.shape[0], o:o + b.shape[0]] = b
            o += b.shape[0]
        return out

    # jointly diagonalisable blocks: A_l diag(d) A_l^H
    A = [rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)) for m in mics]
    Rs = [blkdiag([a @ np.diag(rng.uniform(0.1, 1, a.shape[0])) @ np.conj(a).T for a in A])
          for _ in range(N)]
    assert commutators(Rs) < 1e-9
    # generic PSD blocks: not jointly diagonalisable
    Rg = []
    for _ in range(N):
        bl = []
        for m in mics:
            z = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
            bl.append(z @ np.conj(z).T + 0.1 * np.eye(m))
        Rg.append(blkdiag(bl))
    assert commutators(Rg) > 1e-3


def test_cost_gradient_matches_central_differences():
    """The analytic gradient of Eq. (12) against FP64 central differences of the
    cost itself, entry by entry, on a tiny random state (no floor binding)."""
    p = synth.make_problem(3, 20, (2, 2), 2, 3, seed=71)
    x = p.x.astype(np.complex128)
    st = O.state_from_arrays(synth.random_blocks(p.F, p.mics, seed=72), p.W0, p.H0, p.g0, p.mics)
    st = O.mm_iteration(x, p.mics, st)  # a generic, non-stationary state
    dQ, dW, dH, dg = O.cost_gradient(x, p.mics, st)
    rng = np.random.default_rng(73)
    h = 1e-6

    def cost(Q, W, H, g):
        return O.neg_loglik(x, p.mics, O.State(Q=Q, W=W, H=H, g=g))

    def check(arr_name, grad, cplx):
        base = getattr(st, arr_name)
        for _ in range(6):
            idx = tuple(rng.integers(0, s_) for s_ in base.shape)
            for part in ((1.0,) if not cplx else (1.0, 1j)):
                plus = base.copy(); minus = base.copy()
                plus[idx] += h * part * max(abs(base[idx]), 1.0)
                minus[idx] -= h * part * max(abs(base[idx]), 1.0)
                args = {"Q": st.Q, "W": st.W, "H": st.H, "g": st.g}
                fd = (cost(**{**args, arr_name: plus}) - cost(**{**args, arr_name: minus})) / (2 * h * max(abs(base[idx]), 1.0))
                an = grad[idx].real if part == 1.0 else grad[idx].imag
                assert abs(fd - an) <= 1e-5 * max(abs(an), 1.0), (arr_name, idx, part, fd, an)

    check("W", dW, False)
    check("H", dH, False)
    check("g", dg, False)
    for k in range(len(p.mics)):
        base = st.Q[k]
        for _ in range(6):
            idx = tuple(rng.integers(0, s_) for s_ in base.shape)
            for part in (1.0, 1j):
                Qp = [q.copy() for q in st.Q]; Qm = [q.copy() for q in st.Q]
                Qp[k][idx] += h * part
                Qm[k][idx] -= h * part
                fd = (cost(Qp, st.W, st.H, st.g) - cost(Qm, st.W, st.H, st.g)) / (2 * h)
                an = dQ[k][idx].real if part == 1.0 else dQ[k][idx].imag
                assert abs(fd - an) <= 1e-5 * max(abs(an), 1.0), ("Q", k, idx, part, fd, an)


def _images(F=5, T=60, mics=(4, 4), N=3, seed=90):
    """Soft-masked stand-in images: c_n = (lambda_n / sum lambda) x with the generator's PSDs."""
    p = synth.make_problem(F, T, mics, N, 4, seed=seed, with_images=True)
    lam = O.source_psd(p.W0, p.H0) + 1e-3
    mask = lam / lam.sum(axis=0, keepdims=True)
    return p, mask[..., None] * p.x.astype(np.complex128)[None]


def test_init_gevd_diagonalises_the_last_two_covariances():
    """Step 5: Q R_{N-1} Q^H = I and Q R_{N-2} Q^H diagonal per block; step 6 then
    gives g = 1 for the last source and the generalised eigenvalues (ascending)
    for the one before."""
    p, c = _images()
    h, Q, g = O.init_from_images(c, p.mics)
    N, F, T, M = c.shape
    R = np.einsum("nftm,nftl->nfml", c, np.conj(c)) / T
    off = O.mic_offsets(p.mics)
    for k, mk in enumerate(p.mics):
        sl = slice(off[k], off[k] + mk)
        for f in range(F):
            A = Q[k][f] @ R[N - 2, f][sl, sl] @ np.conj(Q[k][f].T)
            Bm = Q[k][f] @ R[N - 1, f][sl, sl] @ np.conj(Q[k][f].T)
            assert np.abs(Bm - np.eye(mk)).max() < 1e-9
            assert np.abs(A - np.diag(np.diag(A))).max() < 1e-9 * np.abs(A).max()
            ev = np.real(np.diag(A))
            assert np.all(np.diff(ev) >= -1e-12)
            np.testing.assert_allclose(g[f, N - 1, sl], 1.0, rtol=1e-9)
            np.testing.assert_allclose(g[f, N - 2, sl], ev, rtol=1e-9)


def test_init_spectrogram_invariant_to_channel_mixing_and_single_channel_closed_form():
    """Step 3: h = c^H R^{-1} c / M does not change when every frame is mixed by
    the same invertible matrix (R -> A R A^H), its mean over the frames is 1
    (sum_t c^H R^{-1} c / T = trace(R^{-1} R) = M), and for one channel it is
    |c|^2 / mean_t |c|^2."""
    p, c = _images(mics=(4, 4))
    h, _, _ = O.init_from_images(c, p.mics)
    np.testing.assert_allclose(h.mean(axis=2), 1.0, rtol=1e-8)
    rng = np.random.default_rng(91)
    Amix = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    h2, _, _ = O.init_from_images(np.einsum("ab,nftb->nfta", Amix, c), p.mics)
    # R of a masked 3-source, 8-channel mixture has cond ~1e6: FP64 solves agree to ~1e-8
    np.testing.assert_allclose(h2, h, rtol=1e-6)
    c1 = c[..., :1]
    h1, _, _ = O.init_from_images(c1, (1,))
    ref = np.abs(c1[..., 0]) ** 2 / np.mean(np.abs(c1[..., 0]) ** 2, axis=2, keepdims=True)
    np.testing.assert_allclose(h1, ref, rtol=1e-10)
