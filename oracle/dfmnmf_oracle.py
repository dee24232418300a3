"""FP64 CPU oracle of distributed FastMNMF.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may call it.  It shares no code with the CUDA path.

It is a plain, slow, obviously correct restatement of the paper's update
rules in float64, written step by step in the paper's order:

* Eq. (2)            source PSD (NMF model)          -> ``source_psd``
* Eq. (13) / (5)     weighted covariances            -> ``weighted_covariances``
* Eqs. (14)-(15)     iterative projection per block  -> ``ip_update`` / ``ip_update_row``
* Sec. III-B, y = W^H x (block)  projected powers    -> ``projected_power``
* Eq. (8)            basis update (t_ikn)            -> ``update_W``
* Eq. (9)            activation update (v_kjn)       -> ``update_H``
* Eq. (10)           diagonal SCM update             -> ``update_g``
* Eq. (12)           negative log-likelihood         -> ``neg_loglik``
* Sec. II-A/III-B    multichannel Wiener filter      -> ``wiener_filter``
* Sec. III-B         iteration schedule              -> ``mm_iteration``

Notation (paper -> this code): frequency i -> f, frame j -> t, subarray l -> k
(K subarrays, block sizes ``mics``), NMF basis k -> b (B bases), t_ikn ->
W[n,f,b], v_kjn -> H[n,b,t], [Lambda_in]_mm -> g[f,n,m], W_i^H -> Q_f (block
diagonal; row mu of block k is w_{i mu}^{(l) H}), Q_{i mu}^{(l)} -> V[k][f, mu],
eta_ijm -> yhat[f,t,m], |y_ijm|^2 -> P[f,t,m].

Readings of the paper taken here (each also listed in the design notes):
* g is per frequency: [Lambda_in] carries the frequency index (Eq. 10).
* Within an iteration: IP for every block first (Eqs. 13-15, rows mu in
  ascending order, each solve using the rows already updated), then W, H, g in
  equation order (Eqs. 8, 9, 10); yhat is recomputed after each of those three
  rules (the statement after Eq. 10), not after every single element.
* Floors (Sec. IV-A): yhat = max(sum_n lambda g, eps); every MU denominator is
  max(den, eps); the IP normaliser uses max(Re q^H V q, eps); numerators are
  not floored.  eps = 1e-6.
* Singular systems (Sec. IV-A): A = Q V_mu is treated as singular when the
  smallest pivot of Gaussian elimination with partial pivoting has magnitude
  <= ``singular_rtol`` * max|A_ij|; then q = pinv(A) e_mu, with pinv the
  SVD pseudo-inverse that drops singular values <= ``singular_rtol`` * s_max.
* The Wiener filter is the posterior mean of the source image under Eq. (1)
  with the block-diagonal, jointly diagonalised SCMs:
  c_n = Q^{-1} diag(lambda_n g_n / yhat) Q x, applied per subarray block.
* Eq. (12) is reported exactly as printed (no F T M ln(pi) constant).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

EPS = 1e-6                 # Sec. IV-A floor
SINGULAR_RTOL = 1e-12      # relative pivot / singular-value cut-off (FP64 reading)


# ----------------------------------------------------------------------------
# layout helpers (no arithmetic of the method)
# ----------------------------------------------------------------------------
def mic_offsets(mics: Sequence[int]) -> np.ndarray:
    """o_k = sum_{k' < k} M_k' (Sec. III-B: m = mu + sum_{lambda < l} M^(lambda))."""
    return np.concatenate([[0], np.cumsum(np.asarray(mics, dtype=np.int64))])


def unpack_Q(Qp: np.ndarray, mics: Sequence[int]) -> List[np.ndarray]:
    """Packed [F][sum M_k^2] -> list of K arrays [F][M_k][M_k] (complex128)."""
    F = Qp.shape[0]
    out, o = [], 0
    for mk in mics:
        out.append(np.array(Qp[:, o:o + mk * mk], dtype=np.complex128).reshape(F, mk, mk))
        o += mk * mk
    return out


def pack_Q(Q: List[np.ndarray]) -> np.ndarray:
    F = Q[0].shape[0]
    return np.ascontiguousarray(np.concatenate([q.reshape(F, -1) for q in Q], axis=1))


def dense_Q(Q: List[np.ndarray]) -> np.ndarray:
    """Block-diagonal W_i^H as a dense [F][M][M] matrix (Sec. III-B)."""
    F = Q[0].shape[0]
    mics = [q.shape[1] for q in Q]
    M = sum(mics)
    D = np.zeros((F, M, M), dtype=np.complex128)
    o = 0
    for q, mk in zip(Q, mics):
        D[:, o:o + mk, o:o + mk] = q
        o += mk
    return D


@dataclass
class State:
    Q: List[np.ndarray]     # K x [F][M_k][M_k] complex128
    W: np.ndarray           # [N][F][B] float64
    H: np.ndarray           # [N][B][T] float64
    g: np.ndarray           # [F][N][M] float64

    def copy(self) -> "State":
        return State([q.copy() for q in self.Q], self.W.copy(), self.H.copy(), self.g.copy())


def state_from_arrays(Qp, W, H, g, mics) -> State:
    return State(unpack_Q(np.asarray(Qp), mics), np.asarray(W, dtype=np.float64).copy(),
                 np.asarray(H, dtype=np.float64).copy(), np.asarray(g, dtype=np.float64).copy())


# ----------------------------------------------------------------------------
# model (Eq. 2 and the definition of eta after Eq. 7 / Eq. 15)
# ----------------------------------------------------------------------------
def source_psd(W: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Eq. (2): lambda[n,f,t] = sum_b W[n,f,b] H[n,b,t]  (h_ijn = sum_k t_ikn v_kjn)."""
    return np.matmul(W, H)


def model_variance(lam: np.ndarray, g: np.ndarray, eps: float = EPS) -> np.ndarray:
    """eta_ijm = sum_n h_ijn [Lambda_in]_mm, floored at eps (Sec. IV-A).

    yhat[f,t,m] = max(sum_n lambda[n,f,t] g[f,n,m], eps); the sum over n of the
    already-summed lambda is the factorisation stated with Table I."""
    F, N, M = g.shape
    T = lam.shape[2]
    y = np.zeros((F, T, M))
    for n in range(N):
        y += lam[n][:, :, None] * g[:, n, None, :]
    return np.maximum(y, eps)


# ----------------------------------------------------------------------------
# iterative projection (Eqs. 13-15)
# ----------------------------------------------------------------------------
def weighted_covariances(x: np.ndarray, yhat: np.ndarray, mics: Sequence[int]) -> List[np.ndarray]:
    """Eq. (13): V[k][f, mu] = (1/T) sum_t x_ftk x_ftk^H / yhat[f, t, o_k + mu].

    Returns K arrays [F][M_k (mu)][M_k][M_k] complex128."""
    x = np.asarray(x, dtype=np.complex128)
    T = x.shape[1]
    off = mic_offsets(mics)
    out = []
    for k, mk in enumerate(mics):
        xk = x[:, :, off[k]:off[k] + mk]                      # [F][T][M_k]
        outer = xk[:, :, :, None] * np.conj(xk[:, :, None, :])  # [F][T][a][b] = x_a x_b^*
        w = 1.0 / yhat[:, :, off[k]:off[k] + mk]               # [F][T][mu]
        V = np.einsum("ftu,ftab->fuab", w, outer) / T
        out.append(V)
    return out


def ge_solve(A: np.ndarray, b: np.ndarray):
    """Gaussian elimination with partial pivoting, batched over the leading axis.

    A: [S][n][n], b: [S][n].  Returns (x, min_abs_pivot, max_abs_entry)."""
    A = np.array(A, dtype=np.complex128)
    b = np.array(b, dtype=np.complex128)
    S, n, _ = A.shape
    rows = np.arange(S)
    scale = np.abs(A).reshape(S, -1).max(axis=1) if n else np.zeros(S)
    minpiv = np.full(S, np.inf)
    for c in range(n):
        p = c + np.argmax(np.abs(A[:, c:, c]), axis=1)
        Ac, Ap = A[rows, c, :].copy(), A[rows, p, :].copy()
        A[rows, c, :], A[rows, p, :] = Ap, Ac
        bc, bp = b[rows, c].copy(), b[rows, p].copy()
        b[rows, c], b[rows, p] = bp, bc
        piv = A[:, c, c]
        minpiv = np.minimum(minpiv, np.abs(piv))
        safe = np.where(piv == 0, 1.0, piv)
        for i in range(c + 1, n):
            m = A[:, i, c] / safe
            A[:, i, c:] -= m[:, None] * A[:, c, c:]
            b[:, i] -= m * b[:, c]
    xs = np.zeros((S, n), dtype=np.complex128)
    for i in range(n - 1, -1, -1):
        acc = b[:, i] - np.sum(A[:, i, i + 1:] * xs[:, i + 1:], axis=1)
        d = A[:, i, i]
        xs[:, i] = acc / np.where(d == 0, 1.0, d)
    return xs, minpiv, scale


def pinv_apply(A: np.ndarray, b: np.ndarray, rtol: float) -> np.ndarray:
    """q = pinv(A) b with the SVD pseudo-inverse; singular values <= rtol * s_max are dropped."""
    U, s, Vh = np.linalg.svd(A)
    keep = s > rtol * (s[0] if s.size else 0.0)
    sinv = np.where(keep, 1.0 / np.where(keep, s, 1.0), 0.0)
    return np.conj(Vh.T) @ (sinv * (np.conj(U.T) @ b))


def solve_or_pinv(A: np.ndarray, e: np.ndarray, rtol: float = SINGULAR_RTOL):
    """Batched q = A^{-1} e (partial pivoting), pinv where the pivot test says singular."""
    q, minpiv, scale = ge_solve(A, e)
    singular = ~(minpiv > rtol * scale)          # also true when scale == 0 or NaN
    for s_idx in np.nonzero(singular)[0]:
        q[s_idx] = pinv_apply(A[s_idx], e[s_idx], rtol)
    return q, singular


def ip_update_row(Qk: np.ndarray, Vk: np.ndarray, mu: int, eps: float = EPS,
                  rtol: float = SINGULAR_RTOL) -> np.ndarray:
    """Eqs. (14)-(15) for row mu of every block Q_fk (batched over f).

    q = (Q_fk V_fk,mu)^{-1} e_mu ; q <- q / sqrt(max(Re q^H V q, eps)) ; row mu <- q^H.
    Qk: [F][M_k][M_k], Vk: [F][M_k][M_k][M_k] (mu first).  Returns the new Qk."""
    F, mk, _ = Qk.shape
    Vmu = Vk[:, mu]
    A = np.matmul(Qk, Vmu)
    e = np.zeros((F, mk), dtype=np.complex128)
    e[:, mu] = 1.0
    q, _ = solve_or_pinv(A, e, rtol)
    s = np.real(np.einsum("fa,fab,fb->f", np.conj(q), Vmu, q))
    q = q / np.sqrt(np.maximum(s, eps))[:, None]
    Qn = Qk.copy()
    Qn[:, mu, :] = np.conj(q)
    return Qn


def ip_update(Q: List[np.ndarray], V: List[np.ndarray], eps: float = EPS,
              rtol: float = SINGULAR_RTOL) -> List[np.ndarray]:
    """Eqs. (13)-(15) applied independently to each subarray block, mu ascending."""
    out = []
    for Qk, Vk in zip(Q, V):
        Qn = Qk.copy()
        for mu in range(Qk.shape[1]):
            Qn = ip_update_row(Qn, Vk, mu, eps, rtol)
        out.append(Qn)
    return out


def projected_power(x: np.ndarray, Q: List[np.ndarray], mics: Sequence[int]) -> np.ndarray:
    """|y_ftm|^2 with y_ftk = Q_fk x_ftk (y^(l) = W^(l)H x^(l), Sec. III-B)."""
    x = np.asarray(x, dtype=np.complex128)
    F, T, M = x.shape
    off = mic_offsets(mics)
    P = np.empty((F, T, M))
    for k, mk in enumerate(mics):
        xk = x[:, :, off[k]:off[k] + mk]
        y = np.einsum("fuv,ftv->ftu", Q[k], xk)
        P[:, :, off[k]:off[k] + mk] = np.abs(y) ** 2
    return P


# ----------------------------------------------------------------------------
# multiplicative updates (Eqs. 8-10), with the factorised sums of Table I
# ----------------------------------------------------------------------------
def _mu_statistics(W, H, g, P, eps):
    """A[n,f,t] = sum_m g P yhat^-2 and D[n,f,t] = sum_m g yhat^-1 at the current model."""
    lam = source_psd(W, H)
    y = model_variance(lam, g, eps)
    A = np.einsum("fnm,ftm->nft", g, P / y ** 2)
    D = np.einsum("fnm,ftm->nft", g, 1.0 / y)
    return A, D


def update_W(W, H, g, P, eps: float = EPS):
    """Eq. (8): t_ikn <- t_ikn sqrt(sum_{j,m} v [Lambda]_mm |y|^2 eta^-2 / sum_{j,m} v [Lambda]_mm eta^-1)."""
    A, D = _mu_statistics(W, H, g, P, eps)
    num = np.matmul(A, np.transpose(H, (0, 2, 1)))          # [N][F][B] = sum_t A H
    den = np.matmul(D, np.transpose(H, (0, 2, 1)))
    return W * np.sqrt(num / np.maximum(den, eps))


def update_H(W, H, g, P, eps: float = EPS):
    """Eq. (9): v_kjn <- v_kjn sqrt(sum_{i,m} t [Lambda]_mm |y|^2 eta^-2 / sum_{i,m} t [Lambda]_mm eta^-1)."""
    A, D = _mu_statistics(W, H, g, P, eps)
    num = np.matmul(np.transpose(W, (0, 2, 1)), A)          # [N][B][T] = sum_f W A
    den = np.matmul(np.transpose(W, (0, 2, 1)), D)
    return H * np.sqrt(num / np.maximum(den, eps))


def update_g(W, H, g, P, eps: float = EPS):
    """Eq. (10): [Lambda_in]_mm <- [Lambda]_mm sqrt(sum_{j,k} t v |y|^2 eta^-2 / sum_{j,k} t v eta^-1)."""
    lam = source_psd(W, H)
    y = model_variance(lam, g, eps)
    num = np.einsum("nft,ftm->fnm", lam, P / y ** 2)
    den = np.einsum("nft,ftm->fnm", lam, 1.0 / y)
    return g * np.sqrt(num / np.maximum(den, eps))


# ----------------------------------------------------------------------------
# objective (Eq. 12) and Wiener filter
# ----------------------------------------------------------------------------
def log_abs_det_sq(Qk: np.ndarray) -> np.ndarray:
    """ln |det Q_fk|^2 for every f, from the pivots of Gaussian elimination."""
    A = np.array(Qk, dtype=np.complex128)
    F, n, _ = A.shape
    rows = np.arange(F)
    out = np.zeros(F)
    for c in range(n):
        p = c + np.argmax(np.abs(A[:, c:, c]), axis=1)
        Ac, Ap = A[rows, c, :].copy(), A[rows, p, :].copy()
        A[rows, c, :], A[rows, p, :] = Ap, Ac
        piv = A[:, c, c]
        with np.errstate(divide="ignore"):
            out += np.log(np.abs(piv) ** 2)
        safe = np.where(piv == 0, 1.0, piv)
        for i in range(c + 1, n):
            m = A[:, i, c] / safe
            A[:, i, c:] -= m[:, None] * A[:, c, c:]
    return out


def neg_loglik(x, mics, st: State, eps: float = EPS) -> float:
    """Eq. (12): sum_k [ sum_{f,t,mu} (|y|^2/eta + ln eta) - T sum_f ln|det Q_fk|^2 ]."""
    T = x.shape[1]
    P = projected_power(x, st.Q, mics)
    y = model_variance(source_psd(st.W, st.H), st.g, eps)
    data = float(np.sum(P / y + np.log(y)))
    logdet = float(sum(np.sum(log_abs_det_sq(Qk)) for Qk in st.Q))
    return data - T * logdet


def cost_gradient(x, mics, st: State, eps: float = EPS):
    """Gradient of Eq. (12) at the state st (the cost itself, no iteration).

    With y = sum_n lambda g (Eq. 2) and yhat = max(y, eps), the data term
    sum (P / yhat + ln yhat) has dL/dy = 1/y - P/y^2 =: G where y > eps and 0
    where the floor holds.  By the chain rule through lambda = W H:
      dL/dg[f,n,m]   = sum_t lambda[n,f,t] G[f,t,m]
      dL/dlam[n,f,t] = sum_m g[f,n,m] G[f,t,m]
      dL/dW[n,f,b]   = sum_t dL/dlam[n,f,t] H[n,b,t]
      dL/dH[n,b,t]   = sum_f W[n,f,b] dL/dlam[n,f,t]
    For a block Q_fk with z = Q_fk x_ftk (P = |z|^2) and the log-determinant
    term -T ln|det Q_fk|^2, the derivative with respect to the real and
    imaginary parts of each entry, packed as dL/dRe + i dL/dIm (twice the
    derivative with respect to the conjugate entry), is
      dQ[mu, j] = 2 sum_t z_mu conj(x_j) / yhat_mu - 2 T conj(Q^{-1})[j, mu].
    Returns (dQ list of K arrays [F][M_k][M_k] complex128, dW, dH, dg)."""
    x = np.asarray(x, dtype=np.complex128)
    F, T, M = x.shape
    lam = source_psd(st.W, st.H)
    F_, N, M_ = st.g.shape
    y = np.zeros((F, T, M))
    for n in range(N):
        y += lam[n][:, :, None] * st.g[:, n, None, :]
    P = projected_power(x, st.Q, mics)
    G = np.where(y > eps, 1.0 / np.where(y > eps, y, 1.0) - P / np.where(y > eps, y, 1.0) ** 2, 0.0)
    dg = np.einsum("nft,ftm->fnm", lam, G)
    dlam = np.einsum("fnm,ftm->nft", st.g, G)
    dW = np.einsum("nft,nbt->nfb", dlam, st.H)
    dH = np.einsum("nfb,nft->nbt", st.W, dlam)
    yhat = np.maximum(y, eps)
    off = mic_offsets(mics)
    dQ = []
    for k, mk in enumerate(mics):
        xk = x[:, :, off[k]:off[k] + mk]
        z = np.einsum("fuv,ftv->ftu", st.Q[k], xk)
        data = 2.0 * np.einsum("ftu,ftj->fuj", z / yhat[:, :, off[k]:off[k] + mk], np.conj(xk))
        inv = np.linalg.inv(st.Q[k])
        dQ.append(data - 2.0 * T * np.conj(np.swapaxes(inv, -1, -2)))
    return dQ, dW, dH, dg


def init_from_images(c, mics: Sequence[int]):
    """Sec. IV-A initialisation, steps 3, 5 and 6, from given source images.

    c: complex [N][F][T][M] initial images (the paper obtains them by soft
    masking; that step and the IS-NMF of step 4 are not part of this path).
      step 3: R_fn = sum_t c_nft c_nft^H / T (M x M);
              h[n, f, t] = c^H R_fn^{-1} c / M;
      step 5: for every block k, the generalised eigenvectors w of the pair
              (R_f,N-2^(k), R_f,N-1^(k)) -- the diagonal blocks of the last two
              sources' covariances -- which diagonalise both; ascending
              eigenvalues, each w scaled so that w^H R_f,N-1^(k) w = 1;
              Q_fk has rows w^H (it plays W_i^(init)(l)H);
      step 6: g[f, n, o_k + mu] = w_mu^H R_fn^(k) w_mu (ddiag of the
              diagonalised covariance).
    Needs N >= 2.  Returns (h [N][F][T] real, Q list of K [F][M_k][M_k], g [F][N][M])."""
    import scipy.linalg
    c = np.asarray(c, dtype=np.complex128)
    N, F, T, M = c.shape
    R = np.einsum("nftm,nftl->nfml", c, np.conj(c)) / T
    y = np.linalg.solve(R, np.swapaxes(c, 2, 3))                    # [N][F][M][T] = R^{-1} c
    h = np.real(np.einsum("nftm,nfmt->nft", np.conj(c), y)) / M
    off = mic_offsets(mics)
    Q, g = [], np.zeros((F, N, M))
    for k, mk in enumerate(mics):
        sl = slice(off[k], off[k] + mk)
        Qk = np.zeros((F, mk, mk), dtype=np.complex128)
        for f in range(F):
            Ra, Rb = R[N - 2, f][sl, sl], R[N - 1, f][sl, sl]
            lam, Wv = scipy.linalg.eigh(Ra, Rb)                    # ascending; Wv^H Rb Wv = I
            Qk[f] = np.conj(Wv.T)
            for n in range(N):
                g[f, n, sl] = np.real(np.einsum("am,ab,bm->m", np.conj(Wv), R[n, f][sl, sl], Wv))
        Q.append(Qk)
    return h, Q, g


def wiener_filter(x, mics, st: State, eps: float = EPS) -> np.ndarray:
    """Source images per subarray: c_n = Q_fk^{-1} diag(lambda_n g_n / yhat) Q_fk x_ftk.

    Returns complex128 [N][F][T][M]."""
    x = np.asarray(x, dtype=np.complex128)
    F, T, M = x.shape
    lam = source_psd(st.W, st.H)
    y = model_variance(lam, st.g, eps)
    off = mic_offsets(mics)
    N = st.W.shape[0]
    out = np.empty((N, F, T, M), dtype=np.complex128)
    for k, mk in enumerate(mics):
        sl = slice(off[k], off[k] + mk)
        Qk = st.Q[k]
        Qinv = np.linalg.inv(Qk)
        yk = np.einsum("fuv,ftv->ftu", Qk, x[:, :, sl])
        for n in range(N):
            gain = lam[n][:, :, None] * st.g[:, n, None, sl] / y[:, :, sl]
            out[n][:, :, sl] = np.einsum("fuv,ftv->ftu", Qinv, gain * yk)
    return out


# ----------------------------------------------------------------------------
# one iteration (Sec. III-B schedule)
# ----------------------------------------------------------------------------
def mm_iteration(x, mics, st: State, eps: float = EPS, rtol: float = SINGULAR_RTOL,
                 record: dict | None = None) -> State:
    """IP for all blocks (Eqs. 13-15), then W, H, g (Eqs. 8, 9, 10)."""
    lam = source_psd(st.W, st.H)
    y = model_variance(lam, st.g, eps)
    V = weighted_covariances(x, y, mics)
    Q = ip_update(st.Q, V, eps, rtol)
    P = projected_power(x, Q, mics)
    W = update_W(st.W, st.H, st.g, P, eps)
    H = update_H(W, st.H, st.g, P, eps)
    g = update_g(W, H, st.g, P, eps)
    if record is not None:
        record.update(V=V, Q=Q, P=P, W=W, H=H, g=g, lam=source_psd(W, H))
    return State(Q, W, H, g)


def run(x, mics, st: State, n_iter: int, eps: float = EPS) -> State:
    for _ in range(n_iter):
        st = mm_iteration(x, mics, st, eps)
    return st
