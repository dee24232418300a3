"""Shared helpers of the test-suite (comparison metrics, SDR, oracle glue)."""
import itertools

import numpy as np

import oracle as O


def rel_err(a, b):
    """Normwise relative error ||a - b||_F / ||b||_F (b is the reference)."""
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


def v_oracle_layout(V_list):
    """Oracle V (K x [F][Mk][Mk][Mk]) -> GPU layout [F][K][Mk][Mk][Mk]."""
    return np.stack(V_list, axis=1)


def sdr_db(est, ref, mic=0):
    """STFT-domain SDR per source at one microphone, best permutation.

    est, ref: [N][F][T][M] complex.  SDR_n = 10 log10(sum|c|^2 / sum|c_hat - c|^2)
    over (f, t); the permutation maximising the mean SDR is chosen by brute force."""
    N = ref.shape[0]
    e = est[..., mic].reshape(N, -1)
    r = ref[..., mic].reshape(N, -1)
    S = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            S[i, j] = 10 * np.log10(np.sum(np.abs(r[i]) ** 2) / np.sum(np.abs(e[j] - r[i]) ** 2))
    best, bp = -np.inf, None
    for p in itertools.permutations(range(N)):
        v = np.mean([S[i, p[i]] for i in range(N)])
        if v > best:
            best, bp = v, p
    return np.array([S[i, bp[i]] for i in range(N)]), bp


def oracle_state(prob):
    return O.state_from_arrays(prob.Q0, prob.W0, prob.H0, prob.g0, prob.mics)


# ----------------------------------------------------------- element-wise checks
# A normwise error can hide a wrong bin, a wrong partial tile or a wrong small
# entry under large ones, so every parity check also bounds each element:
#     |a_i - b_i| <= tol * max(|b_i|, s_i),
# with a stated scale floor s_i per array (the reference b decides it):
#   V  (Eq. 13, [F][K][mu][Mk][Mk])  the largest |entry| of the same M_k x M_k block;
#   Q  ([F][K][Mk][Mk] or per block)  the largest |entry| of the same row q_mu^H;
#   P, W, H, g, lambda, the Wiener output  the median |entry| of the whole array.
# Entries far below these scales carry the rounding of the sums they come from
# (cancellation in off-diagonal covariances and in projections), so they are
# held to the scale's absolute accuracy, not to their own relative one.
def elem_err(a, b, floor):
    """max_i |a_i - b_i| / max(|b_i|, floor_i) (floor broadcastable to b)."""
    a = np.asarray(a)
    b = np.asarray(b)
    cplx = np.iscomplexobj(a) or np.iscomplexobj(b)
    d = np.abs(a.astype(np.complex128 if cplx else np.float64) - b)
    den = np.maximum(np.abs(b), floor)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(d / den)) if d.size else 0.0


def floor_median(b):
    return float(np.median(np.abs(np.asarray(b))))


def floor_last_axes(b, naxes):
    """Largest |entry| over the last `naxes` axes (kept for broadcasting)."""
    b = np.abs(np.asarray(b))
    return np.max(b, axis=tuple(range(b.ndim - naxes, b.ndim)), keepdims=True)


def elem_err_V(a, b):
    return elem_err(a, b, floor_last_axes(b, 2))


def elem_err_Q(a, b):
    """Q as [..., Mk, Mk] blocks (rows on the second-to-last axis) or a list of such per subarray."""
    if isinstance(b, (list, tuple)):
        return max(elem_err(x, y, floor_last_axes(y, 1)) for x, y in zip(a, b))
    return elem_err(a, b, floor_last_axes(b, 1))


def elem_err_med(a, b):
    return elem_err(a, b, floor_median(b))


def check_both(errs, name, a, b, kind, tol=None):
    """Record the normwise and the element-wise error of one output under `name` and `name`_elem."""
    fn = {"V": elem_err_V, "Q": elem_err_Q, "med": elem_err_med}[kind]
    if isinstance(b, (list, tuple)):
        errs[name] = max(rel_err(x, y) for x, y in zip(a, b))
    else:
        errs[name] = rel_err(a, b)
    errs[name + "_elem"] = fn(a, b)
    return errs
