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
