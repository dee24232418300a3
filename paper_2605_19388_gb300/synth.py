"""Seeded synthetic STFT mixtures for distributed FastMNMF.

This module only draws random inputs: it holds no step of the estimation
method.  Both the CUDA path and the FP64 oracle start from the arrays returned
here, so the two begin from bit-identical state.

Data model (Sec. II-A, Eq. 1 with rank-1 spatial images; Sec. III-B block
structure): each source n has a non-negative PSD lambda_true = W_true H_true
(Eq. 2 shape) with Gamma(0.5, 1) factors, a complex Gaussian STFT signal
s_nft ~ CN(0, lambda_true_nft) and a steering vector that, inside subarray k,
is a unit-modulus random phase per microphone times a per-(source, subarray)
gain gamma_nk ~ U[0.2, 1] and a per-(source, frequency, subarray) phase.  The
mixture is x_ftm = sum_n a_nfm s_nft + CN(0, noise_std^2) white noise.  The
microphones of one subarray are contiguous in m (Sec. III-B).

Initial parameters follow the "initialised with positive values /
transformation matrices nonsingular" requirement of Sec. IV-A: Q = I (per
block), and W0, H0, g0 ~ U[0.1, 1] drawn from a second generator seeded with
seed + 1.

Layouts (all C-contiguous):
  x   complex64 [F][T][M]
  W0  float32   [N][F][B]     (paper t_ikn)
  H0  float32   [N][B][T]     (paper v_kjn)
  g0  float32   [F][N][M]     (paper [Lambda_in]_mm)
  Q0  complex128 [F][sum_k M_k^2], block k row-major M_k x M_k (paper W_i^H)
  c   complex64 [N][F][T][M]  ground-truth source images (optional)
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

# The workloads named by the benchmark: (F, T, mics, N, B, iterations).
WORKLOADS = {
    # K=2 subarrays x 4 mics, N=3, 8 bases, FFT 512 at 16 kHz, 313 frames.
    "small_2x4_n3": dict(F=257, T=313, mics=(4, 4), N=3, B=8, iters=50),
    # K=4 subarrays x 4 mics, N=5, 16 bases, FFT 1024, 10 s at hop 256.
    "paper_4x4_n5": dict(F=513, T=626, mics=(4, 4, 4, 4), N=5, B=16, iters=200),
    # Differentiation-sized case: 4 x 4 mics, N=5, F=257, T=313.
    "grad_4x4_n5": dict(F=257, T=313, mics=(4, 4, 4, 4), N=5, B=16, iters=20),
}


@dataclass
class Problem:
    F: int
    T: int
    mics: tuple
    N: int
    B: int
    x: np.ndarray                 # complex64 [F][T][M]
    W0: np.ndarray                # float32 [N][F][B]
    H0: np.ndarray                # float32 [N][B][T]
    g0: np.ndarray                # float32 [F][N][M]
    Q0: np.ndarray                # complex128 [F][sum M_k^2]
    c: Optional[np.ndarray] = field(default=None, repr=False)  # complex64 [N][F][T][M]
    seed: int = 0

    @property
    def K(self) -> int:
        return len(self.mics)

    @property
    def M(self) -> int:
        return int(sum(self.mics))


def identity_blocks(F: int, mics: Sequence[int]) -> np.ndarray:
    """Packed block-diagonal identity, complex128 [F][sum M_k^2]."""
    parts = [np.broadcast_to(np.eye(mk, dtype=np.complex128).reshape(1, mk * mk),
                             (F, mk * mk)) for mk in mics]
    return np.ascontiguousarray(np.concatenate(parts, axis=1))


def make_problem(F: int, T: int, mics: Sequence[int], N: int, B: int, seed: int = 0,
                 noise_std: float = 1e-3, with_images: bool = False,
                 init_low: float = 0.1, init_high: float = 1.0) -> Problem:
    """Draw one seeded mixture and its initial parameters."""
    mics = tuple(int(m) for m in mics)
    K = len(mics)
    M = sum(mics)
    rng = np.random.default_rng(seed)
    W_true = rng.gamma(0.5, 1.0, size=(N, F, B))
    H_true = rng.gamma(0.5, 1.0, size=(N, B, T))
    psd = np.matmul(W_true, H_true)                       # [N][F][T]
    s = np.sqrt(psd / 2.0) * (rng.standard_normal((N, F, T))
                              + 1j * rng.standard_normal((N, F, T)))
    gain = rng.uniform(0.2, 1.0, size=(N, K))
    psi = rng.uniform(0.0, 2 * np.pi, size=(N, F, K))
    phi = rng.uniform(0.0, 2 * np.pi, size=(N, F, M))
    sub = np.repeat(np.arange(K), mics)                   # subarray of each mic
    a = gain[:, None, sub] * np.exp(1j * psi[:, :, sub]) * np.exp(1j * phi)  # [N][F][M]
    noise = noise_std / np.sqrt(2.0) * (rng.standard_normal((F, T, M))
                                        + 1j * rng.standard_normal((F, T, M)))
    x = noise.astype(np.complex128)
    c = None
    if with_images:
        c = np.empty((N, F, T, M), dtype=np.complex64)
    for n in range(N):
        img = a[n][:, None, :] * s[n][:, :, None]         # [F][T][M]
        x += img
        if with_images:
            c[n] = img
    x = np.ascontiguousarray(x.astype(np.complex64))

    rng0 = np.random.default_rng(seed + 1)
    W0 = rng0.uniform(init_low, init_high, size=(N, F, B)).astype(np.float32)
    H0 = rng0.uniform(init_low, init_high, size=(N, B, T)).astype(np.float32)
    g0 = rng0.uniform(init_low, init_high, size=(F, N, M)).astype(np.float32)
    Q0 = identity_blocks(F, mics)
    return Problem(F=F, T=T, mics=mics, N=N, B=B, x=x, W0=W0, H0=H0, g0=g0, Q0=Q0,
                   c=c, seed=seed)


def make_workload(name: str, seed: int = 0, with_images: bool = False) -> Problem:
    w = WORKLOADS[name]
    return make_problem(w["F"], w["T"], w["mics"], w["N"], w["B"], seed=seed,
                        with_images=with_images)


def random_blocks(F: int, mics: Sequence[int], seed: int, scale: float = 0.3) -> np.ndarray:
    """Packed, well-conditioned random diagonalisers I + scale * Z (complex128)."""
    rng = np.random.default_rng(seed)
    parts = []
    for mk in mics:
        z = rng.standard_normal((F, mk, mk)) + 1j * rng.standard_normal((F, mk, mk))
        parts.append((np.eye(mk)[None] + scale * z).reshape(F, mk * mk))
    return np.ascontiguousarray(np.concatenate(parts, axis=1))
