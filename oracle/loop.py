"""ctypes binding of the plain-C loop oracle (``oracle/c/dfmnmf_loop.c``).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  The C file is a
second, independent FP64 restatement of the paper's updates in plain loops;
the tests hold it and the NumPy oracle against each other.  The shared
library is compiled with gcc into ``oracle/c/_build/`` on first use (or
by ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Sequence

import numpy as np

from .dfmnmf_oracle import EPS, SINGULAR_RTOL, State, pack_Q, unpack_Q

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c", "dfmnmf_loop.c")
LIB = os.path.join(HERE, "c", "_build", "libdfmnmf_loop.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, strict IEEE double: no fast-math, no contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_loop_neg_loglik.restype = ctypes.c_double
        _lib.oracle_loop_iterate.restype = ctypes.c_int
        _lib.oracle_loop_ip_update.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _mics(mics):
    m = np.ascontiguousarray(np.asarray(mics, dtype=np.int32))
    return m, _p(m)


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _v_pack_to_list(Vp, mics, F):
    out, o = [], 0
    for mk in mics:
        out.append(Vp[:, o:o + mk ** 3].reshape(F, mk, mk, mk).copy())
        o += mk ** 3
    return out


def covariances(x, W, H, g, mics: Sequence[int], eps: float = EPS):
    """Eq. (13) at the model of (W, H, g): K arrays [F][mu][a][b]."""
    x = _c128(x)
    F, T, M = x.shape
    N, _, B = W.shape
    m, mp = _mics(mics)
    V = np.zeros((F, int(sum(mk ** 3 for mk in mics))), dtype=np.complex128)
    _load().oracle_loop_covariances(F, T, len(mics), mp, N, B, _p(x), _p(_f64(W)), _p(_f64(H)), _p(_f64(g)),
                                    ctypes.c_double(eps), _p(V))
    return _v_pack_to_list(V, mics, F)


def ip_update(Q, V, mics: Sequence[int], T: int, eps: float = EPS, rtol: float = SINGULAR_RTOL):
    """Eqs. (14)-(15) on every block; returns (Q list, number of pseudo-inverse solves)."""
    Qp = _c128(pack_Q(Q))
    F = Qp.shape[0]
    Vp = _c128(np.concatenate([np.asarray(v).reshape(F, -1) for v in V], axis=1))
    m, mp = _mics(mics)
    ns = _load().oracle_loop_ip_update(F, T, len(mics), mp, _p(Vp), _p(Qp), ctypes.c_double(eps),
                                       ctypes.c_double(rtol))
    return unpack_Q(Qp, mics), ns


def projected_power(x, Q, mics: Sequence[int]):
    x = _c128(x)
    F, T, M = x.shape
    Qp = _c128(pack_Q(Q))
    P = np.zeros((F, T, M))
    m, mp = _mics(mics)
    _load().oracle_loop_projected_power(F, T, len(mics), mp, _p(x), _p(Qp), _p(P))
    return P


def _nmf(fn, W, H, g, P, mics, eps, which):
    W, H, g, P = _f64(W).copy(), _f64(H).copy(), _f64(g).copy(), _f64(P)
    N, F, B = W.shape
    T = H.shape[2]
    m, mp = _mics(mics)
    fn(F, T, len(mics), mp, N, B, _p(W), _p(H), _p(g), _p(P), ctypes.c_double(eps))
    return {"W": W, "H": H, "g": g}[which]


def update_W(W, H, g, P, mics, eps: float = EPS):
    return _nmf(_load().oracle_loop_update_W, W, H, g, P, mics, eps, "W")


def update_H(W, H, g, P, mics, eps: float = EPS):
    return _nmf(_load().oracle_loop_update_H, W, H, g, P, mics, eps, "H")


def update_g(W, H, g, P, mics, eps: float = EPS):
    return _nmf(_load().oracle_loop_update_g, W, H, g, P, mics, eps, "g")


def iterate(x, mics: Sequence[int], st: State, n_iter: int, eps: float = EPS, rtol: float = SINGULAR_RTOL):
    """n_iter MM iterations; returns (State, number of pseudo-inverse solves)."""
    x = _c128(x)
    F, T, M = x.shape
    Qp = _c128(pack_Q(st.Q))
    W, H, g = _f64(st.W).copy(), _f64(st.H).copy(), _f64(st.g).copy()
    N, _, B = W.shape
    m, mp = _mics(mics)
    ns = _load().oracle_loop_iterate(F, T, len(mics), mp, N, B, _p(x), _p(Qp), _p(W), _p(H), _p(g), int(n_iter),
                                     ctypes.c_double(eps), ctypes.c_double(rtol))
    return State(unpack_Q(Qp, mics), W, H, g), ns


def neg_loglik(x, mics: Sequence[int], st: State, eps: float = EPS) -> float:
    x = _c128(x)
    F, T, M = x.shape
    N, _, B = st.W.shape
    m, mp = _mics(mics)
    return float(_load().oracle_loop_neg_loglik(F, T, len(mics), mp, N, B, _p(x), _p(_c128(pack_Q(st.Q))),
                                                _p(_f64(st.W)), _p(_f64(st.H)), _p(_f64(st.g)),
                                                ctypes.c_double(eps)))


def wiener_filter(x, mics: Sequence[int], st: State, eps: float = EPS):
    x = _c128(x)
    F, T, M = x.shape
    N, _, B = st.W.shape
    out = np.zeros((N, F, T, M), dtype=np.complex128)
    m, mp = _mics(mics)
    _load().oracle_loop_wiener(F, T, len(mics), mp, N, B, _p(x), _p(_c128(pack_Q(st.Q))), _p(_f64(st.W)),
                               _p(_f64(st.H)), _p(_f64(st.g)), ctypes.c_double(eps), _p(out))
    return out
