"""The two FP64 oracles against each other (CPU only).

``oracle/dfmnmf_oracle.py`` (NumPy: einsum, matmul, batched elimination) and
``oracle/c/dfmnmf_loop.c`` (plain C loops, one element at a time) restate the
same equations independently; they differ only in the order of their sums.
Every update, the cost of Eq. (12), the Wiener filter and whole trajectories
must agree to within that rounding, so a slip in either one (a dropped term,
a swapped index, a conjugate on the wrong factor) shows up here even where
the invariant pins of ``test_oracle_pins.py`` would let it through.
"""
import numpy as np
import pytest

import oracle as O
from oracle import loop as L
from paper_2605_19388_gb300 import synth
from tests._helpers import rel_err


def random_state(rng, F, T, mics, N, B):
    """A generic state: Q_fk = I + a complex perturbation, W, H, g ~ U[0.1, 1]."""
    Q = [np.eye(mk)[None] + 0.3 * (rng.standard_normal((F, mk, mk)) + 1j * rng.standard_normal((F, mk, mk)))
         for mk in mics]
    W = rng.uniform(0.1, 1.0, (N, F, B))
    H = rng.uniform(0.1, 1.0, (N, B, T))
    g = rng.uniform(0.1, 1.0, (F, N, sum(mics)))
    return O.State(Q, W, H, g)


def random_x(rng, F, T, M):
    return rng.standard_normal((F, T, M)) + 1j * rng.standard_normal((F, T, M))


LAYOUTS = [((2, 3, 1), 3, 4), ((4, 4), 5, 6), ((4,), 2, 3), ((1, 1), 2, 2)]


@pytest.mark.parametrize("mics,N,B", LAYOUTS)
def test_every_update_agrees(mics, N, B):
    rng = np.random.default_rng(7)
    F, T = 5, 23
    x = random_x(rng, F, T, sum(mics))
    st = random_state(rng, F, T, mics, N, B)
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    V_np = O.weighted_covariances(x, y, mics)
    V_c = L.covariances(x, st.W, st.H, st.g, mics)
    for a, b in zip(V_c, V_np):
        assert rel_err(a, b) < 1e-13
    Q_np = O.ip_update(st.Q, V_np)
    Q_c, ns = L.ip_update(st.Q, V_np, mics, T)
    assert ns == 0
    for a, b in zip(Q_c, Q_np):
        assert rel_err(a, b) < 1e-11
    P_np = O.projected_power(x, Q_np, mics)
    assert rel_err(L.projected_power(x, Q_np, mics), P_np) < 1e-13
    W_np = O.update_W(st.W, st.H, st.g, P_np)
    assert rel_err(L.update_W(st.W, st.H, st.g, P_np, mics), W_np) < 1e-13
    H_np = O.update_H(W_np, st.H, st.g, P_np)
    assert rel_err(L.update_H(W_np, st.H, st.g, P_np, mics), H_np) < 1e-13
    g_np = O.update_g(W_np, H_np, st.g, P_np)
    assert rel_err(L.update_g(W_np, H_np, st.g, P_np, mics), g_np) < 1e-13
    st2 = O.State(Q_np, W_np, H_np, g_np)
    nll_np, nll_c = O.neg_loglik(x, mics, st2), L.neg_loglik(x, mics, st2)
    assert abs(nll_c - nll_np) <= 1e-12 * abs(nll_np)
    assert rel_err(L.wiener_filter(x, mics, st2), O.wiener_filter(x, mics, st2)) < 1e-12


@pytest.mark.parametrize("shape,tol", [
    (dict(F=17, T=60, mics=(4, 4, 4, 4), N=5, B=8), 1e-11),  # paper-shaped (N > M_k per subarray)
    (dict(F=13, T=50, mics=(4, 4), N=3, B=8), 1e-7),         # determined per subarray, 60 dB noise floor
])
def test_trajectories_agree(shape, tol):
    """20 MM iterations from the same seeded start: states, Eq. (12) and the Wiener output."""
    p = synth.make_problem(shape["F"], shape["T"], shape["mics"], shape["N"], shape["B"], seed=3)
    x = p.x.astype(np.complex128)
    st0 = O.state_from_arrays(p.Q0, p.W0, p.H0, p.g0, p.mics)
    st_np = O.run(x, p.mics, st0, 20)
    st_c, ns = L.iterate(x, p.mics, st0, 20)
    assert ns == 0
    errs = {"W": rel_err(st_c.W, st_np.W), "H": rel_err(st_c.H, st_np.H), "g": rel_err(st_c.g, st_np.g),
            "Q": max(rel_err(a, b) for a, b in zip(st_c.Q, st_np.Q))}
    assert max(errs.values()) < tol, errs
    nll_np, nll_c = O.neg_loglik(x, p.mics, st_np), L.neg_loglik(x, p.mics, st_c)
    assert abs(nll_c - nll_np) <= tol * abs(nll_np)
    assert rel_err(L.wiener_filter(x, p.mics, st_c), O.wiener_filter(x, p.mics, st_np)) < 10 * tol


def test_cost_never_increases_in_the_loop_oracle():
    """The MM guarantee holds for the loop oracle on its own (Eq. 12 after every iteration)."""
    p = synth.make_problem(9, 40, (4, 4), 5, 6, seed=4)
    x = p.x.astype(np.complex128)
    st = O.state_from_arrays(p.Q0, p.W0, p.H0, p.g0, p.mics)
    prev = L.neg_loglik(x, p.mics, st)
    for _ in range(8):
        st, _ = L.iterate(x, p.mics, st, 1)
        cur = L.neg_loglik(x, p.mics, st)
        assert cur <= prev + 1e-9 * abs(prev)
        prev = cur


def test_singular_systems_take_the_same_pseudo_inverse():
    """A silent microphone makes V_fk,mu singular: both oracles switch to pinv(Q V_mu) e_mu (Sec. IV-A)."""
    rng = np.random.default_rng(11)
    F, T, mics, N, B = 4, 30, (3, 2), 2, 3
    x = random_x(rng, F, T, sum(mics))
    x[1:3, :, 1] = 0.0  # microphone 1 silent in bins 1 and 2
    st = random_state(rng, F, T, mics, N, B)
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    V = O.weighted_covariances(x, y, mics)
    Q_np = O.ip_update(st.Q, V)
    Q_c, ns = L.ip_update(st.Q, V, mics, T)
    assert ns > 0
    for a, b in zip(Q_c, Q_np):
        assert rel_err(a, b) < 1e-10
