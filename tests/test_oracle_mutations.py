"""Planted mistakes in the oracle, each caught by at least one independent pin.

Every mutation below is a plausible one-line slip in a step of the method: a
dropped factor, a wrong sign, a missing power or square root, a transposed or
conjugated operand, an inverse left out.  The test plants it by replacing one
oracle function (in the package namespace the pins call and in the module
namespace the oracle's own functions call), runs the independent pins -- every
test of ``test_oracle_pins.py`` and the closed-form test of
``test_oracle_golden.py`` -- and requires at least one of them to fail.  The
stored-trajectory regression is left out: the oracle wrote it itself.
"""
import contextlib
import inspect

import numpy as np
import pytest

import oracle
import oracle.dfmnmf_oracle as OM
from tests import test_oracle_golden as golden
from tests import test_oracle_pins as pins

ORIG = {name: getattr(OM, name) for name in (
    "weighted_covariances", "model_variance", "ip_update_row", "projected_power", "_mu_statistics",
    "update_W", "update_H", "update_g", "neg_loglik", "wiener_filter", "log_abs_det_sq", "source_psd",
    "init_from_images", "ip_update")}


def _ip_row(Qk, Vk, mu, eps=OM.EPS, rtol=OM.SINGULAR_RTOL, *, normalise=True, conj_row=True, order="QV",
            v_shift=0, root=True):
    """Eqs. (14)-(15) for row mu, with switches that plant the slips below."""
    F, mk, _ = Qk.shape
    Vmu = Vk[:, (mu + v_shift) % mk]
    A = np.matmul(Qk, Vmu) if order == "QV" else np.matmul(Vmu, Qk)
    e = np.zeros((F, mk), dtype=np.complex128)
    e[:, mu] = 1.0
    q, _ = OM.solve_or_pinv(A, e, rtol)
    if normalise:
        s = np.real(np.einsum("fa,fab,fb->f", np.conj(q), Vmu, q))
        nrm = np.maximum(s, eps)
        q = q / (np.sqrt(nrm) if root else nrm)[:, None]
    Qn = Qk.copy()
    Qn[:, mu, :] = np.conj(q) if conj_row else q
    return Qn


def _ip_sweep_from_old_block(Q, V, eps=OM.EPS, rtol=OM.SINGULAR_RTOL):
    """Every row of a block solved from the block as it was before the sweep (all rows at once),
    where Eqs. (14)-(15) update the rows one after another, each from the block with the rows
    before it already replaced."""
    out = []
    for Qk, Vk in zip(Q, V):
        Qn = Qk.copy()
        for mu in range(Qk.shape[1]):
            Qn[:, mu, :] = OM.ip_update_row(Qk, Vk, mu, eps, rtol)[:, mu, :]  # slip: Qk where Qn belongs
        out.append(Qn)
    return out


def _mu_statistics_power1(W, H, g, P, eps):
    lam = OM.source_psd(W, H)
    y = OM.model_variance(lam, g, eps)
    A = np.einsum("fnm,ftm->nft", g, P / y)  # slip: yhat^-1 where Eqs. (8)-(9) have yhat^-2
    D = np.einsum("fnm,ftm->nft", g, 1.0 / y)
    return A, D


def _neg_loglik_variant(x, mics, st, eps=OM.EPS, *, det_sign=-1.0, with_log=True, det_scale="T"):
    """Eq. (12) with switches that plant the slips below."""
    T = x.shape[1]
    P = OM.projected_power(x, st.Q, mics)
    y = OM.model_variance(OM.source_psd(st.W, st.H), st.g, eps)
    data = float(np.sum(P / y + (np.log(y) if with_log else 0.0)))
    logdet = float(sum(np.sum(OM.log_abs_det_sq(Qk)) for Qk in st.Q))
    return data + det_sign * (T if det_scale == "T" else 1) * logdet


def _neg_loglik_flipped(x, mics, st, eps=OM.EPS):
    return _neg_loglik_variant(x, mics, st, eps, det_sign=+1.0)  # slip: the sign of the log-determinant term


def _wiener_without_inverse(x, mics, st, eps=OM.EPS):
    x = np.asarray(x, dtype=np.complex128)
    F, T, M = x.shape
    lam = OM.source_psd(st.W, st.H)
    y = OM.model_variance(lam, st.g, eps)
    off = OM.mic_offsets(mics)
    N = st.W.shape[0]
    out = np.empty((N, F, T, M), dtype=np.complex128)
    for k, mk in enumerate(mics):
        sl = slice(off[k], off[k] + mk)
        Qk = st.Q[k]
        yk = np.einsum("fuv,ftv->ftu", Qk, x[:, :, sl])
        for n in range(N):
            gain = lam[n][:, :, None] * st.g[:, n, None, sl] / y[:, :, sl]
            out[n][:, :, sl] = np.einsum("fuv,ftv->ftu", Qk, gain * yk)  # slip: Q where Q^-1 belongs
    return out


MUTATIONS = {
    "covariance without the 1/T of Eq. (13)":
        ("weighted_covariances", lambda x, y, mics: [V * x.shape[1] for V in ORIG["weighted_covariances"](x, y, mics)]),
    "covariance with the conjugate on the other factor":
        ("weighted_covariances", lambda x, y, mics: [np.conj(V) for V in ORIG["weighted_covariances"](x, y, mics)]),
    "model variance with the microphones of g reversed":
        ("model_variance", lambda lam, g, eps=OM.EPS: ORIG["model_variance"](lam, g[:, :, ::-1], eps)),
    "IP row without the normalisation of Eq. (15)":
        ("ip_update_row", lambda Qk, Vk, mu, eps=OM.EPS, rtol=OM.SINGULAR_RTOL:
            _ip_row(Qk, Vk, mu, eps, rtol, normalise=False)),
    "IP row stored without the conjugate":
        ("ip_update_row", lambda Qk, Vk, mu, eps=OM.EPS, rtol=OM.SINGULAR_RTOL:
            _ip_row(Qk, Vk, mu, eps, rtol, conj_row=False)),
    "IP system V Q instead of Q V":
        ("ip_update_row", lambda Qk, Vk, mu, eps=OM.EPS, rtol=OM.SINGULAR_RTOL:
            _ip_row(Qk, Vk, mu, eps, rtol, order="VQ")),
    "IP row normalised by q^H V q instead of its square root":
        ("ip_update_row", lambda Qk, Vk, mu, eps=OM.EPS, rtol=OM.SINGULAR_RTOL:
            _ip_row(Qk, Vk, mu, eps, rtol, root=False)),
    "IP row solved with the next microphone's covariance":
        ("ip_update_row", lambda Qk, Vk, mu, eps=OM.EPS, rtol=OM.SINGULAR_RTOL:
            _ip_row(Qk, Vk, mu, eps, rtol, v_shift=1)),
    "covariance weighted by yhat^-2 instead of yhat^-1":
        ("weighted_covariances", lambda x, y, mics: ORIG["weighted_covariances"](x, y ** 2, mics)),
    "source model pairing the bases of W and H in reverse":
        ("source_psd", lambda W, H: ORIG["source_psd"](W, H[:, ::-1, :])),
    "IP sweep solving every row from the block before the sweep":
        ("ip_update", _ip_sweep_from_old_block),
    "projected power with Q^H instead of Q":
        ("projected_power", lambda x, Q, mics: ORIG["projected_power"](
            x, [np.conj(np.swapaxes(q, 1, 2)) for q in Q], mics)),
    "projected power |q^H x| without the square":
        ("projected_power", lambda x, Q, mics: np.sqrt(ORIG["projected_power"](x, Q, mics))),
    "MU statistic with yhat^-1 instead of yhat^-2":
        ("_mu_statistics", _mu_statistics_power1),
    "W update with numerator and denominator exchanged":
        ("update_W", lambda W, H, g, P, eps=OM.EPS: W ** 2 / ORIG["update_W"](W, H, g, P, eps)),
    "H update with numerator and denominator exchanged":
        ("update_H", lambda W, H, g, P, eps=OM.EPS: H ** 2 / ORIG["update_H"](W, H, g, P, eps)),
    "log-determinant of Q without its square":
        ("log_abs_det_sq", lambda Qk: 0.5 * ORIG["log_abs_det_sq"](Qk)),
    "g update without the square root":
        ("update_g", lambda W, H, g, P, eps=OM.EPS: ORIG["update_g"](W, H, g, P, eps) ** 2 / g),
    "cost with the sign of the log-determinant flipped":
        ("neg_loglik", _neg_loglik_flipped),
    "cost without the ln yhat term":
        ("neg_loglik", lambda x, mics, st, eps=OM.EPS: _neg_loglik_variant(x, mics, st, eps, with_log=False)),
    "cost with the log-determinant not multiplied by T":
        ("neg_loglik", lambda x, mics, st, eps=OM.EPS: _neg_loglik_variant(x, mics, st, eps, det_scale="1")),
    "Wiener filter without Q^-1":
        ("wiener_filter", _wiener_without_inverse),
}


def _init_variant(c, mics, *, per_mic=True, conj_rows=True, swap_pair=False, g_of_last=False):
    """Steps 3, 5 and 6 of the initialisation (Sec. IV-A) with switches that plant the slips below."""
    import scipy.linalg
    c = np.asarray(c, dtype=np.complex128)
    N, F, T, M = c.shape
    R = np.einsum("nftm,nftl->nfml", c, np.conj(c)) / T
    y = np.linalg.solve(R, np.swapaxes(c, 2, 3))
    h = np.real(np.einsum("nftm,nfmt->nft", np.conj(c), y)) / (M if per_mic else 1)
    off = OM.mic_offsets(mics)
    Q, g = [], np.zeros((F, N, M))
    for k, mk in enumerate(mics):
        sl = slice(off[k], off[k] + mk)
        Qk = np.zeros((F, mk, mk), dtype=np.complex128)
        for f in range(F):
            a, b = (N - 1, N - 2) if swap_pair else (N - 2, N - 1)
            _, Wv = scipy.linalg.eigh(R[a, f][sl, sl], R[b, f][sl, sl])
            Qk[f] = np.conj(Wv.T) if conj_rows else Wv.T
            for n in range(N):
                Rn = R[N - 1 if g_of_last else n, f][sl, sl]
                g[f, n, sl] = np.real(np.einsum("am,ab,bm->m", np.conj(Wv), Rn, Wv))
        Q.append(Qk)
    return h, Q, g


# Slips in the initialisation, which the loop oracle does not restate: the pins alone must catch them.
INIT_MUTATIONS = {
    "initial spectrogram without the 1/M of step 3":
        ("init_from_images", lambda c, mics: _init_variant(c, mics, per_mic=False)),
    "initial Q with rows w^T instead of w^H":
        ("init_from_images", lambda c, mics: _init_variant(c, mics, conj_rows=False)),
    "initial Q from the pair of the last two sources taken in reverse":
        ("init_from_images", lambda c, mics: _init_variant(c, mics, swap_pair=True)),
    "initial g of every source from the last source's covariance":
        ("init_from_images", lambda c, mics: _init_variant(c, mics, g_of_last=True)),
}


def _pins():
    fs = [f for name, f in inspect.getmembers(pins, inspect.isfunction) if name.startswith("test_")]
    fs.append(golden.test_cost_closed_form_identity_and_constant_model)
    return fs


@contextlib.contextmanager
def _planted(name, fn):
    had_pkg = hasattr(oracle, name)
    try:
        setattr(OM, name, fn)
        if had_pkg:
            setattr(oracle, name, fn)
        yield
    finally:
        setattr(OM, name, ORIG[name])
        if had_pkg:
            setattr(oracle, name, ORIG[name])


def test_unmutated_oracle_passes_every_pin():
    for f in _pins():
        with np.errstate(all="ignore"):
            f()


def test_unmutated_initialisation_variant_is_the_oracle():
    """The switch-free variant reproduces the oracle's initialisation, so each slip below is one change."""
    from tests.test_oracle_pins import _images
    p, c = _images()
    ref, got = OM.init_from_images(c, p.mics), _init_variant(c, p.mics)
    np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
    for a, b in zip(got[1], ref[1]):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(got[2], ref[2], rtol=1e-12)


@pytest.mark.parametrize("slip", list(INIT_MUTATIONS))
def test_planted_initialisation_mistake_is_caught(slip):
    name, fn = INIT_MUTATIONS[slip]
    caught = []
    with _planted(name, fn), np.errstate(all="ignore"):
        for f in _pins():
            try:
                f()
            except AssertionError:
                caught.append(f.__name__)
    assert caught, f"no pin fails with the planted mistake: {slip}"


@pytest.mark.parametrize("slip", list(MUTATIONS))
def test_planted_mistake_is_caught(slip):
    name, fn = MUTATIONS[slip]
    caught = []
    with _planted(name, fn), np.errstate(all="ignore"):
        for f in _pins():
            try:
                f()
            except Exception:  # an assertion, or a numerical error the slip provokes
                caught.append(f.__name__)
    assert caught, f"no pin fails with the planted mistake: {slip}"


@pytest.mark.parametrize("slip", list(MUTATIONS))
def test_planted_mistake_is_caught_by_the_loop_oracle(slip):
    """The plain-C loop oracle alone catches each planted mistake too (one layout, one trajectory)."""
    from tests import test_oracle_loop as loop
    name, fn = MUTATIONS[slip]
    checks = [lambda: loop.test_every_update_agrees((4, 4), 5, 6),
              lambda: loop.test_trajectories_agree(dict(F=17, T=60, mics=(4, 4, 4, 4), N=5, B=8), 1e-11)]
    caught = 0
    with _planted(name, fn), np.errstate(all="ignore"):
        for check in checks:
            try:
                check()
            except Exception:
                caught += 1
    assert caught, f"the loop oracle agrees with the planted mistake: {slip}"
