"""Oracle regression fixture and closed forms of Eq. (12)."""
import json
import os

import numpy as np

import oracle as O
from paper_2605_19388_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_stored_trajectory():
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(HERE, "golden", "make_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(os.path.join(HERE, "golden", "oracle_tiny_trajectory.json")) as fh:
        ref = json.load(fh)
    got = mk.compute()
    np.testing.assert_allclose(got["nll"], ref["nll"], rtol=1e-10)
    for key in ("sum_abs_Q", "sum_W", "sum_H", "sum_g"):
        np.testing.assert_allclose(got[key], ref[key], rtol=1e-10)
    assert np.all(np.diff(ref["nll"]) <= 0)


def test_cost_closed_form_identity_and_constant_model():
    """Q = I and yhat = c everywhere: Eq. (12) = sum |x|^2 / c + F T M ln c."""
    F, T, mics, N, B = 3, 11, (2, 2), 1, 1
    p = synth.make_problem(F, T, mics, N, B, seed=3)
    c = 2.5
    st = O.State(O.unpack_Q(synth.identity_blocks(F, mics), mics),
                 np.ones((N, F, B)), np.full((N, B, T), c), np.ones((F, N, sum(mics))))
    x = p.x.astype(np.complex128)
    ref = np.sum(np.abs(x) ** 2) / c + F * T * sum(mics) * np.log(c)
    np.testing.assert_allclose(O.neg_loglik(x, mics, st), ref, rtol=1e-13)
