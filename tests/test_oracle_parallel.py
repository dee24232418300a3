"""The all-core timing harness around the oracle (oracle/parallel.py) runs the
oracle's own iteration: on a small mixture its bin slices, spread over two
worker processes, give the state of O.mm_iteration up to the order of the
Eq. (9) sum over bins."""
import numpy as np

import oracle as O
from oracle.parallel import SlicedOracle
from paper_2605_19388_gb300 import synth


def test_sliced_oracle_equals_oracle_iteration():
    p = synth.make_problem(13, 40, (4, 4), 3, 4, seed=41)
    x = p.x.astype(np.complex128)
    st0 = O.state_from_arrays(synth.random_blocks(p.F, p.mics, seed=42), p.W0, p.H0, p.g0, p.mics)
    ref = O.run(x, p.mics, st0.copy(), 2)
    with SlicedOracle(x, p.mics, st0, workers=2) as so:
        assert len(so.slices) == 2
        so.iterate(2)
        got = so.state()
    for k in range(p.K):
        np.testing.assert_allclose(got.Q[k], ref.Q[k], rtol=1e-9, atol=1e-12)
    for name in ("W", "H", "g"):
        np.testing.assert_allclose(getattr(got, name), getattr(ref, name), rtol=1e-9)
