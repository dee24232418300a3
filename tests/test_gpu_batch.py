"""Many mixtures in one graph launch per iteration, and measured launch
shapes: both must leave the arithmetic of every mixture unchanged."""
import numpy as np
import pytest

import oracle as O
from paper_2605_19388_gb300 import synth
from tests._helpers import rel_err, oracle_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_19388_gb300 import dfmnmf as D  # noqa: E402

SHAPES = [dict(F=33, T=70, mics=(4, 4), N=3, B=8, precision=D.DFMNMF_FP32),
          dict(F=41, T=150, mics=(4, 4, 4, 4), N=5, B=16, precision=D.DFMNMF_BF16_TC),
          dict(F=19, T=97, mics=(2, 2), N=2, B=4, precision=D.DFMNMF_FP32),
          dict(F=9, T=200, mics=(16,), N=3, B=4, precision=D.DFMNMF_FP32)]


def ctx_of(p, precision):
    return D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0, p.Q0, precision=precision)


def test_batch_iterate_equals_per_context_iterate():
    probs = [synth.make_problem(s["F"], s["T"], s["mics"], s["N"], s["B"], seed=50 + i) for i, s in enumerate(SHAPES)]
    solo = [ctx_of(p, s["precision"]) for p, s in zip(probs, SHAPES)]
    batched = [ctx_of(p, s["precision"]) for p, s in zip(probs, SHAPES)]
    b = D.dfmnmf_batch_create(batched)
    D.dfmnmf_batch_iterate(b, 4)
    for c in solo:
        D.dfmnmf_iterate(c, 4)
    torch.cuda.synchronize()
    for cs, cb in zip(solo, batched):
        for u, v in zip(D.params_numpy(cs), D.params_numpy(cb)):
            np.testing.assert_array_equal(u, v)
    D.dfmnmf_batch_destroy(b)


def test_autotune_restores_state_and_keeps_parity():
    p = synth.make_problem(45, 130, (4, 4, 4), 4, 8, seed=60)
    ctx = ctx_of(p, D.DFMNMF_FP32)
    D.dfmnmf_iterate(ctx, 2)
    before = D.params_numpy(ctx)
    br, ct = D.dfmnmf_autotune(ctx, 3)
    assert br in (1, 2) and ct in (2, 4, 8)
    for u, v in zip(before, D.params_numpy(ctx)):
        np.testing.assert_array_equal(u, v)
    # one iteration with the chosen shapes against the oracle from the same state
    st = O.state_from_arrays(*before, p.mics)
    D.dfmnmf_iterate(ctx, 1)
    ref = O.mm_iteration(p.x.astype(np.complex128), p.mics, st)
    Q, W, H, g = D.params_numpy(ctx)
    got = O.state_from_arrays(Q, W, H, g, p.mics)
    for k in range(len(p.mics)):
        assert rel_err(got.Q[k], ref.Q[k]) < 1e-5
    assert rel_err(got.W, ref.W) < 1e-5 and rel_err(got.H, ref.H) < 1e-5 and rel_err(got.g, ref.g) < 1e-5
