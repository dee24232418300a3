"""The allocation-free cost entry point against the context-based one.

dfmnmf_loglik_noalloc serves callers that may not allocate device memory when
they need the cost (a real-time audio thread, a plug-in inside a host that owns
the GPU memory budget): it keeps its partial sums in one static device array.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2605_19388_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_19388_gb300 import build as B  # noqa: E402
from paper_2605_19388_gb300 import dfmnmf as D  # noqa: E402

B.build()


def _device_state(ctx, p):
    Q = torch.empty((p.F, sum(m * m for m in p.mics)), dtype=torch.complex128, device="cuda")
    W = torch.empty((p.N, p.F, p.B), dtype=torch.float32, device="cuda")
    H = torch.empty((p.N, p.B, p.T), dtype=torch.float32, device="cuda")
    g = torch.empty((p.F, p.N, p.M), dtype=torch.float32, device="cuda")
    D.dfmnmf_get_params(ctx, Q, W, H, g)
    torch.cuda.synchronize()
    return Q, W, H, g


@pytest.mark.parametrize("shape", [dict(F=29, T=83, mics=(4, 4), N=3, B=4),
                                   dict(F=513, T=626, mics=(4, 4, 4, 4), N=5, B=16)])
def test_noalloc_cost_matches_context_cost_on_two_calls(shape):
    p = synth.make_problem(shape["F"], shape["T"], shape["mics"], shape["N"], shape["B"], seed=21)
    x = torch.from_numpy(p.x).cuda()
    ctx = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, x, p.W0, p.H0, p.g0,
                        synth.random_blocks(p.F, p.mics, seed=22))
    tol = 1e-5 * p.F * p.T * p.M
    refs, gots = [], []
    for n_iter in (1, 2):                      # two calls in a row, on two different states
        D.dfmnmf_iterate(ctx, n_iter)
        ref = D.dfmnmf_loglik(ctx)
        Q, W, H, g = _device_state(ctx, p)
        got = D.dfmnmf_loglik_noalloc(p.F, p.T, p.mics, p.N, p.B, x, Q, W, H, g)
        refs.append(ref)
        gots.append(got)
        assert abs(got - ref) <= 1e-5 * max(abs(ref), p.F * p.T * p.M), (got, ref)
    assert abs(refs[0] - refs[1]) > tol            # the two states really differ
    # the same state again: the shared array holds the previous call's partials
    again = D.dfmnmf_loglik_noalloc(p.F, p.T, p.mics, p.N, p.B, x, Q, W, H, g)
    assert again == gots[-1]


def test_noalloc_rejects_sizes_beyond_its_array():
    F, T, mics, N, Bn = 4000, 2048, (4, 4), 1, 1      # 4000*16 + 4000*2 + 1 > 65536
    x = torch.zeros((1,), dtype=torch.complex64, device="cuda")
    Q = torch.zeros((1,), dtype=torch.complex128, device="cuda")
    f = torch.zeros((1,), dtype=torch.float32, device="cuda")
    with pytest.raises(D.DfmnmfError) as ei:
        D.dfmnmf_loglik_noalloc(F, T, mics, N, Bn, x, Q, f, f, f)
    assert ei.value.code == D.DFMNMF_EINVAL
    assert "exceeds the maximum" in str(ei.value)
