"""The allocation-free cost entry point against the context-based one and the oracle.

dfmnmf_loglik_noalloc serves callers that may not allocate device memory when
they need the cost (a real-time audio thread, where cudaMalloc can block and
synchronise the device; a plug-in inside a host that owns the GPU memory
budget): it keeps its partial sums in one static device array.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
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


def _bar(p, ref):
    """The cost tolerance of the parity tests: 1e-5 relative, floored at F T M."""
    return 1e-5 * max(abs(ref), p.F * p.T * p.M)


SHAPES = [dict(F=29, T=83, mics=(4, 4), N=3, B=4),
          dict(F=513, T=626, mics=(4, 4, 4, 4), N=5, B=16),
          dict(F=17, T=200, mics=(2, 2, 2), N=3, B=5),     # M_k = 2, three subarrays
          dict(F=11, T=130, mics=(3,), N=2, B=3),          # one subarray of three microphones
          dict(F=9, T=129, mics=(1, 1, 1, 1), N=2, B=2)]   # M_k = 1, a ragged last 128-frame chunk


@pytest.mark.parametrize("shape", SHAPES)
def test_noalloc_cost_matches_context_cost_on_two_calls(shape):
    p = synth.make_problem(shape["F"], shape["T"], shape["mics"], shape["N"], shape["B"], seed=21)
    x = torch.from_numpy(p.x).cuda()
    ctx = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, x, p.W0, p.H0, p.g0,
                        synth.random_blocks(p.F, p.mics, seed=22))
    refs, gots = [], []
    for n_iter in (1, 2):                      # two calls in a row, on two different states
        D.dfmnmf_iterate(ctx, n_iter)
        ref = D.dfmnmf_loglik(ctx)
        Q, W, H, g = _device_state(ctx, p)
        got = D.dfmnmf_loglik_noalloc(p.F, p.T, p.mics, p.N, p.B, x, Q, W, H, g)
        refs.append(ref)
        gots.append(got)
        assert abs(got - ref) <= _bar(p, ref), (got, ref)
        # and against the oracle's Eq. (12) on the same state
        st = O.state_from_arrays(Q.cpu().numpy(), W.cpu().numpy(), H.cpu().numpy(), g.cpu().numpy(), p.mics)
        orc = O.neg_loglik(p.x.astype(np.complex128), p.mics, st)
        assert abs(got - orc) <= _bar(p, orc), (got, orc)
    assert abs(refs[0] - refs[1]) > 1e-5 * p.F * p.T * p.M   # the two states really differ
    # the same state again: the shared array holds the previous call's partials
    again = D.dfmnmf_loglik_noalloc(p.F, p.T, p.mics, p.N, p.B, x, Q, W, H, g)
    assert again == gots[-1]


def test_noalloc_on_a_side_stream():
    """Called on a non-default stream, ordered after the writes of the state on that stream."""
    p = synth.make_problem(23, 150, (4, 4), 3, 4, seed=24)
    x = torch.from_numpy(p.x).cuda()
    ctx = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, x, p.W0, p.H0, p.g0, None)
    D.dfmnmf_iterate(ctx, 3)
    ref = D.dfmnmf_loglik(ctx)
    Q, W, H, g = _device_state(ctx, p)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        got1 = D.dfmnmf_loglik_noalloc(p.F, p.T, p.mics, p.N, p.B, x, Q, W, H, g, stream=side)
        got2 = D.dfmnmf_loglik_noalloc(p.F, p.T, p.mics, p.N, p.B, x, Q, W, H, g, stream=side)
    assert abs(got1 - ref) <= _bar(p, ref), (got1, ref)
    assert got1 == got2


def test_noalloc_rejects_sizes_beyond_its_array():
    """Through the C ABI with real device pointers: the size check comes before any device work."""
    F, T, mics, N, Bn = 4000, 2048, (4, 4), 1, 1      # 4000*16 + 4000*2 + 1 > 65536
    buf = torch.zeros((16,), dtype=torch.complex128, device="cuda")
    ptr = ctypes.c_void_p(buf.data_ptr())
    lib = D.load_library()
    m = (ctypes.c_int * len(mics))(*mics)
    d = D.dfmnmf_desc(F, T, len(mics), m, N, Bn, 0, 0, 0.0)
    out = ctypes.c_double()
    assert lib.dfmnmf_loglik_noalloc(ctypes.byref(d), ptr, ptr, ptr, ptr, ptr, ctypes.byref(out),
                                     None) == D.DFMNMF_EINVAL
    assert b"exceeds the maximum" in lib.dfmnmf_last_error()
