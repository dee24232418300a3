"""Conventional all-microphone FastMNMF (K = 1, one 16 x 16 diagonaliser per
frequency, Sec. II-A) on the GPU against the FP64 oracle, which runs the same
equations at K = 1 (the distributed method reduces to it there, Sec. III-B).

Tolerances are those of the FP32 form: every single update within 1e-5
normwise relative error, Eq. (12) within 1e-3 and the SDR within 0.1 dB after
the iterations.  With 16 microphones and at most 5 sources the weighted
covariances are far more ill-conditioned (cond ~ 1e7) than per-subarray ones,
which is what the float-float covariances and IP solves are for.
"""
import numpy as np
import pytest

import oracle as O
from paper_2605_19388_gb300 import synth
from tests._helpers import rel_err, v_oracle_layout, sdr_db, oracle_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_19388_gb300 import dfmnmf as D  # noqa: E402

TOL = 1e-5
ALLMIC = (16,)


def make_ctx(p, Q0=None, ip=D.DFMNMF_IP_F32X2):
    return D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0,
                         Q0 if Q0 is not None else p.Q0, ip_arith=ip)


def gpu_state(ctx):
    Q, W, H, g = D.params_numpy(ctx)
    return O.state_from_arrays(Q, W, H, g, ctx.mics)


@pytest.mark.parametrize("ip", [D.DFMNMF_IP_F32X2, D.DFMNMF_IP_F64])
def test_allmic_stage_parity(ip):
    """The five stages once, each against the oracle fed the GPU's own inputs."""
    p = synth.make_problem(13, 150, ALLMIC, 4, 6, seed=41)
    Q0 = synth.random_blocks(p.F, p.mics, seed=42, scale=0.2)
    x = p.x.astype(np.complex128)
    ctx = make_ctx(p, Q0, ip)
    st = gpu_state(ctx)
    errs = {}
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_COV)
    V_gpu = D.buffer_numpy(ctx, D.DFMNMF_BUF_V)
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    errs["V"] = rel_err(V_gpu, v_oracle_layout(O.weighted_covariances(x, y, p.mics)))
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_IP)
    st2 = gpu_state(ctx)
    errs["Q"] = rel_err(st2.Q[0], O.ip_update(st.Q, [V_gpu[:, 0].astype(np.complex128)])[0])
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_W)
    st3 = gpu_state(ctx)
    P_ref = O.projected_power(x, st2.Q, p.mics)
    errs["P"] = rel_err(D.buffer_numpy(ctx, D.DFMNMF_BUF_P), P_ref)
    errs["W"] = rel_err(st3.W, O.update_W(st2.W, st2.H, st2.g, P_ref))
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_H)
    st4 = gpu_state(ctx)
    errs["H"] = rel_err(st4.H, O.update_H(st3.W, st3.H, st3.g, P_ref))
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_G)
    errs["g"] = rel_err(gpu_state(ctx).g, O.update_g(st4.W, st4.H, st4.g, P_ref))
    for k, v in errs.items():
        assert v <= TOL, (k, v, errs)


def test_allmic_covariances_ragged_frames():
    """Frame counts that leave a partial chunk and odd bin counts."""
    p = synth.make_problem(5, 97, ALLMIC, 3, 4, seed=43)
    ctx = make_ctx(p)
    st = gpu_state(ctx)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_COV)
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    V_ref = v_oracle_layout(O.weighted_covariances(p.x.astype(np.complex128), y, p.mics))
    # exact float-float sums of exact products; the weights 1/yhat are FP32 (relative 6e-8 each)
    assert rel_err(D.buffer_numpy(ctx, D.DFMNMF_BUF_V), V_ref) < 1e-6


@pytest.mark.parametrize("ip", [D.DFMNMF_IP_F32X2, D.DFMNMF_IP_F64])
def test_allmic_singular_uses_pseudo_inverse(ip):
    """T < 16 frames: every V_mu has rank 6 (the pseudo-inverse rule, Sec. IV-A).

    Sixteen successive pseudo-inverse rows on rank-6 covariances amplify any
    change of V enormously (the FP32 weights' 3e-8 moves the oracle's own
    result by orders of magnitude), so the oracle is fed the GPU's V, as in
    the stage-by-stage checks."""
    p = synth.make_problem(2, 6, ALLMIC, 2, 2, seed=44)
    ctx = make_ctx(p, ip=ip)
    st = gpu_state(ctx)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_COV)
    V_gpu = D.buffer_numpy(ctx, D.DFMNMF_BUF_V)[:, 0].astype(np.complex128)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_IP)
    Q_ref = O.ip_update(st.Q, [V_gpu])
    assert rel_err(gpu_state(ctx).Q[0], Q_ref[0]) < 1e-4


def test_allmic_trajectory_loglik_and_wiener():
    """20 iterations, then Eq. (12) and the Wiener filter against the oracle's run."""
    p = synth.make_problem(17, 200, ALLMIC, 3, 4, seed=45, with_images=True)
    x = p.x.astype(np.complex128)
    ctx = make_ctx(p)
    D.dfmnmf_iterate(ctx, 20)
    nll_gpu = D.dfmnmf_loglik(ctx)
    c_gpu = torch.empty((p.N, p.F, p.T, p.M), dtype=torch.complex64, device="cuda")
    D.dfmnmf_separate(ctx, c_gpu)
    st = oracle_state(p)
    for _ in range(20):
        st = O.mm_iteration(x, p.mics, st)
    nll_ref = O.neg_loglik(x, p.mics, st)
    assert abs(nll_gpu - nll_ref) <= 1e-3 * abs(nll_ref), (nll_gpu, nll_ref)
    c_ref = O.wiener_filter(x, p.mics, st)
    sdr_gpu, _ = sdr_db(c_gpu.cpu().numpy(), p.c)
    sdr_ref, _ = sdr_db(c_ref, p.c)
    assert np.max(np.abs(np.sort(sdr_gpu) - np.sort(sdr_ref))) <= 0.1, (sdr_gpu, sdr_ref)


def test_allmic_rejects_tensor_core_form_and_two_blocks():
    p = synth.make_problem(3, 20, ALLMIC, 2, 2, seed=46)
    with pytest.raises(D.DfmnmfError) as ei:
        D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0, precision=D.DFMNMF_BF16_TC)
    assert ei.value.code == D.DFMNMF_EINVAL
