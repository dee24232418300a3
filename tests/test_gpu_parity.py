"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances are those of the acceptance bar for the FP32 form: every single
update within 1e-5 normwise relative error, the cost of Eq. (12) after 50
iterations within 1e-3 relative and the separated sources' SDR within 0.1 dB.
"""
import numpy as np
import pytest

import oracle as O
from paper_2605_19388_gb300 import synth
from tests._helpers import rel_err, v_oracle_layout, sdr_db, oracle_state, check_both

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_19388_gb300 import dfmnmf as D  # noqa: E402

TOL_UPDATE = 1e-5


def make_ctx(p, Q0=None, ip=D.DFMNMF_IP_F32X2, precision=D.DFMNMF_FP32):
    return D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0,
                         Q0 if Q0 is not None else p.Q0, precision=precision, ip_arith=ip)


def gpu_state(ctx):
    Q, W, H, g = D.params_numpy(ctx)
    return O.state_from_arrays(Q, W, H, g, ctx.mics)


def stage_parity(p, Q0, ip=D.DFMNMF_IP_F32X2, tol=TOL_UPDATE, tol_ip=TOL_UPDATE):
    """Run the five stages once; check each against the oracle fed the GPU's own inputs."""
    x = p.x.astype(np.complex128)
    ctx = make_ctx(p, Q0, ip)
    st = gpu_state(ctx)
    errs = {}
    # stage 1: yhat and V (Eq. 13)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_COV)
    V_gpu = D.buffer_numpy(ctx, D.DFMNMF_BUF_V)
    lam_gpu = D.buffer_numpy(ctx, D.DFMNMF_BUF_LAMBDA)
    check_both(errs, "lambda", lam_gpu, O.source_psd(st.W, st.H), "med")
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    V_ref = O.weighted_covariances(x, y, p.mics)
    check_both(errs, "V", V_gpu, v_oracle_layout(V_ref), "V")
    # stage 2: IP (Eqs. 14-15) on the GPU's V
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_IP)
    st2 = gpu_state(ctx)
    V_in = [V_gpu[:, k].astype(np.complex128) for k in range(p.K)]
    Q_ref = O.ip_update(st.Q, V_in)
    check_both(errs, "Q", list(st2.Q), list(Q_ref), "Q")
    # stage 3: P and W (Eq. 8) from the GPU's Q
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_W)
    st3 = gpu_state(ctx)
    P_gpu = D.buffer_numpy(ctx, D.DFMNMF_BUF_P)
    P_ref = O.projected_power(x, st2.Q, p.mics)
    check_both(errs, "P", P_gpu, P_ref, "med")
    check_both(errs, "W", st3.W, O.update_W(st2.W, st2.H, st2.g, P_ref), "med")
    # stage 4: H (Eq. 9)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_H)
    st4 = gpu_state(ctx)
    check_both(errs, "H", st4.H, O.update_H(st3.W, st3.H, st3.g, P_ref), "med")
    # stage 5: g (Eq. 10)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_G)
    st5 = gpu_state(ctx)
    check_both(errs, "g", st5.g, O.update_g(st4.W, st4.H, st4.g, P_ref), "med")
    lam5 = D.buffer_numpy(ctx, D.DFMNMF_BUF_LAMBDA)
    check_both(errs, "lambda_end", lam5, O.source_psd(st5.W, st5.H), "med")
    for k, v in errs.items():
        lim = tol_ip if k.startswith("Q") else tol
        assert v <= lim, (k, v, errs)
    return errs


@pytest.mark.parametrize("ip", [D.DFMNMF_IP_F32X2, D.DFMNMF_IP_F64])
def test_stage_parity_two_subarrays_ragged(ip):
    p = synth.make_problem(37, 150, (4, 4), 3, 8, seed=1)
    Q0 = synth.random_blocks(p.F, p.mics, seed=3)
    stage_parity(p, Q0, ip)


def test_stage_parity_plain_fp32_ip_well_conditioned():
    """Plain binary32 solves are only a study mode: they hold on well-conditioned
    covariances (more sources than microphones per subarray, 26 dB noise floor)."""
    p = synth.make_problem(23, 97, (4, 4, 4), 6, 5, seed=2, noise_std=0.05)
    Q0 = synth.random_blocks(p.F, p.mics, seed=4)
    stage_parity(p, Q0, D.DFMNMF_IP_F32, tol_ip=1e-4)


@pytest.mark.parametrize("mics", [(1, 1, 1), (2, 2), (3, 3), (4,), (4, 4, 4, 4), (4,) * 8])
def test_stage_parity_block_sizes(mics):
    p = synth.make_problem(19, 71, mics, 3, 6, seed=5)
    Q0 = synth.random_blocks(p.F, p.mics, seed=6)
    stage_parity(p, Q0)


@pytest.mark.parametrize("N,B", [(1, 1), (5, 16), (9, 20), (16, 33)])
def test_stage_parity_source_and_basis_counts(N, B):
    p = synth.make_problem(21, 45, (4, 4), N, B, seed=7)
    stage_parity(p, synth.random_blocks(p.F, p.mics, seed=8))


def test_minimal_sizes():
    p = synth.make_problem(1, 5, (2,), 1, 1, seed=9)
    stage_parity(p, synth.random_blocks(p.F, p.mics, seed=1))


def test_singular_systems_use_pseudo_inverse():
    """T < M_k makes every V_mu rank deficient: the pseudo-inverse rule (Sec. IV-A)."""
    p = synth.make_problem(6, 2, (4, 4), 2, 3, seed=10)
    x = p.x.astype(np.complex128)
    ctx = make_ctx(p)
    st = gpu_state(ctx)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_COV)
    V_gpu = D.buffer_numpy(ctx, D.DFMNMF_BUF_V)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_IP)
    Q_gpu = gpu_state(ctx).Q
    # oracle on the exactly rank-deficient FP64 covariances
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    V_ref = O.weighted_covariances(x, y, p.mics)
    Q_ref = O.ip_update(st.Q, V_ref)
    errs = check_both({}, "Q", list(Q_gpu), list(Q_ref), "Q")
    assert max(errs.values()) < 1e-4, errs
    assert np.all(np.isfinite(V_gpu))


def test_silent_subarray_bin():
    """x = 0 on one subarray at one bin: V = 0, the pseudo-inverse gives q = 0."""
    p = synth.make_problem(5, 40, (4, 4), 2, 3, seed=11)
    p.x[2, :, 4:8] = 0
    ctx = make_ctx(p)
    st = gpu_state(ctx)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_COV)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_IP)
    Q_gpu = gpu_state(ctx).Q
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    Q_ref = O.ip_update(st.Q, O.weighted_covariances(p.x.astype(np.complex128), y, p.mics))
    assert np.all(Q_gpu[1][2] == 0) and np.all(Q_ref[1][2] == 0)
    errs = check_both({}, "Q", list(Q_gpu), list(Q_ref), "Q")
    assert max(errs.values()) < TOL_UPDATE, errs


def test_loglik_and_wiener_parity():
    p = synth.make_problem(29, 83, (4, 4), 3, 4, seed=12)
    Q0 = synth.random_blocks(p.F, p.mics, seed=2)
    ctx = make_ctx(p, Q0)
    D.dfmnmf_iterate(ctx, 2)
    st = gpu_state(ctx)
    x = p.x.astype(np.complex128)
    nll_gpu = D.dfmnmf_loglik(ctx)
    nll_ref = O.neg_loglik(x, p.mics, st)
    assert abs(nll_gpu - nll_ref) <= 1e-5 * max(abs(nll_ref), p.F * p.T * p.M)
    c = torch.empty((p.N, p.F, p.T, p.M), dtype=torch.complex64, device="cuda")
    D.dfmnmf_separate(ctx, c)
    torch.cuda.synchronize()
    c_ref = O.wiener_filter(x, p.mics, st)
    errs = check_both({}, "c", c.cpu().numpy(), c_ref, "med")
    assert max(errs.values()) < 1e-5, errs


def test_iterate_equals_stages():
    p = synth.make_problem(17, 60, (4, 4), 2, 4, seed=13)
    a, b = make_ctx(p), make_ctx(p)
    D.dfmnmf_iterate(a, 3)
    for _ in range(3):
        for s in range(1, 6):
            D.dfmnmf_run_stage(b, s)
    for u, v in zip(D.params_numpy(a), D.params_numpy(b)):
        np.testing.assert_array_equal(u, v)


def test_trajectory_50_iterations_small_workload():
    """50 MM iterations on the 2 x 4-mic, N = 3, F = 257, T = 313 workload."""
    p = synth.make_workload("small_2x4_n3", seed=0, with_images=True)
    x = p.x.astype(np.complex128)
    ctx = make_ctx(p)
    D.dfmnmf_iterate(ctx, 50)
    nll_gpu = D.dfmnmf_loglik(ctx)
    c_gpu = torch.empty((p.N, p.F, p.T, p.M), dtype=torch.complex64, device="cuda")
    D.dfmnmf_separate(ctx, c_gpu)
    st = oracle_state(p)
    for _ in range(50):
        st = O.mm_iteration(x, p.mics, st)
    nll_ref = O.neg_loglik(x, p.mics, st)
    assert abs(nll_gpu - nll_ref) <= 1e-3 * abs(nll_ref), (nll_gpu, nll_ref)
    c_ref = O.wiener_filter(x, p.mics, st)
    sdr_gpu, _ = sdr_db(c_gpu.cpu().numpy(), p.c)
    sdr_ref, _ = sdr_db(c_ref, p.c)
    assert np.max(np.abs(np.sort(sdr_gpu) - np.sort(sdr_ref))) <= 0.1, (sdr_gpu, sdr_ref)


def test_paper_workload_one_iteration_full_size():
    """The 4 x 4-mic, N = 5, F = 513, T = 626 workload in the benchmark's launch
    configuration: one iteration from identical state, every output compared."""
    p = synth.make_workload("paper_4x4_n5", seed=0)
    x = p.x.astype(np.complex128)
    ctx = make_ctx(p)
    D.dfmnmf_iterate(ctx, 1)
    got = gpu_state(ctx)
    rec = {}
    ref = O.mm_iteration(x, p.mics, oracle_state(p), record=rec)
    errs = check_both({}, "Q", list(got.Q), list(ref.Q), "Q")
    for name in ("W", "H", "g"):
        check_both(errs, name, getattr(got, name), getattr(ref, name), "med")
    check_both(errs, "P", D.buffer_numpy(ctx, D.DFMNMF_BUF_P), rec["P"], "med")
    print("FP32 form, one full-size iteration", errs)
    assert max(errs.values()) < TOL_UPDATE, errs


def test_nonfinite_input_reports_enumeric():
    p = synth.make_problem(7, 30, (4, 4), 2, 3, seed=14)
    p.x[3, 5, 2] = np.nan
    ctx = make_ctx(p)
    D.dfmnmf_iterate(ctx, 1)
    with pytest.raises(D.DfmnmfError) as ei:
        D.dfmnmf_loglik(ctx)
    assert ei.value.code == D.DFMNMF_ENUMERIC


def test_fp32_form_200_iterations_paper_workload():
    """The 4 x 4-mic, N = 5, F = 513, T = 626 workload for its full 200 iterations in the FP32 form:
    Eq. (12) within 1e-3 relative and the SDR within 0.1 dB of the oracle's.  The oracle runs on
    every host core (its bins split over worker processes; oracle/parallel.py)."""
    import os
    from oracle.parallel import SlicedOracle
    p = synth.make_workload("paper_4x4_n5", seed=0, with_images=True)
    x = p.x.astype(np.complex128)
    ctx = make_ctx(p)
    D.dfmnmf_iterate(ctx, 200)
    nll_gpu = D.dfmnmf_loglik(ctx)
    c_gpu = torch.empty((p.N, p.F, p.T, p.M), dtype=torch.complex64, device="cuda")
    D.dfmnmf_separate(ctx, c_gpu)
    with SlicedOracle(x, p.mics, oracle_state(p), workers=os.cpu_count() or 1) as so:
        so.iterate(200)
        st = so.state()
    nll_ref = O.neg_loglik(x, p.mics, st)
    sdr_gpu, _ = sdr_db(c_gpu.cpu().numpy(), p.c)
    sdr_ref, _ = sdr_db(O.wiener_filter(x, p.mics, st), p.c)
    print("FP32 form, 200 iterations: nll", nll_gpu, nll_ref, "SDR", sdr_gpu, sdr_ref)
    assert abs(nll_gpu - nll_ref) <= 1e-3 * abs(nll_ref), (nll_gpu, nll_ref)
    assert np.max(np.abs(np.sort(sdr_gpu) - np.sort(sdr_ref))) <= 0.1, (sdr_gpu, sdr_ref)


def test_w_update_fallback_when_the_fused_tile_does_not_fit():
    """B = 64 bases and T = 1000 frames: H[n] and ten A, D rows (B Tp + 20 Tp floats, 336 KB) exceed the
    shared memory of one CTA, so the W stage runs the split products (k_wupd) and the separate lambda
    refresh instead of the fused k_wlam; both paths match the oracle stage by stage."""
    p = synth.make_problem(9, 1000, (4, 4), 4, 64, seed=81)
    Q0 = synth.random_blocks(p.F, p.mics, seed=82, scale=0.2)
    stage_parity(p, Q0)
    ctx = make_ctx(p, Q0)
    names = [n for n, _ in D.dfmnmf_kernel_times(ctx, 1)]
    assert "k_wupd" in names and "k_wlam" not in names, names
    q = synth.make_problem(9, 300, (4, 4), 4, 16, seed=83)
    names = [n for n, _ in D.dfmnmf_kernel_times(make_ctx(q), 1)]
    assert "k_wlam" in names and "k_wupd" not in names, names
