"""Tensor-core form (split-bfloat16 weighted covariances on tcgen05) against
the FP32 form and the FP64 oracle.

Tolerances are those of the acceptance bar for the tensor-core form: every
single update within 3e-3 normwise relative error, the cost of Eq. (12) after
50 iterations within 1e-2 relative and the SDR within 0.2 dB.  The form is
meant for mixtures with at least as many sources as microphones per subarray
(the 4 x 4-mic, N = 5 workload): its covariances keep condition numbers
below ~1e4 there, which split bfloat16 resolves.
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

TOL_TC = 3e-3


def ctx_for(p, precision, Q0=None):
    return D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0,
                         Q0 if Q0 is not None else p.Q0, precision=precision)


def state(ctx):
    Q, W, H, g = D.params_numpy(ctx)
    return O.state_from_arrays(Q, W, H, g, ctx.mics)


FORMS = [D.DFMNMF_BF16_TC, D.DFMNMF_TF32_TC]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("shape", [dict(F=37, T=150, mics=(4, 4, 4, 4), N=5, B=8),
                                   dict(F=20, T=64, mics=(4, 4), N=6, B=4),
                                   dict(F=9, T=200, mics=(4,), N=5, B=3),
                                   dict(F=11, T=77, mics=(4,) * 8, N=9, B=5)])
def test_tc_covariances_match_oracle(shape, form):
    """k_vtc's V against the oracle's Eq. (13) on the same state (ragged T, odd F), both operand types."""
    p = synth.make_problem(shape["F"], shape["T"], shape["mics"], shape["N"], shape["B"], seed=31)
    ctx = ctx_for(p, form)
    st = state(ctx)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_COV)
    V = D.buffer_numpy(ctx, D.DFMNMF_BUF_V)
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    V_ref = v_oracle_layout(O.weighted_covariances(p.x.astype(np.complex128), y, p.mics))
    errs = check_both({}, "V", V, V_ref, "V")
    assert max(errs.values()) < 1e-4, errs


def tc_stage_errors(p, form=D.DFMNMF_BF16_TC):
    """Every update of one iteration against the oracle fed the GPU's inputs."""
    x = p.x.astype(np.complex128)
    ctx = ctx_for(p, form)
    st = state(ctx)
    errs = {}
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_COV)
    V = D.buffer_numpy(ctx, D.DFMNMF_BUF_V)
    y = O.model_variance(O.source_psd(st.W, st.H), st.g)
    check_both(errs, "V", V, v_oracle_layout(O.weighted_covariances(x, y, p.mics)), "V")
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_IP)
    st2 = state(ctx)
    Q_ref = O.ip_update(st.Q, [V[:, k] for k in range(p.K)])
    check_both(errs, "Q", list(st2.Q), list(Q_ref), "Q")
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_W)
    st3 = state(ctx)
    P = O.projected_power(x, st2.Q, p.mics)
    check_both(errs, "P", D.buffer_numpy(ctx, D.DFMNMF_BUF_P), P, "med")
    check_both(errs, "W", st3.W, O.update_W(st2.W, st2.H, st2.g, P), "med")
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_H)
    st4 = state(ctx)
    check_both(errs, "H", st4.H, O.update_H(st3.W, st3.H, st3.g, P), "med")
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_G)
    st5 = state(ctx)
    check_both(errs, "g", st5.g, O.update_g(st4.W, st4.H, st4.g, P), "med")
    return errs


@pytest.mark.parametrize("form", FORMS)
def test_tc_stage_parity_paper_shaped(form):
    """Every update of one iteration within 3e-3 (oracle fed the GPU's inputs)."""
    errs = tc_stage_errors(synth.make_problem(41, 120, (4, 4, 4, 4), 5, 16, seed=32), form)
    print("tensor-core form", form, "stage errors", errs)
    assert max(errs.values()) < TOL_TC, errs


@pytest.mark.parametrize("shape", [
    dict(F=1, T=65, mics=(4, 4, 4, 4), N=5, B=1),       # one bin (partial operand tile), one frame in the last chunk
    dict(F=9, T=100, mics=(4, 4, 4, 4), N=16, B=64),    # the largest source and basis counts
    dict(F=3, T=64, mics=(4,) * 8, N=12, B=2),          # eight subarrays, exactly one 64-frame chunk
])
@pytest.mark.parametrize("form", FORMS)
def test_tc_stage_parity_edge_sizes(shape, form):
    p = synth.make_problem(shape["F"], shape["T"], shape["mics"], shape["N"], shape["B"], seed=33)
    errs = tc_stage_errors(p, form)
    assert max(errs.values()) < TOL_TC, (shape, errs)


@pytest.fixture(scope="module")
def paper_oracle_50():
    """The oracle's state after 50 iterations of the paper-shaped workload (bins split over host cores)."""
    import os
    from oracle.parallel import SlicedOracle
    p = synth.make_workload("paper_4x4_n5", seed=0, with_images=True)
    x = p.x.astype(np.complex128)
    with SlicedOracle(x, p.mics, oracle_state(p), workers=os.cpu_count() or 1) as so:
        so.iterate(50)
        st = so.state()
    return p, x, st


@pytest.mark.parametrize("form", FORMS)
def test_tc_trajectory_50_iterations_paper_workload(form, paper_oracle_50):
    """50 iterations on the 4 x 4-mic, N = 5, F = 513, T = 626 workload."""
    p, x, st = paper_oracle_50
    ctx = ctx_for(p, form)
    D.dfmnmf_iterate(ctx, 50)
    nll = D.dfmnmf_loglik(ctx)
    c = torch.empty((p.N, p.F, p.T, p.M), dtype=torch.complex64, device="cuda")
    D.dfmnmf_separate(ctx, c)
    ref = O.neg_loglik(x, p.mics, st)
    s_gpu, _ = sdr_db(c.cpu().numpy(), p.c)
    s_ref, _ = sdr_db(O.wiener_filter(x, p.mics, st), p.c)
    print("tensor-core form", form, "50 iterations: nll", nll, ref, "SDR", s_gpu, s_ref)
    assert abs(nll - ref) <= 1e-2 * abs(ref), (nll, ref)
    assert np.max(np.abs(np.sort(s_gpu) - np.sort(s_ref))) <= 0.2, (s_gpu, s_ref)


def block_errors(a, b):
    """Per-(f, k) normwise relative error of [F][K][...] arrays (b is the reference)."""
    F, K = b.shape[:2]
    d = np.linalg.norm((np.asarray(a, np.complex128) - b).reshape(F, K, -1), axis=2)
    return d / np.maximum(np.linalg.norm(b.reshape(F, K, -1), axis=2), 1e-300)


@pytest.mark.parametrize("form", FORMS)
def test_tc_error_distribution_per_block_paper_workload(form, paper_oracle_50):
    """The distribution over the F x K = 2052 blocks of the 4 x 4-mic, N = 5, F = 513, T = 626 workload,
    at the oracle's state after 50 iterations: the covariances' error (Eq. 13, block-wise relative to the
    oracle's FP64 V on the same state), the IP update's error (Eqs. 14-15: the GPU's rows from its own V
    against the oracle's rows from the exact V, so the covariance error enters amplified by cond(Q V_mu)),
    and that condition number.  Every block's IP update stays within the 3e-3 bar."""
    p, x, st = paper_oracle_50
    ctx = ctx_for(p, form, Q0=O.pack_Q(st.Q))
    D.dfmnmf_set_params(ctx, O.pack_Q(st.Q), st.W.astype(np.float32), st.H.astype(np.float32),
                        st.g.astype(np.float32))
    g_st = state(ctx)  # the state as the GPU holds it (W, H, g rounded to FP32)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_COV)
    V = D.buffer_numpy(ctx, D.DFMNMF_BUF_V)
    y = O.model_variance(O.source_psd(g_st.W, g_st.H), g_st.g)
    V_list = O.weighted_covariances(x, y, p.mics)
    V_ref = v_oracle_layout(V_list)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_IP)
    Q_gpu = np.stack(state(ctx).Q, axis=1)
    Q_ref = np.stack(O.ip_update(g_st.Q, V_list), axis=1)
    ev = block_errors(V, V_ref)
    eq = block_errors(Q_gpu, Q_ref)
    cond = np.stack([np.max(np.linalg.cond(np.matmul(g_st.Q[k][:, None], V_list[k])), axis=1)
                     for k in range(p.K)], axis=1)  # [F][K]: the largest over mu
    stats = {}
    for name, e in (("V", ev), ("Q", eq), ("cond_QV", cond)):
        stats[name] = {"max": float(e.max()), "p99": float(np.quantile(e, 0.99)),
                       "median": float(np.median(e))}
    worst = np.unravel_index(np.argmax(eq), eq.shape)
    print("tensor-core form", form, "per-(f,k) distribution over", eq.size, "blocks:", stats,
          "worst IP block (f, k) =", tuple(int(i) for i in worst), "cond", float(cond[worst]))
    assert stats["V"]["max"] < 1e-4, stats
    assert stats["Q"]["max"] < TOL_TC, stats


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("autotune", [False, True])
def test_tc_paper_workload_one_iteration_full_size(autotune, form):
    """The 4 x 4-mic, N = 5, F = 513, T = 626 workload: one captured iteration
    from identical state, every output within the 3e-3 bar.  Without the
    autotuner the per-frequency kernels run on two graph branches (one per
    half of the band); with it, in the launch shapes the benchmark uses."""
    p = synth.make_workload("paper_4x4_n5", seed=0)
    x = p.x.astype(np.complex128)
    ctx = ctx_for(p, form)
    if autotune:
        D.dfmnmf_autotune(ctx, 2)  # restores the initial state
    D.dfmnmf_iterate(ctx, 1)
    got = state(ctx)
    rec = {}
    ref = O.mm_iteration(x, p.mics, oracle_state(p), record=rec)
    errs = check_both({}, "Q", list(got.Q), list(ref.Q), "Q")
    for name in ("W", "H", "g"):
        check_both(errs, name, getattr(got, name), getattr(ref, name), "med")
    check_both(errs, "P", D.buffer_numpy(ctx, D.DFMNMF_BUF_P), rec["P"], "med")
    print("tensor-core form", form, "one full-size iteration, autotune", autotune, errs)
    norm = {k: v for k, v in errs.items() if not k.endswith("_elem")}
    elem = {k: v for k, v in errs.items() if k.endswith("_elem")}
    assert max(norm.values()) < TOL_TC, errs
    # the split-bfloat16 form also meets the bar element by element; the TF32 form's sums come out about
    # three times less accurate on this workload (V 4.0e-6 against 1.3e-6 normwise), and its element-wise
    # P error (3.1e-3 measured) is held to 5e-3
    assert max(elem.values()) < (TOL_TC if form == D.DFMNMF_BF16_TC else 5e-3), errs


def test_tc_w_update_on_tensor_cores_stage_parity():
    """The W-update products on the tensor cores (tcgen05 kind::tf32, DFMNMF_OPT_WUPD_TC = 1): every
    update of one iteration within 3e-3 of the oracle fed the GPU's inputs, normwise and element-wise."""
    p = synth.make_problem(41, 120, (4, 4, 4, 4), 5, 16, seed=32)
    x = p.x.astype(np.complex128)
    ctx = ctx_for(p, D.DFMNMF_BF16_TC)
    D.dfmnmf_set_option(ctx, D.DFMNMF_OPT_WUPD_TC, 1)
    assert D.dfmnmf_get_option(ctx, D.DFMNMF_OPT_WUPD_TC) == 1
    st = state(ctx)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_COV)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_IP)
    st2 = state(ctx)
    D.dfmnmf_run_stage(ctx, D.DFMNMF_STAGE_W)
    st3 = state(ctx)
    P = O.projected_power(x, st2.Q, p.mics)
    errs = check_both({}, "W", st3.W, O.update_W(st2.W, st2.H, st2.g, P), "med")
    print("tensor-core W update", errs)
    assert max(errs.values()) < TOL_TC, errs
    # the full-size workload in the captured iteration, both engines from the same state
    q = synth.make_workload("paper_4x4_n5", seed=0)
    a, b = ctx_for(q, D.DFMNMF_BF16_TC), ctx_for(q, D.DFMNMF_BF16_TC)
    D.dfmnmf_set_option(b, D.DFMNMF_OPT_WUPD_TC, 1)
    D.dfmnmf_iterate(a, 1)
    D.dfmnmf_iterate(b, 1)
    Wa, Wb = D.params_numpy(a)[1], D.params_numpy(b)[1]
    errs = check_both({}, "W", Wb, Wa, "med")
    print("tensor-core W update against the CUDA-core one, full size", errs)
    assert max(errs.values()) < TOL_TC, errs


def test_launch_options_rejected_values():
    p = synth.make_problem(9, 40, (4, 4), 3, 4, seed=34)
    fp32 = ctx_for(p, D.DFMNMF_FP32)
    for opt, val in ((D.DFMNMF_OPT_BRANCHES, 3), (D.DFMNMF_OPT_NMF_CTAS, 5), (D.DFMNMF_OPT_VX_GROUPS, 0),
                     (D.DFMNMF_OPT_WUPD_TC, 1), (99, 1)):
        with pytest.raises(D.DfmnmfError) as ei:
            D.dfmnmf_set_option(fp32, opt, val)
        assert ei.value.code == D.DFMNMF_EINVAL, (opt, val)
    D.dfmnmf_set_option(fp32, D.DFMNMF_OPT_BRANCHES, 1)
    assert D.dfmnmf_get_option(fp32, D.DFMNMF_OPT_BRANCHES) == 1
    assert D.dfmnmf_get_option(fp32, 99) == -1


@pytest.mark.parametrize("form", FORMS)
def test_tc_form_rejects_unsupported_layouts(form):
    p = synth.make_problem(5, 20, (2, 2), 2, 3, seed=1)
    with pytest.raises(D.DfmnmfError) as ei:
        ctx_for(p, form)
    assert ei.value.code == D.DFMNMF_EINVAL
