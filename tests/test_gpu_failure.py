"""Failure detection on the GPU without a fault.

The tensor-core covariance kernel bounds every mbarrier wait.  With the
pipeline-wait budget set to one clock cycle (DFMNMF_OPT_WAIT_CYCLES) its first
waits give up at once: the kernel records FLAG_TIMEOUT, still waits -- with the
full budget -- for the copies and tensor-core work it has in flight, frees its
tensor memory and returns.  The next synchronising call reports
DFMNMF_ETIMEOUT, and the GPU goes on working for a new context.  Nothing here
traps, faults or waits on a flag that nothing sets without a bound.
"""
import numpy as np
import pytest

from paper_2605_19388_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_19388_gb300 import dfmnmf as D  # noqa: E402


@pytest.mark.parametrize("form", [D.DFMNMF_BF16_TC, D.DFMNMF_TF32_TC])
def test_pipeline_wait_that_runs_out_reports_etimeout(form):
    p = synth.make_problem(41, 300, (4, 4, 4, 4), 5, 8, seed=51)
    ctx = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0, p.Q0, precision=form)
    D.dfmnmf_set_option(ctx, D.DFMNMF_OPT_WAIT_CYCLES, 1)
    assert D.dfmnmf_get_option(ctx, D.DFMNMF_OPT_WAIT_CYCLES) == 1
    D.dfmnmf_iterate(ctx, 1)
    with pytest.raises(D.DfmnmfError) as ei:
        D.dfmnmf_loglik(ctx)
    assert ei.value.code == D.DFMNMF_ETIMEOUT
    D.dfmnmf_destroy(ctx)
    torch.cuda.synchronize()
    # the device is healthy: a new context iterates and reports a finite cost
    ctx2 = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, p.x, p.W0, p.H0, p.g0, p.Q0, precision=form)
    D.dfmnmf_iterate(ctx2, 2)
    assert np.isfinite(D.dfmnmf_loglik(ctx2))
