"""FP64 CPU oracle of distributed FastMNMF -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library never does.

Two independent restatements of the method live here: ``dfmnmf_oracle`` in
NumPy and ``c/dfmnmf_loop.c`` in plain C loops (binding: ``oracle.loop``);
``tests/test_oracle_loop.py`` holds them against each other.
"""
from .dfmnmf_oracle import *  # noqa: F401,F403
from .dfmnmf_oracle import (EPS, SINGULAR_RTOL, State, state_from_arrays, unpack_Q, pack_Q,
                            dense_Q, mic_offsets, source_psd, model_variance,
                            weighted_covariances, ge_solve, pinv_apply, solve_or_pinv,
                            ip_update_row, ip_update, projected_power, update_W, update_H,
                            update_g, log_abs_det_sq, neg_loglik, wiener_filter,
                            mm_iteration, run)
