"""Write tests/golden/oracle_tiny_trajectory.json from the FP64 oracle alone.

The paper prints no worked numerical example, so this fixture is a regression
guard on the oracle: the cost of Eq. (12) over five iterations of the Sec. III-B
schedule on a tiny seeded mixture, plus parameter checksums.  Any later change
of the oracle's arithmetic that moves these numbers must name the passage that
justifies it.  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2605_19388_gb300 import synth  # noqa: E402

CASE = dict(F=4, T=24, mics=[2, 3], N=2, B=3, seed=0, noise_std=0.05, iters=5)


def compute():
    p = synth.make_problem(CASE["F"], CASE["T"], CASE["mics"], CASE["N"], CASE["B"],
                           seed=CASE["seed"], noise_std=CASE["noise_std"])
    st = O.state_from_arrays(p.Q0, p.W0, p.H0, p.g0, p.mics)
    x = p.x.astype(np.complex128)
    nll = [O.neg_loglik(x, p.mics, st)]
    for _ in range(CASE["iters"]):
        st = O.mm_iteration(x, p.mics, st)
        nll.append(O.neg_loglik(x, p.mics, st))
    return dict(case=CASE, nll=nll,
                sum_abs_Q=float(sum(np.abs(q).sum() for q in st.Q)),
                sum_W=float(st.W.sum()), sum_H=float(st.H.sum()), sum_g=float(st.g.sum()))


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny_trajectory.json")
    with open(out, "w") as fh:
        json.dump(compute(), fh, indent=1)
    print("wrote", out)
