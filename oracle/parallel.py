"""All-core timing harness around the FP64 oracle (test and benchmark infrastructure).

The oracle itself stays single-threaded and plain.  This module only runs it
on slices of the frequency axis in separate processes, so that its MM
iterations can be timed on every host core:

* every step of an iteration except the H update (Eq. 9) is local to a
  frequency bin -- Eq. 2, Eq. 13, Eqs. 14-15, the projected power, the W
  update of Eq. 8 (its sums run over frames) and the g update of Eq. 10 --
  so each worker applies the oracle's own functions to its bins;
* Eq. 9 sums over all bins: each worker returns its bins' share of the
  numerator and denominator sums, the parent adds the shares in worker order
  and applies the update, exactly as the oracle's update_H does with the
  whole sum (the result differs from one process only by the order of that
  sum).

Workers start with the ``spawn`` method (safe after CUDA is initialised in
the parent) and keep their slice of x, Q, W and g between iterations; only H
and the Eq. 9 shares cross the pipes.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from typing import List, Sequence

import numpy as np

from . import dfmnmf_oracle as O


def _worker(conn, x, Qp, W, H, g, mics, eps):
    """Serve one slice of bins: 'p1' -> (num, den) shares of Eq. 9; 'p2', H -> g update; 'get' -> state."""
    # one thread per worker process: the parent runs one worker per core
    x = np.asarray(x, dtype=np.complex128)
    Q = O.unpack_Q(Qp, mics)
    W = np.asarray(W, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    P = None
    while True:
        msg = conn.recv()
        if msg[0] == "p1":
            lam = O.source_psd(W, H)
            y = O.model_variance(lam, g, eps)
            V = O.weighted_covariances(x, y, mics)
            Q = O.ip_update(Q, V, eps)
            P = O.projected_power(x, Q, mics)
            W = O.update_W(W, H, g, P, eps)
            A, D = O._mu_statistics(W, H, g, P, eps)
            Wt = np.transpose(W, (0, 2, 1))
            conn.send((np.matmul(Wt, A), np.matmul(Wt, D)))
        elif msg[0] == "p2":
            H = msg[1]
            g = O.update_g(W, H, g, P, eps)
            conn.send(True)
        elif msg[0] == "get":
            conn.send((O.pack_Q(Q), W, g))
        else:
            conn.close()
            return


class SlicedOracle:
    """The oracle's MM iteration on `workers` processes, each holding a contiguous slice of bins."""

    def __init__(self, x, mics: Sequence[int], st: O.State, workers: int, eps: float = O.EPS):
        F = x.shape[0]
        self.workers = max(1, min(int(workers), F))
        self.mics, self.eps = tuple(mics), eps
        self.H = np.array(st.H, dtype=np.float64)
        bounds = np.linspace(0, F, self.workers + 1).astype(int)
        self.slices = [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:])]
        ctx = mp.get_context("spawn")
        Qp = O.pack_Q(st.Q)
        self.conns, self.procs = [], []
        env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env_keep:
            os.environ[k] = "1"
        try:
            for a, b in self.slices:
                parent, child = ctx.Pipe()
                p = ctx.Process(target=_worker, args=(child, x[a:b], Qp[a:b], st.W[:, a:b], self.H, st.g[a:b],
                                                      self.mics, eps), daemon=True)
                p.start()
                child.close()
                self.conns.append(parent)
                self.procs.append(p)
        finally:
            for k, v in env_keep.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def iterate(self, n: int = 1):
        for _ in range(n):
            for c in self.conns:
                c.send(("p1",))
            shares = [c.recv() for c in self.conns]
            num = shares[0][0].copy()
            den = shares[0][1].copy()
            for s_num, s_den in shares[1:]:
                num += s_num
                den += s_den
            self.H = self.H * np.sqrt(num / np.maximum(den, self.eps))
            for c in self.conns:
                c.send(("p2", self.H))
            for c in self.conns:
                c.recv()

    def state(self) -> O.State:
        parts = []
        for c in self.conns:
            c.send(("get",))
            parts.append(c.recv())
        Qp = np.concatenate([p[0] for p in parts], axis=0)
        W = np.concatenate([p[1] for p in parts], axis=1)
        g = np.concatenate([p[2] for p in parts], axis=0)
        return O.state_from_arrays(Qp, W, self.H, g, self.mics)

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
                c.close()
            except (OSError, BrokenPipeError):
                pass
        for p in self.procs:
            p.join(timeout=10)
            if p.is_alive():
                p.terminate()
        self.conns, self.procs = [], []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
