#!/usr/bin/env python
"""Benchmark: MM iterations/s of distributed FastMNMF on one GB300.

Workload (default): 4 subarrays x 4 microphones (M = 16), N = 5 sources,
B = 16 bases, F = 513 bins, T = 626 frames, seeded synthetic mixtures.
One timed step is the whole job of the paper on one mixture: reset to the
initial state, 200 MM iterations (IP of every block, then the W, H, g
multiplicative updates), the negative log-likelihood (read back to the host)
and the per-subarray Wiener filter.  value = MM iterations/s over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank separates its own mixture on its own GPU (replicas:
the mixture does not shard), timing is bracketed by a barrier and a device
synchronise, and rank 0 prints one JSON line with the max time over ranks.
L2 is flushed (a 256 MB write) before every timed step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MM iter/s at 4\u00d74 mics,N=5,F=513,T=626: BF16-TC vs FP32 plain, % roofline"
UNIT = "MM iter/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="paper_4x4_n5")
    ap.add_argument("--iters", type=int, default=None, help="MM iterations per step (default: the workload's)")
    ap.add_argument("--ip", choices=["f32x2", "f64", "f32"], default="f32x2")
    ap.add_argument("--forms", default="bf16tc,tf32tc,fp32,allmic",
                    help="comma list of forms to time (allmic: conventional FastMNMF with one full M x M "
                         "diagonaliser, the comparator); the first is the headline value")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the gradient through 20 unrolled iterations (4 x 4 mics, N = 5, F = 257, T = 313)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only the gradient through 20 unrolled iterations and print it (no headline line)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batched", type=int, default=64,
                    help="also time this many mixtures of mixed length and layout (T in [150, 1250], K in {2, 4, 8} "
                         "x 4 mics, N in {3, 5, 8}, F = 513) in one graph launch per iteration (0: skip)")
    ap.add_argument("--concurrent", type=int, default=8,
                    help="also time this many independent mixtures run concurrently on separate streams (0: skip)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            try:
                os.unlink(self.path)
            except OSError:
                pass
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            out = parse_clock_samples(fh)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        return out


def parse_clock_samples(lines) -> dict:
    """Median SM clock, the largest maximum clock and the throttle reasons seen, from lines of
    `nvidia-smi --query-gpu=<ClockSampler.FIELDS> --format=csv,noheader,nounits`; a line without
    numeric clocks (or too short) is skipped."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            cur, top = float(parts[1]), float(parts[2])
        except ValueError:
            continue
        sm.append(cur)
        smax.append(top)
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------- algorithmic bytes
def kernel_bytes(F, T, M, N, B, K, MK):
    """Algorithmic DRAM bytes of one launch of each kernel (each operand once)."""
    q = F * K * MK * MK
    return {
        # Eq. 13 in either form: x once, lambda and g once, V once (complex64 count)
        "k_vtc": 8 * F * T * M + 4 * N * F * T + 4 * F * N * M + 8 * q * MK,
        "k_cov": 8 * F * T * M + 4 * N * F * T + 4 * F * N * M + 8 * q * MK,
        "k_ip": 8 * q * MK + 32 * q + 8 * q,
        "k_pstats": 8 * F * T * M + 4 * N * F * T + 4 * F * N * M + 8 * q + 4 * F * T * M + 8 * N * F * T,
        "k_wupd": 8 * N * F * T + 4 * N * B * T + 8 * N * F * B + 4 * N * F * T,
        "k_wupd_tc": 8 * N * F * T + 4 * N * B * T + 8 * N * F * B,
        "k_wlam": 12 * N * F * T + 4 * N * B * T + 8 * N * F * B,
        "k_stats": 4 * F * T * M + 4 * N * F * T + 4 * F * N * M + 8 * N * F * T,
        "k_hupd": 8 * N * F * T + 4 * N * F * B + 8 * N * B * T + 4 * N * F * T,
        "k_gupd": 4 * N * F * T + 4 * F * T * M + 8 * F * N * M,
        "k_lambda": 4 * N * F * B + 4 * N * B * T + 4 * N * F * T,
    }


# DRAM bytes (read + write) of one band-wide launch, from a full-section ncu
# capture of one iteration of the tensor-core form (caches flushed before
# each launch, so reads are cold).  A figure holds only while the
# kernel's sources are the ones captured: the digest is the first 16 hex
# digits of sha256 over csrc/<file>, csrc/common.cuh and csrc/internal.h, and
# `traffic` is null when it no longer matches.
NCU_TRAFFIC = {
    "paper_4x4_n5": {
        "k_vtc": (47760896 + 113408, "kernels_tc.cu", "aa8cbc1fdd39f821"),  # k_vtc<4, 2, 0>
        "k_pstats": (48014592 + 2304256, "kernels_tc.cu", "aa8cbc1fdd39f821"),  # k_pstats_tma<0>
        "k_stats": (27194112 + 1280, "kernels_model.cu", "2a06519bbda944e8"),
        "k_gupd": (27193344 + 0, "kernels_model.cu", "2a06519bbda944e8"),
        "k_lambda": (388096 + 0, "kernels_model.cu", "2a06519bbda944e8"),
        "k_ip": (2692096 + 0, "kernels_ip.cu", "a29c23b8fb31e383"),
        "k_wlam": (13277440 + 0, "kernels_nmf.cu", "adf34c7a08fb1dbe"),
        "k_hupd": (13270272 + 0, "kernels_nmf.cu", "adf34c7a08fb1dbe"),
        # FP32 form, the two half-band launches of one iteration added
        "k_cov": (23855360 + 23948288, "kernels_cov.cu", "451a396ec67f3273"),
    },
}


# Kernels bound by instruction issue (float-pair arithmetic chains), not by
# HBM: their roofline is the issue rate, 4 warp-instructions per clock per SM
# (one per scheduler) at the maximum SM clock.  Executed warp instructions of
# one band-wide launch (smsp__inst_executed.sum of the same captures, with the
# same digest rule as NCU_TRAFFIC).
ALU_KERNELS = ("k_ip", "k_cov")
NCU_INST = {  # keyed by (kernel, form): k_ip refines three times in the FP32 form, once in the tensor-core form
    "paper_4x4_n5": {
        ("k_ip", "bf16tc"): (6536940, "kernels_ip.cu", "a29c23b8fb31e383"),
        # the FP32 form's capture ran the per-frequency kernels on two graph branches: the two halves' sum
        ("k_ip", "fp32"): (4366836 + 4400978, "kernels_ip.cu", "34f0aab99e2d0c80"),
        ("k_cov", "fp32"): (28044032 + 28153579, "kernels_cov.cu", "451a396ec67f3273"),
    },
}


def source_digest(src):
    """First 16 hex digits of sha256 over csrc/<src>, csrc/common.cuh and csrc/internal.h."""
    import hashlib
    h = hashlib.sha256()
    for name in (src, "common.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_2605_19388_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_inst(workload, kernel, form):
    ent = NCU_INST.get(workload, {}).get((kernel, form))
    if ent is None:
        return None
    n, src, digest = ent
    return n if source_digest(src) == digest else None


def issue_peak_ginst(sm_count):
    """Warp instructions per second, in G: SMs x 4 schedulers x 1 per clock x the maximum SM clock."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mhz = float(json.load(fh)["sm_max_mhz"])
    except Exception:
        mhz = 2070.0
    return sm_count * 4 * mhz * 1e6 / 1e9, mhz


def ncu_traffic(workload, kernel, form):
    ent = NCU_TRAFFIC.get(workload, {}).get(kernel)
    if ent is None or (kernel in ("k_pstats", "k_vtc") and form != "bf16tc"):  # captured in the bfloat16 form
        return None
    nbytes, src, digest = ent
    return nbytes if source_digest(src) == digest else None


def iteration_bytes(F, T, M, N):
    """B_alg = 28 F T M + 56 F T N: bytes of one MM iteration with each kernel's operands read once."""
    return 28 * F * T * M + 56 * F * T * N


# ------------------------------------------------------ replicas (N > 1)
def ranks_max(v: float, device) -> float:
    """Largest value over the ranks of the default process group (v itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(max_ms: float, world: int, iters: int, steps: int) -> float:
    """Whole-job MM iterations/s: every rank runs its own mixture for `steps` steps of `iters`
    iterations; the job takes the slowest rank's time."""
    return world * iters * steps / (max_ms / 1000.0)


# --------------------------------------------------------- CPU oracle arm
def run_oracle_sample(workload: str, seconds: float, max_iters: int = 1000) -> dict:
    """Time the FP64 oracle (single thread) for about `seconds` of MM iterations."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
import oracle as O
from paper_2605_19388_gb300 import synth
p = synth.make_workload({workload!r}, seed=0)
x = p.x.astype(np.complex128)
st = O.state_from_arrays(p.Q0, p.W0, p.H0, p.g0, p.mics)
t0 = time.perf_counter(); n = 0
while True:
    st = O.mm_iteration(x, p.mics, st); n += 1
    el = time.perf_counter() - t0
    if el >= {seconds} or n >= {max_iters}:
        break
print(json.dumps(dict(iters=n, seconds=el)))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=10 * seconds + 300)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_sample_allcores(workload: str, seconds: float, workers: int | None = None) -> dict:
    """Time the FP64 oracle's MM iterations on every host core for about `seconds`: its bins are split into
    one contiguous slice per core, each slice iterated by the oracle's own functions in a worker process,
    the Eq. 9 sum over bins added in the parent (oracle/parallel.py).  One warm-up iteration is untimed."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle as O
    from oracle.parallel import SlicedOracle
    from paper_2605_19388_gb300 import synth
    p = synth.make_workload(workload, seed=0)
    workers = workers or os.cpu_count() or 1
    st = O.state_from_arrays(p.Q0, p.W0, p.H0, p.g0, p.mics)
    with SlicedOracle(p.x.astype(np.complex128), p.mics, st, workers) as so:
        so.iterate(1)
        t0 = time.perf_counter()
        n = 0
        while True:
            so.iterate(1)
            n += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                break
        return {"iters": n, "seconds": el, "workers": so.workers}


def reference_arm(args, rank, world):
    """The FP64 oracle as it stands, on every host core (its bins split over one worker process per core,
    oracle/parallel.py); each step is one MM iteration of the workload, a bounded sample of its
    200-iteration job.  Under torchrun rank 0 alone runs."""
    if rank != 0:
        return
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle as O
    from oracle.parallel import SlicedOracle
    from paper_2605_19388_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    F, T, M = w["F"], w["T"], sum(w["mics"])
    p = synth.make_workload(args.workload, seed=0)
    st = O.state_from_arrays(p.Q0, p.W0, p.H0, p.g0, p.mics)
    workers = os.cpu_count() or 1
    times = []
    with SlicedOracle(p.x.astype(np.complex128), p.mics, st, workers) as so:
        for _ in range(args.warmup):
            so.iterate(1)
        for _ in range(args.steps):
            t0 = time.perf_counter()
            so.iterate(1)
            times.append(time.perf_counter() - t0)
        workers = so.workers
    total = sum(times)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded STFT mixtures, stand-in for the paper's simulated JNAS rooms)",
        "config": {"workload": args.workload, "F": F, "T": T, "mics": list(w["mics"]), "N": w["N"],
                   "B": w["B"], "step": "one MM iteration of the FP64 oracle (bounded sample of the 200-iteration job)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": f"{args.steps} MM iterations of the {args.workload} workload, one per step, "
                                   f"its bins split over {workers} worker processes, one thread each"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "tf_bin_mic_updates_per_s": F * T * M * value,
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------- gradient through unrolled iterations
def adjoint_measurement(D, synth, torch, timed):
    """Reverse pass through 20 iterations of the FP32 form, checkpoints every 5, on 4 x 4 mics, N = 5,
    B = 16, F = 257, T = 313 (seeded), for Eq. 12 and for the Wiener-filter MSE against the seeded images.
    Each timed gradient runs the 20 forward iterations, the loss, the reverse sweep with its
    recomputation, and copies the gradients to device arrays; the forward alone (the state reset and
    20 iterations) is timed beside it."""
    import numpy as np
    p = synth.make_problem(257, 313, (4, 4, 4, 4), 5, 16, seed=27, with_images=True)
    dev = torch.device("cuda")
    x, W0, H0, g0 = (torch.from_numpy(a).to(dev) for a in (p.x, p.W0, p.H0, p.g0))
    Q0 = torch.from_numpy(p.Q0).to(dev)
    ct = torch.from_numpy(p.c).to(dev)
    ctx = D.dfmnmf_init(p.F, p.T, p.mics, p.N, p.B, x, W0, H0, g0, Q0)
    adj = D.dfmnmf_adjoint_create(ctx, 20, 5)
    dQ = torch.empty_like(Q0)
    dW, dH, dg = (torch.empty(a.shape, dtype=torch.float64, device=dev) for a in (W0, H0, g0))
    out = {"workload": "diff_4x4_n5_f257_t313", "n_iter": 20, "every": 5, "form": "fp32",
           "note": "ms_per_gradient: forward iterations + loss + reverse sweep with segment recomputation; "
                   "forward_ms: state reset + the same 20 iterations"}

    def fwd(_):
        D.dfmnmf_set_params(ctx, Q0, W0, H0, g0)
        D.dfmnmf_iterate(ctx, 20)

    for name, code in (("nll", D.DFMNMF_LOSS_NLL), ("wiener_mse", D.DFMNMF_LOSS_WIENER_MSE)):
        def grad(_):
            D.dfmnmf_set_params(ctx, Q0, W0, H0, g0)
            D.dfmnmf_adjoint_run(adj, code, ct if code == D.DFMNMF_LOSS_WIENER_MSE else None, dQ, dW, dH, dg)

        for _ in range(2):
            grad(None)
        out[name] = {"ms_per_gradient": timed(grad, None, 5) / 5}
    for _ in range(2):
        fwd(None)
    out["forward_ms"] = timed(fwd, None, 5) / 5
    out["nll"]["ratio_to_forward"] = out["nll"]["ms_per_gradient"] / out["forward_ms"]
    D.dfmnmf_adjoint_destroy(adj)
    D.dfmnmf_destroy(ctx)
    return out


# ----------------------------------------------------------- batched form
def batched_measurement(args, D, synth, torch, dev, timed, precision, ip):
    """args.batched mixtures: T ~ U[150, 1250], K in {2, 4, 8} subarrays of 4 mics, N in {3, 5, 8}, F = 513,
    B = 16, seeded.  The observations are the first T frames of one generated mixture per (K, N) pair (the
    generator's cost grows with T; the values do not change the work).  Each context's launch shapes come
    from dfmnmf_autotune; the batch advances all mixtures with one graph launch per iteration.  Reported:
    aggregate TF-bin.mic updates/s, against the same contexts iterated one after another."""
    import numpy as np
    rng = np.random.default_rng(2026)
    n = args.batched
    Ts = rng.integers(150, 1251, size=n)
    Ks = rng.choice([2, 4, 8], size=n)
    Ns = rng.choice([3, 5, 8], size=n)
    F, B, iters = 513, 16, 20
    base = {}
    for K, N in sorted(set(zip(Ks.tolist(), Ns.tolist()))):
        base[(K, N)] = synth.make_problem(F, int(Ts.max()), (4,) * K, N, B, seed=100 + 10 * K + N)
    ctxs, tune, forms_used = [], {}, {}
    for T, K, N in zip(Ts.tolist(), Ks.tolist(), Ns.tolist()):
        p = base[(K, N)]
        x = np.ascontiguousarray(p.x[:, :T])
        H0 = np.ascontiguousarray(p.H0[:, :, :T])
        # tensor-core covariances where the subarrays are underdetermined (N >= 4 sources for 4 microphones);
        # determined ones keep the float-float covariances (their V reach cond 1e6..1e8)
        prec = precision if (precision != D.DFMNMF_BF16_TC or N >= 4) else D.DFMNMF_FP32
        forms_used[prec] = forms_used.get(prec, 0) + 1
        c = D.dfmnmf_init(F, T, (4,) * K, N, B, x, p.W0, H0, p.g0, None, precision=prec, ip_arith=ip)
        shape = D.dfmnmf_autotune(c, 3)
        tune[str(shape)] = tune.get(str(shape), 0) + 1
        ctxs.append(c)
    batch = D.dfmnmf_batch_create(ctxs)
    work = float(sum(F * T * 4 * K for T, K in zip(Ts.tolist(), Ks.tolist()))) * iters  # TF-bin.mic updates per step

    def step_batch(_):
        D.dfmnmf_batch_iterate(batch, iters)

    def step_loop(_):
        for c in ctxs:
            D.dfmnmf_iterate(c, iters)

    for _ in range(2):
        step_batch(None)
        step_loop(None)
    torch.cuda.synchronize()
    nsteps = max(2, args.steps // 2)
    tb = timed(step_batch, None, nsteps)
    tl = timed(step_loop, None, nsteps)
    res = {"mixtures": n, "iters_per_step": iters, "unit": "TF-bin.mic updates/s",
           "value": work * nsteps / (tb / 1000.0), "loop_value": work * nsteps / (tl / 1000.0),
           "speedup_vs_loop": tl / tb, "ms_per_step": tb / nsteps, "loop_ms_per_step": tl / nsteps,
           "mm_iter_per_s_aggregate": n * iters * nsteps / (tb / 1000.0),
           "T_range": [int(Ts.min()), int(Ts.max())], "launch_shapes": tune,
           "forms": {("bf16tc" if k == D.DFMNMF_BF16_TC else "fp32"): v for k, v in forms_used.items()},
           "note": "per-mixture launch loop = the same contexts' graphs launched one after another on one stream"}
    del batch
    for c in ctxs:
        D.dfmnmf_destroy(c)
    return res


# ------------------------------------------- all-microphone comparator at M = 32
def allmic32_measurement(args, D, synth, torch, timed, precision, ip):
    """One mixture of the batched workload's largest layout (K = 8 subarrays x 4 mics, M = 32, N = 5, B = 16,
    F = 513, T = 626): the distributed form (headline precision, 8 diagonalisers of 4 x 4 per bin) against
    conventional all-microphone FastMNMF (K = 1, one 32 x 32 diagonaliser per bin, float-float covariances
    and IP solves: its covariances are far too ill-conditioned for the tensor-core split operands), each
    timed as 10 captured iterations per step."""
    import numpy as np
    F, T, N, B, iters = 513, 626, 5, 16, 10
    p = synth.make_problem(F, T, (4,) * 8, N, B, seed=77)
    res = {"workload": "F=513, T=626, M=32 (8 x 4 mics), N=5, B=16", "iters_per_step": iters,
           "unit": "MM iter/s"}
    for name, mics, prec in (("distributed_8x4", (4,) * 8, precision), ("allmic_32", (32,), D.DFMNMF_FP32)):
        Q0 = torch.from_numpy(synth.identity_blocks(F, mics)).cuda()
        W0, H0, g0 = (torch.from_numpy(a).cuda() for a in (p.W0, p.H0, p.g0))
        c = D.dfmnmf_init(F, T, mics, N, B, p.x, p.W0, p.H0, p.g0, Q0, precision=prec, ip_arith=ip)

        def step(_, c=c, st=(Q0, W0, H0, g0)):
            D.dfmnmf_set_params(c, *st)  # device to device
            D.dfmnmf_iterate(c, iters)

        for _ in range(2):
            step(None)
        torch.cuda.synchronize()
        nsteps = 3
        ms = timed(step, None, nsteps)
        nll = D.dfmnmf_loglik(c)
        res[name] = {"value": iters * nsteps / (ms / 1000.0), "ms_per_iter": ms / (nsteps * iters),
                     "tf_bin_mic_updates_per_s": F * T * 32 * iters * nsteps / (ms / 1000.0), "nll_after": nll,
                     "launches_per_iter": D.dfmnmf_launches_per_iteration(c)}
        D.dfmnmf_destroy(c)
    res["distributed_vs_allmic"] = res["distributed_8x4"]["value"] / res["allmic_32"]["value"]
    return res


# ---------------------------------------------------------------- our arm
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    from paper_2605_19388_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
        dist.barrier()
    from paper_2605_19388_gb300 import dfmnmf as D
    from paper_2605_19388_gb300 import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.adjoint_only:
        def timed_plain(fn, c, nsteps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(nsteps):
                fn(c)
            e1.record()
            e1.synchronize()
            return e0.elapsed_time(e1)
        if rank == 0:
            print(json.dumps({"adjoint": adjoint_measurement(D, synth, torch, timed_plain)}), flush=True)
        return
    ip = {"f32x2": D.DFMNMF_IP_F32X2, "f64": D.DFMNMF_IP_F64, "f32": D.DFMNMF_IP_F32}[args.ip]
    wl = synth.WORKLOADS[args.workload]
    iters = args.iters or wl["iters"]
    p = synth.make_workload(args.workload, seed=rank)
    F, T, M, N, Bb, K, MK = p.F, p.T, p.M, p.N, p.B, p.K, p.mics[0]

    x_d = torch.from_numpy(p.x).to(dev)
    W0_d, H0_d, g0_d = (torch.from_numpy(a).to(dev) for a in (p.W0, p.H0, p.g0))
    Q0_d = torch.from_numpy(p.Q0).to(dev)
    c_out = torch.empty((N, F, T, M), dtype=torch.complex64, device=dev)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    precisions = {"bf16tc": D.DFMNMF_BF16_TC, "tf32tc": D.DFMNMF_TF32_TC, "fp32": D.DFMNMF_FP32,
                  "allmic": D.DFMNMF_FP32}
    # conventional all-microphone FastMNMF on the same observation: one 16 x 16 block per bin
    allmic = (M,)
    Q0_all_d = torch.from_numpy(synth.identity_blocks(F, allmic)).to(dev)
    form_mics = {"bf16tc": p.mics, "tf32tc": p.mics, "fp32": p.mics, "allmic": allmic}
    form_q0 = {"bf16tc": Q0_d, "tf32tc": Q0_d, "fp32": Q0_d, "allmic": Q0_all_d}
    ctx_q0 = {}
    shapes = {}
    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    nll_box = []

    def step(c):
        D.dfmnmf_set_observation(c, x_d)          # observation in place (TC form: x x^H split anew)
        D.dfmnmf_set_params(c, ctx_q0.get(id(c), Q0_d), W0_d, H0_d, g0_d)
        D.dfmnmf_iterate(c, iters)
        nll_box.append(D.dfmnmf_loglik(c))
        D.dfmnmf_separate(c, c_out)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(fn, c, nsteps):
        tot = 0.0
        for _ in range(nsteps):
            flush_buf.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(c)
            e1.record()
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot

    def max_over_ranks(v):
        return ranks_max(v, dev)

    kb_form = {f: (kernel_bytes(F, T, M, N, Bb, 1, M) if f == "allmic" else kernel_bytes(F, T, M, N, Bb, K, MK))
               for f in forms}
    kb = kb_form[forms[0]]
    peak, peak_kind = peaks()
    ib = iteration_bytes(F, T, M, N)
    results = {}
    ctxs = {}
    clocks = None
    for form in forms:
        c = D.dfmnmf_init(F, T, form_mics[form], N, Bb, x_d, W0_d, H0_d, g0_d, form_q0[form], ip_arith=ip,
                          precision=precisions[form])
        ctx_q0[id(c)] = form_q0[form]
        ctxs[form] = c
        shapes[form] = D.dfmnmf_autotune(c, 5)  # launch shapes measured on this context (state restored)
        for _ in range(args.warmup):
            step(c)
        torch.cuda.synchronize()
        sampler = ClockSampler(local if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
        barrier()
        torch.cuda.synchronize()
        sampler.start()
        total_ms = timed(step, c, args.steps)
        torch.cuda.synchronize()
        barrier()
        ck = sampler.stop()
        total_ms = max_over_ranks(total_ms)
        launches_iter = D.dfmnmf_launches_per_iteration(c)
        # steady-state iteration time of the captured graph (back-to-back launches)
        D.dfmnmf_set_params(c, form_q0[form], W0_d, H0_d, g0_d)
        D.dfmnmf_iterate(c, 5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        D.dfmnmf_iterate(c, 50)
        e1.record()
        e1.synchronize()
        graph_iter_ms = e0.elapsed_time(e1) / 50
        # per-kernel times: the same iteration replayed as a linear graph with an event after every kernel
        kt = D.dfmnmf_kernel_times(c, 50)
        seen = {}
        kt_u = []
        for name, ms in kt:  # a kernel launched twice per iteration gets a suffix the second time
            seen[name] = seen.get(name, 0) + 1
            kt_u.append((name if seen[name] == 1 else f"{name}#{seen[name]}", ms))
        kt = kt_u
        iter_ms = sum(ms for _, ms in kt)
        # each kernel alone, 20 launches back to back in one graph between two events: its launch duration
        # without the timing event that the in-iteration replay puts after every kernel (which adds a few us
        # to each); the state is reset by the next step's set_params
        ki = D.dfmnmf_kernel_times_isolated(c, 20)
        seen, ki_u = {}, []
        for name, ms in ki:
            seen[name] = seen.get(name, 0) + 1
            ki_u.append((name if seen[name] == 1 else f"{name}#{seen[name]}", ms))
        dom_name, dom_ms = max(ki_u, key=lambda e: e[1])
        results[form] = dict(
            value=replica_value(total_ms, world, iters, args.steps), ms_per_step=total_ms / args.steps,
            launches_iter=launches_iter, kernels=kt, kernels_isolated=ki_u, iter_ms=iter_ms,
            graph_iter_ms=graph_iter_ms, dominant=(dom_name, dom_ms),
            nll=nll_box[-1], clocks=ck)
        if clocks is None:
            clocks = ck
    head = results[forms[0]]
    dom_name, dom_ms = head["dominant"]
    base = lambda n: n.split("#")[0]

    def hbm_roofline(name, ms):
        ach = kb[base(name)] / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": ncu_traffic(args.workload, base(name), forms[0]),
                "peak_kind": f"{peak_kind} hbm_gbs (burst copy)", "alg_bytes_per_launch": kb[base(name)],
                "launch_ms": ms, "timing": "CUDA events around 20 launches of this kernel alone in one graph"}

    if base(dom_name) in ALU_KERNELS:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        ipeak, mhz = issue_peak_ginst(sms)
        inst = ncu_inst(args.workload, base(dom_name), forms[0])
        ach = inst / (dom_ms * 1e-3) / 1e9 if inst else None
        roofline = {"bound": "alu", "kernel": dom_name, "achieved": ach, "peak": ipeak,
                    "unit": "G warp-instructions/s", "frac": (ach / ipeak) if ach else None,
                    "traffic": ncu_traffic(args.workload, base(dom_name), forms[0]),
                    "peak_kind": f"derived: {sms} SMs x 4 schedulers x 1 warp-instruction/clock x {mhz:.0f} MHz",
                    "instructions_per_launch": inst}
    else:
        roofline = hbm_roofline(dom_name, dom_ms)
    hbm_kernels = [(n, ms) for n, ms in head["kernels_isolated"] if base(n) not in ALU_KERNELS]
    roofline_hbm = hbm_roofline(*max(hbm_kernels, key=lambda e: e[1]))

    def kernel_table(kt, iter_ms, kbf=None):
        kbf = kb if kbf is None else kbf
        return {n: {"ms": ms, "share": ms / iter_ms, "alg_bytes": kbf.get(base(n)),
                    "GBps": (kbf[base(n)] / (ms * 1e-3) / 1e9) if base(n) in kbf else None} for n, ms in kt}

    launches_step = iters * head["launches_iter"] + 2 + 3 + 2
    out = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("bf16x3 tensor-core covariances, f32 updates, f32x2 IP" if forms[0] == "bf16tc"
                  else "f32 (float-float covariances, f32x2 IP)"),
        "data": "synthetic (seeded STFT mixtures, stand-in for the paper's simulated JNAS rooms)",
        "config": {"workload": args.workload, "F": F, "T": T, "mics": list(p.mics), "N": N, "B": Bb,
                   "iters_per_step": iters, "form": forms[0], "ip_arith": args.ip,
                   "step": "observation + state reset, iterations, loglik (D2H), Wiener filter",
                   "l2": "flushed before every timed step (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "tf_bin_mic_updates_per_s": F * T * M * head["value"],
        "roofline": roofline,
        "roofline_hbm": roofline_hbm,
        "iteration": {"ms": head["graph_iter_ms"], "alg_bytes": ib,
                      "GBps": ib / (head["graph_iter_ms"] * 1e-3) / 1e9,
                      "frac_of_hbm_peak": ib / (head["graph_iter_ms"] * 1e-3) / 1e9 / peak,
                      "kernel_sum_ms": head["iter_ms"], "launches": head["launches_iter"],
                      "note": "ms: captured iteration graph replayed back to back (L2 warm); kernel_sum_ms: "
                              "the per-kernel event times below, band-wide launches in order"},
        "kernels": kernel_table(head["kernels"], head["iter_ms"]),
        "kernels_isolated": {"note": "each kernel alone, 20 launches back to back between two events (the "
                                     "roofline's launch duration); the table above times them inside the "
                                     "iteration with an event after every kernel",
                             **kernel_table(head["kernels_isolated"],
                                            sum(ms for _, ms in head["kernels_isolated"]))},
        "forms": {f: {"value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
                      "launch_shapes": {"branches": shapes[f][0], "nmf_ctas_per_sm": shapes[f][1]},
                      "iter_ms": r["graph_iter_ms"], "kernel_sum_ms": r["iter_ms"],
                      "kernels": kernel_table(r["kernels"], r["iter_ms"], kb_form[f]), "nll_last": r["nll"],
                      "clocks": r["clocks"]} for f, r in results.items()},
        "clocks": clocks,
        "distributed_vs_allmic": (results[forms[0]]["value"] / results["allmic"]["value"]) if "allmic" in results else None,
        "gpu_launches": launches_step * args.steps,
        "nll_last": head["nll"],
    }
    ctx = ctxs[forms[0]]

    # end to end through the public API with host buffers (pinned): the observation and the initial state
    # go in, the separated images (Wiener filter output) and the final state come back, every step
    if not args.no_e2e:
        xh = torch.from_numpy(p.x).pin_memory()
        W0h, H0h, g0h = (torch.from_numpy(a).pin_memory() for a in (p.W0, p.H0, p.g0))
        Q0h = torch.from_numpy(p.Q0).pin_memory()
        c_h = torch.empty((N, F, T, M), dtype=torch.complex64).pin_memory()
        Q_h = torch.empty_like(Q0h).pin_memory()
        W_h, H_h, g_h = (torch.empty_like(a).pin_memory() for a in (W0h, H0h, g0h))
        nll_e2e = []

        def step_e2e(c):
            D.dfmnmf_set_observation(c, xh)           # pinned host -> device, inside the timed region
            D.dfmnmf_set_params(c, Q0h, W0h, H0h, g0h)
            D.dfmnmf_iterate(c, iters)
            nll_e2e.append(D.dfmnmf_loglik(c))        # Eq. 12 to the host (synchronises)
            D.dfmnmf_separate(c, c_out)
            c_h.copy_(c_out, non_blocking=True)       # separated images, device -> pinned host
            D.dfmnmf_get_params(c, Q_h, W_h, H_h, g_h)  # final state, device -> pinned host

        for _ in range(2):
            step_e2e(ctx)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = timed(step_e2e, ctx, args.steps)
        barrier()
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        h2d = xh.numel() * 8 + (W0h.numel() + H0h.numel() + g0h.numel()) * 4 + Q0h.numel() * 16
        d2h = (8 + 16 + c_h.numel() * 8 + Q_h.numel() * 16 + (W_h.numel() + H_h.numel() + g_h.numel()) * 4)
        out["e2e"] = {"value": replica_value(e2e_ms, world, iters, args.steps), "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "ms_per_step": e2e_ms / args.steps,
                      "d2h": "the cost (8 B) and device flags (16 B), the separated images complex64 [N][F][T][M], "
                             "the final Q, W, H and g"}

    # independent mixtures of the same shape run concurrently, one stream and one context each
    if args.concurrent > 1:
        nmix = args.concurrent
        cctx, cstreams, couts = [], [], []
        for _ in range(nmix):
            cctx.append(D.dfmnmf_init(F, T, p.mics, N, Bb, x_d, W0_d, H0_d, g0_d, Q0_d, ip_arith=ip,
                                      precision=precisions[forms[0]]))
            cstreams.append(torch.cuda.Stream(device=dev))
            couts.append(torch.empty((N, F, T, M), dtype=torch.complex64, device=dev))

        def step_many(_):
            cur = torch.cuda.current_stream()
            start = torch.cuda.Event()
            start.record(cur)
            for c, st in zip(cctx, cstreams):
                st.wait_event(start)
                D.dfmnmf_set_observation(c, x_d, stream=st)
                D.dfmnmf_set_params(c, Q0_d, W0_d, H0_d, g0_d, stream=st)
                D.dfmnmf_iterate(c, iters, stream=st)
            for c, st, co in zip(cctx, cstreams, couts):
                D.dfmnmf_loglik(c, stream=st)
                D.dfmnmf_separate(c, co, stream=st)
                ev = torch.cuda.Event()
                ev.record(st)
                cur.wait_event(ev)

        for _ in range(2):
            step_many(None)
        torch.cuda.synchronize()
        barrier()
        many_ms = max_over_ranks(timed(step_many, None, max(2, args.steps // 2)))
        n_many = max(2, args.steps // 2)
        val = world * nmix * iters * n_many / (many_ms / 1000.0)
        out["concurrent"] = {"mixtures": nmix, "value": val, "unit": UNIT, "ms_per_step": many_ms / n_many,
                             "tf_bin_mic_updates_per_s": F * T * M * val,
                             "alg_GBps_per_iteration_bytes": ib * val / world / 1e9,
                             "frac_of_hbm_peak": ib * val / world / 1e9 / peak}
        for c in cctx:
            D.dfmnmf_destroy(c)

    # many mixtures of uneven length and layout, one graph launch per iteration, launch shapes autotuned
    if args.batched > 0 and world == 1:
        out["batched"] = batched_measurement(args, D, synth, torch, dev, timed, precisions[forms[0]], ip)
        out["allmic32"] = allmic32_measurement(args, D, synth, torch, timed, precisions[forms[0]], ip)

    if not args.no_adjoint and world == 1:
        out["adjoint"] = adjoint_measurement(D, synth, torch, timed)

    # variants on the same GPU: native-FP64 and plain-FP32 IP solves (FP32 form), and the tensor-core form
    # with native-FP64 IP solves (the headline tensor-core form solves in float pairs)
    if not args.no_variants:
        var = {}
        for name, ipv, prec, wtc in (("ip_f64", D.DFMNMF_IP_F64, D.DFMNMF_FP32, 0),
                                     ("ip_f32", D.DFMNMF_IP_F32, D.DFMNMF_FP32, 0),
                                     ("bf16tc_ip_f64", D.DFMNMF_IP_F64, D.DFMNMF_BF16_TC, 0),
                                     ("bf16tc_wupd_tc", ip, D.DFMNMF_BF16_TC, 1)):
            if ipv == ip and prec == precisions[forms[0]] and not wtc:
                continue
            c2 = D.dfmnmf_init(F, T, p.mics, N, Bb, x_d, W0_d, H0_d, g0_d, Q0_d, ip_arith=ipv, precision=prec)
            D.dfmnmf_autotune(c2, 3)
            if wtc:  # W-update products on the tensor cores (tcgen05 kind::tf32) instead of the CUDA cores
                D.dfmnmf_set_option(c2, D.DFMNMF_OPT_WUPD_TC, 1)
            for _ in range(2):
                step(c2)
            ms = timed(step, c2, max(2, args.steps // 2))
            n2 = max(2, args.steps // 2)
            var[name] = {"value": world * iters * n2 / (ms / 1000.0), "unit": UNIT,
                         "form": "bf16tc" if prec == D.DFMNMF_BF16_TC else "fp32",
                         "ip_arith": {D.DFMNMF_IP_F64: "f64", D.DFMNMF_IP_F32: "f32",
                                      D.DFMNMF_IP_F32X2: "f32x2"}[ipv],
                         "nll_last": nll_box[-1],
                         "k_ip_ms": dict(D.dfmnmf_kernel_times(c2, 10)).get("k_ip"),
                         "w_update_ms": {k: v for k, v in D.dfmnmf_kernel_times(c2, 10)
                                         if k.startswith(("k_wupd", "k_wlam")) or k == "k_lambda"}}
            D.dfmnmf_destroy(c2)
        out["variants"] = var

    if rank == 0 and world == 1 and not args.no_cpu:
        s = run_oracle_sample(args.workload, args.cpu_seconds)
        sa = run_oracle_sample_allcores(args.workload, args.cpu_seconds)
        out["cpu_baseline"] = {
            "value": sa["iters"] / sa["seconds"], "unit": UNIT, "cores": sa["workers"], "kind": "oracle",
            "sample": f"{sa['iters']} MM iterations of the FP64 oracle on the same workload ({sa['seconds']:.1f} s), "
                      f"its bins split over {sa['workers']} worker processes, one thread each",
            "single_thread": {"value": s["iters"] / s["seconds"], "unit": UNIT, "cores": 1,
                              "sample": f"{s['iters']} MM iterations of the FP64 oracle ({s['seconds']:.1f} s, "
                                        f"one thread)"}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
