"""Host-side logic of bench.py (no GPU): the algorithmic byte counts behind
the roofline, the rule that ties stored ncu traffic to the captured sources,
the whole-job throughput, the clock and throttle-reason parsing that decides
whether a run is kept, and the JSON line of the reference arm (the FP64
oracle on the host cores) on the small workload."""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

# the paper-sized workload: 4 subarrays x 4 mics, N = 5, B = 16, F = 513, T = 626
F, T, K, MK, N, B = 513, 626, 4, 4, 5, 16
M = K * MK


def test_covariance_bytes_are_the_methods_own():
    """Eq. 13 moves x once (complex64), lambda and g once, and V once as complex64."""
    kb = bench.kernel_bytes(F, T, M, N, B, K, MK)
    x = 8 * F * T * M
    lam = 4 * N * F * T
    g = 4 * F * N * M
    v = 8 * F * K * MK ** 3
    assert kb["k_vtc"] == kb["k_cov"] == x + lam + g + v
    assert kb["k_vtc"] == 48_743_208  # 48.7 MB


def test_iteration_bytes_and_the_kernels_of_one_iteration():
    """B_alg = 28 F T M + 56 F T N (233.8 MB here) is the best fused schedule: the
    kernels of the tensor-core iteration, each counted alone, move at least that."""
    ib = bench.iteration_bytes(F, T, M, N)
    assert ib == 28 * F * T * M + 56 * F * T * N == 233_788_464
    kb = bench.kernel_bytes(F, T, M, N, B, K, MK)
    tc_iteration = ("k_vtc", "k_ip", "k_pstats", "k_wlam", "k_stats", "k_hupd", "k_lambda", "k_gupd")
    assert sum(kb[k] for k in tc_iteration) >= ib
    unfused = ("k_vtc", "k_ip", "k_pstats", "k_wupd", "k_lambda", "k_stats", "k_hupd", "k_lambda", "k_gupd")
    assert sum(kb[k] for k in unfused) > sum(kb[k] for k in tc_iteration)  # the fusion saves the W reread


def test_whole_job_throughput_counts_every_rank():
    assert bench.replica_value(2000.0, 1, 200, 30) == pytest.approx(3000.0)
    assert bench.replica_value(2000.0, 4, 200, 30) == pytest.approx(12000.0)


def _fake_root(tmp_path):
    csrc = tmp_path / "paper_2605_19388_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in ("kernels_tc.cu", "common.cuh", "internal.h"):
        shutil.copy(os.path.join(ROOT, "paper_2605_19388_gb300", "csrc", name), csrc / name)
    return csrc


def test_stored_traffic_holds_only_for_the_captured_sources(tmp_path, monkeypatch):
    nbytes, src, digest = bench.NCU_TRAFFIC["paper_4x4_n5"]["k_vtc"]
    real = bench.source_digest(src)
    csrc = _fake_root(tmp_path)
    assert bench_digest(csrc, src) == real  # the copies hash like the sources
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.NCU_TRAFFIC["paper_4x4_n5"], "k_vtc", (nbytes, src, bench_digest(csrc, src)))
    assert bench.ncu_traffic("paper_4x4_n5", "k_vtc", "bf16tc") == nbytes
    assert bench.ncu_traffic("paper_4x4_n5", "k_vtc", "tf32tc") is None  # captured in the bfloat16 form
    assert bench.ncu_traffic("other_workload", "k_vtc", "bf16tc") is None
    with open(csrc / "internal.h", "a") as fh:  # any change to a hashed file voids the figure
        fh.write("\n")
    assert bench.ncu_traffic("paper_4x4_n5", "k_vtc", "bf16tc") is None


def bench_digest(csrc, src):
    import hashlib
    h = hashlib.sha256()
    for name in (src, "common.cuh", "internal.h"):
        h.update((csrc / name).read_bytes())
    return h.hexdigest()[:16]


def test_stored_traffic_is_near_the_algorithmic_bytes():
    """The committed capture of the covariance kernel: DRAM traffic within 5 % of Eq. 13's bytes
    (nothing read twice), and never a figure below what the method must read."""
    nbytes = bench.NCU_TRAFFIC["paper_4x4_n5"]["k_vtc"][0]
    alg = bench.kernel_bytes(F, T, M, N, B, K, MK)["k_vtc"]
    reads_needed = 8 * F * T * M + 4 * N * F * T  # x and lambda must come from DRAM once
    assert reads_needed <= nbytes <= 1.05 * alg


def test_clock_samples_parse_reasons_and_skip_bad_lines():
    lines = [
        "0, 2070, 2070, 912.31, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1398.02, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 1398.02, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, [N/A], 1398.02, 0x0, Active, Not Active, Not Active, Not Active",
        "garbage line",
        "",
        "0, 1890, 2070, 1401.50, 0x0000000000000008, Not Active, Not Active, Active, Not Active",
    ]
    out = bench.parse_clock_samples(lines)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 1980.0
    assert out["sm_max_mhz"] == 2070.0
    # the reason of the skipped line (no numeric maximum clock) is not counted
    assert out["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]
    empty = bench.parse_clock_samples([])
    assert empty == {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "reasons": []}


def test_clock_sampler_runs_the_query_and_parses_its_output(tmp_path, monkeypatch):
    """start() runs nvidia-smi with the sampling loop, stop() ends it and parses what it wrote
    (a stand-in nvidia-smi on PATH prints two samples); without nvidia-smi stop() says so."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 2010, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")
    cs = bench.ClockSampler(0)
    cs.start()
    import time
    for _ in range(100):  # until both samples are on disk
        with open(cs.path) as fh:
            if len(fh.read().splitlines()) >= 2:
                break
        time.sleep(0.05)
    out = cs.stop()
    assert out == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "samples": 2, "reasons": ["sw_power_cap"]}
    assert not os.path.exists(cs.path)
    monkeypatch.setenv("PATH", str(tmp_path / "empty"))
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]
    assert not os.path.exists(cs.path)


def test_cpu_baseline_samples_time_the_oracle():
    """The bench's cpu_baseline legs: the FP64 oracle in a single-thread subprocess, and split over
    worker processes; each reports whole MM iterations and the seconds they took."""
    one = bench.run_oracle_sample("small_2x4_n3", 0.2, max_iters=2)
    assert 1 <= one["iters"] <= 2 and one["seconds"] > 0
    many = bench.run_oracle_sample_allcores("small_2x4_n3", 0.2, workers=2)
    assert many["iters"] >= 1 and many["seconds"] >= 0.2 and many["workers"] == 2


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference`: the FP64 oracle on the host cores, one JSON line carrying the
    metric, unit and direction of the GPU arm, no host-device bytes and no GPU launches."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "small_2x4_n3", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT == "MM iter/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] == pytest.approx(1000.0 / d["value"])
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["gpu_launches"] == 0 and d["dtype"] == "f64"
    assert d["config"]["workload"] == "small_2x4_n3"
    assert (d["config"]["F"], d["config"]["T"], d["config"]["mics"]) == (257, 313, [4, 4])
