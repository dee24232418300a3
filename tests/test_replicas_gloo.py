"""The N > 1 path of bench.py on the CPU: independent replicas, one per rank,
with the job time taken as the slowest rank's (gloo process group, two ranks
on 127.0.0.1), and the reference arm under torchrun (rank 0 alone prints)."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 * (rank + 1)            # rank r took (r + 1) x 100 ms
        m = bench.ranks_max(local_ms, "cpu")
        out[rank] = (m, bench.replica_value(m, world, iters=200, steps=5))
    finally:
        dist.destroy_process_group()


def test_ranks_take_the_slowest_rank_and_count_every_replica():
    world, port = 2, 29517
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        m, v = res[r]
        assert m == 200.0                          # max over ranks, the same on every rank
        assert v == pytest.approx(2 * 200 * 5 / 0.2)  # both replicas' iterations over the slowest time


def test_single_process_without_group_is_identity():
    assert bench.ranks_max(3.5, "cpu") == 3.5
    assert bench.replica_value(1000.0, 1, 10, 2) == pytest.approx(20.0)


@pytest.mark.slow
def test_reference_arm_under_torchrun_two_ranks_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", "29519", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "small_2x4_n3"]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=600,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
