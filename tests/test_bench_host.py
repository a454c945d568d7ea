"""Host logic of bench.py without a GPU: the multi-rank reduction (gloo, two CPU ranks
under torchrun, as a multi-GPU launch runs the bench) and the reference arm, which runs the
FP64 oracle on the host and, under torchrun, prints from rank 0 only."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def torchrun(nproc, *args, timeout=240):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), *args]
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def json_lines(text):
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def test_reduce_max_and_weak_scaling_value_on_two_gloo_ranks():
    r = torchrun(2, os.path.join(ROOT, "tests", "gloo_bench_ranks.py"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert sorted(l["rank"] for l in lines) == [0, 1]
    for l in lines:
        assert l["world"] == 2
        assert l["ms"] == pytest.approx(13.0)                  # the max over ranks, on every rank
        assert l["value"] == pytest.approx(2 * 5 * 4 / 13e-3)   # both ranks' right-hand sides


def test_reduce_max_without_process_group_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    import torch
    assert bench.reduce_max(7.5, torch.device("cpu")) == 7.5
    assert bench.aggregate_value(1, 10, 64, 2.0) == pytest.approx(320.0)


def test_reference_arm_single_rank():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "c1_ring64",
                        "--steps", "3", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=240,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr[-2000:]
    (line,) = json_lines(r.stdout)
    assert line["impl"] == "reference" and line["unit"] == "vectors/s" and line["value"] > 0
    assert line["steps"] == 3 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "vectors/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_under_torchrun_prints_from_rank_zero_only():
    r = torchrun(2, "bench.py", "--impl", "reference", "--workload", "c1_ring64", "--steps", "2", "--warmup", "1",
                 "--gpus", "2")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference"


@pytest.mark.parametrize("ny,world", [(256, 1), (256, 3), (128, 8), (7, 3), (2, 4)])
def test_slab_rows_cover_the_grid_once(ny, world):
    """bench.py --partition slabs: the ranks' row ranges are disjoint, cover 0..ny-1 in order,
    and differ in size by at most one row (a rank may get none when world > ny)."""
    import bench
    cuts = [bench.slab_rows(ny, world, r) for r in range(world)]
    assert cuts[0][0] == 0 and cuts[-1][1] == ny
    for (a0, a1), (b0, b1) in zip(cuts[:-1], cuts[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in cuts]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0
