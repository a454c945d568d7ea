"""The y-slab partition of the left inverse (a multi-GPU layout in which each rank owns a
slab of grid rows and one all-reduce of K L partial sums per right-hand side joins them),
exercised on three gloo CPU ranks (uneven slabs of 5, 5 and 4 rows) with the FP64 oracle's building blocks: each rank touches
only its own rows, and the reduced result equals the whole-grid oracle."""

import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slab_partial_sums_all_reduce_to_the_whole_grid_left_inverse():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=3",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "tests", "gloo_slab_ranks.py")]
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert [l["case"] for l in lines] == ["slab_wide", "slab_tall"]
    for l in lines:
        assert l["rows"] == [[0, 5], [5, 10], [10, 14]]    # every row in exactly one slab, uneven
        assert l["err"] <= 1e-12, l
