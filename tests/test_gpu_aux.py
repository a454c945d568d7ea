"""Auxiliary subsystems on the GPU: the allocation-failure hook (every allocation of a
setup made to fail in turn: ZL_ERR_ALLOC, no plan, nothing leaked) and the ZL_LOG lines."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import basis
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
W = synth.Workload("aux_mixed", 32, 24, 16, 40, 4.0, 0.7, 3.0, 9, "mixed", 71)


@pytest.fixture(scope="module")
def zl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_13327_b300 import zl as mod
    return mod


def test_every_setup_allocation_failing_is_reported_and_cleaned_up(zl):
    Z = torch.from_numpy(synth.ensemble(W).astype(np.float32)).cuda()
    lam = basis.spectrum_2d(W.Nx, W.Ny, W.ell_loc)
    ok = zl.zl_setup(Z, lam, tau=W.tau, prec="mixed", max_rhs=W.R, nx=W.Nx, ny=W.Ny)   # loads every module
    assert ok.uses_tc()
    ok.destroy()
    torch.cuda.synchronize()
    free = []
    failures = 0
    try:
        for n in range(1, 80):
            assert zl._lib.zl_set_test_alloc_failure(n) == zl.ZL_OK
            try:
                plan = zl.zl_setup(Z, lam, tau=W.tau, prec="mixed", max_rhs=W.R, nx=W.Nx, ny=W.Ny)
            except zl.ZLError as err:
                assert err.code == zl.ZL_ERR_ALLOC, (n, err)
                failures += 1
                torch.cuda.synchronize()
                free.append(torch.cuda.mem_get_info()[0])
                continue
            plan.destroy()                      # n is past the setup's last allocation
            break
    finally:
        zl._lib.zl_set_test_alloc_failure(0)
    assert failures >= 15                       # plan buffers, tables, tensor-core operands
    assert max(free) - min(free) <= 2 << 20     # repeated failed setups leak nothing
    assert zl._lib.zl_set_test_alloc_failure(-1) == zl.ZL_ERR_ARG


def test_log_lines(tmp_path):
    code = (
        "import numpy as np, torch\n"
        "from oracle import basis\n"
        "from paper_2609_13327_b300 import synth, zl\n"
        "w = synth.Workload('log', 32, 24, 16, 40, 4.0, 0.7, 3.0, 3, 'mixed', 71)\n"
        "Z = torch.from_numpy(synth.ensemble(w).astype(np.float32)).cuda()\n"
        "plan = zl.zl_setup(Z, basis.spectrum_2d(32, 24, 3.0), tau=w.tau, prec='mixed', max_rhs=3, nx=32, ny=24)\n"
        "x = torch.from_numpy(synth.rhs(w, dtype=np.float32)).cuda()\n"
        "xt = zl.zl_apply_left_inverse(plan, x)\n"
        "zl.zl_apply_sqrt(plan, xt)\n"
        "torch.cuda.synchronize()\n")
    env = dict(os.environ, ZL_LOG="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stderr.splitlines() if l.startswith('{"zl"')]
    assert [l["zl"] for l in lines] == ["left_inverse", "sqrt"]
    assert lines[0]["column"] == "tcgen05" and lines[0]["R"] == 3 and lines[0]["K"] == 40
    assert lines[1]["column"] == "cuda-core" and lines[1]["prec"] == "mixed"
