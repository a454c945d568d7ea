"""Plan checkpoints: zl_plan_save / zl_plan_load restore a plan whose applies give the
saved plan's bits, and reject malformed files before any device work."""

import os

import numpy as np
import pytest

from oracle import basis
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")

CASES = [
    (synth.Workload("io_fp64", 24, 20, 6, 9, 3.0, 0.6, 3.0, 5, "fp64", 65), "fp64"),
    (synth.Workload("io_fp32", 32, 24, 10, 32, 4.0, 0.7, 3.0, 7, "fp32", 66), "fp32"),
    (synth.Workload("io_mixed", 32, 24, 16, 40, 4.0, 0.7, 3.0, 9, "mixed", 67), "mixed"),
]


@pytest.fixture(scope="module")
def zl():
    from paper_2609_13327_b300 import zl as mod
    return mod


@pytest.mark.gpu
@pytest.mark.parametrize("w,prec", CASES, ids=[p for _, p in CASES])
def test_saved_plan_gives_the_same_bits(zl, w, prec, tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dt = synth.storage_dtype(prec)
    Z = torch.from_numpy(synth.ensemble(w).astype(dt)).cuda()
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(Z, lam, tau=w.tau, prec=prec, max_rhs=w.R, nx=w.Nx, ny=w.Ny)
    path = str(tmp_path / "plan.zl")
    zl.zl_plan_save(plan, path)
    back = zl.zl_plan_load(path)
    assert (back.L, back.nw, back.K, back.nh, back.nx, back.ny, back.prec) == \
        (plan.L, plan.nw, plan.K, plan.nh, plan.nx, plan.ny, plan.prec)
    assert np.array_equal(back.modes(), plan.modes())
    assert back.uses_tc() == plan.uses_tc()
    x = torch.from_numpy(synth.rhs(w, dtype=dt)).cuda()
    xt = torch.from_numpy(synth.coefficients(w, plan.L, dtype=dt)).cuda()
    for fn, v in ((zl.zl_apply_left_inverse, x), (zl.zl_apply_sqrt, xt), (zl.zl_apply_adjoint, xt),
                  (zl.zl_apply_sqrt_adjoint, x)):
        assert torch.equal(fn(plan, v), fn(back, v)), fn.__name__


def test_malformed_files_are_rejected_before_device_work(zl, tmp_path):
    import ctypes
    h = ctypes.c_void_p(123)
    lib = zl._lib
    assert lib.zl_plan_load(os.fsencode(str(tmp_path / "missing")), None, ctypes.byref(h)) == zl.ZL_ERR_ARG
    assert h.value is None
    bad = tmp_path / "bad"
    bad.write_bytes(b"NOTAPLAN" + b"\0" * 64)
    assert lib.zl_plan_load(os.fsencode(str(bad)), None, ctypes.byref(h)) == zl.ZL_ERR_ARG
    short = tmp_path / "short"
    short.write_bytes(b"ZLPLAN1\0" + b"\0" * 8)
    assert lib.zl_plan_load(os.fsencode(str(short)), None, ctypes.byref(h)) == zl.ZL_ERR_ARG
    assert lib.zl_plan_load(None, None, ctypes.byref(h)) == zl.ZL_ERR_ARG
    assert lib.zl_plan_save(None, os.fsencode(str(bad))) == zl.ZL_ERR_ARG
