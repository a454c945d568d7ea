"""Standardized forecast ensemble (Sec. 2.1-2.2): zl_standardize_ensemble against the FP64
oracle applied to the centred, scaled members, in every precision.  The members carry a
common offset field, which the centring must remove exactly; the output's member mean is
zero to rounding."""

import numpy as np
import pytest

from oracle import basis, compare, swift
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    (synth.WORKLOADS["c0a_plane"], "fp64", 1e-10),
    (synth.Workload("ens_fp32", 32, 20, 10, 32, 4.0, 0.7, 4.0, 9, "fp32", 71), "fp32", 1e-6),
    (synth.Workload("ens_mixed", 48, 40, 32, 64, 8.0, 0.8, 6.0, 13, "mixed", 72, var_range=(0.1, 10.0)), "mixed", 1e-5),
]


@pytest.fixture(scope="module")
def zl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_13327_b300 import zl as mod
    return mod


@pytest.mark.parametrize("w,prec,tol", CASES, ids=[c[1] for c in CASES])
def test_standardized_forecast_ensemble(zl, w, prec, tol):
    dt = synth.storage_dtype(prec)
    Z = synth.ensemble(w).astype(dt)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec=prec, max_rhs=8, nx=w.Nx, ny=w.Ny)
    if prec == "mixed":
        assert plan.uses_tc()
    Kf = 20                                                   # more members than max_rhs: passes
    offset = 3.0 * synth.rhs(w, R=1, seed=w.seed + 5)[0]
    members = (synth.rhs(w, R=Kf, seed=w.seed + 6) + offset[None]).astype(dt)
    out = zl.zl_standardize_ensemble(plan, torch.from_numpy(members).cuda()).cpu().numpy().astype(np.float64)
    oracle = swift.Plan(Z.astype(np.float64), w.Nx, w.Ny, lam, w.tau)
    m = members.astype(np.float64)
    ref = swift.apply_left_inverse(oracle, (m - m.mean(axis=0, keepdims=True)) / np.sqrt(Kf - 1))
    compare.check(out, ref, tol, 2, f"standardized ensemble {prec}")
    assert np.abs(out.mean(axis=0)).max() <= 1e-6 * np.abs(out).max()


def test_too_few_members_rejected(zl):
    w = synth.WORKLOADS["c0a_plane"]
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(synth.ensemble(w)).cuda(), lam, tau=w.tau, prec="fp64", max_rhs=4,
                       nx=w.Nx, ny=w.Ny)
    one = torch.zeros((1, w.nw, w.nh), dtype=torch.float64, device="cuda")
    out = torch.zeros((1, plan.K, plan.L), dtype=torch.float64, device="cuda")
    assert zl._lib.zl_standardize_ensemble(plan.handle, zl._vp(one.data_ptr()), zl._vp(out.data_ptr()), 1, None) \
        == zl.ZL_ERR_ARG
