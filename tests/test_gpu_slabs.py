"""The horizontal domain in slabs of grid rows (the paper's parallel decomposition, Sec.
3.10) through the library: each slab's rows of x go through zl_apply_left_inverse_rows,
the partial sums are added (what one all-reduce of K L values per right-hand side does
across GPUs) and scaled by zl_scale_modes.  The result must equal the oracle's left
inverse of the whole grid, on the CUDA-core and the tensor-core kernels, for uneven slabs
(one of them a single row)."""

import numpy as np
import pytest

from oracle import basis, compare, swift
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-6, "mixed": 1e-5}
C2 = synth.WORKLOADS["c2_128x128x10"]


@pytest.fixture(scope="module")
def zl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_13327_b300 import zl as mod
    return mod


CASES = [
    (C2, "fp32", [0, 40, 90, 128]),
    (C2, "mixed", [0, 40, 90, 128]),
    (synth.Workload("slab_fp64", 24, 20, 6, 9, 3.0, 0.6, 3.0, 5, "fp64", 65), "fp64", [0, 1, 13, 20]),
    (synth.Workload("slab_mixed_small", 32, 24, 16, 40, 4.0, 0.7, 3.0, 19, "mixed", 66), "mixed", [0, 7, 8, 24]),
]


@pytest.mark.parametrize("w,prec,cuts", CASES, ids=[f"{w.name}-{p}" for w, p, _ in CASES])
def test_slab_partials_sum_to_the_left_inverse(zl, w, prec, cuts):
    dt = synth.storage_dtype(prec)
    R = min(w.R, 16)
    Z = synth.ensemble(w).astype(dt)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec=prec, max_rhs=R, nx=w.Nx, ny=w.Ny)
    if prec == "mixed":
        assert plan.uses_tc()
    x = synth.rhs(w, R=R, dtype=dt)
    total = None
    for y0, y1 in zip(cuts[:-1], cuts[1:]):
        xs = torch.from_numpy(np.ascontiguousarray(x[:, :, y0 * w.Nx:y1 * w.Nx])).cuda()
        part = zl.zl_apply_left_inverse_rows(plan, y0, y1, xs)
        total = part if total is None else total + part
    xt = zl.zl_scale_modes(plan, total, out=total)             # in place
    oracle = swift.Plan(Z.astype(np.float64), w.Nx, w.Ny, lam, w.tau)
    ref = swift.apply_left_inverse(oracle, x.astype(np.float64))
    compare.check(xt.cpu().numpy(), ref, TOL[prec], 2, f"{w.name} {prec} slabs {cuts}")
    # one slab covering the grid is the ordinary entry point, bit for bit
    whole = zl.zl_scale_modes(plan, zl.zl_apply_left_inverse_rows(plan, 0, w.Ny, torch.from_numpy(x).cuda()))
    assert torch.equal(whole, zl.zl_apply_left_inverse(plan, torch.from_numpy(x).cuda()))


def test_row_range_errors(zl):
    w = CASES[2][0]
    Z = synth.ensemble(w)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec="fp64", max_rhs=4, nx=w.Nx, ny=w.Ny)
    x = torch.zeros((2, w.nw, w.nh), dtype=torch.float64, device="cuda")
    out = torch.zeros((2, plan.K, plan.L), dtype=torch.float64, device="cuda")
    lib = zl._lib
    for y0, y1 in ((-1, 3), (3, 3), (5, 2), (0, w.Ny + 1)):
        assert lib.zl_apply_left_inverse_rows(plan.handle, y0, y1, zl._vp(x.data_ptr()), zl._vp(out.data_ptr()), 2,
                                              None) == zl.ZL_ERR_SHAPE
