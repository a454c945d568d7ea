"""zl_apply_left_inverse_static, the entry point that allocates nothing.

Some callers cannot allocate device memory at the moment they apply the
operator (a real-time loop with a memory budget fixed at start-up, a host
callback, a process whose device memory belongs to another framework's pool).
For them the library keeps the transform's intermediate in a static device
array; zl_setup resolves the array's address and loads the kernels, so an
apply only launches kernels.  This file is collected last so a failure here
comes after every other test has run; it passes alone in a fresh process as
well as after the rest.
"""

import numpy as np
import pytest

from oracle import basis, swift
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the static path runs the CUDA-core kernels: FP32 accuracy for FP32 and mixed plans
TOL = {"fp64": 1e-10, "fp32": 1e-6, "mixed": 1e-6}


@pytest.fixture(scope="module")
def zl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_13327_b300 import zl as mod
    return mod


def rel_err(out, ref):
    out = out.reshape(len(out), -1)
    ref = ref.reshape(len(ref), -1)
    return float(np.max(np.linalg.norm(out - ref, axis=1) / np.linalg.norm(ref, axis=1)))


CASES = [
    (synth.WORKLOADS["c2_128x128x10"], "fp32", 64),     # 442 KB per rhs: two passes through the 16 MiB array
    (synth.Workload("ragged_fp64", 40, 24, 6, 9, 4.0, 0.6, 3.0, 7, "fp64", 61), "fp64", 7),
    # a mixed plan (its own apply runs the tensor-core kernel): the static path uses the FP32 kernels
    (synth.Workload("ragged_mixed", 48, 40, 32, 64, 8.0, 0.8, 6.0, 13, "mixed", 31, var_range=(0.1, 10.0)),
     "mixed", 13),
]


@pytest.mark.parametrize("w,prec,R", CASES, ids=[f"{w.name}-{p}" for w, p, _ in CASES])
def test_static_scratch_matches_workspace_entry_point_and_oracle(zl, w, prec, R):
    dt = synth.storage_dtype(prec)
    Z = synth.ensemble(w).astype(dt)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec=prec, max_rhs=R, nx=w.Nx, ny=w.Ny)
    x = torch.from_numpy(synth.rhs(w, R=R, dtype=dt)).cuda()
    ref_ws = zl.zl_apply_left_inverse(plan, x).cpu().numpy().astype(np.float64)
    oracle = swift.Plan(Z.astype(np.float64), w.Nx, w.Ny, lam, w.tau)
    ref = swift.apply_left_inverse(oracle, x.cpu().numpy().astype(np.float64))
    outs = [torch.empty((R, plan.K, plan.L), dtype=x.dtype, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for out in outs:   # the array keeps the previous call's contents: a second call must not depend on them
        zl.zl_apply_left_inverse_static(plan, x, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0          # nothing allocated, no module loaded
    tol_ws = TOL[prec] if prec != "mixed" else 1e-5       # the workspace path of a mixed plan is the tensor-core one
    for out in outs:
        got = out.cpu().numpy().astype(np.float64)
        assert rel_err(got, ref) <= TOL[prec]
        assert rel_err(got, ref_ws) <= tol_ws


def test_static_scratch_rejects_plans_beyond_its_size(zl):
    """One right-hand side needing more than 16 MiB of intermediate is refused before any work.

    64 x 520 grid, K = 64, FP64, a spectrum that keeps all 64 x-frequencies of the
    first 150 y-frequencies: 64 * 520 * 64 * 8 bytes = 17.0 MB per right-hand side.
    """
    w = synth.Workload("tall_grid", 64, 520, 1, 64, 2.0, 0.0, 1.5, 1, "fp64", 62)
    Z = synth.ensemble(w)
    lam = np.zeros((w.Ny, w.Nx))
    lam[:150, :] = 1.0
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam.reshape(-1), tau=0.5, prec="fp64", max_rhs=1,
                       nx=w.Nx, ny=w.Ny)
    x = torch.zeros((1, w.nw, w.nh), dtype=torch.float64, device="cuda")
    out = torch.full((1, w.K, plan.L), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(zl.ZLError) as ei:
        zl.zl_apply_left_inverse_static(plan, x, out)
    assert ei.value.code == zl.ZL_ERR_SHAPE
    assert torch.all(out == 7.0)
