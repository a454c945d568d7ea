"""zl_apply_left_inverse_static, the entry point that allocates nothing.

Some callers cannot allocate device memory at the moment they apply the
operator (a real-time loop with a memory budget fixed at start-up, a host
callback, a process whose device memory belongs to another framework's pool).
For them the library keeps the transform's intermediate in a static device
array.  This file is collected last so a failure here comes after every other
test has run; it passes alone in a fresh process as well as after the rest.
"""

import numpy as np
import pytest

from oracle import basis
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-6}


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
]


@pytest.mark.parametrize("w,prec,R", CASES, ids=[f"{w.name}-{p}" for w, p, _ in CASES])
def test_static_scratch_matches_workspace_entry_point(zl, w, prec, R):
    dt = synth.storage_dtype(prec)
    Z = synth.ensemble(w).astype(dt)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec=prec, max_rhs=R, nx=w.Nx, ny=w.Ny)
    x = torch.from_numpy(synth.rhs(w, R=R, dtype=dt)).cuda()
    ref = zl.zl_apply_left_inverse(plan, x).cpu().numpy().astype(np.float64)
    for _ in range(2):   # the array keeps the previous call's contents: a second call must not depend on them
        out = zl.zl_apply_left_inverse_static(plan, x).cpu().numpy().astype(np.float64)
        assert rel_err(out, ref) <= TOL[prec]


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
