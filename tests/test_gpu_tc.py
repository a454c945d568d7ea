"""The tcgen05 tensor-core left inverse (ZL_MIXED plans) against the FP64 oracle.

Checks that the tensor-core kernel is really the one that runs
(``uses_tc``), that it recorded no device-side timeout, and that its result
matches the oracle within the mixed-precision tolerance 1e-5 (relative 2-norm
per right-hand side) on shapes that exercise every padded path: ragged numbers
of right-hand sides (partial 16-rhs units), fewer than 64 members, fewer than
16 levels, several rows per CTA, and every row tier (16 to 48 kept
y-frequencies) of the y-pass.
"""

import numpy as np
import pytest

from oracle import basis, swift
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-5


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
    synth.Workload("tc_c3_like", 48, 40, 32, 64, 8.0, 0.8, 6.0, 13, "mixed", 31, var_range=(0.1, 10.0)),
    synth.Workload("tc_small_K", 32, 12, 10, 40, 4.0, 0.7, 3.0, 21, "mixed", 32),
    synth.Workload("tc_16_levels", 64, 24, 16, 48, 6.0, 0.75, 5.0, 35, "mixed", 33),
    synth.Workload("tc_one_row_many_rhs", 128, 2, 24, 64, 6.0, 0.7, 8.0, 64, "mixed", 34),
    # 47, 31 and 17 kept y-frequencies: the 48-, 32- and 24-row tiers of the y-pass
    synth.Workload("tc_py47", 64, 64, 16, 48, 6.0, 0.7, 3.0, 19, "mixed", 36),
    synth.Workload("tc_py31", 64, 64, 24, 40, 6.0, 0.75, 4.5, 23, "mixed", 37),
    synth.Workload("tc_py17", 64, 48, 8, 32, 4.0, 0.7, 6.0, 11, "mixed", 38),
]


@pytest.mark.parametrize("w", CASES, ids=[w.name for w in CASES])
def test_tensor_core_left_inverse(zl, w):
    Z = synth.ensemble(w).astype(np.float32)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    oracle = swift.Plan(Z.astype(np.float64), w.Nx, w.Ny, lam, w.tau)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec="mixed", max_rhs=w.R, nx=w.Nx, ny=w.Ny)
    assert plan.uses_tc()
    x = synth.rhs(w, dtype=np.float32)
    out = zl.zl_apply_left_inverse(plan, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    assert plan.device_error() == 0
    ref = swift.apply_left_inverse(oracle, x.astype(np.float64))
    assert rel_err(out, ref) <= TOL_MIXED


def test_tensor_core_repeated_calls_and_chunking(zl):
    """Two calls in a row give the same bits; R above max_rhs runs in passes."""
    w = CASES[0]
    Z = synth.ensemble(w).astype(np.float32)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec="mixed", max_rhs=8, nx=w.Nx, ny=w.Ny)
    x = torch.from_numpy(synth.rhs(w, R=19, dtype=np.float32)).cuda()
    a = zl.zl_apply_left_inverse(plan, x)
    b = zl.zl_apply_left_inverse(plan, x)
    assert torch.equal(a, b)
    oracle = swift.Plan(Z.astype(np.float64), w.Nx, w.Ny, lam, w.tau)
    ref = swift.apply_left_inverse(oracle, x.cpu().numpy().astype(np.float64))
    assert rel_err(a.cpu().numpy().astype(np.float64), ref) <= TOL_MIXED
    assert plan.device_error() == 0


def test_unsupported_shape_runs_cuda_cores(zl):
    """A mixed plan the tensor-core kernel cannot take (nx not a multiple of 16) uses the FP32 kernels."""
    w = synth.Workload("odd_mixed", 17, 9, 5, 7, 2.0, 0.5, 1.5, 6, "mixed", 41)
    Z = synth.ensemble(w).astype(np.float32)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec="mixed", max_rhs=w.R, nx=w.Nx, ny=w.Ny)
    assert not plan.uses_tc()


FULL_TC = [("c2_128x128x10", [0, 255]), ("c3_256x256x32", [1, 62]), ("c5_512x512x16", [2])]


@pytest.mark.parametrize("name,sample", FULL_TC, ids=[n for n, _ in FULL_TC])
def test_tensor_core_full_size_sampled(zl, name, sample):
    """The 1-GPU benchmark shapes in mixed precision, at full size, sampled right-hand sides."""
    w = synth.WORKLOADS[name]
    Z = synth.ensemble(w).astype(np.float32)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec="mixed", max_rhs=w.R, nx=w.Nx, ny=w.Ny)
    assert plan.uses_tc()
    x = synth.rhs(w, dtype=np.float32)
    out = zl.zl_apply_left_inverse(plan, torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.device_error() == 0
    oracle = swift.Plan(Z.astype(np.float64), w.Nx, w.Ny, lam, w.tau)
    ref = swift.apply_left_inverse(oracle, x[sample].astype(np.float64))
    assert rel_err(out[sample].astype(np.float64), ref) <= TOL_MIXED


def test_host_buffer_pipeline_matches_device_path(zl):
    """The host-buffer entry point runs the right-hand sides in pieces (16 here: 16, 16, 5,
    so a staging slot is reused) with the copies on their own streams; each piece is the
    same kernel launch as the device entry point's max_rhs chunk, so the bits agree."""
    w = CASES[1]
    Z = synth.ensemble(w).astype(np.float32)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec="mixed", max_rhs=16, nx=w.Nx, ny=w.Ny)
    assert plan.uses_tc()
    x = synth.rhs(w, R=37, dtype=np.float32)
    dev = zl.zl_apply_left_inverse(plan, torch.from_numpy(x).cuda()).cpu()
    for _ in range(2):                                    # the second call reuses streams and staging
        host = zl.zl_apply_left_inverse_host(plan, torch.from_numpy(x).pin_memory())
        assert torch.equal(host, dev)
    oracle = swift.Plan(Z.astype(np.float64), w.Nx, w.Ny, lam, w.tau)
    assert rel_err(host.numpy().astype(np.float64), swift.apply_left_inverse(oracle, x.astype(np.float64))) <= TOL_MIXED
