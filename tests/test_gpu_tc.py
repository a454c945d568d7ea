"""The tcgen05 tensor-core left inverse (ZL_MIXED plans) against the FP64 oracle.

Checks that the tensor-core kernel is really the one that runs
(``uses_tc``), that it recorded no device-side timeout, and that its result
matches the oracle within the mixed-precision tolerance 1e-5 (relative 2-norm
per right-hand side, and per mode and element through ``oracle.compare.check``) on shapes that exercise every padded path: ragged numbers
of right-hand sides (partial 16-rhs units), fewer than 64 members, fewer than
16 levels, several rows per CTA, and every row tier (16 to 48 kept
y-frequencies) of the y-pass.
"""

import numpy as np
import pytest

from oracle import basis, compare, swift
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


CASES = [
    synth.Workload("tc_c3_like", 48, 40, 32, 64, 8.0, 0.8, 6.0, 13, "mixed", 31, var_range=(0.1, 10.0)),
    synth.Workload("tc_small_K", 32, 12, 10, 40, 4.0, 0.7, 3.0, 21, "mixed", 32),
    synth.Workload("tc_16_levels", 64, 24, 16, 48, 6.0, 0.75, 5.0, 35, "mixed", 33),
    synth.Workload("tc_one_row_many_rhs", 128, 2, 24, 64, 6.0, 0.7, 8.0, 64, "mixed", 34),
    # 47, 31 and 17 kept y-frequencies: the 48-, 32- and 24-row tiers of the y-pass
    synth.Workload("tc_py47", 64, 64, 16, 48, 6.0, 0.7, 3.0, 19, "mixed", 36),
    synth.Workload("tc_py31", 64, 64, 24, 40, 6.0, 0.75, 4.5, 23, "mixed", 37),
    synth.Workload("tc_py17", 64, 48, 8, 32, 4.0, 0.7, 6.0, 11, "mixed", 38),
    # n_w = K (the paper's square A_m, Eq. nwEqualsK): Zh^- is a true left inverse there
    synth.Workload("tc_square_16", 32, 16, 16, 16, 3.0, 0.7, 3.0, 16, "mixed", 51),
    synth.Workload("tc_square_32", 32, 8, 32, 32, 3.0, 0.7, 3.0, 16, "mixed", 52),
    # n_w > K: the least-squares pseudo-inverse (AᵀA)^{-1} Aᵀ of each column
    synth.Workload("tc_tall_24_16", 48, 16, 24, 16, 4.0, 0.7, 4.0, 16, "mixed", 54),
    synth.Workload("tc_tall_32_20", 32, 16, 32, 20, 4.0, 0.7, 4.0, 19, "mixed", 55),
]

# n_w = K with every mode kept (tau = 0): Zh is square and Zh^- Zh = I (Sec. 3.9)
SQUARE_ALL_MODES = [
    synth.Workload("tc_square_16_all_modes", 16, 8, 16, 16, 3.0, 0.7, 1.0, 16, "mixed", 61, tau=0.0),
    synth.Workload("tc_square_32_all_modes", 32, 8, 32, 32, 3.0, 0.7, 1.0, 16, "mixed", 62, tau=0.0),
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
    compare.check(out, ref, TOL_MIXED, 2, w.name)


def _rel(a, b):
    R = b.shape[0]
    return float(np.max(np.linalg.norm((a - b).reshape(R, -1), axis=1) / np.linalg.norm(b.reshape(R, -1), axis=1)))


@pytest.mark.parametrize("w", SQUARE_ALL_MODES, ids=[w.name for w in SQUARE_ALL_MODES])
def test_tensor_core_left_inverse_property_square(zl, w):
    """Zh^- (Zh x~0) = x~0 on the tensor cores where A_m is square and all modes are kept.

    x = Zh x~0 is formed by the oracle in FP64 and rounded to FP32, the library's input
    type.  On such range-space inputs the rounding of x is amplified by cond(A_m) and by
    (lambda_max / lambda_min)^{1/2}, so even exact arithmetic on the FP32 x misses x~0 by
    err_ref (1e-5 to 1e-4 here).  The tensor-core path works on 22-bit operand splits
    (FP16 hi + lo) of x and of A_m^+, about 4x coarser than FP32's 24 bits, so it must
    recover x~0 to within a small multiple of err_ref; and it must match the oracle on
    the same FP32 input to the mixed tolerance scaled by the same amplification.
    """
    Z = synth.ensemble(w).astype(np.float32)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    oracle = swift.Plan(Z.astype(np.float64), w.Nx, w.Ny, lam, w.tau)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec="mixed", max_rhs=w.R, nx=w.Nx, ny=w.Ny)
    assert plan.uses_tc()
    assert plan.L == w.nh and w.nw == w.K
    xt0 = synth.coefficients(w, plan.L)
    x32 = np.ascontiguousarray(swift.apply_sqrt(oracle, xt0), dtype=np.float32)
    got = zl.zl_apply_left_inverse(plan, torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
    assert plan.device_error() == 0
    ref = swift.apply_left_inverse(oracle, x32.astype(np.float64))
    err_ref = _rel(ref, xt0)
    assert err_ref < 1e-3, f"the FP32 rounding of Zh x~0 alone misses x~0 by {err_ref:.2e}"
    err_gpu = _rel(got, xt0)
    assert err_gpu <= 16.0 * err_ref + 1e-6, f"{w.name}: {err_gpu:.3e} vs exact arithmetic {err_ref:.3e}"
    compare.check(got, ref, max(TOL_MIXED, 16.0 * err_ref), 2, w.name)


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
    compare.check(a.cpu().numpy(), ref, TOL_MIXED, 2, "chunked")
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
    compare.check(out[sample], ref, TOL_MIXED, 2, name)


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
    compare.check(host.numpy(), swift.apply_left_inverse(oracle, x.astype(np.float64)), TOL_MIXED, 2, "host pipeline")


# n_w = K (the paper's assumption, Eq. nwEqualsK: every A_m square, Zh^- a genuine left
# inverse) and n_w > K (least squares), forced onto the tensor-core kernel
SQUARE_TALL = [
    synth.Workload("tc_square16", 16, 16, 16, 16, 2.0, 0.6, 1.0, 13, "mixed", 81, tau=0.0),
    synth.Workload("tc_square32", 16, 16, 32, 32, 2.0, 0.6, 1.0, 21, "mixed", 82, tau=0.0),
    synth.Workload("tc_tall24x16", 32, 24, 24, 16, 3.0, 0.7, 3.0, 19, "mixed", 83),
]


@pytest.mark.parametrize("w", SQUARE_TALL, ids=[w.name for w in SQUARE_TALL])
def test_tensor_core_square_and_tall_columns(zl, w):
    """Parity with the oracle on random x, and the left-inverse property on x = Zh x~0.

    For x in the range of Zh the problem's own conditioning sets the accuracy: rounding
    x to FP32 (2^-24) already moves the FP64 oracle's Zh^- x away from x~0 by e_or,
    about eps cond(A_m) sqrt(lambda_max/lambda_min) (the bound of the delta pin).  The
    tensor-core path represents x and A_m^+ to 2^-22 (FP16 hi/lo) and accumulates the
    n_w-term sums of V1 in FP32 on the tensor cores, whose rounding error is amplified by
    the same cancellation (up to about 2 sqrt(n_w) times the input rounding's effect), so
    it must recover x~0 within 16 e_or plus the mixed tolerance."""
    Z = synth.ensemble(w).astype(np.float32)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    oracle = swift.Plan(Z.astype(np.float64), w.Nx, w.Ny, lam, w.tau)
    assert oracle.ok and w.nw >= w.K
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec="mixed", max_rhs=w.R, nx=w.Nx, ny=w.Ny)
    assert plan.uses_tc()
    x = synth.rhs(w, dtype=np.float32)
    out = zl.zl_apply_left_inverse(plan, torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.device_error() == 0
    compare.check(out, swift.apply_left_inverse(oracle, x.astype(np.float64)), TOL_MIXED, 2, w.name)
    # left-inverse property
    xt0 = synth.coefficients(w, plan.L)
    xr = np.ascontiguousarray(swift.apply_sqrt(oracle, xt0), dtype=np.float32)
    back = zl.zl_apply_left_inverse(plan, torch.from_numpy(xr).cuda()).cpu().numpy().astype(np.float64)
    ref = swift.apply_left_inverse(oracle, xr.astype(np.float64))
    e_or = np.linalg.norm((ref - xt0).reshape(w.R, -1), axis=1)
    e_gpu = np.linalg.norm((back - xt0).reshape(w.R, -1), axis=1)
    scale = np.linalg.norm(xt0.reshape(w.R, -1), axis=1)
    assert np.all(e_or <= 1e-3 * scale)
    assert np.all(e_gpu <= 16 * e_or + 2 * TOL_MIXED * scale), (e_gpu / scale, e_or / scale)
