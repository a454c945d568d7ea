"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every input is seeded and synthetic (paper_2609_13327_b300.synth); the
localization spectrum given to both sides is the oracle's.  The tolerance tol
bounds the relative 2-norm error per right-hand side, max over right-hand sides:
  FP64 plans   <= 1e-10   (the FP64 path is the same algorithm in the same precision)
  FP32 plans   <= 1e-6
  MIXED plans  <= 1e-5
and, through ``oracle.compare.check``, also every mode (outputs [R][K][L]) or
level (outputs [R][n_w][n_h]) in relative terms and every element against its
mode's or level's scale.
Small cases span several CTAs and ragged tails and are compared in full; the
1-GPU benchmark shapes run at full size on the GPU and are compared on a
sample of right-hand sides.
"""

import dataclasses

import numpy as np
import pytest

from oracle import basis, compare, swift
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-6, "mixed": 1e-5}
W = synth.WORKLOADS


@pytest.fixture(scope="module")
def zl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_13327_b300 import zl as mod
    return mod


# the axis of an operator's output whose entries have their own scale: modes or levels
SLICE = {"left_inverse": 2, "sqrt": 1, "adjoint": 1, "sqrt_adjoint": 2}


class Case:
    """One workload set up on both sides (oracle from the same rounded inputs)."""

    def __init__(self, zl, w, prec, tau=None, max_rhs=None, spectrum=None):
        self.w, self.prec = w, prec
        self.tau = w.tau if tau is None else tau
        dt = synth.storage_dtype(prec)
        self.dt = dt
        self.Z = synth.ensemble(w).astype(dt)
        self.lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc) if spectrum is None else spectrum
        self.oracle = swift.Plan(self.Z.astype(np.float64), w.Nx, w.Ny, self.lam, self.tau)
        self.plan = zl.zl_setup(torch.from_numpy(self.Z).cuda(), self.lam, tau=self.tau, prec=prec,
                                max_rhs=max_rhs or max(1, w.R), nx=w.Nx, ny=w.Ny)

    def tol(self):
        return TOL[self.prec]


def check_all_ops(zl, c, R=None):
    w = c.w
    R = w.R if R is None else R
    assert c.plan.L == c.oracle.L
    assert np.array_equal(c.plan.modes(), c.oracle.S)
    x = synth.rhs(w, R=R, dtype=c.dt)
    xt = synth.coefficients(w, c.plan.L, R=R, dtype=c.dt)
    xg, xtg = torch.from_numpy(x).cuda(), torch.from_numpy(xt).cuda()
    x64, xt64 = x.astype(np.float64), xt.astype(np.float64)
    # every output buffer starts NaN-poisoned: an element a kernel fails to write fails the check
    nan = lambda shape: torch.full(shape, float("nan"), dtype=xg.dtype, device="cuda")  # noqa: E731
    got = {
        "left_inverse": zl.zl_apply_left_inverse(c.plan, xg, nan(xtg.shape)),
        "sqrt": zl.zl_apply_sqrt(c.plan, xtg, nan(xg.shape)),
        "adjoint": zl.zl_apply_adjoint(c.plan, xtg, nan(xg.shape)),
        "sqrt_adjoint": zl.zl_apply_sqrt_adjoint(c.plan, xg, nan(xtg.shape)),
    }
    torch.cuda.synchronize()
    ref = {
        "left_inverse": swift.apply_left_inverse(c.oracle, x64),
        "sqrt": swift.apply_sqrt(c.oracle, xt64),
        "adjoint": swift.apply_adjoint(c.oracle, xt64),
        "sqrt_adjoint": swift.apply_sqrt_adjoint(c.oracle, x64),
    }
    tol = TOL["fp32"] if c.prec == "mixed" else c.tol()   # only the left inverse uses tensor cores
    for op in got:
        t = c.tol() if op == "left_inverse" else tol
        compare.check(got[op].cpu().numpy(), ref[op], t, SLICE[op], f"{w.name} {c.prec} {op}")


# ------------------------------------------------------------------ small cases, all four operators

RAGGED_C2 = synth.Workload("ragged_c2", 40, 24, 10, 32, 6.0, 0.7, 5.0, 19, "fp32", 21)
RAGGED_C3 = synth.Workload("ragged_c3", 48, 40, 32, 64, 8.0, 0.8, 6.0, 13, "mixed", 31, var_range=(0.1, 10.0))
ODD = synth.Workload("odd", 17, 9, 5, 7, 2.0, 0.5, 1.5, 6, "fp32", 41)
WIDE = synth.Workload("wide", 8, 6, 3, 7, 2.0, 0.6, 1.2, 5, "fp64", 11, tau=0.0)
TALL = synth.Workload("tall", 8, 6, 6, 3, 2.0, 0.6, 1.2, 5, "fp64", 12, tau=0.0)
LONG_RING = synth.Workload("long_ring", 300, 1, 3, 12, 9.0, 0.5, 12.0, 9, "fp32", 51)
# P_x = 60 kept x-frequencies (the widest tile of the register-tiled FP32 column kernel)
# and P_x = 72 (past it: the per-column kernel)
PX60 = synth.Workload("px60", 60, 8, 4, 20, 1.5, 0.6, 1.5, 10, "fp32", 61)
PX72 = synth.Workload("px72", 72, 6, 3, 9, 1.5, 0.6, 1.5, 3, "fp32", 62)
# 40 levels: 10 level groups of the TMA-fed forward kernel, 2 rhs per CTA in the TMA-fed
# inverse pass; in mixed precision the tensor-core kernel does not take n_w > 32, so the
# mixed plan runs the FP32 CUDA-core kernels
LEVELS40 = synth.Workload("levels40", 24, 16, 40, 56, 3.0, 0.7, 3.0, 6, "fp32", 71)

SMALL = [
    (W["c0a_ring"], "fp64"), (W["c0a_plane"], "fp64"), (W["c0b_paper_shape"], "fp64"), (W["c1_ring64"], "fp64"),
    (WIDE, "fp64"), (TALL, "fp64"), (WIDE, "fp32"), (TALL, "fp32"), (ODD, "fp64"), (ODD, "fp32"),
    (RAGGED_C2, "fp32"), (RAGGED_C2, "fp64"), (RAGGED_C3, "fp32"), (RAGGED_C3, "mixed"), (LONG_RING, "fp32"),
    (PX60, "fp32"), (PX72, "fp32"), (LEVELS40, "fp32"), (LEVELS40, "mixed"),
]


@pytest.mark.parametrize("w,prec", SMALL, ids=[f"{w.name}-{p}" for w, p in SMALL])
def test_all_operators_match_oracle(zl, w, prec):
    check_all_ops(zl, Case(zl, w, prec))


def test_untruncated_ring_closed_form_spectrum(zl):
    """64-point ring, K = 8, tau = 0 with the closed-form spectrum: L = n_h = 64 (right inverse)."""
    w = W["c1_ring64"]
    lam = basis.spectrum_1d_closed_form(w.Nx, w.ell_loc)
    c = Case(zl, w, "fp64", tau=0.0, spectrum=lam)
    assert c.plan.L == 64
    check_all_ops(zl, c)


def test_rhs_chunking_and_ragged_batches(zl):
    """R larger than the plan's pass size, and not a multiple of it or of the CTA's rhs tile."""
    c = Case(zl, RAGGED_C2, "fp32", max_rhs=5)
    check_all_ops(zl, c, R=23)
    check_all_ops(zl, c, R=1)


def test_zero_rhs_is_a_no_op(zl):
    c = Case(zl, ODD, "fp32")
    x = torch.zeros((0, ODD.nw, ODD.nh), dtype=torch.float32, device="cuda")
    out = zl.zl_apply_left_inverse(c.plan, x)
    assert out.shape == (0, ODD.K, c.plan.L)


def test_rank_deficient_ensemble_is_reported(zl):
    """A self-centred ensemble with n_w >= K has singular A_m (Sec. 4.2): ZL_ERR_RANK."""
    w = W["c0a_plane"]
    Z = synth.centred_ensemble(w)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    with pytest.raises(zl.ZLError) as ei:
        zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=1e-10, prec="fp64", max_rhs=4, nx=w.Nx, ny=w.Ny)
    assert ei.value.code == zl.ZL_ERR_RANK
    assert ei.value.bad_column == 0


def test_aliasing_and_shape_errors(zl):
    c = Case(zl, ODD, "fp32")
    x = torch.zeros((2, ODD.nw, ODD.nh), dtype=torch.float32, device="cuda")
    lib = zl._lib
    import ctypes
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.zl_apply_left_inverse(c.plan.handle, p, p, 2, None) == zl.ZL_ERR_ARG
    with pytest.raises(ValueError):
        zl.zl_apply_left_inverse(c.plan, x.double())
    with pytest.raises(ValueError):
        zl.zl_apply_left_inverse(c.plan, x[:, :1])


def test_host_buffer_entry_point(zl):
    c = Case(zl, RAGGED_C2, "fp32", max_rhs=8)
    x = synth.rhs(RAGGED_C2, R=11, dtype=np.float32)
    out = zl.zl_apply_left_inverse_host(c.plan, torch.from_numpy(x).pin_memory())
    ref = swift.apply_left_inverse(c.oracle, x.astype(np.float64))
    compare.check(out.numpy(), ref, TOL["fp32"], 2, "host-buffer entry point")


# ------------------------------------------------------------------ full-size 1-GPU shapes, sampled

FULL = [("c2_128x128x10", "fp32", [0, 131, 255]), ("c3_256x256x32", "mixed", [0, 37, 63]),
        ("c3_256x256x32", "fp32", [5]), ("c5_512x512x16", "fp32", [0, 7])]


@pytest.mark.parametrize("name,prec,sample", FULL, ids=[f"{n}-{p}" for n, p, _ in FULL])
def test_full_size_left_inverse_sampled(zl, name, prec, sample):
    w = W[name]
    c = Case(zl, w, prec, max_rhs=w.R)
    x = synth.rhs(w, dtype=np.float32)
    out = zl.zl_apply_left_inverse(c.plan, torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.all(np.isfinite(out))
    if prec == "mixed":
        assert c.plan.uses_tc() and c.plan.device_error() == 0
    ref = swift.apply_left_inverse(c.oracle, x[sample].astype(np.float64))
    compare.check(out[sample], ref, TOL[prec], 2, f"{name} {prec} sampled")


def test_full_size_adjoint_sampled(zl):
    """The 512 x 512 x 16 shape (K = 48, 8 rhs) through the adjoint, sampled."""
    w = W["c5_512x512x16"]
    c = Case(zl, w, "fp32", max_rhs=w.R)
    y = synth.coefficients(w, c.plan.L, dtype=np.float32)
    out = zl.zl_apply_adjoint(c.plan, torch.from_numpy(y).cuda()).cpu().numpy()
    ref = swift.apply_adjoint(c.oracle, y[[3]].astype(np.float64))
    compare.check(out[[3]], ref, TOL["fp32"], 1, "512x512x16 adjoint sampled")
