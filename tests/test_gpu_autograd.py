"""Differentiation through the library (torch.autograd wrappers, adjoint kernels).

J(x) = 1/2 ||Zh^- x||^2 has the gradient (Zh^-)^T Zh^- x.  Checked on a 32 x 32 x 2
sub-instance of the 512 x 512 x 16 recipe (K = 48, AR(1) 0.75 between levels; localization
length 6 points so that the dense operator, 48 x 101 by 2048, stays small):
* against the oracle's dense transpose: Zh^- formed column by column by the FP64 oracle
  (the swift algorithm applied to every unit vector, which the oracle pins equate with
  the dense pseudo-inverse definition), then (Zh^-)^T (Zh^- x);
* against central finite differences with h = 1e-3 (exact for a quadratic J up to
  rounding) on an FP64 plan, along x itself (where the directional derivative is 2J/||x||),
  the gradient direction and random directions;
* by torch.autograd.gradcheck (every direction) on a tiny FP64 plan;
and at full size (512 x 512 x 16, K = 48, 8 rhs, FP32) against the oracle on a sampled
right-hand side.  The square root's wrapper is checked the same way against the dense
Zh of the oracle.
"""

import numpy as np
import pytest

from oracle import basis, compare, dense, swift
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SUB = synth.Workload("c5_sub_32x32x2", 32, 32, 2, 48, 2.0, 0.75, 6.0, 4, "fp32", 51)   # L = 101
TINY = synth.Workload("tiny_8x8x2", 8, 8, 2, 4, 1.5, 0.5, 1.0, 2, "fp64", 52)


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_13327_b300 import autograd, zl
    return zl, autograd


def make(zl, w, prec):
    dt = np.float64 if prec == "fp64" else np.float32
    Z = synth.ensemble(w)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z.astype(dt)).cuda(), lam, tau=w.tau, prec=prec, max_rhs=64, nx=w.Nx, ny=w.Ny)
    oracle = swift.Plan(Z.astype(dt).astype(np.float64), w.Nx, w.Ny, lam, w.tau)
    return plan, oracle


def dense_left_inverse(oracle, w):
    """Zh^- (K L x n) from the oracle applied to the n unit vectors."""
    n = w.nw * w.nh
    eye = np.eye(n).reshape(n, w.nw, w.nh)
    cols = swift.apply_left_inverse(oracle, eye)          # [n][K][L]
    return cols.reshape(n, -1).T


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-10)])
def test_gradient_matches_dense_transpose(mods, prec, tol):
    zl, ag = mods
    plan, oracle = make(zl, SUB, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    x = torch.from_numpy(synth.rhs(SUB)).to(dt).cuda().requires_grad_(True)
    xt = ag.left_inverse(plan, x)
    J = 0.5 * (xt.double() ** 2).sum()
    J.backward()
    Zinv = dense_left_inverse(oracle, SUB)
    xs = x.detach().cpu().numpy().astype(np.float64).reshape(SUB.R, -1)
    g_ref = (Zinv.T @ (Zinv @ xs.T)).T
    compare.check(x.grad.cpu().numpy(), g_ref.reshape(SUB.R, SUB.nw, SUB.nh), tol, 1, f"gradient {prec}")
    compare.check(xt.detach().cpu().numpy(), (Zinv @ xs.T).T.reshape(SUB.R, SUB.K, -1), tol, 2, f"forward {prec}")


def test_gradient_central_differences(mods):
    zl, ag = mods
    plan, _ = make(zl, SUB, "fp64")
    x0 = torch.from_numpy(synth.rhs(SUB, R=1)).cuda()

    def J(x):
        return 0.5 * float((zl.zl_apply_left_inverse(plan, x) ** 2).sum())

    x = x0.clone().requires_grad_(True)
    (0.5 * (ag.left_inverse(plan, x) ** 2).sum()).backward()
    g = x.grad
    rng = np.random.default_rng(7)
    dirs = [x0 / x0.norm(), g / g.norm()] + [torch.from_numpy(rng.standard_normal(x0.shape)).cuda() for _ in range(3)]
    h = 1e-3
    for d in dirs:
        d = d / d.norm()
        fd = (J(x0 + h * d) - J(x0 - h * d)) / (2 * h)
        assert abs(fd - float((g * d).sum())) <= 1e-7 * J(x0) + 1e-6 * abs(fd)
    # J is homogeneous of degree 2: the derivative along x is 2 J / ||x||
    assert float((g * x0).sum()) / float(x0.norm()) == pytest.approx(2 * J(x0) / float(x0.norm()), rel=1e-10)


def test_gradcheck_tiny_fp64(mods):
    zl, ag = mods
    plan, _ = make(zl, TINY, "fp64")
    x = torch.from_numpy(synth.rhs(TINY)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v: ag.left_inverse(plan, v), (x,), eps=1e-6, atol=1e-8, rtol=1e-6)
    xt = torch.from_numpy(synth.coefficients(TINY, plan.L)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v: ag.sqrt(plan, v), (xt,), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_sqrt_wrapper_matches_dense_zh(mods):
    zl, ag = mods
    plan, oracle = make(zl, SUB, "fp64")
    lam = basis.spectrum_2d(SUB.Nx, SUB.Ny, SUB.ell_loc)
    S = basis.kept_modes(lam, SUB.tau)
    Zh = dense.modulated_sqrt(synth.ensemble(SUB), SUB.Nx, SUB.Ny, lam, S)      # n x K L, columns (k, j)
    xt = torch.from_numpy(synth.coefficients(SUB, plan.L)).cuda().requires_grad_(True)
    x = ag.sqrt(plan, xt)
    (0.5 * (x ** 2).sum()).backward()
    xts = xt.detach().cpu().numpy().reshape(SUB.R, -1)
    compare.check(x.detach().cpu().numpy(), (Zh @ xts.T).T.reshape(SUB.R, SUB.nw, SUB.nh), 1e-10, 1, "sqrt")
    compare.check(xt.grad.cpu().numpy(), (Zh.T @ (Zh @ xts.T)).T.reshape(SUB.R, SUB.K, -1), 1e-10, 2,
                  "sqrt gradient")


def test_full_size_gradient_sampled(mods):
    """512 x 512 x 16 (K = 48, 8 rhs, FP32): autograd gradient vs the oracle on one rhs."""
    zl, ag = mods
    w = synth.WORKLOADS["c5_512x512x16"]
    plan, oracle = make(zl, w, "fp32")
    x = torch.from_numpy(synth.rhs(w, dtype=np.float32)).cuda().requires_grad_(True)
    (0.5 * (ag.left_inverse(plan, x).double() ** 2).sum()).backward()
    assert plan.device_error() == 0
    xs = x.detach()[[5]].cpu().numpy().astype(np.float64)
    g_ref = swift.apply_adjoint(oracle, swift.apply_left_inverse(oracle, xs))
    compare.check(x.grad[[5]].cpu().numpy(), g_ref, 1e-5, 1, "512x512x16 gradient")
