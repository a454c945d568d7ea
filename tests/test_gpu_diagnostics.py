"""Matrix-form diagnostics on the GPU (Xi indicators and delta, Sec. 4.8-4.9) against the
oracle's dense brute force: Zh and Zh^- formed explicitly (dense SVD pseudo-inverse).

With n_w < K and truncated modes, M = Zh^- Zh = Delta^{-1/2} V^T (A^+ A) V Delta^{1/2} is a
projection conjugated by the eigenvalue scaling, so Xi = I - M M^T has entries up to the
ratio of the extreme eigenvalues; the indicators are compared in relative terms on FP64
plans.  With n_w = K (the paper's setting) the left inverse is exact and both indicators
vanish to rounding."""

import numpy as np
import pytest

from oracle import basis, dense
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WIDE = synth.Workload("diag_wide", 16, 16, 8, 12, 3.0, 0.7, 3.0, 4, "fp64", 61)    # n_w < K
SQUARE = synth.WORKLOADS["c0a_plane"]                                               # n_w = K


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_13327_b300 import diagnostics, zl
    return zl, diagnostics


def dense_pair(w, Z):
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    S = basis.kept_modes(lam, w.tau)
    return dense.left_inverse_matrix(Z, w.Nx, w.Ny, lam, S), dense.modulated_sqrt(Z, w.Nx, w.Ny, lam, S), lam


def test_xi_indicators_match_dense(mods):
    zl, diag = mods
    Z = synth.ensemble(WIDE)
    Zinv, Zh, lam = dense_pair(WIDE, Z)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=WIDE.tau, prec="fp64", max_rhs=256, nx=WIDE.Nx, ny=WIDE.Ny)
    fro, mx = diag.xi_indicators(plan)
    fro_ref, mx_ref = dense.xi_indicators(Zinv, Zh)
    assert fro_ref > 1.0 and mx_ref > 0.1                    # a genuinely non-trivial Xi
    assert abs(fro - fro_ref) <= 1e-9 * fro_ref
    assert abs(mx - mx_ref) <= 1e-9 * mx_ref


def test_xi_vanishes_for_a_square_left_inverse(mods):
    """n_w = K: Xi is rounding only.  Each column of M carries the FP64 path's relative error
    (at most 1e-10, the parity tolerance) amplified by the eigenvalue scaling
    sqrt(lambda_max / lambda_min), so ||Xi||_F <= 2e-10 sqrt(lambda_max/lambda_min) sqrt(K L)
    and max |Xi_ij| <= 2e-10 sqrt(lambda_max/lambda_min); the dense FP64 SVD brute force sits
    below the same bound."""
    zl, diag = mods
    Z = synth.ensemble(SQUARE)
    lam = basis.spectrum_2d(SQUARE.Nx, SQUARE.Ny, SQUARE.ell_loc)
    S = basis.kept_modes(lam, SQUARE.tau)
    amp = float(np.sqrt(lam[S].max() / lam[S].min()))
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=SQUARE.tau, prec="fp64", max_rhs=256,
                       nx=SQUARE.Nx, ny=SQUARE.Ny)
    fro, mx = diag.xi_indicators(plan)
    KL = plan.K * plan.L
    assert fro <= 2e-10 * amp * np.sqrt(KL)
    assert mx <= 2e-10 * amp
    fro_ref, mx_ref = dense.xi_indicators(*dense_pair(SQUARE, Z)[:2])
    assert fro_ref <= 2e-10 * amp * np.sqrt(KL) and mx_ref <= 2e-10 * amp


def test_delta_matches_dense(mods):
    zl, diag = mods
    Z = synth.ensemble(WIDE)
    Zinv, Zh, lam = dense_pair(WIDE, Z)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=WIDE.tau, prec="fp64", max_rhs=8, nx=WIDE.Nx, ny=WIDE.Ny)
    xt = synth.coefficients(WIDE, plan.L)
    d, norms = diag.delta(plan, torch.from_numpy(xt).cuda())
    for r in range(len(xt)):
        ref = dense.rmse_delta(Zinv, Zh, xt[r].reshape(-1))
        assert abs(float(norms[r]) - ref) <= 1e-9 * ref
