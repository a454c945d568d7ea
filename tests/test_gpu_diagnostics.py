"""Matrix-form diagnostics on the GPU (Xi indicators and delta, Sec. 4.8-4.9) against the
oracle's dense brute force: Zh and Zh^- formed explicitly (dense SVD pseudo-inverse).

With n_w < K and truncated modes, M = Zh^- Zh = Delta^{-1/2} V^T (A^+ A) V Delta^{1/2} is a
projection conjugated by the eigenvalue scaling, so Xi = I - M M^T has entries up to the
ratio of the extreme eigenvalues; the indicators are compared in relative terms on FP64
plans.  With n_w = K (the paper's setting) the left inverse is exact and both indicators
vanish to rounding."""

import numpy as np
import pytest

from oracle import basis, compare, dense, swift
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
    # the difference vector itself, element by element, against the dense brute force
    d_ref = xt - (Zinv @ (Zh @ xt.reshape(len(xt), -1).T)).T.reshape(xt.shape)
    compare.check(d.cpu().numpy(), d_ref, 1e-9, 2, "delta vector")


# ---------------------------------------------------------------- per-column SVD (Eq. svdOfAm)

SVD_CASES = [
    (WIDE, "fp64"),                                                                     # n_w < K
    (synth.Workload("svd_tall", 16, 12, 24, 16, 2.0, 0.7, 2.0, 2, "fp64", 63), "fp64"),  # n_w > K
    (synth.WORKLOADS["c0b_paper_shape"], "fp64"),                                       # n_w = K = 64
    (synth.Workload("svd_odd", 9, 7, 5, 11, 2.0, 0.6, 2.0, 2, "fp32", 64), "fp32"),       # odd g, FP32 copy
]


def sign_fixed(E, lam, F):
    """The library's convention: the entry of largest magnitude of each F column is positive."""
    idx = np.argmax(np.abs(F), axis=1)                                  # [n_h][g]
    sgn = np.sign(np.take_along_axis(F, idx[:, None, :], axis=1))[:, 0, :]
    sgn[sgn == 0] = 1.0
    return E * sgn[:, None, :], lam, F * sgn[:, None, :]


@pytest.mark.parametrize("w,prec", SVD_CASES, ids=[f"{w.name}-{p}" for w, p in SVD_CASES])
def test_column_svd_matches_numpy(mods, w, prec):
    """E_m, Lambda_m, F_m of every column against numpy.linalg.svd of the oracle's A_m (same
    rounded ensemble), after fixing each singular pair's sign by the same rule; plus the
    factorisation A_m = E_m Lambda_m F_m^T and the orthonormality of E_m and F_m."""
    zl, diag = mods
    dt = synth.storage_dtype(prec)
    Z = synth.ensemble(w).astype(dt)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=w.tau, prec=prec, max_rhs=4, nx=w.Nx, ny=w.Ny)
    E, L, F = (t.cpu().numpy() for t in diag.column_svd(plan))
    oracle = swift.Plan(Z.astype(np.float64), w.Nx, w.Ny, lam, w.tau)
    Eo, Lo, Fo = sign_fixed(oracle.E, oracle.Lam, oracle.F)
    smax = Lo[:, :1]
    assert np.all(np.abs(L - Lo) <= 1e-12 * smax)
    assert np.all(np.diff(L, axis=1) <= 0)
    A = oracle.A                                                      # [n_h][n_w][K]
    rec = np.einsum("mli,mi,mki->mlk", E, L, F)
    assert np.abs(rec - A).max() <= 1e-12 * np.abs(A).max()
    g = L.shape[1]
    for Q in (E, F):
        G = np.einsum("mai,maj->mij", Q, Q)
        assert np.abs(G - np.eye(g)[None]).max() <= 1e-12
    assert np.abs(E - Eo).max() <= 1e-8 and np.abs(F - Fo).max() <= 1e-8


def test_xi_kernel_against_its_definition(mods):
    """zl_xi_indicators on a random non-square-like M: sum of squares and max of I - M M^T."""
    zl, _ = mods
    rng = np.random.default_rng(5)
    for n in (1, 31, 70):
        M = rng.standard_normal((n, n)) / np.sqrt(n)
        Xi = np.eye(n) - M @ M.T
        out = zl.zl_xi_indicators(torch.from_numpy(M).cuda()).cpu().numpy()
        assert abs(out[0] - np.sum(Xi ** 2)) <= 1e-12 * np.sum(Xi ** 2)
        assert out[1] == pytest.approx(np.abs(Xi).max(), rel=1e-13)
