"""The parity criteria (oracle/compare.py) catch what a per-right-hand-side norm hides.

Mistakes are planted in a copy of an oracle output, on the CPU: a whole mode with a
large eigenvalue (small lambda^{-1/2}, so it carries almost none of the norm), a
single (member, mode) slot, one level of a model-space field.  Each passes the norm
bound and fails the slice or element bound; a uniform relative perturbation of half
the tolerance passes all three.
"""

import numpy as np
import pytest

from oracle import basis, compare, swift
from paper_2609_13327_b300 import synth

W = synth.Workload("cmp", 32, 24, 6, 12, 3.0, 0.7, 3.0, 5, "fp64", 91, var_range=(0.1, 10.0))


@pytest.fixture(scope="module")
def outputs():
    Z = synth.ensemble(W)
    lam = basis.spectrum_2d(W.Nx, W.Ny, W.ell_loc)
    plan = swift.Plan(Z, W.Nx, W.Ny, lam, W.tau)
    xt = swift.apply_left_inverse(plan, synth.rhs(W))
    xs = swift.apply_sqrt(plan, synth.coefficients(W, plan.L))
    return plan, xt, xs


def test_uniform_relative_noise_passes(outputs):
    plan, xt, xs = outputs
    rng = np.random.default_rng(0)
    tol = 1e-5
    for ref, axis in ((xt, 2), (xs, 1)):
        got = ref * (1 + 0.5 * tol * rng.standard_normal(ref.shape) / 3)
        compare.check(got, ref, tol, axis, "noise")


def test_a_wrong_large_eigenvalue_mode_is_caught(outputs):
    plan, xt, _ = outputs
    j = int(np.argmax(plan.lamS))                       # lambda^{-1/2} smallest: the mode hides in the norm
    got = xt.copy()
    got[:, :, j] *= 1.5
    rhs_err, (js, s_err), _ = compare.measures(got, xt, 2)
    assert rhs_err < 1e-5 and js == j
    with pytest.raises(AssertionError):
        compare.check(got, xt, 1e-5, 2, "planted mode")


def test_a_single_wrong_slot_is_caught(outputs):
    plan, xt, _ = outputs
    got = xt.copy()
    j = int(np.argsort(plan.lamS)[len(plan.lamS) // 2])
    got[2, 5, j] += 1e-3 * abs(got[2, 5, j]) + 1e-3 * np.sqrt(np.mean(xt[:, :, j] ** 2))
    assert compare.measures(got, xt, 2)[0] < 1e-5
    with pytest.raises(AssertionError):
        compare.check(got, xt, 1e-5, 2, "planted slot")


def test_a_wrong_level_is_caught(outputs):
    _, _, xs = outputs
    scale = np.linalg.norm(xs, axis=(0, 2))
    lq = int(np.argmin(scale))                          # the level with the smallest variance
    got = xs.copy()
    got[:, lq, :] *= 1 + 6e-5                          # 6e-5 of that level: above the slice bound 4e-5
    rhs_err, (ls, s_err), _ = compare.measures(got, xs, 1)
    assert rhs_err < 1e-5 and ls == lq
    with pytest.raises(AssertionError):
        compare.check(got, xs, 1e-5, 1, "planted level")


def test_non_finite_output_fails(outputs):
    _, xt, _ = outputs
    got = xt.copy()
    got[0, 0, 0] = np.nan
    with pytest.raises(AssertionError):
        compare.check(got, xt, 1e-5, 2, "nan")
