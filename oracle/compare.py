"""Parity criteria of a result against the oracle's (test infrastructure).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): used by ``tests/`` and
``__graft_entry__.smoke()``; it holds no arithmetic of the method.

A result ``got`` and the oracle's ``ref`` are arrays [R][A][B] (R right-hand
sides).  The ``slice_axis`` (1 or 2) names the axis whose entries have their
own scale:

* outputs in standardized variables [R][K][L]: the modes (axis 2).  Mode j is
  scaled by lambda_j^{-1/2}, which spans five decades at tau = 1e-10, so a
  norm over a right-hand side is dominated by the smallest-lambda modes and
  says nothing about the others;
* outputs in model space [R][n_w][n_h]: the levels (axis 1), whose variances
  differ by two decades in the mixed-precision workloads.

Three bounds, all required (d = got - ref):

1. per right-hand side  ||d_r||_2 <= tol ||ref_r||_2
   (the relative error of the metric);
2. per slice s          ||d_s||_2 <= C_SLICE tol ||ref_s||_2
   (an error confined to a few modes or levels, invisible in 1, fails here);
3. per element i        |d_i| <= C_ELEM tol rms(ref_s(i))
   (a single wrong slot fails here).

The rounding errors of every path are about uniform in relative terms across
modes (the per-mode scale is applied once, after the transform) and levels,
so the slice bound holds with the same margin as the norm bound; C_ELEM
leaves room for the largest of a few thousand Gaussian-distributed element
errors (about four times their rms).
"""

import numpy as np

C_SLICE = 4.0
C_ELEM = 16.0


def measures(got, ref, slice_axis):
    """(per-rhs max relative error, worst slice (index, relative error), worst element (index, ratio))."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.shape != ref.shape or got.ndim != 3:
        raise ValueError(f"shape mismatch or not [R][A][B]: {got.shape} vs {ref.shape}")
    R = got.shape[0]
    d = got - ref
    if not np.all(np.isfinite(got)):
        bad = np.argwhere(~np.isfinite(got))[0]
        return np.inf, (int(bad[slice_axis]), np.inf), (tuple(int(v) for v in bad), np.inf)
    rn = np.linalg.norm(ref.reshape(R, -1), axis=1)
    dn = np.linalg.norm(d.reshape(R, -1), axis=1)
    rhs_err = float(np.max(np.where(rn > 0, dn / np.where(rn > 0, rn, 1.0), np.where(dn > 0, np.inf, 0.0))))
    other = tuple(a for a in range(3) if a != slice_axis)
    sref = np.sqrt(np.sum(ref ** 2, axis=other))
    sd = np.sqrt(np.sum(d ** 2, axis=other))
    # a slice whose reference is exactly zero is measured against the mean slice scale
    floor = np.sqrt(np.mean(sref ** 2)) if np.any(sref > 0) else 1.0
    sscale = np.where(sref > 0, sref, floor)
    srel = sd / sscale
    js = int(np.argmax(srel))
    count = R * got.shape[other[1]]
    rms = sscale / np.sqrt(count)
    shape = [1, 1, 1]
    shape[slice_axis] = -1
    ratio = np.abs(d) / rms.reshape(shape)
    ie = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    return rhs_err, (js, float(srel[js])), (tuple(int(v) for v in ie), float(ratio[ie]))


def check(got, ref, tol, slice_axis, what=""):
    """Assert the three bounds; the message names the worst slice and element."""
    rhs_err, (js, s_err), (ie, e_ratio) = measures(got, ref, slice_axis)
    msg = (f"{what}: per-rhs rel. err {rhs_err:.3e} (tol {tol:.1e}); worst slice {js} (axis {slice_axis}) "
           f"rel. err {s_err:.3e} (bound {C_SLICE * tol:.1e}); worst element {ie} at {e_ratio:.3e} x its "
           f"slice rms (bound {C_ELEM * tol:.1e})")
    assert rhs_err <= tol and s_err <= C_SLICE * tol and e_ratio <= C_ELEM * tol, msg
    return rhs_err
