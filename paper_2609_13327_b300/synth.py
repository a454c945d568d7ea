"""Seeded synthetic workloads: ensembles and right-hand sides.

This module only draws random inputs; it contains none of the swift
algorithm's arithmetic (no Gram matrices, no eigenbasis, no spectrum of the
localization).  Both the CUDA library's tests/benchmark and the FP64 oracle
receive the arrays it returns.

Ensemble recipe (the paper's experiment uses a spherical grid and a
spherical-harmonics covariance that it does not specify completely, Sec. 4.1-4.3
and S4-S5; these doubly periodic stand-ins keep the structure):

* every member e_k' is a Gaussian random field, horizontally correlated with a
  Gaussian correlation of length ell_c (white noise circularly convolved with a
  periodized Gaussian kernel, normalised to unit variance), vertically an AR(1)
  process with lag-one correlation rho across the n_w levels, then scaled by a
  per-level standard deviation sigma_l;
* the paper's rank-safe draw (Sec. 4.2): draw K' = K + 4 members, subtract the
  mean over all K', discard 4 of them at random, scale by 1/sqrt(K-1) so that
  P^s = Z Z^T (Sec. 3.3).
"""

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    Nx: int
    Ny: int
    nw: int
    K: int
    ell_c: float
    rho: float
    ell_loc: float
    R: int
    prec: str            # "fp64", "fp32" or "mixed"
    seed: int
    tau: float = 1e-10
    var_range: tuple = (1.0, 1.0)   # sigma_l^2 drawn log-uniformly in this range
    extra: dict = field(default_factory=dict)

    @property
    def nh(self):
        return self.Nx * self.Ny

    @property
    def n(self):
        return self.nw * self.nh


# The named workloads.  C0a/C0b satisfy the paper's n_w = K; C1-C5 are the
# 1-GPU benchmark shapes (ring, 128^2 x 10, 256^2 x 32, batched, 512^2 x 16).
WORKLOADS = {
    "c0a_ring": Workload("c0a_ring", 16, 1, 4, 4, 3.0, 0.7, 1.5, 16, "fp64", 100, tau=0.0),
    "c0a_plane": Workload("c0a_plane", 16, 16, 8, 8, 3.0, 0.7, 3.0, 16, "fp64", 100),
    "c0b_paper_shape": Workload("c0b_paper_shape", 16, 12, 64, 64, 2.0, 0.8, 2.0, 50, "fp64", 101),
    "c1_ring64": Workload("c1_ring64", 64, 1, 1, 8, 5.0, 0.0, 8.0, 16, "fp64", 0),
    "c2_128x128x10": Workload("c2_128x128x10", 128, 128, 10, 32, 6.0, 0.7, 10.0, 256, "fp32", 2),
    "c3_256x256x32": Workload("c3_256x256x32", 256, 256, 32, 64, 8.0, 0.8, 16.0, 64, "mixed", 3,
                              var_range=(0.1, 10.0)),
    "c5_512x512x16": Workload("c5_512x512x16", 512, 512, 16, 48, 12.0, 0.75, 24.0, 8, "fp32", 5),
}


def _axis_kernel(N, ell):
    """Periodized Gaussian smoothing kernel along one axis, unit l2 norm.

    Convolving white noise with exp(-t^2/ell^2) gives a field whose
    correlation is exp(-d^2/(2 ell^2)) (the autocorrelation of the kernel).
    """
    if N == 1:
        return np.ones(1)
    t = np.arange(N, dtype=np.float64)
    P = int(np.ceil(8.0 * ell / N)) + 2
    k = np.zeros(N)
    for p in range(-P, P + 1):
        k += np.exp(-((t + p * N) ** 2) / (ell * ell))
    return k / np.sqrt(np.sum(k * k))


def correlated_fields(rng, count, nw, Nx, Ny, ell_c, rho, sigma):
    """`count` fields of shape [n_w][Ny*Nx]: horizontal Gaussian x vertical AR(1)."""
    kx = _axis_kernel(Nx, ell_c)
    ky = _axis_kernel(Ny, ell_c)
    H = np.fft.rfft2(np.outer(ky, kx))
    out = np.empty((count, nw, Ny * Nx))
    a = np.sqrt(max(0.0, 1.0 - rho * rho))
    for c in range(count):
        xi = rng.standard_normal((nw, Ny, Nx))
        f = np.fft.irfft2(np.fft.rfft2(xi) * H, s=(Ny, Nx))     # circular convolution
        prev = None
        for l in range(nw):
            cur = f[l] if prev is None else rho * prev + a * f[l]
            out[c, l] = (sigma[l] * cur).reshape(-1)
            prev = cur
    return out


def ensemble(w, seed=None):
    """Z [K][n_w][n_h] in float64 by the rank-safe K' = K + 4 draw."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    lo, hi = w.var_range
    if lo == hi:
        sigma = np.full(w.nw, np.sqrt(lo))
    else:
        sigma = np.sqrt(np.exp(rng.uniform(np.log(lo), np.log(hi), size=w.nw)))
    Kp = w.K + 4
    E = correlated_fields(rng, Kp, w.nw, w.Nx, w.Ny, w.ell_c, w.rho, sigma)
    E -= E.mean(axis=0, keepdims=True)
    drop = rng.choice(Kp, size=Kp - w.K, replace=False)
    keep = np.setdiff1d(np.arange(Kp), drop)
    return E[keep] / np.sqrt(w.K - 1)


def centred_ensemble(w, seed=None):
    """K members centred on their own mean (the singular case of Sec. 4.2)."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    E = correlated_fields(rng, w.K, w.nw, w.Nx, w.Ny, w.ell_c, w.rho, np.ones(w.nw))
    E -= E.mean(axis=0, keepdims=True)
    return E / np.sqrt(w.K - 1)


def rhs(w, R=None, seed=None, dtype=np.float64):
    """R i.i.d. N(0, 1) state vectors, [R][n_w][n_h]."""
    rng = np.random.default_rng((w.seed if seed is None else seed) + 7919)
    R = w.R if R is None else R
    return rng.standard_normal((R, w.nw, w.nh), dtype=dtype)


def coefficients(w, L, R=None, seed=None, dtype=np.float64):
    """R i.i.d. N(0, 1) vectors in the standardized space, [R][K][L]."""
    rng = np.random.default_rng((w.seed if seed is None else seed) + 104729)
    R = w.R if R is None else R
    return rng.standard_normal((R, w.K, L), dtype=dtype)


def batched_instances(count=200, seed=4):
    """Uneven independent instances for the batched left inverse: square periodic grids of
    side 32, 48, ..., 192, 4-24 levels, K in [16, 64] members (so n_w > K occurs), a
    localization length 0.05-0.15 of the side, 1-32 right-hand sides, mixed precision.
    The member correlation length is half the localization length, the vertical AR(1)
    correlation 0.75, unit variances (the recipe leaves them open; these follow the other
    workloads)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(rng.choice(np.arange(32, 193, 16)))
        nw = int(rng.integers(4, 25))
        K = int(rng.integers(16, 65))
        ell_loc = float(rng.uniform(0.05, 0.15) * side)
        R = int(rng.integers(1, 33))
        out.append(Workload(f"c4_{i:03d}", side, side, nw, K, 0.5 * ell_loc, 0.75, ell_loc, R, "mixed", seed * 1000 + i))
    return out


def storage_dtype(prec):
    """Element type of every caller-visible buffer for a precision mode."""
    return np.float64 if prec == "fp64" else np.float32
