"""Horizontal eigenbasis and spectrum of a circulant localization (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 3.9 of the paper writes the localization block as an economical
eigendecomposition C_b = V_b Delta_b V_b^T, keeping only the columns of the
orthogonal eigenvector matrix whose eigenvalue is non-zero; Sec. 3.11 notes
that V_b can be generated analytically instead of stored.  On a doubly
periodic grid with an even, separable correlation function the eigenvectors
are the real Fourier modes, so the oracle fixes that basis explicitly:

Per axis of length N the packed real-Fourier basis is
    b_0(m)      = 1/sqrt(N)
    b_{2j-1}(m) = sqrt(2/N) cos(2 pi j m / N)      j = 1 .. ceil(N/2)-1
    b_{2j}(m)   = sqrt(2/N) sin(2 pi j m / N)
    b_{N-1}(m)  = (-1)^m / sqrt(N)                 (N even only)
with frequency f(p) = 0, j, j, N/2.  In 2-D the basis is the Kronecker product
B_y (x) B_x, grid point m = y*N_x + x, packed mode s = p_y*N_x + p_x.

The paper gives no threshold for "non-zero" eigenvalues; the oracle keeps
S = {s : lambda_s > tau * max(lambda)}, sorted ascending in s.
"""

import numpy as np


def packed_frequency(N):
    """Frequency f(p) of every packed index p for an axis of length N."""
    f = np.zeros(N, dtype=np.int64)
    for p in range(1, N):
        if N % 2 == 0 and p == N - 1:
            f[p] = N // 2
        else:
            f[p] = (p + 1) // 2
    return f


def basis_1d(N):
    """N x N orthogonal matrix whose column p is the packed basis vector b_p."""
    m = np.arange(N, dtype=np.float64)
    B = np.empty((N, N), dtype=np.float64)
    B[:, 0] = 1.0 / np.sqrt(N)
    for p in range(1, N):
        if N % 2 == 0 and p == N - 1:
            B[:, p] = np.where(np.arange(N) % 2 == 0, 1.0, -1.0) / np.sqrt(N)
        else:
            j = (p + 1) // 2
            arg = 2.0 * np.pi * j * m / N
            B[:, p] = np.sqrt(2.0 / N) * (np.cos(arg) if p % 2 == 1 else np.sin(arg))
    return B


def basis_2d(Nx, Ny):
    """Dense n_h x n_h basis V = B_y (x) B_x (rows: m = y*Nx+x, cols: s = py*Nx+px)."""
    return np.kron(basis_1d(Ny), basis_1d(Nx))


def _images(N, ell):
    """How many periodic images make exp(-(d+pN)^2 / 2 ell^2) negligible."""
    return int(np.ceil(12.0 * ell / N)) + 2


def periodized_gaussian(N, ell):
    """c(d), d = 0..N-1: sum_p exp(-(d+pN)^2/(2 ell^2)) normalised to c(0) = 1.

    The paper requires a localization with unit diagonal (Sec. 2, Sec. 4.4);
    periodizing the Gaussian makes it positive semi-definite on the ring.
    N == 1 (an axis that does not exist) gives c = [1].
    """
    if N == 1:
        return np.ones(1)
    P = _images(N, ell)
    d = np.arange(N, dtype=np.float64)
    num = np.zeros(N)
    den = 0.0
    for p in range(-P, P + 1):
        num += np.exp(-((d + p * N) ** 2) / (2.0 * ell * ell))
        den += np.exp(-((p * N) ** 2) / (2.0 * ell * ell))
    return num / den


def circulant(c):
    """Dense symmetric circulant matrix C[i, j] = c((i - j) mod N)."""
    N = len(c)
    idx = (np.arange(N)[:, None] - np.arange(N)[None, :]) % N
    return c[idx]


def spectrum_1d_direct(N, ell):
    """The definition: lambda(f(p)) = sum_d c(d) cos(2 pi f d / N) for every packed basis vector.

    In FP64 this sum cancels to about 1e-16 of the largest eigenvalue, i.e. it keeps only
    ~1e-6 relative accuracy for the smallest eigenvalues above the threshold tau = 1e-10,
    which the left inverse scales by lambda^{-1/2}; ``spectrum_1d`` therefore evaluates the
    same eigenvalues by Poisson summation, and this sum pins it."""
    c = periodized_gaussian(N, ell)
    f = packed_frequency(N)
    d = np.arange(N, dtype=np.float64)
    return np.array([np.sum(c * np.cos(2.0 * np.pi * fp * d / N)) for fp in f])


def spectrum_1d(N, ell):
    """Eigenvalue of every packed basis vector of the periodized Gaussian (Poisson closed form)."""
    return spectrum_1d_closed_form(N, ell)


def spectrum_1d_closed_form(N, ell):
    """The eigenvalues of ``spectrum_1d_direct`` by Poisson summation, a sum of positive terms
    (accurate in relative terms down to the smallest eigenvalue):

    sum_{t in Z} exp(-t^2/2ell^2) e^{-2 pi i f t / N}
        = sqrt(2 pi) ell sum_q exp(-2 pi^2 ell^2 (f/N - q)^2).
    """
    if N == 1:
        return np.ones(1)
    f = packed_frequency(N).astype(np.float64)
    Q = int(np.ceil(4.0 / max(ell, 1e-3))) + 3
    s = np.zeros(N)
    for q in range(-Q, Q + 1):
        s += np.exp(-2.0 * np.pi ** 2 * ell ** 2 * (f / N - q) ** 2)
    P = _images(N, ell)
    den = sum(np.exp(-((p * N) ** 2) / (2.0 * ell * ell)) for p in range(-P, P + 1))
    return np.sqrt(2.0 * np.pi) * ell * s / den


def spectrum_2d(Nx, Ny, ell):
    """lambda[s], s = py*Nx + px, of the separable periodized Gaussian of length ell."""
    lx = spectrum_1d(Nx, ell)
    ly = spectrum_1d(Ny, ell)
    return np.outer(ly, lx).reshape(-1)


def localization_block(Nx, Ny, ell):
    """Dense n_h x n_h localization block C_b (direct from c(d), no basis)."""
    return np.kron(circulant(periodized_gaussian(Ny, ell)), circulant(periodized_gaussian(Nx, ell)))


def kept_modes(lam, tau):
    """Indices s with lambda_s > tau * max(lambda), ascending (the economical basis)."""
    lam = np.asarray(lam, dtype=np.float64)
    return np.nonzero(lam > tau * lam.max())[0]
