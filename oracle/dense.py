"""Dense brute force at tiny sizes (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Forms the paper's matrices explicitly, with state index i = l*n_h + m
(segment order, Sec. 3.4) and square-root column index (k, j) -> k*L + j:

* C^{1/2}   n x L, L stacked copies of C_b^{1/2} = V_b Delta_b^{1/2} (Eq. SqrtOfC)
* Zh        n x K L, Zh = [diag(z_1) C^{1/2}, ..., diag(z_K) C^{1/2}]
            (Eq. SQRTofPCModulation, the modulated-ensemble square root)
* A         n x K n_h, block (l, k) = diag(z_{l,k}) (Eq. ADef)
* V, Delta  block diagonal with K copies of V_b and Delta_b (Eq. VBlocks, DeltaBlocks)
* Zh^-      Delta^{-1/2} V^T A^+ (Eq. InverseSquareRootAlmost with A^{-1} -> A^+,
            A^+ by dense SVD, i.e. ``numpy.linalg.pinv``)
* Xi        I - Zh^- (Zh Zh^T) Zh^-^T and its two indicators (Sec. 4.8)
* delta     x~ - Zh^- Zh x~ and its 2-norm (Sec. 4.9)
"""

import numpy as np

from . import basis as _basis


def member_matrix(Z):
    """Z as the n x K matrix whose columns are the members z_k."""
    Z = np.asarray(Z, dtype=np.float64)
    K = Z.shape[0]
    return Z.reshape(K, -1).T


def sqrt_localization(Nx, Ny, lam, S, nw):
    """C^{1/2}: n_w stacked copies of V_b Delta_b^{1/2} (n x L)."""
    Vb = _basis.basis_2d(Nx, Ny)[:, S]
    Cb_half = Vb * np.sqrt(np.asarray(lam)[S])[None, :]
    return np.vstack([Cb_half] * nw)


def modulated_sqrt(Z, Nx, Ny, lam, S):
    """Zh = C^{1/2} (triangle) Z: columns c_j (.) z_k, ordered (k, j)."""
    Zm = member_matrix(Z)
    K, nw = Z.shape[0], Z.shape[1]
    Ch = sqrt_localization(Nx, Ny, lam, S, nw)
    return np.hstack([Zm[:, k:k + 1] * Ch for k in range(K)])


def matrix_A(Z):
    """A (n x K n_h): block (l, k) is diag(z_{l,k})."""
    Z = np.asarray(Z, dtype=np.float64)
    K, nw, nh = Z.shape
    A = np.zeros((nw * nh, K * nh))
    for l in range(nw):
        for k in range(K):
            A[l * nh:(l + 1) * nh, k * nh:(k + 1) * nh] = np.diag(Z[k, l])
    return A


def block_V(Nx, Ny, S, K):
    """V: K diagonal copies of V_b (K n_h x K L)."""
    Vb = _basis.basis_2d(Nx, Ny)[:, S]
    return np.kron(np.eye(K), Vb)


def left_inverse_matrix(Z, Nx, Ny, lam, S):
    """Dense Zh^- = Delta^{-1/2} V^T A^+, A^+ from a dense SVD."""
    K = Z.shape[0]
    Apinv = np.linalg.pinv(matrix_A(Z), rcond=1e-13)
    V = block_V(Nx, Ny, S, K)
    dinv = np.tile(1.0 / np.sqrt(np.asarray(lam)[S]), K)
    return dinv[:, None] * (V.T @ Apinv)


def xi_indicators(Zinv, Zh):
    """Xi = I - Zh^- Ph Zh^-^T with Ph = Zh Zh^T; returns (||Xi||_F, max |Xi_ij|).

    The paper calls the first one RMSE_Xi but defines it without a mean, i.e.
    the Frobenius norm (Sec. 4.8); it is reported as such.
    """
    M = Zinv @ Zh
    Xi = np.eye(M.shape[0]) - M @ M.T
    return float(np.sqrt(np.sum(Xi ** 2))), float(np.max(np.abs(Xi)))


def rmse_delta(Zinv, Zh, xt):
    """||x~ - Zh^- Zh x~||_2 (Sec. 4.9; again a 2-norm, not a mean)."""
    return float(np.linalg.norm(xt - Zinv @ (Zh @ xt)))
