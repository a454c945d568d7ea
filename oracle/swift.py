"""Vector-form swift algorithm, in FP64 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation follows the paper (Sec. 3.2-3.10):
  Z      ensemble, array [K][n_w][n_h]; member k is z_k, segment l is z_{l,k}
         (the segment ordering of Sec. 3.4), so z_k[l*n_h + m] = Z[k, l, m].
  A_m    the n_w x K matrix of the m-th grid vertical column, A_m[l, k] =
         Z[k, l, m] (Sec. 3.9: Z with every row deleted except those of column m).
  x      a batch of state vectors, array [R][n_w][n_h] (same segment order).
  xt     standardized variables x~ = Zh^- x, array [R][K][L] (Sec. 3.10, V5).

The paper assumes n_w = K so that every A_m is square and invertible
(Sec. 3.8, Eq. nwEqualsK), and computes A_m^{-1} from the per-column singular
value decomposition A_m = E_m Lambda_m F_m^T (Eq. svdOfAm; step V1 writes
w^(m) = F_m Lambda_m^{-1} E_m^T x^(m)).  The oracle does exactly that with the
thin SVD, which for n_w != K yields the pseudo-inverse
A_m^+ = F_m Lambda_m^{-1} E_m^T (minimum norm for n_w < K, least squares for
n_w > K) and equals A_m^{-1} when n_w = K.  Column m is reported as
rank-deficient when sigma_min^2 <= rank_eps * sum_i sigma_i^2 (Supporting
information S2: rank(A) = sum_m rank(A_m), so invertibility is decided column
by column).

A second route, through the Gram matrix and its Cholesky factor,
  n_w <= K:  G_m = A_m A_m^T,  A_m^+ = A_m^T G_m^{-1}
  n_w >  K:  G_m = A_m^T A_m,  A_m^+ = G_m^{-1} A_m^T
is kept for pinning (it agrees with the SVD route up to cond(A_m)^2 * eps).
"""

import numpy as np

from . import basis as _basis


class Plan:
    """Everything the swift algorithm precomputes (experiment steps (a)-(e), Sec. 4.7)."""

    def __init__(self, Z, Nx, Ny, lam, tau, rank_eps=1e-13):
        Z = np.asarray(Z, dtype=np.float64)
        K, nw, nh = Z.shape
        if nh != Nx * Ny:
            raise ValueError("n_h must equal Nx*Ny")
        self.Z, self.K, self.nw, self.nh, self.Nx, self.Ny = Z, K, nw, nh, Nx, Ny
        # step (a): the column matrices A_m, stored as A[m, l, k]
        self.A = np.transpose(Z, (2, 1, 0)).copy()
        self.g = min(nw, K)
        # step (b): thin SVD of every A_m (E_m: n_w x g, Lambda_m: g, F_m: K x g)
        U, sig, Vh = np.linalg.svd(self.A, full_matrices=False)
        self.E, self.Lam, self.F = U, sig, np.transpose(Vh, (0, 2, 1))
        tr = np.sum(sig ** 2, axis=1)
        bad = ~(sig[:, -1] ** 2 > rank_eps * tr)
        idx = np.nonzero(bad)[0]
        self.bad_column = int(idx[0]) if len(idx) else -1
        self.rank_eps = rank_eps
        # steps (d)-(e): economical eigendecomposition of C_b
        lam = np.asarray(lam, dtype=np.float64)
        self.lam_full = lam
        self.S = _basis.kept_modes(lam, tau)
        self.lamS = lam[self.S]
        self.L = len(self.S)
        self.Bx = _basis.basis_1d(Nx)
        self.By = _basis.basis_1d(Ny)

    @property
    def ok(self):
        return self.bad_column < 0


def cholesky_columns(G, rank_eps):
    """Lower Cholesky factor of every G[m]; returns (Lc, first bad column or -1).

    Plain right-looking factorisation, vectorised over the columns m only.
    A pivot d_j <= rank_eps * trace(G_m) marks column m as rank-deficient; its
    factor is then filled with NaN.
    """
    nh, g, _ = G.shape
    Lc = np.zeros_like(G)
    tr = np.trace(G, axis1=1, axis2=2)
    bad = np.zeros(nh, dtype=bool)
    for j in range(g):
        d = G[:, j, j] - np.sum(Lc[:, j, :j] ** 2, axis=1)
        bad |= ~(d > rank_eps * tr)
        d = np.where(bad, 1.0, d)
        Lc[:, j, j] = np.sqrt(d)
        if j + 1 < g:
            Lc[:, j + 1:, j] = (G[:, j + 1:, j] - np.einsum("mik,mk->mi", Lc[:, j + 1:, :j], Lc[:, j, :j])) / Lc[:, j, j][:, None]
    Lc[bad] = np.nan
    idx = np.nonzero(bad)[0]
    return Lc, (int(idx[0]) if len(idx) else -1)


def cholesky_solve(Lc, b):
    """Solve G_m u = b_m for every column m (G_m = Lc_m Lc_m^T); b is [n_h][g][R]."""
    nh, g, _ = Lc.shape
    y = np.zeros_like(b)
    for i in range(g):
        y[:, i, :] = (b[:, i, :] - np.einsum("mj,mjr->mr", Lc[:, i, :i], y[:, :i, :])) / Lc[:, i, i][:, None]
    u = np.zeros_like(b)
    for i in reversed(range(g)):
        u[:, i, :] = (y[:, i, :] - np.einsum("mj,mjr->mr", Lc[:, i + 1:, i], u[:, i + 1:, :])) / Lc[:, i, i][:, None]
    return u


# ---------------------------------------------------------------------------
# V_b^T and V_b: the horizontal transform in the packed real-Fourier basis
# ---------------------------------------------------------------------------

def forward_transform(plan, w):
    """V_b^T w for every field w[..., n_h]; returns [..., L] (kept modes only)."""
    lead = w.shape[:-1]
    f = w.reshape(lead + (plan.Ny, plan.Nx))
    c = f @ plan.Bx                                     # along x: [..., y, p_x]
    c = np.swapaxes(np.swapaxes(c, -1, -2) @ plan.By, -1, -2)  # along y: [..., p_y, p_x]
    return c.reshape(lead + (plan.nh,))[..., plan.S]


def inverse_transform(plan, c):
    """V_b c for every coefficient vector c[..., L]; returns [..., n_h]."""
    lead = c.shape[:-1]
    full = np.zeros(lead + (plan.nh,))
    full[..., plan.S] = c
    f = full.reshape(lead + (plan.Ny, plan.Nx))
    f = f @ plan.Bx.T                                   # x: sum over p_x
    f = np.swapaxes(np.swapaxes(f, -1, -2) @ plan.By.T, -1, -2)
    return f.reshape(lead + (plan.nh,))


# ---------------------------------------------------------------------------
# Per-column pseudo-inverse and its transpose (step V1 and its adjoint)
# ---------------------------------------------------------------------------

def column_pinv_apply(plan, X):
    """w^(m) = A_m^+ x^(m) = F_m Lambda_m^{-1} E_m^T x^(m); X is [n_h][n_w][R] -> [n_h][K][R]."""
    Et = np.transpose(plan.E, (0, 2, 1))
    return plan.F @ ((Et @ X) / plan.Lam[:, :, None])


def column_pinv_transpose_apply(plan, V):
    """g^(m) = (A_m^+)^T v^(m) = E_m Lambda_m^{-1} F_m^T v^(m); V is [n_h][K][R] -> [n_h][n_w][R]."""
    Ft = np.transpose(plan.F, (0, 2, 1))
    return plan.E @ ((Ft @ V) / plan.Lam[:, :, None])


def gram(A):
    """G_m = A_m A_m^T if n_w <= K else A_m^T A_m, for every column."""
    nw, K = A.shape[1], A.shape[2]
    At = np.transpose(A, (0, 2, 1))
    return A @ At if nw <= K else At @ A


def gram_route_pinv_apply(A, X, rank_eps=1e-13):
    """A_m^+ x^(m) through G_m and its Cholesky factor (second route, for pins).

    Returns (W, first bad column or -1); W is [n_h][K][R].
    """
    nw, K = A.shape[1], A.shape[2]
    Lc, bad = cholesky_columns(gram(A), rank_eps)
    At = np.transpose(A, (0, 2, 1))
    if nw <= K:
        return At @ cholesky_solve(Lc, X), bad
    return cholesky_solve(Lc, At @ X), bad


# ---------------------------------------------------------------------------
# The four operators
# ---------------------------------------------------------------------------

def apply_left_inverse(plan, x):
    """x~ = Zh^- x = Delta^{-1/2} V^T A^+ x by steps V1-V5 (Sec. 3.10).

    V1: w^(m) = A_m^+ x^(m) for every column m;
    V2/V3: regroup w into its K segments w_k (one per member);
    V4: x~_k = Delta_b^{-1/2} V_b^T w_k;
    V5: concatenate -> [R][K][L].
    """
    x = np.asarray(x, dtype=np.float64)
    R = x.shape[0]
    X = np.transpose(x, (2, 1, 0))                      # x^(m): [n_h][n_w][R]
    W = column_pinv_apply(plan, X)                      # w^(m): [n_h][K][R]
    w = np.transpose(W, (2, 1, 0))                      # segments w_k: [R][K][n_h]
    return forward_transform(plan, w) / np.sqrt(plan.lamS)


def apply_sqrt(plan, xt):
    """x = Zh x~ = A V Delta^{1/2} x~ (Sec. 3.9)."""
    xt = np.asarray(xt, dtype=np.float64)
    y = inverse_transform(plan, xt * np.sqrt(plan.lamS))  # y_k = V_b Delta_b^{1/2} x~_k
    Y = np.transpose(y, (2, 1, 0))                      # [n_h][K][R]
    X = plan.A @ Y                                      # x^(m) = A_m y^(m)
    return np.transpose(X, (2, 1, 0))


def apply_adjoint(plan, y):
    """g = (Zh^-)^T y = (A^+)^T V Delta^{-1/2} y (transpose of Eq. InverseSquareRootAlmost)."""
    y = np.asarray(y, dtype=np.float64)
    v = inverse_transform(plan, y / np.sqrt(plan.lamS))
    V = np.transpose(v, (2, 1, 0))
    return np.transpose(column_pinv_transpose_apply(plan, V), (2, 1, 0))


def apply_sqrt_adjoint(plan, x):
    """Zh^T x = Delta^{1/2} V^T A^T x."""
    x = np.asarray(x, dtype=np.float64)
    X = np.transpose(x, (2, 1, 0))
    T = np.transpose(plan.A, (0, 2, 1)) @ X             # A_m^T x^(m): [n_h][K][R]
    t = np.transpose(T, (2, 1, 0))
    return forward_transform(plan, t) * np.sqrt(plan.lamS)
