"""Matrix-form accuracy diagnostics of a plan (the paper's Sec. 4.8-4.9 measures).

* ``xi_indicators(plan)``: Xi = I - Zh^- (Zh Zh^T) Zh^-T, the deviation of the left
  inverse from whitening the modulated-ensemble covariance P^ = Zh Zh^T (Sec. 4.8), and
  its two indicators: the Frobenius norm (the paper's "RMSE_Xi", defined without a mean)
  and max |Xi_ij|.  M = Zh^- Zh is formed column by column on the GPU by the library's
  own kernels (the square root of every standardized unit vector, then the left
  inverse), in chunks of the plan's max_rhs; Xi = I - M M^T and its two reductions run
  in libzl's FP64 kernel (``zl_xi_indicators``).  Memory and time grow as (K L)^2 and
  (K L)^3: meant for moderate sizes (K L of a few thousand).
* ``delta(plan, xt)``: x~ - Zh^- Zh x~ per right-hand side and its 2-norm (Sec. 4.9),
  the difference and norms in libzl's kernel (``zl_delta``).
* ``column_svd(plan)``: the per-column SVD A_m = E_m Lambda_m F_m^T (Eq. svdOfAm).

Every computation runs in libzl's kernels; PyTorch supplies device memory (and builds
the unit vectors whose images are M's columns).
"""

import torch

from . import zl


def zh_inverse_zh(plan, stream=None):
    """M = Zh^- Zh (K L x K L, float64 on the plan's device), built in chunks of max_rhs."""
    KL = plan.K * plan.L
    dev = torch.device("cuda")
    M = torch.empty((KL, KL), dtype=torch.float64, device=dev)
    chunk = max(1, plan.desc.max_rhs)
    for j0 in range(0, KL, chunk):
        n = min(chunk, KL - j0)
        e = torch.zeros((n, plan.K, plan.L), dtype=plan.dtype, device=dev)
        e.view(n, KL)[torch.arange(n, device=dev), j0 + torch.arange(n, device=dev)] = 1
        cols = zl.zl_apply_left_inverse(plan, zl.zl_apply_sqrt(plan, e, stream=stream), stream=stream)
        M[:, j0:j0 + n] = cols.view(n, KL).T.to(torch.float64)
    return M


def xi_indicators(plan, stream=None):
    """(||Xi||_F, max |Xi_ij|) with Xi = I - M M^T, M = Zh^- Zh."""
    M = zh_inverse_zh(plan, stream)
    sq, mx = zl.zl_xi_indicators(M, stream=stream).cpu().tolist()
    return sq ** 0.5, mx


def delta(plan, xt, stream=None):
    """x~ - Zh^- Zh x~ for x~ [R][K][L] and the 2-norm of each right-hand side."""
    xt = xt.contiguous()
    back = zl.zl_apply_left_inverse(plan, zl.zl_apply_sqrt(plan, xt, stream=stream), stream=stream)
    return zl.zl_delta(plan, xt, back, stream=stream)


def column_svd(plan, stream=None):
    """(E [n_h][n_w][g], Lambda [n_h][g], F [n_h][K][g]): A_m = E_m diag(Lambda_m) F_m^T per column."""
    return zl.zl_column_svd(plan, stream=stream)
