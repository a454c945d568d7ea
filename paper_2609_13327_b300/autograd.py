"""torch.autograd wrappers of the library's operators (argument marshalling only).

``left_inverse(plan, x)`` is x~ = Zh^- x (the vector algorithm V1-V5, Sec. 3.10) with its
vector-Jacobian product (Zh^-)^T g computed by the library's adjoint kernels
(``zl_apply_adjoint``), so a variational cost such as J(x) = 1/2 ||Zh^- x||^2 can be
differentiated through it.  ``sqrt(plan, xt)`` is x = Zh x~ (Sec. 3.9, Zh = A V Delta^{1/2})
with its vector-Jacobian product Zh^T g (``zl_apply_sqrt_adjoint``).  Every computation
runs in libzl's CUDA kernels; there is no fallback.
"""

import torch

from . import zl


class _LeftInverse(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return zl.zl_apply_left_inverse(plan, x.contiguous())

    @staticmethod
    def backward(ctx, g):
        return zl.zl_apply_adjoint(ctx.plan, g.contiguous()), None


class _Sqrt(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xt, plan):
        ctx.plan = plan
        return zl.zl_apply_sqrt(plan, xt.contiguous())

    @staticmethod
    def backward(ctx, g):
        return zl.zl_apply_sqrt_adjoint(ctx.plan, g.contiguous()), None


def left_inverse(plan, x):
    """x~ = Zh^- x for x [R][n_w][n_h] on the plan's device and dtype, differentiable in x."""
    return _LeftInverse.apply(x, plan)


def sqrt(plan, xt):
    """x = Zh x~ for x~ [R][K][L], differentiable in x~."""
    return _Sqrt.apply(xt, plan)
