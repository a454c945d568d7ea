"""Failure detection of the TMA-fed kernels without a GPU fault.

Every wait in the tensor-core column kernel and in the TMA-fed FP32 column
kernel is bounded.  The test hook makes the copy-issuing thread issue no
copies, so the first wait for a copy runs out (about 2 s); the kernel records
a nonzero device error (the tensor-core kernel frees its TMEM) and returns.
The host reads the error through zl_get_runtime_info (ZL_ERR_TIMEOUT), then
switches the hook off, which clears the error, and the same plan and context
give oracle-exact results again.
"""

import numpy as np
import pytest

from oracle import basis, compare, swift
from paper_2609_13327_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"mixed": 1e-5, "fp32": 1e-6}
W = synth.Workload("timeout_case", 32, 12, 10, 40, 4.0, 0.7, 3.0, 21, "mixed", 32)
W32 = synth.Workload("timeout_f32", 32, 12, 10, 40, 4.0, 0.7, 3.0, 21, "fp32", 33)


@pytest.fixture(scope="module")
def zl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_13327_b300 import zl as mod
    return mod


@pytest.mark.parametrize("w", [W, W32], ids=["tensor-core", "fp32-tma"])
def test_bounded_wait_times_out_and_the_context_stays_usable(zl, w):
    W = w
    Z = synth.ensemble(W).astype(np.float32)
    lam = basis.spectrum_2d(W.Nx, W.Ny, W.ell_loc)
    plan = zl.zl_setup(torch.from_numpy(Z).cuda(), lam, tau=W.tau, prec=W.prec, max_rhs=W.R, nx=W.Nx, ny=W.Ny)
    assert plan.uses_tc() == (W.prec == "mixed")
    x = torch.from_numpy(synth.rhs(W, dtype=np.float32)).cuda()
    ref = swift.apply_left_inverse(swift.Plan(Z.astype(np.float64), W.Nx, W.Ny, lam, W.tau),
                                   x.cpu().numpy().astype(np.float64))
    assert plan.device_error() == 0

    plan.set_test_wait_timeout(True)
    zl.zl_apply_left_inverse(plan, x)
    torch.cuda.synchronize()                         # the kernel ended by itself
    code = plan.device_error()
    assert code != 0
    if W.prec == "fp32":
        assert code == 32 + 2                        # the FP32 kernel's compute warps gave up
    info = zl._lib.zl_get_runtime_info(plan.handle, None, None)
    assert info == zl.ZL_OK                          # no error pointer: nothing read
    import ctypes
    c = ctypes.c_int()
    assert zl._lib.zl_get_runtime_info(plan.handle, None, ctypes.byref(c)) == zl.ZL_ERR_TIMEOUT
    assert c.value == code

    plan.set_test_wait_timeout(False)
    assert plan.device_error() == 0
    out = zl.zl_apply_left_inverse(plan, x).cpu().numpy().astype(np.float64)
    assert plan.device_error() == 0
    compare.check(out, ref, TOL[W.prec], 2, "after the timeout")
    # an unrelated allocation and kernel on the same context still work
    t = torch.ones(1 << 20, device="cuda")
    assert float(t.sum()) == float(1 << 20)
