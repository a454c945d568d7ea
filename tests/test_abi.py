"""Host-side tests of the C ABI: the library loads, exports what include/zl.h
declares, rejects bad arguments before touching the GPU, and its host helper
spectrum matches the oracle.  No kernel is launched here (no GPU needed)."""

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import basis

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def zl():
    from paper_2609_13327_b300 import zl as mod
    return mod


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "zl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(zl_[a-z_]+)\s*\(", text)))


def test_header_declares_the_documented_entry_points():
    names = declared_symbols()
    for must in ("zl_setup", "zl_apply_left_inverse", "zl_apply_sqrt", "zl_apply_adjoint", "zl_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(zl):
    lib = ctypes.CDLL(zl.LIBPATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(zl.EXPORTS) == declared_symbols()


def test_status_strings(zl):
    for code in range(8):
        assert zl.zl_status_string(code).startswith("ZL_")
    assert "unknown" in zl.zl_status_string(99)


@pytest.mark.parametrize("nx,ny,ell", [(64, 1, 8.0), (16, 12, 2.0), (128, 128, 10.0), (48, 48, 5.5), (7, 5, 1.3),
                                       (512, 512, 24.0)])
def test_host_spectrum_matches_oracle(zl, nx, ny, ell):
    """Per eigenvalue in relative terms, down to the smallest kept one (tau = 1e-10)."""
    lam = zl.zl_gaussian_spectrum(nx, ny, ell)
    ref = basis.spectrum_2d(nx, ny, ell)
    assert np.abs(lam - ref).max() <= 1e-13 * ref.max()
    kept = ref > 1e-10 * ref.max()
    assert np.max(np.abs(lam[kept] - ref[kept]) / ref[kept]) <= 1e-12


def test_host_spectrum_rejects_bad_arguments(zl):
    lib = zl._lib
    out = np.empty(4)
    ptr = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.zl_gaussian_spectrum(2, 2, -1.0, ptr) == zl.ZL_ERR_ARG
    assert lib.zl_gaussian_spectrum(2, 2, 1.0, None) == zl.ZL_ERR_ARG
    assert lib.zl_gaussian_spectrum(0, 2, 1.0, ptr) == zl.ZL_ERR_SHAPE


def test_setup_rejects_bad_arguments_before_any_gpu_work(zl):
    lib = zl._lib
    spec = np.ones(16)
    sp = spec.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p(123)
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
    assert lib.zl_setup(None, fake, sp, None, ctypes.byref(h)) == zl.ZL_ERR_ARG
    assert h.value is None
    d = zl.zl_desc(16, 1, 2, 4, zl.ZL_FP32, 1e-10, 8)
    assert lib.zl_setup(ctypes.byref(d), None, sp, None, ctypes.byref(h)) == zl.ZL_ERR_ARG
    assert lib.zl_setup(ctypes.byref(d), fake, None, None, ctypes.byref(h)) == zl.ZL_ERR_ARG
    assert lib.zl_setup(ctypes.byref(d), fake, sp, None, None) == zl.ZL_ERR_ARG
    for bad in (zl.zl_desc(0, 1, 2, 4, 1, 1e-10, 8), zl.zl_desc(16, 1, 0, 4, 1, 1e-10, 8),
                zl.zl_desc(16, 1, 2, 0, 1, 1e-10, 8), zl.zl_desc(16, 1, 2, 4, 1, 1e-10, 0),
                zl.zl_desc(16, 1, 200, 200, 1, 1e-10, 8)):
        assert lib.zl_setup(ctypes.byref(bad), fake, sp, None, ctypes.byref(h)) == zl.ZL_ERR_SHAPE
    for bad in (zl.zl_desc(16, 1, 2, 4, 9, 1e-10, 8), zl.zl_desc(16, 1, 2, 4, 1, -1.0, 8),
                zl.zl_desc(16, 1, 2, 4, 1, float("nan"), 8)):
        assert lib.zl_setup(ctypes.byref(bad), fake, sp, None, ctypes.byref(h)) == zl.ZL_ERR_ARG
    nan_spec = np.ones(16)
    nan_spec[3] = np.nan
    assert lib.zl_setup(ctypes.byref(d), fake, nan_spec.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None,
                        ctypes.byref(h)) == zl.ZL_ERR_ARG
    zero_spec = np.zeros(16)
    assert lib.zl_setup(ctypes.byref(d), fake, zero_spec.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None,
                        ctypes.byref(h)) == zl.ZL_ERR_ARG


def test_applies_reject_null_plan(zl):
    lib = zl._lib
    for name in ("zl_apply_left_inverse", "zl_apply_left_inverse_host", "zl_apply_sqrt", "zl_apply_adjoint",
                 "zl_apply_sqrt_adjoint"):
        assert getattr(lib, name)(None, None, None, 4, None) == zl.ZL_ERR_ARG
    assert lib.zl_get_info(None, None, None, None, None, None) == zl.ZL_ERR_ARG
    assert lib.zl_destroy(None) == zl.ZL_OK


def test_batch_argument_errors_need_no_gpu(zl):
    """Every batch entry point rejects bad arguments before touching the device."""
    lib = zl._lib
    out = ctypes.c_void_p()
    failed = ctypes.c_int(7)
    assert lib.zl_setup_batch(0, None, None, None, None, ctypes.byref(out), ctypes.byref(failed)) == zl.ZL_ERR_ARG
    assert failed.value == -1 and not out.value
    assert lib.zl_setup_batch(2, None, None, None, None, ctypes.byref(out), None) == zl.ZL_ERR_ARG
    assert lib.zl_setup_batch(1, None, None, None, None, None, None) == zl.ZL_ERR_ARG
    assert lib.zl_apply_left_inverse_batch(None, None, None, None, None) == zl.ZL_ERR_ARG
    assert lib.zl_batch_get_info(None, 0, None, None) == zl.ZL_ERR_ARG
    assert lib.zl_destroy_batch(None) == zl.ZL_ERR_ARG


def test_standardize_ensemble_rejects_null_plan(zl):
    assert zl._lib.zl_standardize_ensemble(None, None, None, 4, None) == zl.ZL_ERR_ARG


def test_wait_timeout_hook_rejects_bad_arguments(zl):
    lib = zl._lib
    assert lib.zl_set_test_wait_timeout(None, 1) == zl.ZL_ERR_ARG
    assert lib.zl_set_test_wait_timeout(None, 0) == zl.ZL_ERR_ARG


def test_setup_rejects_a_threshold_that_keeps_no_mode(zl):
    """tau >= 1: no eigenvalue exceeds tau * max, L would be 0 (nothing to apply, and
    per-mode sizes of zero).  Rejected as a shape error before any device work."""
    lib = zl._lib
    spec = np.linspace(1.0, 2.0, 16)
    sp = spec.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p(123)
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
    for prec in (zl.ZL_FP64, zl.ZL_FP32, zl.ZL_MIXED):
        for tau in (1.0, 2.5):
            d = zl.zl_desc(16, 1, 2, 4, prec, tau, 8)
            assert lib.zl_setup(ctypes.byref(d), fake, sp, None, ctypes.byref(h)) == zl.ZL_ERR_SHAPE
            assert h.value is None


def test_static_entry_point_rejects_null_plan(zl):
    assert zl._lib.zl_apply_left_inverse_static(None, None, None, 4, None) == zl.ZL_ERR_ARG
