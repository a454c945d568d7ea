"""Thin Python binding of libzl (ctypes).  Argument marshalling only.

Every computation runs in libzl's CUDA kernels; this module checks tensor
dtypes, devices, shapes and contiguity, passes raw device pointers and the
current CUDA stream, and turns status codes into exceptions.  PyTorch is used
only for device memory and streams.  If ``libzl.so`` has not been built the
import of this module fails loudly: there is no CPU fallback.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libzl.so")

if not os.path.exists(LIBPATH):
    raise ImportError(f"libzl.so is not built ({LIBPATH}); run `python -m paper_2609_13327_b300.build`")

_lib = ctypes.CDLL(LIBPATH)

ZL_OK, ZL_ERR_ARG, ZL_ERR_SHAPE, ZL_ERR_RANK, ZL_ERR_ALLOC, ZL_ERR_CUDA, ZL_ERR_TIMEOUT, ZL_ERR_UNSUPPORTED = range(8)
ZL_FP64, ZL_FP32, ZL_MIXED = 0, 1, 2
PRECISIONS = {"fp64": ZL_FP64, "fp32": ZL_FP32, "mixed": ZL_MIXED}

# every symbol declared in include/zl.h
EXPORTS = ["zl_setup", "zl_get_info", "zl_get_modes", "zl_apply_left_inverse", "zl_apply_left_inverse_host",
           "zl_apply_sqrt", "zl_apply_adjoint", "zl_apply_sqrt_adjoint", "zl_destroy", "zl_status_string",
           "zl_gaussian_spectrum", "zl_set_stage_timing", "zl_get_stage_times", "zl_get_runtime_info",
           "zl_apply_left_inverse_static", "zl_setup_batch", "zl_batch_get_info", "zl_apply_left_inverse_batch",
           "zl_destroy_batch", "zl_standardize_ensemble", "zl_set_test_wait_timeout", "zl_column_svd",
           "zl_xi_indicators", "zl_delta", "zl_apply_left_inverse_rows", "zl_scale_modes",
           "zl_set_test_alloc_failure", "zl_plan_save", "zl_plan_load", "zl_get_desc"]
STAGES = {"fwd_column": 0, "fwd_ypass": 1, "inv_ypass": 2, "inv_column": 3}


class zl_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nw", ctypes.c_int), ("K", ctypes.c_int),
                ("prec", ctypes.c_int), ("tau", ctypes.c_double), ("max_rhs", ctypes.c_int)]


_vp, _int, _ip, _llp, _dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), \
    ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)
_lib.zl_setup.argtypes = [ctypes.POINTER(zl_desc), _vp, _dp, _vp, ctypes.POINTER(_vp)]
_lib.zl_get_info.argtypes = [_vp, _ip, _ip, _ip, _llp, _ip]
_lib.zl_get_modes.argtypes = [_vp, _ip]
for _name in ("zl_apply_left_inverse", "zl_apply_left_inverse_host", "zl_apply_sqrt", "zl_apply_adjoint",
              "zl_apply_sqrt_adjoint", "zl_apply_left_inverse_static", "zl_standardize_ensemble"):
    getattr(_lib, _name).argtypes = [_vp, _vp, _vp, _int, _vp]
_lib.zl_destroy.argtypes = [_vp]
_lib.zl_status_string.argtypes = [_int]
_lib.zl_status_string.restype = ctypes.c_char_p
_lib.zl_gaussian_spectrum.argtypes = [_int, _int, ctypes.c_double, _dp]
_lib.zl_set_stage_timing.argtypes = [_vp, _int]
_lib.zl_get_runtime_info.argtypes = [_vp, _ip, _ip]
_lib.zl_set_test_wait_timeout.argtypes = [_vp, _int]
_lib.zl_get_stage_times.argtypes = [_vp, _int, _ip, _dp]
_lib.zl_setup_batch.argtypes = [_int, ctypes.POINTER(zl_desc), ctypes.POINTER(_vp), ctypes.POINTER(_dp), _vp,
                                ctypes.POINTER(_vp), _ip]
_lib.zl_batch_get_info.argtypes = [_vp, _int, ctypes.POINTER(_vp), _ip]
_lib.zl_apply_left_inverse_batch.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _ip, _vp]
_lib.zl_destroy_batch.argtypes = [_vp]
_lib.zl_column_svd.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.zl_apply_left_inverse_rows.argtypes = [_vp, _int, _int, _vp, _vp, _int, _vp]
_lib.zl_scale_modes.argtypes = [_vp, _vp, _vp, _int, _vp]
_lib.zl_set_test_alloc_failure.argtypes = [_int]
_lib.zl_plan_save.argtypes = [_vp, ctypes.c_char_p]
_lib.zl_plan_load.argtypes = [ctypes.c_char_p, _vp, ctypes.POINTER(_vp)]
_lib.zl_get_desc.argtypes = [_vp, ctypes.c_void_p]
_lib.zl_xi_indicators.argtypes = [_vp, _int, _vp, _vp]
_lib.zl_delta.argtypes = [_vp, _vp, _vp, _vp, _vp, _int, _vp]
for _name in EXPORTS:
    if _name != "zl_status_string":
        getattr(_lib, _name).restype = _int


class ZLError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {zl_status_string(code)}")


def zl_status_string(code):
    return _lib.zl_status_string(int(code)).decode()


def _check(code, where):
    if code != ZL_OK:
        raise ZLError(code, where)


def zl_gaussian_spectrum(nx, ny, ell):
    """Eigenvalues of the separable periodized-Gaussian localization, packed order (host, float64)."""
    out = np.empty(nx * ny, dtype=np.float64)
    _check(_lib.zl_gaussian_spectrum(nx, ny, float(ell), out.ctypes.data_as(_dp)), "zl_gaussian_spectrum")
    return out


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """Owns a zl_plan handle; freed by ``destroy()`` or garbage collection."""

    def __init__(self, handle, desc, owned=True):
        self.handle = handle
        self.desc = desc
        self.owned = owned          # False for the plans of a batch (freed with the batch)
        L, nw, K, nh, bad = _int(), _int(), _int(), ctypes.c_longlong(), _int()
        _check(_lib.zl_get_info(handle, ctypes.byref(L), ctypes.byref(nw), ctypes.byref(K), ctypes.byref(nh),
                                ctypes.byref(bad)), "zl_get_info")
        self.L, self.nw, self.K, self.nh, self.bad_column = L.value, nw.value, K.value, nh.value, bad.value
        self.prec = desc.prec
        self.nx, self.ny = desc.nx, desc.ny

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.prec == ZL_FP64 else torch.float32

    def modes(self):
        out = np.empty(self.L, dtype=np.int32)
        _check(_lib.zl_get_modes(self.handle, out.ctypes.data_as(_ip)), "zl_get_modes")
        return out

    def uses_tc(self):
        """True if the left inverse runs the tcgen05 tensor-core kernel."""
        f = _int()
        _check(_lib.zl_get_runtime_info(self.handle, ctypes.byref(f), None), "zl_get_runtime_info")
        return bool(f.value)

    def device_error(self):
        """0, or the code of a bounded device wait that gave up (synchronises the device)."""
        code = _int()
        rc = _lib.zl_get_runtime_info(self.handle, None, ctypes.byref(code))
        if rc not in (ZL_OK, ZL_ERR_TIMEOUT):
            _check(rc, "zl_get_runtime_info")
        return code.value

    def set_test_wait_timeout(self, enable):
        """Test hook: the tensor-core kernel's bounded wait runs out (enable) / normal
        operation with the device error cleared (disable).  Synchronises the device."""
        _check(_lib.zl_set_test_wait_timeout(self.handle, 1 if enable else 0), "zl_set_test_wait_timeout")

    def set_stage_timing(self, enable):
        _check(_lib.zl_set_stage_timing(self.handle, 1 if enable else 0), "zl_set_stage_timing")

    def stage_times(self):
        """{stage name: (launches, total ms)} of the recorded stage launches."""
        out = {}
        for name, sid in STAGES.items():
            n, ms = _int(), ctypes.c_double()
            _check(_lib.zl_get_stage_times(self.handle, sid, ctypes.byref(n), ctypes.byref(ms)), "zl_get_stage_times")
            out[name] = (n.value, ms.value)
        return out

    def destroy(self):
        if self.handle and self.owned:
            _lib.zl_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def zl_setup(Z, spectrum, tau=1e-10, prec="fp32", max_rhs=64, stream=None, nx=None, ny=None):
    """Build a plan from a device ensemble Z [K][n_w][n_h] and a host spectrum [n_h].

    ``nx``/``ny`` give the grid (default: a ring, ny = 1).  Raises ZLError; on a
    rank-deficient ensemble the error carries ``code == ZL_ERR_RANK`` and the
    offending column is available as ``err.bad_column``.
    """
    import torch
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    want = torch.float64 if p == ZL_FP64 else torch.float32
    if not (isinstance(Z, torch.Tensor) and Z.is_cuda and Z.dtype == want and Z.dim() == 3 and Z.is_contiguous()):
        raise ValueError(f"Z must be a contiguous CUDA {want} tensor [K][n_w][n_h]")
    K, nw, nh = Z.shape
    if nx is None:
        nx, ny = nh, 1
    if nx * ny != nh:
        raise ValueError("nx * ny must equal Z.shape[2]")
    spec = np.ascontiguousarray(spectrum, dtype=np.float64)
    if spec.shape != (nh,):
        raise ValueError("spectrum must have n_h entries")
    d = zl_desc(nx, ny, nw, K, p, float(tau), int(max_rhs))
    h = _vp()
    code = _lib.zl_setup(ctypes.byref(d), _vp(Z.data_ptr()), spec.ctypes.data_as(_dp), _stream_handle(stream),
                         ctypes.byref(h))
    if code == ZL_ERR_RANK:
        plan = Plan(h, d)
        err = ZLError(code, "zl_setup")
        err.bad_column = plan.bad_column
        plan.destroy()
        raise err
    _check(code, "zl_setup")
    return Plan(h, d)


def zl_plan_save(plan, path):
    """Write the plan's descriptor, modes, Z copy and pseudo-inverse to `path`."""
    _check(_lib.zl_plan_save(plan.handle, os.fsencode(path)), "zl_plan_save")


def zl_plan_load(path, stream=None):
    """Restore a plan saved by zl_plan_save (no per-column factorisation)."""
    h = _vp()
    code = _lib.zl_plan_load(os.fsencode(path), _stream_handle(stream), ctypes.byref(h))
    if code == ZL_ERR_RANK:
        plan = Plan(h, _desc_of(h))
        err = ZLError(code, "zl_plan_load")
        err.bad_column = plan.bad_column
        plan.destroy()
        raise err
    _check(code, "zl_plan_load")
    return Plan(h, _desc_of(h))


def _desc_of(handle):
    d = zl_desc()
    _check(_lib.zl_get_desc(handle, ctypes.byref(d)), "zl_get_desc")
    return d


def _apply(fn, plan, inp, in_shape, out_shape, out, stream, where):
    import torch
    if not (isinstance(inp, torch.Tensor) and inp.is_cuda and inp.dtype == plan.dtype and inp.is_contiguous()):
        raise ValueError(f"{where}: input must be a contiguous CUDA {plan.dtype} tensor")
    if inp.dim() != 3 or tuple(inp.shape[1:]) != in_shape:
        raise ValueError(f"{where}: input shape must be [R]{list(in_shape)}")
    R = inp.shape[0]
    if out is None:
        out = torch.empty((R,) + out_shape, dtype=plan.dtype, device=inp.device)
    elif not (out.is_cuda and out.dtype == plan.dtype and out.is_contiguous() and tuple(out.shape) == (R,) + out_shape):
        raise ValueError(f"{where}: bad output tensor")
    _check(fn(plan.handle, _vp(inp.data_ptr()), _vp(out.data_ptr()), R, _stream_handle(stream)), where)
    return out


def zl_apply_left_inverse(plan, x, out=None, stream=None):
    """x~ = Zh^- x: x [R][n_w][n_h] -> x~ [R][K][L]."""
    return _apply(_lib.zl_apply_left_inverse, plan, x, (plan.nw, plan.nh), (plan.K, plan.L), out, stream,
                  "zl_apply_left_inverse")


def zl_standardize_ensemble(plan, members, out=None, stream=None):
    """Forecast members e [K_f][n_w][n_h] -> Zh^- (e_j - mean) / sqrt(K_f - 1), [K_f][K][L]."""
    if members.dim() == 3 and members.shape[0] < 2:
        raise ValueError("zl_standardize_ensemble: at least two members")
    return _apply(_lib.zl_standardize_ensemble, plan, members, (plan.nw, plan.nh), (plan.K, plan.L), out, stream,
                  "zl_standardize_ensemble")


def zl_apply_left_inverse_static(plan, x, out=None, stream=None):
    """x~ = Zh^- x without any device allocation (scratch in the library's static array)."""
    return _apply(_lib.zl_apply_left_inverse_static, plan, x, (plan.nw, plan.nh), (plan.K, plan.L), out, stream,
                  "zl_apply_left_inverse_static")


def zl_apply_sqrt_adjoint(plan, x, out=None, stream=None):
    """Zh^T x: x [R][n_w][n_h] -> [R][K][L]."""
    return _apply(_lib.zl_apply_sqrt_adjoint, plan, x, (plan.nw, plan.nh), (plan.K, plan.L), out, stream,
                  "zl_apply_sqrt_adjoint")


def zl_apply_sqrt(plan, xt, out=None, stream=None):
    """x = Zh x~: x~ [R][K][L] -> x [R][n_w][n_h]."""
    return _apply(_lib.zl_apply_sqrt, plan, xt, (plan.K, plan.L), (plan.nw, plan.nh), out, stream, "zl_apply_sqrt")


def zl_apply_adjoint(plan, y, out=None, stream=None):
    """g = (Zh^-)^T y: y [R][K][L] -> g [R][n_w][n_h]."""
    return _apply(_lib.zl_apply_adjoint, plan, y, (plan.K, plan.L), (plan.nw, plan.nh), out, stream,
                  "zl_apply_adjoint")


def zl_apply_left_inverse_rows(plan, y0, y1, x, out=None, stream=None):
    """One slab's unscaled share of x~: x [R][n_w][(y1 - y0) nx] (the slab's rows) -> [R][K][L]."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == plan.dtype and x.is_contiguous()
            and x.dim() == 3 and tuple(x.shape[1:]) == (plan.nw, (y1 - y0) * plan.nx)):
        raise ValueError("zl_apply_left_inverse_rows: x must be a contiguous CUDA tensor [R][n_w][(y1 - y0) nx]")
    R = x.shape[0]
    if out is None:
        out = torch.empty((R, plan.K, plan.L), dtype=plan.dtype, device=x.device)
    elif not (out.is_cuda and out.dtype == plan.dtype and out.is_contiguous() and tuple(out.shape) == (R, plan.K, plan.L)):
        raise ValueError("zl_apply_left_inverse_rows: bad output tensor")
    _check(_lib.zl_apply_left_inverse_rows(plan.handle, int(y0), int(y1), _vp(x.data_ptr()), _vp(out.data_ptr()), R,
                                           _stream_handle(stream)), "zl_apply_left_inverse_rows")
    return out


def zl_scale_modes(plan, partial, out=None, stream=None):
    """x~ = Delta^{-1/2} partial ([R][K][L]); out may be partial itself."""
    import torch
    if not (isinstance(partial, torch.Tensor) and partial.is_cuda and partial.dtype == plan.dtype
            and partial.is_contiguous() and partial.dim() == 3 and tuple(partial.shape[1:]) == (plan.K, plan.L)):
        raise ValueError("zl_scale_modes: partial must be a contiguous CUDA tensor [R][K][L]")
    if out is None:
        out = torch.empty_like(partial)
    elif not (out.is_cuda and out.dtype == plan.dtype and out.is_contiguous() and out.shape == partial.shape):
        raise ValueError("zl_scale_modes: bad output tensor")
    _check(_lib.zl_scale_modes(plan.handle, _vp(partial.data_ptr()), _vp(out.data_ptr()), partial.shape[0],
                               _stream_handle(stream)), "zl_scale_modes")
    return out


def zl_column_svd(plan, stream=None):
    """Per-column SVD A_m = E_m Lambda_m F_m^T (Eq. svdOfAm): (E [n_h][n_w][g], lam [n_h][g],
    F [n_h][K][g]), float64 CUDA tensors, singular values descending."""
    import torch
    g = min(plan.nw, plan.K)
    E = torch.empty((plan.nh, plan.nw, g), dtype=torch.float64, device="cuda")
    lam = torch.empty((plan.nh, g), dtype=torch.float64, device="cuda")
    F = torch.empty((plan.nh, plan.K, g), dtype=torch.float64, device="cuda")
    _check(_lib.zl_column_svd(plan.handle, _vp(E.data_ptr()), _vp(lam.data_ptr()), _vp(F.data_ptr()),
                              _stream_handle(stream)), "zl_column_svd")
    return E, lam, F


def zl_xi_indicators(M, stream=None):
    """(sum of Xi_ij^2, max |Xi_ij|) of Xi = I - M M^T as a float64 CUDA tensor [2]."""
    import torch
    if not (isinstance(M, torch.Tensor) and M.is_cuda and M.dtype == torch.float64 and M.is_contiguous()
            and M.dim() == 2 and M.shape[0] == M.shape[1]):
        raise ValueError("zl_xi_indicators: M must be a contiguous square CUDA float64 tensor")
    out = torch.empty(2, dtype=torch.float64, device=M.device)
    _check(_lib.zl_xi_indicators(_vp(M.data_ptr()), M.shape[0], _vp(out.data_ptr()), _stream_handle(stream)),
           "zl_xi_indicators")
    return out


def zl_delta(plan, xt, back, stream=None):
    """d = x~ - back and ||d_r||_2 per right-hand side (back = Zh^- Zh x~)."""
    import torch
    for t in (xt, back):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == plan.dtype and t.is_contiguous()
                and t.dim() == 3 and tuple(t.shape[1:]) == (plan.K, plan.L)):
            raise ValueError(f"zl_delta: inputs must be contiguous CUDA {plan.dtype} tensors [R][K][L]")
    if back.shape != xt.shape:
        raise ValueError("zl_delta: x~ and back differ in shape")
    R = xt.shape[0]
    d = torch.empty_like(xt)
    norms = torch.empty(R, dtype=torch.float64, device=xt.device)
    _check(_lib.zl_delta(plan.handle, _vp(xt.data_ptr()), _vp(back.data_ptr()), _vp(d.data_ptr()),
                         _vp(norms.data_ptr()), R, _stream_handle(stream)), "zl_delta")
    return d, norms


def zl_apply_left_inverse_host(plan, x, out=None, stream=None):
    """Host-buffer variant: x and out are CPU tensors (pinned for asynchronous copies)."""
    import torch
    if not (isinstance(x, torch.Tensor) and not x.is_cuda and x.dtype == plan.dtype and x.is_contiguous()):
        raise ValueError("zl_apply_left_inverse_host: x must be a contiguous CPU tensor")
    if x.dim() != 3 or tuple(x.shape[1:]) != (plan.nw, plan.nh):
        raise ValueError("zl_apply_left_inverse_host: bad input shape")
    R = x.shape[0]
    if out is None:
        out = torch.empty((R, plan.K, plan.L), dtype=plan.dtype, pin_memory=x.is_pinned())
    _check(_lib.zl_apply_left_inverse_host(plan.handle, _vp(x.data_ptr()), _vp(out.data_ptr()), R,
                                           _stream_handle(stream)), "zl_apply_left_inverse_host")
    return out


class Batch:
    """Owns a zl_batch handle: independent instances applied together (one CUDA graph)."""

    def __init__(self, handle, descs):
        self.handle = handle
        self.plans = []
        self.variants = []
        for i, d in enumerate(descs):
            ph, v = _vp(), _int()
            _check(_lib.zl_batch_get_info(handle, i, ctypes.byref(ph), ctypes.byref(v)), "zl_batch_get_info")
            self.plans.append(Plan(ph, d, owned=False))
            self.variants.append(v.value)

    def __len__(self):
        return len(self.plans)

    def apply_left_inverse(self, xs, outs=None, stream=None):
        """x~_i = Zh_i^- x_i for every instance; xs[i] [R_i][n_w][n_h] (R_i = 0 allowed)."""
        import torch
        n = len(self.plans)
        if len(xs) != n:
            raise ValueError("one input per instance")
        if outs is None:
            outs = [torch.empty((x.shape[0], p.K, p.L), dtype=p.dtype, device=x.device) for x, p in zip(xs, self.plans)]
        xp, op, R = (_vp * n)(), (_vp * n)(), (_int * n)()
        for i, (x, o, p) in enumerate(zip(xs, outs, self.plans)):
            if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == p.dtype and x.is_contiguous()
                    and x.dim() == 3 and tuple(x.shape[1:]) == (p.nw, p.nh)):
                raise ValueError(f"instance {i}: input must be a contiguous CUDA {p.dtype} tensor [R][{p.nw}][{p.nh}]")
            if not (o.is_cuda and o.dtype == p.dtype and o.is_contiguous() and tuple(o.shape) == (x.shape[0], p.K, p.L)):
                raise ValueError(f"instance {i}: bad output tensor")
            xp[i], op[i], R[i] = x.data_ptr(), o.data_ptr(), x.shape[0]
        _check(_lib.zl_apply_left_inverse_batch(self.handle, xp, op, R, _stream_handle(stream)),
               "zl_apply_left_inverse_batch")
        return outs

    def destroy(self):
        if self.handle:
            for p in self.plans:
                p.handle = None
            _lib.zl_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def zl_setup_batch(instances, stream=None):
    """Build a batch from a list of instances, each a dict with keys Z (device tensor
    [K][n_w][n_h]), spectrum (host [n_h]), nx, ny, and optionally prec, tau, max_rhs.
    Raises ZLError; ``err.failed_instance`` names the instance whose setup failed."""
    import torch
    n = len(instances)
    descs = (zl_desc * n)()
    zs, specs, keep = (_vp * n)(), (_dp * n)(), []
    for i, inst in enumerate(instances):
        Z = inst["Z"]
        p = PRECISIONS[inst.get("prec", "fp32")]
        want = torch.float64 if p == ZL_FP64 else torch.float32
        if not (isinstance(Z, torch.Tensor) and Z.is_cuda and Z.dtype == want and Z.dim() == 3 and Z.is_contiguous()):
            raise ValueError(f"instance {i}: Z must be a contiguous CUDA {want} tensor [K][n_w][n_h]")
        K, nw, nh = Z.shape
        if inst["nx"] * inst["ny"] != nh:
            raise ValueError(f"instance {i}: nx * ny must equal Z.shape[2]")
        spec = np.ascontiguousarray(inst["spectrum"], dtype=np.float64)
        if spec.shape != (nh,):
            raise ValueError(f"instance {i}: spectrum must have n_h entries")
        keep.append(spec)
        descs[i] = zl_desc(inst["nx"], inst["ny"], nw, K, p, float(inst.get("tau", 1e-10)), int(inst.get("max_rhs", 32)))
        zs[i] = Z.data_ptr()
        specs[i] = spec.ctypes.data_as(_dp)
    h, failed = _vp(), _int()
    code = _lib.zl_setup_batch(n, descs, zs, specs, _stream_handle(stream), ctypes.byref(h), ctypes.byref(failed))
    if code != ZL_OK:
        err = ZLError(code, "zl_setup_batch")
        err.failed_instance = failed.value
        raise err
    return Batch(h, [descs[i] for i in range(n)])
