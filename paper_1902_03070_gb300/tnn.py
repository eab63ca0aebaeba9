"""Thin ctypes binding of libtnn (include/tnn.h), same names as the C ABI.

Only argument marshalling happens here: every step of every call runs in the
library's CUDA kernels.  Importing this module fails if libtnn.so has not been
built (there is no CPU fallback).

Tensors follow the paper's MATLAB layout: an n1 x n2 x n3 tensor is a
torch.Tensor or numpy.ndarray of shape (n1, n2, n3) whose element (i, j, k)
sits at offset i + n1*(j + n2*k) (Fortran order; see `fortran_empty`).
CUDA tensors are passed as device pointers on torch's current stream; NumPy
arrays and CPU tensors are passed as host pointers (the library stages them and
synchronises).
"""
import ctypes as _ct
import os as _os

import numpy as _np

_HERE = _os.path.dirname(_os.path.abspath(__file__))
LIB_PATH = _os.path.join(_HERE, "libtnn.so")

if not _os.path.exists(LIB_PATH):
    raise ImportError("libtnn.so is not built (run `python -c 'import __graft_entry__ as g; g.build()'`)")

_lib = _ct.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ENONFINITE, ENODEV = range(7)
OPT_JACOBI_MAX_SWEEPS, OPT_TC_WAIT_POLLS, OPT_JACOBI_FP64_ANGLES, OPT_ADMM_WARM_START = 1, 2, 3, 4
OPT_JACOBI_SMALL_STOP, OPT_JACOBI_SWEEP_LOG = 5, 6
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32x3": 2, "bf16split": 3}
OP_TDCT3, OP_TSVT, OP_TSVD, OP_TPROD, OP_COMPLETE = range(5)


class Shape(_ct.Structure):
    _fields_ = [("n1", _ct.c_int64), ("n2", _ct.c_int64), ("n3", _ct.c_int64)]


class AdmmParams(_ct.Structure):
    _fields_ = [("beta0", _ct.c_double), ("rho", _ct.c_double), ("beta_max", _ct.c_double), ("tol", _ct.c_double),
                ("max_iter", _ct.c_int32), ("jacobi_max_sweeps", _ct.c_int32)]


class AdmmReport(_ct.Structure):
    _fields_ = [("iters", _ct.c_int32), ("converged", _ct.c_int32), ("rel_change", _ct.c_double),
                ("primal_res", _ct.c_double), ("beta_final", _ct.c_double), ("jacobi_sweeps_max", _ct.c_int32),
                ("jacobi_unconverged", _ct.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_vp = _ct.c_void_p
_st = _ct.c_int
_lib.tnn_create.argtypes = [_ct.POINTER(_vp), _ct.c_int]
_lib.tnn_create.restype = _st
_lib.tnn_destroy.argtypes = [_vp]
_lib.tnn_destroy.restype = None
_lib.tnn_status_string.argtypes = [_st]
_lib.tnn_status_string.restype = _ct.c_char_p
_lib.tnn_last_error.argtypes = [_vp]
_lib.tnn_last_error.restype = _ct.c_char_p
_lib.tnn_reserve.argtypes = [_vp, _ct.c_size_t]
_lib.tnn_reserve.restype = _st
_lib.tnn_set_option.argtypes = [_vp, _ct.c_int, _ct.c_int64]
_lib.tnn_set_option.restype = _st
_lib.tnn_workspace_size.argtypes = [_vp, _ct.c_int, Shape, _ct.c_int, _ct.POINTER(_ct.c_size_t)]
_lib.tnn_workspace_size.restype = _st
_lib.tdct3.argtypes = [_vp, _vp, Shape, _ct.c_int, _ct.c_int, _ct.c_int, _vp, _vp]
_lib.tdct3.restype = _st
_lib.tsvt_dct.argtypes = [_vp, _vp, Shape, _ct.c_double, _ct.c_int, _vp, _ct.POINTER(_ct.c_double), _vp]
_lib.tsvt_dct.restype = _st
_lib.tsvd_dct_forward.argtypes = [_vp, _vp, Shape, _ct.c_int, _vp, _vp, _vp, _vp]
_lib.tsvd_dct_forward.restype = _st
_lib.tsvd_dct_inverse.argtypes = [_vp, _vp, _vp, _vp, Shape, _ct.c_int, _vp, _vp]
_lib.tsvd_dct_inverse.restype = _st
_lib.tprod_dct.argtypes = [_vp, _vp, _vp, _ct.c_int64, _ct.c_int64, _ct.c_int64, _ct.c_int64, _ct.c_int, _vp, _vp]
_lib.tprod_dct.restype = _st
_lib.tnn_complete.argtypes = [_vp, _vp, _vp, Shape, _ct.POINTER(AdmmParams), _ct.c_int, _vp,
                              _ct.POINTER(AdmmReport), _vp]
_lib.tnn_complete.restype = _st
_lib.tnn_admm_iterate.argtypes = [_vp, _vp, _vp, Shape, _ct.POINTER(AdmmParams), _ct.c_int, _vp, _vp,
                                  _ct.POINTER(_ct.c_double), _ct.c_int32, _vp, _ct.POINTER(AdmmReport), _vp]
_lib.tnn_admm_iterate.restype = _st
_lib.tnn_admm_warm_size.argtypes = [Shape, _ct.c_int, _ct.POINTER(_ct.c_size_t)]
_lib.tnn_admm_warm_size.restype = _st
_lib.tnn_last_jacobi_stats.argtypes = [_vp, _ct.POINTER(_ct.c_int64)]
_lib.tnn_last_jacobi_stats.restype = _st
_lib.tnn_last_slice_stats.argtypes = [_vp, _ct.c_int64, _ct.POINTER(_ct.c_int32), _ct.POINTER(_ct.c_int32),
                                      _ct.POINTER(_ct.c_int64)]
_lib.tnn_last_slice_stats.restype = _st
_lib.tnn_last_sweep_log.argtypes = [_vp, _ct.c_int64, _ct.POINTER(_ct.c_float)]
_lib.tnn_last_sweep_log.restype = _st
_lib.tnn_fma_peak.argtypes = [_ct.c_int32, _ct.c_int32, _ct.POINTER(_ct.c_double)]
_lib.tnn_fma_peak.restype = _st
_lib.tnn_jacobi_plan_info.argtypes = [Shape, _ct.c_int, _ct.POINTER(_ct.c_int64)]
_lib.tnn_jacobi_plan_info.restype = _st
_lib.tnn_server_footprint.argtypes = [Shape, _ct.c_int, _ct.POINTER(_ct.c_uint64)]
_lib.tnn_server_footprint.restype = _st
_lib.tnn_profile.argtypes = [_vp, _ct.c_int]
_lib.tnn_profile.restype = _st
_lib.tnn_profile_read.argtypes = [_vp, _ct.POINTER(_ct.c_double), _ct.POINTER(_ct.c_int64)]
_lib.tnn_profile_read.restype = _st
_lib.tsvt_dct_static.argtypes = [_vp, Shape, _ct.c_double, _ct.c_int, _vp, _vp]
_lib.tsvt_dct_static.restype = _st


class TsvtItem(_ct.Structure):
    _fields_ = [("Z", _vp), ("Y", _vp), ("shape", Shape), ("tau", _ct.c_double)]


_lib.tnn_tsvt_batch_create.argtypes = [_vp, _ct.POINTER(TsvtItem), _ct.c_int32, _ct.c_int, _ct.c_int32, _vp,
                                       _ct.POINTER(_vp)]
_lib.tnn_tsvt_batch_create.restype = _st
_lib.tnn_tsvt_batch_run.argtypes = [_vp, _vp]
_lib.tnn_tsvt_batch_run.restype = _st
_lib.tnn_tsvt_batch_info.argtypes = [_vp, _ct.POINTER(_ct.c_int32)]
_lib.tnn_tsvt_batch_info.restype = _st
_lib.tnn_tsvt_batch_group.argtypes = [_vp, _ct.c_int32, _ct.POINTER(_ct.c_int32)]
_lib.tnn_tsvt_batch_group.restype = _st
_lib.tnn_tsvt_batch_profile.argtypes = [_vp, _vp, _ct.POINTER(_ct.c_double)]
_lib.tnn_tsvt_batch_profile.restype = _st
_lib.tnn_tsvt_batch_stats.argtypes = [_vp, _vp, _ct.POINTER(_ct.c_int64)]
_lib.tnn_tsvt_batch_stats.restype = _st
_lib.tnn_tsvt_batch_destroy.argtypes = [_vp]
_lib.tnn_tsvt_batch_destroy.restype = None


class ServerParams(_ct.Structure):
    _fields_ = [("hbm_cap_bytes", _ct.c_uint64), ("max_active", _ct.c_int32), ("streams", _ct.c_int32),
                ("chunk", _ct.c_int32), ("device", _ct.c_int32), ("policy", _ct.c_int32), ("flags", _ct.c_int32)]


_lib.tnn_server_create.argtypes = [_ct.POINTER(ServerParams), _ct.POINTER(_vp)]
_lib.tnn_server_create.restype = _st
_lib.tnn_server_submit.argtypes = [_vp, _vp, _vp, Shape, _ct.POINTER(AdmmParams), _ct.c_int, _ct.POINTER(_ct.c_int64)]
_lib.tnn_server_submit.restype = _st
_lib.tnn_server_step.argtypes = [_vp, _ct.POINTER(_ct.c_int32)]
_lib.tnn_server_step.restype = _st
_lib.tnn_server_job_state.argtypes = [_vp, _ct.c_int64, _ct.POINTER(_ct.c_int32)]
_lib.tnn_server_job_state.restype = _st
_lib.tnn_server_take.argtypes = [_vp, _ct.c_int64, _vp, _ct.POINTER(AdmmReport), _ct.POINTER(_ct.c_double)]
_lib.tnn_server_take.restype = _st
_lib.tnn_server_stats.argtypes = [_vp, _ct.POINTER(_ct.c_int64)]
_lib.tnn_server_stats.restype = _st
_lib.tnn_server_destroy.argtypes = [_vp]
_lib.tnn_server_destroy.restype = None


class AdmmItem(_ct.Structure):
    _fields_ = [("B", _vp), ("mask", _vp), ("X", _vp), ("M", _vp), ("shape", Shape)]


_lib.tnn_admm_batch_create.argtypes = [_vp, _ct.POINTER(AdmmItem), _ct.c_int32, _ct.POINTER(AdmmParams), _ct.c_int,
                                       _ct.c_int32, _vp, _ct.POINTER(_vp)]
_lib.tnn_admm_batch_create.restype = _st
_lib.tnn_admm_batch_reset.argtypes = [_vp, _vp]
_lib.tnn_admm_batch_reset.restype = _st
_lib.tnn_admm_batch_step.argtypes = [_vp, _ct.c_int32, _vp]
_lib.tnn_admm_batch_step.restype = _st
_lib.tnn_admm_batch_sync.argtypes = [_vp, _vp, _ct.POINTER(_ct.c_int32)]
_lib.tnn_admm_batch_sync.restype = _st
_lib.tnn_admm_batch_run.argtypes = [_vp, _vp]
_lib.tnn_admm_batch_run.restype = _st
_lib.tnn_admm_batch_report.argtypes = [_vp, _ct.c_int32, _ct.POINTER(AdmmReport)]
_lib.tnn_admm_batch_report.restype = _st
_lib.tnn_admm_batch_destroy.argtypes = [_vp]
_lib.tnn_admm_batch_destroy.restype = None
BATCH_GRAPH = 1
BATCH_AUTOTUNE = 2
NKERNELS = 13
KERNEL_KINDS = ["tube", "tube_fwd_admm", "jacobi_svt", "tube_inv_admm", "admm_finalize", "ctl_init", "admm_init",
                "jacobi_svd", "facewise", "dft", "jacobi_plain", "warm", "svt_tail"]
_lib.tsvt_dft.argtypes = [_vp, _vp, Shape, _ct.c_double, _ct.c_int, _vp, _ct.POINTER(_ct.c_double), _vp]
_lib.tsvt_dft.restype = _st
_lib.tsvt_dct_plain.argtypes = [_vp, _vp, Shape, _ct.c_double, _ct.c_int, _vp, _ct.POINTER(_ct.c_double), _vp]
_lib.tsvt_dct_plain.restype = _st

EXPORTS = ["tnn_create", "tnn_destroy", "tnn_status_string", "tnn_last_error", "tnn_reserve", "tnn_set_option",
           "tnn_workspace_size",
           "tdct3", "tsvt_dct", "tsvd_dct_forward", "tsvd_dct_inverse", "tprod_dct", "tnn_complete",
           "tnn_admm_iterate", "tnn_admm_warm_size", "tnn_last_jacobi_stats", "tnn_last_slice_stats", "tnn_last_sweep_log", "tnn_profile", "tnn_profile_read", "tsvt_dct_static",
           "tnn_tsvt_batch_create", "tnn_tsvt_batch_run", "tnn_tsvt_batch_info", "tnn_tsvt_batch_group",
           "tnn_tsvt_batch_profile", "tnn_tsvt_batch_stats", "tnn_tsvt_batch_destroy",
           "tnn_server_create", "tnn_server_submit", "tnn_server_step", "tnn_server_job_state", "tnn_server_take",
           "tnn_server_stats", "tnn_server_destroy", "tsvt_dft", "tsvt_dct_plain", "tnn_admm_batch_create",
           "tnn_admm_batch_reset", "tnn_admm_batch_step", "tnn_admm_batch_sync", "tnn_admm_batch_run",
           "tnn_admm_batch_report", "tnn_admm_batch_destroy", "tnn_fma_peak", "tnn_jacobi_plan_info",
           "tnn_server_footprint"]


class TnnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_lib.tnn_status_string(status).decode(), msg))
        self.status = status


FMA_KINDS = {"fp32": 0, "fp32x2": 1, "fp64": 2}


def jacobi_plan_info(shape, prec="fp32"):
    """The Jacobi SVT launch planned for slices of `shape` (host only;
    tnn_jacobi_plan_info)."""
    out = (_ct.c_int64 * 9)()
    st = _lib.tnn_jacobi_plan_info(Shape(*shape), PRECISIONS[prec], out)
    if st != OK:
        raise TnnError(st, "tnn_jacobi_plan_info")
    keys = ["L", "R", "K", "nb", "W", "in_smem", "cluster", "smem_bytes", "work_bytes"]
    return dict(zip(keys, list(out)))


def server_footprint(shape, prec="fp32"):
    """Device bytes a completion job of `shape` holds in the server (host
    only; tnn_server_footprint)."""
    out = _ct.c_uint64(0)
    st = _lib.tnn_server_footprint(Shape(*shape), PRECISIONS[prec], _ct.byref(out))
    if st != OK:
        raise TnnError(st, "tnn_server_footprint")
    return out.value


def fma_peak(kind="fp32", device=0):
    """Measured FMA-pipe rate of the device in flop/s (tnn_fma_peak)."""
    out = _ct.c_double(0.0)
    st = _lib.tnn_fma_peak(int(device), FMA_KINDS[kind], _ct.byref(out))
    if st != OK:
        raise TnnError(st, "tnn_fma_peak")
    return out.value


def status_string(s):
    return _lib.tnn_status_string(int(s)).decode()


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _check_layout(x, shape):
    """x must be (n1, n2, n3) with element (i, j, k) at i + n1*(j + n2*k)."""
    if tuple(x.shape) != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (tuple(shape), tuple(x.shape)))
    if _is_torch(x):
        exp, acc = [], 1
        for d in shape:
            exp.append(acc)
            acc *= d
        ok = all(st == e for st, e, d in zip(x.stride(), exp, shape) if d > 1)
    else:
        ok = x.flags.f_contiguous
    if not ok:
        raise ValueError("tensor must be in Fortran (MATLAB) order; use fortran_empty / to_fortran")


def _ptr(x):
    if _is_torch(x):
        return x.data_ptr(), x.is_cuda
    return x.ctypes.data, False


def _dtype_ok(x, prec):
    want = "float64" if prec == "fp64" else "float32"
    name = str(x.dtype).replace("torch.", "")
    if name != want:
        raise TypeError("precision %s needs %s data, got %s" % (prec, want, name))


def _stream(args):
    for a in args:
        if _is_torch(a) and a.is_cuda:
            import torch
            return _ct.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return _ct.c_void_p(0)


def fortran_empty(shape, dtype, device="cuda"):
    """Uninitialised torch tensor of `shape` in Fortran order."""
    import torch
    return torch.empty(tuple(reversed(shape)), dtype=dtype, device=device).permute(*reversed(range(len(shape))))


def to_fortran(x, device="cuda", dtype=None):
    """Copy a NumPy array or tensor into a Fortran-ordered torch tensor."""
    import torch
    a = _np.asarray(x.cpu().numpy() if _is_torch(x) else x)
    if dtype is None:
        dtype = torch.float64 if a.dtype == _np.float64 else (torch.uint8 if a.dtype == _np.uint8 else torch.float32)
    t = torch.from_numpy(_np.ascontiguousarray(_np.transpose(a, tuple(reversed(range(a.ndim))))))
    t = t.to(device=device, dtype=dtype)
    return t.permute(*reversed(range(a.ndim)))


def to_numpy(t):
    """Fortran-ordered NumPy copy of a tensor produced by this binding."""
    if _is_torch(t):
        return _np.asfortranarray(t.detach().cpu().numpy())
    return _np.asfortranarray(t)


class Context:
    """A libtnn context (device workspace, DCT operator cache)."""

    def __init__(self, device=0):
        h = _vp()
        st = _lib.tnn_create(_ct.byref(h), int(device))
        if st != OK:
            raise TnnError(st, "tnn_create(device=%d)" % device)
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            _lib.tnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _chk(self, st, what, allow=()):
        if st != OK and st not in allow:
            raise TnnError(st, "%s: %s" % (what, _lib.tnn_last_error(self._h).decode()))
        return st

    def last_error(self):
        return _lib.tnn_last_error(self._h).decode()

    def reserve(self, nbytes):
        self._chk(_lib.tnn_reserve(self._h, int(nbytes)), "tnn_reserve")

    def set_option(self, option, value):
        """tnn_set_option: OPT_JACOBI_MAX_SWEEPS, OPT_TC_WAIT_POLLS,
        OPT_JACOBI_FP64_ANGLES, OPT_ADMM_WARM_START, OPT_JACOBI_SMALL_STOP or
        OPT_JACOBI_SWEEP_LOG."""
        self._chk(_lib.tnn_set_option(self._h, int(option), int(value)), "tnn_set_option")

    def workspace_size(self, op, shape, prec="fp32"):
        out = _ct.c_size_t(0)
        self._chk(_lib.tnn_workspace_size(self._h, int(op), Shape(*shape), PRECISIONS[prec], _ct.byref(out)),
                  "tnn_workspace_size")
        return out.value

    def tdct3(self, X, Y, inverse=False, scaled=False, prec="fp32"):
        _check_layout(Y, X.shape)
        _check_layout(X, X.shape)
        _dtype_ok(X, prec)
        self._chk(_lib.tdct3(self._h, _ptr(X)[0], Shape(*X.shape), int(inverse), int(scaled), PRECISIONS[prec],
                             _ptr(Y)[0], _stream([X, Y])), "tdct3")
        return Y

    def tsvt(self, Z, tau, Y=None, prec="fp32", want_tnn=False, allow_noconv=False):
        """Y = t-SVT_tau(Z) (Theorem 5).  Returns Y, or (Y, tnn) with want_tnn."""
        if len(Z.shape) == 2:
            raise ValueError("pass a 3-way tensor (n1, n2, n3)")
        _check_layout(Z, Z.shape)
        _dtype_ok(Z, prec)
        if Y is None:
            Y = Z
        _check_layout(Y, Z.shape)
        out = _ct.c_double(0.0)
        st = _lib.tsvt_dct(self._h, _ptr(Z)[0], Shape(*Z.shape), float(tau), PRECISIONS[prec], _ptr(Y)[0],
                           _ct.byref(out) if want_tnn else None, _stream([Z, Y]))
        self._chk(st, "tsvt_dct", allow=(ENOCONV,) if allow_noconv else ())
        return (Y, out.value) if want_tnn else Y

    def _tsvt_plain(self, fn, name, Z, tau, Y, prec, want_tnn, allow_noconv):
        _check_layout(Z, Z.shape)
        _dtype_ok(Z, prec)
        if Y is None:
            Y = Z
        _check_layout(Y, Z.shape)
        out = _ct.c_double(0.0)
        st = fn(self._h, _ptr(Z)[0], Shape(*Z.shape), float(tau), PRECISIONS[prec], _ptr(Y)[0],
                _ct.byref(out) if want_tnn else None, _stream([Z, Y]))
        self._chk(st, name, allow=(ENOCONV,) if allow_noconv else ())
        return (Y, out.value) if want_tnn else Y

    def tsvt_dft(self, Z, tau, Y=None, prec="fp32", want_tnn=False, allow_noconv=False):
        """Y = ifft(SVT_tau(fft(Z))) along the tubes: the proximal operator of
        tau * TNN-F (the DFT comparison path).  With want_tnn: (Y, TNN-F(Y))."""
        return self._tsvt_plain(_lib.tsvt_dft, "tsvt_dft", Z, tau, Y, prec, want_tnn, allow_noconv)

    def tsvt_dct_plain(self, Z, tau, Y=None, prec="fp32", want_tnn=False, allow_noconv=False):
        """The DCT t-SVT with the DFT path's plain Jacobi kernel (like-for-like
        comparison)."""
        return self._tsvt_plain(_lib.tsvt_dct_plain, "tsvt_dct_plain", Z, tau, Y, prec, want_tnn, allow_noconv)

    def tsvd(self, X, U, S, V, prec="fp32"):
        n1, n2, n3 = X.shape
        r = min(n1, n2)
        _check_layout(X, (n1, n2, n3))
        _check_layout(U, (n1, r, n3))
        _check_layout(V, (n2, r, n3))
        _check_layout(S, (r, n3))
        _dtype_ok(X, prec)
        self._chk(_lib.tsvd_dct_forward(self._h, _ptr(X)[0], Shape(n1, n2, n3), PRECISIONS[prec], _ptr(U)[0],
                                        _ptr(S)[0], _ptr(V)[0], _stream([X, U, S, V])), "tsvd_dct_forward")
        return U, S, V

    def tsvd_inverse(self, U, S, V, X, prec="fp32"):
        n1, n2, n3 = X.shape
        r = min(n1, n2)
        _check_layout(X, (n1, n2, n3))
        _check_layout(U, (n1, r, n3))
        _check_layout(V, (n2, r, n3))
        _check_layout(S, (r, n3))
        self._chk(_lib.tsvd_dct_inverse(self._h, _ptr(U)[0], _ptr(S)[0], _ptr(V)[0], Shape(n1, n2, n3),
                                        PRECISIONS[prec], _ptr(X)[0], _stream([X, U, S, V])), "tsvd_dct_inverse")
        return X

    def tprod(self, X, Y, Z, prec="fp32"):
        m1, m2, m3 = X.shape
        m2b, m4, m3b = Y.shape
        if m2 != m2b or m3 != m3b:
            raise ValueError("t-product shape mismatch")
        _check_layout(X, (m1, m2, m3))
        _check_layout(Y, (m2, m4, m3))
        _check_layout(Z, (m1, m4, m3))
        self._chk(_lib.tprod_dct(self._h, _ptr(X)[0], _ptr(Y)[0], m1, m2, m4, m3, PRECISIONS[prec], _ptr(Z)[0],
                                 _stream([X, Y, Z])), "tprod_dct")
        return Z

    @staticmethod
    def params(beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-8, max_iter=300, jacobi_max_sweeps=0):
        return AdmmParams(float(beta0), float(rho), float(beta_max), float(tol), int(max_iter),
                          int(jacobi_max_sweeps))

    def complete(self, B, mask, X_out, params, prec="fp32"):
        """Algorithm 1.  Returns (status, report dict); TNN_ENOCONV is not raised."""
        _check_layout(B, B.shape)
        _check_layout(X_out, B.shape)
        _check_layout(mask, B.shape)
        rep = AdmmReport()
        st = _lib.tnn_complete(self._h, _ptr(B)[0], _ptr(mask)[0], Shape(*B.shape), _ct.byref(params),
                               PRECISIONS[prec], _ptr(X_out)[0], _ct.byref(rep), _stream([B, mask, X_out]))
        self._chk(st, "tnn_complete", allow=(ENOCONV,))
        return st, rep.as_dict()

    def admm_iterate(self, B, mask, X, M, beta, iters, params, prec="fp32", warm=None):
        """Advance a caller-held ADMM state (X, M, beta and, optionally, the
        warm-start buffer of admm_warm_state) by up to `iters` iterations.
        Returns (beta, report dict)."""
        for t in (B, X, M, mask):
            _check_layout(t, B.shape)
        b = _ct.c_double(float(beta))
        rep = AdmmReport()
        wp = None if warm is None else warm.data_ptr()
        st = _lib.tnn_admm_iterate(self._h, _ptr(B)[0], _ptr(mask)[0], Shape(*B.shape), _ct.byref(params),
                                   PRECISIONS[prec], _ptr(X)[0], _ptr(M)[0], _ct.byref(b), int(iters), wp,
                                   _ct.byref(rep), _stream([B, mask, X, M]))
        self._chk(st, "tnn_admm_iterate")
        return b.value, rep.as_dict()

    @staticmethod
    def admm_warm_state(shape, prec="fp32", device="cuda"):
        """A zero-filled warm-start buffer for admm_iterate (torch uint8
        tensor on the device), or None where the precision or slice size does
        not use one (tnn_admm_warm_size)."""
        import torch
        n = _ct.c_size_t(0)
        st = _lib.tnn_admm_warm_size(Shape(*shape), PRECISIONS[prec], _ct.byref(n))
        if st != OK:
            raise TnnError(st, "tnn_admm_warm_size")
        return torch.zeros(n.value, dtype=torch.uint8, device=device) if n.value else None

    def tsvt_batch(self, Zs, taus, Ys=None, prec="fp32", graph=True, autotune=False):
        """Plan for Y_i = t-SVT_{tau_i}(Z_i) over device tensors of different
        shapes (Theorem 5 per tensor).  Returns a TsvtBatch; call .run()."""
        if Ys is None:
            Ys = Zs
        if not (len(Zs) == len(Ys) == len(taus)) or not Zs:
            raise ValueError("Zs, Ys and taus must be non-empty and of equal length")
        arr = (TsvtItem * len(Zs))()
        for i, (Z, Y, t) in enumerate(zip(Zs, Ys, taus)):
            if len(Z.shape) != 3:
                raise ValueError("pass 3-way tensors (n1, n2, n3)")
            _check_layout(Z, Z.shape)
            _check_layout(Y, Z.shape)
            _dtype_ok(Z, prec)
            _dtype_ok(Y, prec)
            arr[i] = TsvtItem(_ptr(Z)[0], _ptr(Y)[0], Shape(*Z.shape), float(t))
        flags = (BATCH_GRAPH if graph else 0) | (BATCH_AUTOTUNE if autotune else 0)
        h = _vp()
        stream = _stream(list(Zs) + list(Ys))
        self._chk(_lib.tnn_tsvt_batch_create(self._h, arr, len(Zs), PRECISIONS[prec], flags, stream, _ct.byref(h)),
                  "tnn_tsvt_batch_create")
        return TsvtBatch(h, list(Zs), list(Ys))

    def admm_batch(self, Bs, masks, Xs, Ms, params, prec="fp32", graph=True):
        """Plan for Algorithm 1 over many device problems at once (initialises
        X = B on the mask and M = 0).  Returns an AdmmBatch."""
        if not (len(Bs) == len(masks) == len(Xs) == len(Ms)) or not Bs:
            raise ValueError("Bs, masks, Xs and Ms must be non-empty and of equal length")
        arr = (AdmmItem * len(Bs))()
        for i, (B, m, X, M) in enumerate(zip(Bs, masks, Xs, Ms)):
            for t in (B, m, X, M):
                _check_layout(t, B.shape)
            for t in (B, X, M):
                _dtype_ok(t, prec)
            arr[i] = AdmmItem(_ptr(B)[0], _ptr(m)[0], _ptr(X)[0], _ptr(M)[0], Shape(*B.shape))
        h = _vp()
        stream = _stream(list(Bs) + list(Xs))
        self._chk(_lib.tnn_admm_batch_create(self._h, arr, len(Bs), _ct.byref(params), PRECISIONS[prec],
                                             BATCH_GRAPH if graph else 0, stream, _ct.byref(h)),
                  "tnn_admm_batch_create")
        return AdmmBatch(h, (list(Bs), list(masks), list(Xs), list(Ms)))

    def last_jacobi_stats(self):
        out = (_ct.c_int64 * 6)()
        self._chk(_lib.tnn_last_jacobi_stats(self._h, out), "tnn_last_jacobi_stats")
        keys = ["slices", "pairs", "rotations", "max_sweeps", "unconverged", "kept"]
        return dict(zip(keys, list(out)))

    def last_slice_stats(self):
        """Per-slice sweeps, kept singular values and rotations of the last
        Jacobi launch: {"sweeps": [...], "kept": [...], "rotations": [...]}."""
        n = self.last_jacobi_stats()["slices"]
        sw = (_ct.c_int32 * max(n, 1))()
        kp = (_ct.c_int32 * max(n, 1))()
        rt = (_ct.c_int64 * max(n, 1))()
        self._chk(_lib.tnn_last_slice_stats(self._h, n, sw, kp, rt), "tnn_last_slice_stats")
        return {"sweeps": list(sw)[:n], "kept": list(kp)[:n], "rotations": list(rt)[:n]}

    def last_sweep_log(self):
        """Per-sweep log of the last Jacobi launch (OPT_JACOBI_SWEEP_LOG on):
        a numpy array (slices, 9, 8).  Rows 0-7 are sweeps: big rotations,
        wide rotations, big low-low rotations, largest |gamma|/sqrt(alpha
        beta) of the big ones, largest |t| of the big ones and of all, the
        sweep's clock cycles, the stopping tests' cycles.  Row 8: cycles of
        the load, the sweeps, the tail and the whole slice."""
        n = self.last_jacobi_stats()["slices"]
        out = _np.zeros((max(n, 1), 9, 8), dtype=_np.float32)
        self._chk(_lib.tnn_last_sweep_log(self._h, n, out.ctypes.data_as(_ct.POINTER(_ct.c_float))),
                  "tnn_last_sweep_log")
        return out[:n]

    def profile(self, enable=True):
        """Bracket every kernel launch of later calls with CUDA events."""
        self._chk(_lib.tnn_profile(self._h, int(bool(enable))), "tnn_profile")

    def profile_read(self):
        """{kind: (ms, launches)} since the last read (synchronises)."""
        ms = (_ct.c_double * NKERNELS)()
        cnt = (_ct.c_int64 * NKERNELS)()
        self._chk(_lib.tnn_profile_read(self._h, ms, cnt), "tnn_profile_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS) if cnt[i]}


class TsvtBatch:
    """A batched t-SVT plan (tnn_tsvt_batch_*); keeps its tensors alive."""

    def __init__(self, h, Zs, Ys):
        self._h = h
        self._keep = (Zs, Ys)

    def _stream(self):
        return _stream(self._keep[0])

    def run(self):
        st = _lib.tnn_tsvt_batch_run(self._h, self._stream())
        if st != OK:
            raise TnnError(st, "tnn_tsvt_batch_run")

    def info(self):
        out = (_ct.c_int32 * 4)()
        st = _lib.tnn_tsvt_batch_info(self._h, out)
        if st != OK:
            raise TnnError(st, "tnn_tsvt_batch_info")
        return dict(zip(["groups", "launches", "slices", "graph"], list(out)))

    def groups(self):
        res = []
        for g in range(self.info()["groups"]):
            out = (_ct.c_int32 * 6)()
            st = _lib.tnn_tsvt_batch_group(self._h, g, out)
            if st != OK:
                raise TnnError(st, "tnn_tsvt_batch_group")
            res.append(dict(zip(["L", "R", "K", "slices", "in_smem", "m"], list(out))))
        return res

    def profile(self):
        """Milliseconds of each launch of one serial run:
        {"forward": ms, "groups": [ms, ...], "inverse": ms}."""
        n = self.info()["groups"]
        ms = (_ct.c_double * (n + 2))()
        st = _lib.tnn_tsvt_batch_profile(self._h, self._stream(), ms)
        if st != OK:
            raise TnnError(st, "tnn_tsvt_batch_profile")
        return {"forward": ms[0], "groups": list(ms[1:n + 1]), "inverse": ms[n + 1]}

    def stats(self):
        out = (_ct.c_int64 * 4)()
        st = _lib.tnn_tsvt_batch_stats(self._h, self._stream(), out)
        if st not in (OK, ENONFINITE):
            raise TnnError(st, "tnn_tsvt_batch_stats")
        return dict(zip(["unconverged", "nonfinite", "rotations", "max_sweeps"], list(out)))

    def close(self):
        if self._h:
            _lib.tnn_tsvt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Completion server (tnn_server_*): continuous batching of completion
    jobs with device-resident state and HBM-footprint admission."""

    QUEUED, RUNNING, FINISHED, FAILED = range(4)

    FIFO, SHORTEST_FIRST = 0, 1
    BATCH_KERNELS = 1

    def __init__(self, hbm_cap_bytes=0, max_active=0, streams=0, chunk=0, device=0, policy=0, batch_kernels=False):
        p = ServerParams(int(hbm_cap_bytes), int(max_active), int(streams), int(chunk), int(device), int(policy),
                         self.BATCH_KERNELS if batch_kernels else 0)
        h = _vp()
        st = _lib.tnn_server_create(_ct.byref(p), _ct.byref(h))
        if st != OK:
            raise TnnError(st, "tnn_server_create")
        self._h = h
        self._keep = {}

    def submit(self, B, mask, params, prec="fp32"):
        """Queue a completion job (B and mask are kept referenced until the
        result is taken).  Returns the job id."""
        _check_layout(B, B.shape)
        _check_layout(mask, B.shape)
        _dtype_ok(B, prec)
        jid = _ct.c_int64(0)
        st = _lib.tnn_server_submit(self._h, _ptr(B)[0], _ptr(mask)[0], Shape(*B.shape), _ct.byref(params),
                                    PRECISIONS[prec], _ct.byref(jid))
        if st != OK:
            raise TnnError(st, "tnn_server_submit")
        self._keep[jid.value] = (B, mask, tuple(B.shape), prec)
        return jid.value

    def step(self):
        """One scheduling pass; returns how many jobs finished in it."""
        fin = _ct.c_int32(0)
        st = _lib.tnn_server_step(self._h, _ct.byref(fin))
        if st != OK:
            raise TnnError(st, "tnn_server_step")
        return fin.value

    def state(self, jid):
        out = _ct.c_int32(0)
        st = _lib.tnn_server_job_state(self._h, int(jid), _ct.byref(out))
        if st != OK:
            raise TnnError(st, "tnn_server_job_state")
        return out.value

    def take(self, jid, X_out=None):
        """(status, X, report, (t_submit, t_admit, t_finish)) of a finished
        job; X is X_out, or a new host array when X_out is None."""
        import numpy as np
        B, mask, shape, prec = self._keep[jid]
        if X_out is None:
            X_out = np.empty(shape, dtype=np.float64 if prec == "fp64" else np.float32, order="F")
        rep = AdmmReport()
        t = (_ct.c_double * 3)()
        st = _lib.tnn_server_take(self._h, int(jid), _ptr(X_out)[0], _ct.byref(rep), t)
        if st == EINVAL and self.state(jid) < 2:
            raise TnnError(st, "tnn_server_take: job %d not finished" % jid)
        del self._keep[jid]
        return st, X_out, rep.as_dict(), (t[0], t[1], t[2])

    def stats(self):
        out = (_ct.c_int64 * 6)()
        st = _lib.tnn_server_stats(self._h, out)
        if st != OK:
            raise TnnError(st, "tnn_server_stats")
        return dict(zip(["queued", "running", "finished", "bytes", "peak_bytes", "completed"], list(out)))

    def close(self):
        if self._h:
            _lib.tnn_server_destroy(self._h)
            self._h = None
            self._keep = {}

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AdmmBatch:
    """A batched ADMM plan (tnn_admm_batch_*); keeps its tensors alive."""

    def __init__(self, h, keep):
        self._h = h
        self._keep = keep

    def _stream(self):
        return _stream(self._keep[0])

    def _call(self, st, what):
        if st != OK:
            raise TnnError(st, what)

    def reset(self):
        self._call(_lib.tnn_admm_batch_reset(self._h, self._stream()), "tnn_admm_batch_reset")

    def step(self, iters=1):
        self._call(_lib.tnn_admm_batch_step(self._h, int(iters), self._stream()), "tnn_admm_batch_step")

    def sync(self):
        r = _ct.c_int32(0)
        self._call(_lib.tnn_admm_batch_sync(self._h, self._stream(), _ct.byref(r)), "tnn_admm_batch_sync")
        return r.value

    def run(self):
        self._call(_lib.tnn_admm_batch_run(self._h, self._stream()), "tnn_admm_batch_run")

    def report(self, i):
        rep = AdmmReport()
        st = _lib.tnn_admm_batch_report(self._h, int(i), _ct.byref(rep))
        if st not in (OK, ENOCONV, ENONFINITE):
            raise TnnError(st, "tnn_admm_batch_report")
        return st, rep.as_dict()

    def close(self):
        if self._h:
            _lib.tnn_admm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

