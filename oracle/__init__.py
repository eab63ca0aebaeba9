"""FP64 CPU oracle (test infrastructure only).

NumPy front end of oracle.c.  Only tests/, the smoke check and the benchmark's
CPU-baseline leg import this package; the CUDA library never does, and the two
share no code.  Arrays use the paper's MATLAB layout: a tensor of size
n1 x n2 x n3 is an array of shape (n1, n2, n3) in Fortran order, so element
(i, j, k) sits at i + n1*(j + n2*k).
"""
import contextlib as _contextlib
import ctypes as _ct

import numpy as _np

from . import build as _build

_lib = None


def _open(path):
    L = _ct.CDLL(path)
    d = _ct.POINTER(_ct.c_double)
    i64 = _ct.c_int64
    ip = _ct.POINTER(_ct.c_int)
    L.or_dct_matrix.argtypes = [i64, d]
    L.or_tube_transform.argtypes = [i64, i64, i64, d, _ct.c_int, _ct.c_int, d]
    L.or_btph.argtypes = [i64, i64, i64, d, d]
    L.or_tprod_btph.argtypes = [i64, i64, i64, i64, d, d, d]
    L.or_tprod.argtypes = [i64, i64, i64, i64, d, d, d]
    L.or_jacobi_svd.argtypes = [i64, i64, d, i64, d, d, d, _ct.c_int, ip]
    L.or_jacobi_svd.restype = _ct.c_int
    L.or_svt_matrix.argtypes = [i64, i64, d, i64, _ct.c_double, d, i64, d, _ct.c_int, ip]
    L.or_svt_matrix.restype = _ct.c_int
    L.or_tsvt.argtypes = [i64, i64, i64, d, _ct.c_double, d, d, _ct.c_int, _ct.c_int, ip, ip]
    L.or_tsvt.restype = _ct.c_int
    L.or_tsvd.argtypes = [i64, i64, i64, d, d, d, d, _ct.c_int, _ct.c_int]
    L.or_tsvd.restype = _ct.c_int
    L.or_admm.argtypes = [i64, i64, i64, d, _ct.POINTER(_ct.c_uint8), _ct.c_double, _ct.c_double,
                          _ct.c_double, _ct.c_double, _ct.c_int, _ct.c_int, _ct.c_int, _ct.c_int, d, d, d]
    L.or_threads.argtypes = [_ct.c_int]
    L.or_threads.restype = _ct.c_int
    return L


def _load():
    global _lib
    if _lib is None:
        _lib = _open(_build.build())
    return _lib


@_contextlib.contextmanager
def using_library(path):
    """Temporarily route every call to another build of oracle.c (the
    mutation tests load deliberately broken copies this way)."""
    global _lib
    old = _lib
    _lib = _open(path)
    try:
        yield
    finally:
        _lib = old


def _dp(a):
    return a.ctypes.data_as(_ct.POINTER(_ct.c_double))


def _f64(a):
    return _np.asfortranarray(_np.asarray(a, dtype=_np.float64))


def _shape3(a):
    a = _np.asarray(a)
    if a.ndim == 2:
        return a.shape[0], a.shape[1], 1
    return a.shape


def dct_matrix(n):
    """Orthonormal DCT-II matrix C (n x n), C[k, j] (MATLAB dct; Section 3)."""
    C = _np.zeros((n, n), order="F")
    _load().or_dct_matrix(n, _dp(C))
    return C


def tube_transform(X, inverse=False, scaled=False):
    """dct / idct along mode 3 (Algorithm 1); scaled=True gives the transform L
    under which Theorem 3 and Example 1 hold as printed (L(X)_k = dct(X)_k / w_k)."""
    X = _f64(X)
    n1, n2, n3 = _shape3(X)
    Y = _np.zeros((n1, n2, n3), order="F")
    _load().or_tube_transform(n1, n2, n3, _dp(X), int(inverse), int(scaled), _dp(Y))
    return Y


def btph(X):
    """Dense block Toeplitz-plus-Hankel matrix of Eqs. 9-11, (m1 m3) x (m2 m3)."""
    X = _f64(X)
    m1, m2, m3 = _shape3(X)
    out = _np.zeros((m1 * m3, m2 * m3), order="F")
    _load().or_btph(m1, m2, m3, _dp(X), _dp(out))
    return out


def tprod_btph(X, Y):
    """DCT-based t-product by Definition 7 / Eq. 13: fold(btph(A) unfold(Y))."""
    X, Y = _f64(X), _f64(Y)
    m1, m2, m3 = _shape3(X)
    m2b, m4, m3b = _shape3(Y)
    assert m2 == m2b and m3 == m3b
    Z = _np.zeros((m1, m4, m3), order="F")
    _load().or_tprod_btph(m1, m2, m4, m3, _dp(X), _dp(Y), _dp(Z))
    return Z


def tprod(X, Y):
    """DCT-based t-product through the transform (Eq. 14), facewise in L."""
    X, Y = _f64(X), _f64(Y)
    m1, m2, m3 = _shape3(X)
    m2b, m4, m3b = _shape3(Y)
    assert m2 == m2b and m3 == m3b
    Z = _np.zeros((m1, m4, m3), order="F")
    _load().or_tprod(m1, m2, m4, m3, _dp(X), _dp(Y), _dp(Z))
    return Z


def jacobi_svd(A, max_sweeps=100):
    """One-sided Jacobi SVD of an m x n matrix, m >= n.
    Returns (U m x n, sigma (n,), V n x n, sweeps, converged)."""
    A = _f64(A)
    m, n = A.shape
    assert m >= n
    U = _np.zeros((m, n), order="F")
    V = _np.zeros((n, n), order="F")
    s = _np.zeros(n)
    cv = _ct.c_int(0)
    sw = _load().or_jacobi_svd(m, n, _dp(A), m, _dp(s), _dp(U), _dp(V), max_sweeps, _ct.byref(cv))
    return U, s, V, sw, bool(cv.value)


def svt_matrix(A, tau, max_sweeps=100):
    """Matrix SVT: U (S - tau)_+ V^T.  Returns (Y, nuclear norm of Y)."""
    A = _f64(A)
    m, n = A.shape
    Y = _np.zeros((m, n), order="F")
    nuc = _ct.c_double(0)
    cv = _ct.c_int(0)
    _load().or_svt_matrix(m, n, _dp(A), m, float(tau), _dp(Y), m, _ct.byref(nuc), max_sweeps, _ct.byref(cv))
    return Y, nuc.value


def tsvt(Z, tau, max_sweeps=100, nthreads=1, return_info=False):
    """t-SVT of Theorem 5 as computed in Algorithm 1.  Returns Y, or
    (Y, tnn, info) with tnn = sum_k ||dct(Y)_k||_* and info a dict."""
    Z = _f64(Z)
    n1, n2, n3 = _shape3(Z)
    Y = _np.zeros((n1, n2, n3), order="F")
    tnn = _ct.c_double(0)
    cv = _ct.c_int(0)
    sw = _np.zeros(n3, dtype=_np.intc)
    smax = _load().or_tsvt(n1, n2, n3, _dp(Z), float(tau), _dp(Y), _ct.byref(tnn), max_sweeps, nthreads,
                           _ct.byref(cv), sw.ctypes.data_as(_ct.POINTER(_ct.c_int)))
    if return_info:
        return Y, tnn.value, {"max_sweeps": smax, "converged": bool(cv.value), "sweeps": sw}
    return Y


def tsvd(X, max_sweeps=100, nthreads=1):
    """Thin DCT-based t-SVD (Theorem 4).  Returns U (m1 x r x m3),
    S (r x m3, the tubes S(i,i,:)), V (m2 x r x m3) with r = min(m1, m2)."""
    X = _f64(X)
    m1, m2, m3 = _shape3(X)
    r = min(m1, m2)
    U = _np.zeros((m1, r, m3), order="F")
    V = _np.zeros((m2, r, m3), order="F")
    S = _np.zeros((r, m3), order="F")
    _load().or_tsvd(m1, m2, m3, _dp(X), _dp(U), _dp(S), _dp(V), max_sweeps, nthreads)
    return U, S, V


def fdiag(S, r=None):
    """f-diagonal tensor (r x r x m3) whose tube (i, i, :) is S[i, :]."""
    S = _np.asarray(S)
    r = S.shape[0] if r is None else r
    out = _np.zeros((r, r, S.shape[1]), order="F")
    for i in range(S.shape[0]):
        out[i, i, :] = S[i, :]
    return out


def ttranspose(X):
    """Tensor transpose: transpose every frontal slice (Theorem 4)."""
    return _np.asfortranarray(_np.transpose(_np.asarray(X), (1, 0, 2)))


def admm(B, mask, beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-8, max_iter=300, max_sweeps=100, nthreads=1,
         X0=None, M0=None):
    """Algorithm 1 with the schedule beta <- min(rho beta, beta_max), from
    X = B on the mask, M = 0, or (with X0 and M0) continuing from that state
    with beta0 as the next iteration's beta.  Returns (X, M, report dict);
    report["beta_final"] is the beta a further iteration would use."""
    B = _f64(B)
    n1, n2, n3 = _shape3(B)
    mk = _np.asfortranarray(_np.asarray(mask, dtype=_np.uint8).reshape((n1, n2, n3), order="F"))
    resume = X0 is not None
    if resume != (M0 is not None):
        raise ValueError("X0 and M0 go together")
    X = _np.array(_f64(X0).reshape((n1, n2, n3), order="F"), order="F") if resume else \
        _np.zeros((n1, n2, n3), order="F")
    M = _np.array(_f64(M0).reshape((n1, n2, n3), order="F"), order="F") if resume else \
        _np.zeros((n1, n2, n3), order="F")
    out = _np.zeros(5)
    _load().or_admm(n1, n2, n3, _dp(B), mk.ctypes.data_as(_ct.POINTER(_ct.c_uint8)), beta0, rho, beta_max,
                    tol, int(max_iter), int(max_sweeps), int(nthreads), int(resume), _dp(X), _dp(M), _dp(out))
    rep = {"iters": int(out[0]), "rel_change": out[1], "primal_res": out[2], "beta_final": out[3],
           "converged": bool(out[4])}
    return X, M, rep


def threads(n):
    """Number of OpenMP threads granted for a request of n."""
    return _load().or_threads(int(n))
