"""FP64 oracle of the DFT-based comparison path (test infrastructure only).

The t-SVD of Kilmer and Martin that the paper compares against: the DFT along
every tube (Section 2: the tensor X~ = fft(X, [], 3)), the t-product of
Definition 1 / Eq. (5) in its Fourier-domain form Eq. (6), the tensor
nuclear norm TNN-F of Definition 6 (the mean over the n3 DFT slices of
their nuclear norms),
and its proximal operator, the DFT t-SVT: every DFT slice of Z has its
singular values shrunk by tau, and the inverse DFT brings the result back.
For a real Z the DFT slices k and n3 - k are complex conjugates, so the
shrunk slices keep that symmetry and the result is real.

Written from those definitions with library primitives as steps (NumPy's
FFT and LAPACK's SVD); it shares nothing with the CUDA path.
"""
import numpy as np


def tnn_f(X):
    """TNN-F (Definition 6): (1/n3) sum_k ||X~^(k)||_*, X~ = fft along tubes."""
    X = np.asarray(X, dtype=np.float64)
    Xf = np.fft.fft(X, axis=2)
    return float(sum(np.linalg.svd(Xf[:, :, k], compute_uv=False).sum() for k in range(X.shape[2])) / X.shape[2])


def tprod_dft(X, Y):
    """t-product through the DFT (Eq. (6)): the DFT slices of X * Y are the
    products of the DFT slices of X and Y."""
    Xf = np.fft.fft(np.asarray(X, dtype=np.float64), axis=2)
    Yf = np.fft.fft(np.asarray(Y, dtype=np.float64), axis=2)
    Zf = np.einsum("ijk,jlk->ilk", Xf, Yf)
    return np.asfortranarray(np.real(np.fft.ifft(Zf, axis=2)))


def tsvt_dft(Z, tau, return_info=False):
    """Proximal operator of tau * TNN-F at Z: Y = ifft(SVT_tau(fft(Z))) slice
    by slice.  With the unnormalised DFT, ||Y - Z||_F^2 = (1/n3) sum_k
    ||Y~_k - Z~_k||_F^2, so the threshold of every DFT slice is tau itself.
    With return_info, also returns TNN-F of Y."""
    Z = np.asarray(Z, dtype=np.float64)
    n3 = Z.shape[2]
    Zf = np.fft.fft(Z, axis=2)
    Yf = np.empty_like(Zf)
    for k in range(n3):
        U, s, Vh = np.linalg.svd(Zf[:, :, k], full_matrices=False)
        Yf[:, :, k] = (U * np.maximum(s - tau, 0.0)) @ Vh
    Y = np.asfortranarray(np.real(np.fft.ifft(Yf, axis=2)))
    if return_info:
        return Y, tnn_f(Y)
    return Y
