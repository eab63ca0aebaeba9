"""Pins of the DFT comparison path's oracle (oracle/dft.py) against facts the
definitions fix: a single slice is the matrix SVT (checked against the
independent Jacobi oracle in oracle.c), the DFT t-product agrees with the
block-circulant definition written out, the result is real and is the
proximal point of tau * TNN-F (no perturbation lowers the objective), and
TNN-F matches its definition on a tensor with a known spectrum."""
import numpy as np

import oracle as O
from oracle import dft as D


def _bcirc_tprod(X, Y):
    # Eq. (5): fold(bcirc(X) unfold(Y)), block (r, c) of bcirc(X) (Eq. (1)) = X^((r - c) mod n3)
    n1, n2, n3 = X.shape
    n4 = Y.shape[1]
    Z = np.zeros((n1, n4, n3))
    for r in range(n3):
        for c in range(n3):
            Z[:, :, r] += X[:, :, (r - c) % n3] @ Y[:, :, c]
    return Z


def test_single_slice_is_matrix_svt():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((9, 6))
    tau = 0.8
    Y = D.tsvt_dft(A[:, :, None], tau)[:, :, 0]
    assert np.allclose(Y, O.svt_matrix(A, tau)[0], atol=1e-12)


def test_tprod_dft_matches_block_circulant():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((4, 3, 5))
    Y = rng.standard_normal((3, 2, 5))
    assert np.allclose(D.tprod_dft(X, Y), _bcirc_tprod(X, Y), atol=1e-12)


def test_result_is_real_and_conjugate_symmetric():
    rng = np.random.default_rng(3)
    Z = rng.standard_normal((7, 5, 6))
    Zf = np.fft.fft(Z, axis=2)
    Yf = np.empty_like(Zf)
    for k in range(6):
        U, s, Vh = np.linalg.svd(Zf[:, :, k], full_matrices=False)
        Yf[:, :, k] = (U * np.maximum(s - 1.0, 0)) @ Vh
    assert np.abs(np.imag(np.fft.ifft(Yf, axis=2))).max() < 1e-12
    for k in range(1, 6):
        assert np.allclose(Yf[:, :, k], np.conj(Yf[:, :, 6 - k]), atol=1e-12)


def test_prox_optimality():
    # Y = argmin tau TNN-F(Y) + 1/2 ||Y - Z||^2: random perturbations never lower it
    rng = np.random.default_rng(4)
    Z = rng.standard_normal((6, 5, 4))
    tau = 1.3
    Y = D.tsvt_dft(Z, tau)
    f = lambda W: tau * D.tnn_f(W) + 0.5 * np.sum((W - Z) ** 2)
    f0 = f(Y)
    for _ in range(40):
        E = rng.standard_normal(Z.shape)
        for h in (1e-2, 1e-4):
            assert f(Y + h * E) >= f0 - 1e-12


def test_tnn_f_of_constant_tubes():
    # X(:, :, k) = A for all k: the DFT puts n3 A in slice 0 and zeros elsewhere,
    # so TNN-F = ||A||_* (Definition 6)
    rng = np.random.default_rng(5)
    A = rng.standard_normal((5, 4))
    X = np.repeat(A[:, :, None], 7, axis=2)
    assert abs(D.tnn_f(X) - np.linalg.svd(A, compute_uv=False).sum()) < 1e-12


def test_homogeneity_and_zero_threshold():
    rng = np.random.default_rng(6)
    Z = rng.standard_normal((5, 8, 3))
    assert np.allclose(D.tsvt_dft(Z, 0.0), Z, atol=1e-12)
    assert np.allclose(D.tsvt_dft(3.0 * Z, 3.0 * 0.7), 3.0 * D.tsvt_dft(Z, 0.7), atol=1e-12)
