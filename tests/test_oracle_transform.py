"""Pins of the oracle's transform layer against what the paper and the
mathematics fix: the DCT matrix (Section 3), Example 1's printed numbers,
Theorem 3 by brute force, and the two routes to the DCT t-product (Eqs. 13-14).
"""
import numpy as np
import pytest
import scipy.fft

import oracle as O
from conftest import load_golden


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 31, 64, 100])
def test_dct_matrix_orthogonal(n):
    C = O.dct_matrix(n)
    assert np.abs(C.T @ C - np.eye(n)).max() <= 1e-15 * max(n, 4)
    assert np.abs(C @ C.T - np.eye(n)).max() <= 1e-15 * max(n, 4)


@pytest.mark.parametrize("n", [1, 2, 5, 16, 31, 100])
def test_dct_matrix_is_scipy_dct2_ortho(n):
    # MATLAB's dct is the orthonormal DCT-II; scipy's type-2 'ortho' DCT is the same map.
    C = O.dct_matrix(n)
    ref = scipy.fft.dct(np.eye(n), type=2, norm="ortho", axis=0)
    assert np.abs(C - ref).max() <= 1e-15 * max(n, 4)


@pytest.mark.parametrize("shape", [(3, 4, 1), (5, 2, 7), (4, 6, 16), (2, 3, 31)])
def test_tube_transform_matches_scipy(shape):
    rng = np.random.default_rng(11)
    X = rng.standard_normal(shape)
    tol = 1e-15 * shape[2] * np.abs(X).max()   # direct O(n3) sums of n3 terms
    Y = O.tube_transform(X)
    assert np.abs(Y - scipy.fft.dct(X, type=2, norm="ortho", axis=2)).max() <= tol
    Xi = O.tube_transform(X, inverse=True)
    assert np.abs(Xi - scipy.fft.idct(X, type=2, norm="ortho", axis=2)).max() <= tol
    # scaled transform L and its inverse are inverse maps
    Lx = O.tube_transform(X, scaled=True)
    assert np.abs(O.tube_transform(Lx, inverse=True, scaled=True) - X).max() <= 1e-13
    # L(X)_k = dct(X)_k / w_k with w the first column of C (all entries > 0)
    w = O.dct_matrix(shape[2])[:, 0]
    assert (w > 0).all()
    assert np.abs(Lx - Y / w[None, None, :]).max() <= 1e-13


def _example1_tensor(g):
    X = np.zeros((2, 2, 2), order="F")
    X[:, :, 0] = g["X1"]
    X[:, :, 1] = g["X2"]
    return X


def test_example1_btph_printed_values():
    g = load_golden("example1.txt")
    X = _example1_tensor(g)
    B = O.btph(X)
    assert np.array_equal(B, g["btph"])
    # the printed decomposition: btph = bt + bh, with A^(1) = X^(1) - X^(2), A^(2) = X^(2)
    assert np.array_equal(g["A1"], g["X1"] - g["X2"])
    assert np.array_equal(g["A2"], g["X2"])
    assert np.array_equal(g["bt"] + g["bh"], g["btph"])
    # stride permutation as printed
    P = g["P"]
    assert np.array_equal(P @ B @ P, g["PbtphP"])


def test_example1_block_diagonalisation_printed_values():
    g = load_golden("example1.txt")
    X = _example1_tensor(g)
    C = O.dct_matrix(2)
    lhs = np.kron(C, np.eye(2)) @ O.btph(X) @ np.kron(C.T, np.eye(2))
    assert np.abs(lhs - g["CbtphCt"]).max() <= 1e-14
    # Theorem 3's diagonal blocks are the scaled transform of X (not plain dct(X))
    L = O.tube_transform(X, scaled=True)
    assert np.abs(L[:, :, 0] - g["CbtphCt"][0:2, 0:2]).max() <= 1e-14
    assert np.abs(L[:, :, 1] - g["CbtphCt"][2:4, 2:4]).max() <= 1e-14


@pytest.mark.parametrize("n3", [1, 2, 3, 4, 5, 6, 7, 8])
def test_theorem3_brute_force(n3):
    rng = np.random.default_rng(100 + n3)
    m1, m2 = 3, 4
    X = rng.standard_normal((m1, m2, n3))
    C = O.dct_matrix(n3)
    lhs = np.kron(C, np.eye(m1)) @ O.btph(X) @ np.kron(C.T, np.eye(m2))
    L = O.tube_transform(X, scaled=True)
    bd = np.zeros_like(lhs)
    for k in range(n3):
        bd[m1 * k:m1 * (k + 1), m2 * k:m2 * (k + 1)] = L[:, :, k]
    assert np.abs(lhs - bd).max() <= 1e-13 * max(1.0, np.abs(X).max())


@pytest.mark.parametrize("dims", [(3, 4, 2, 1), (2, 3, 4, 5), (4, 4, 4, 8), (5, 2, 3, 6)])
def test_tproduct_definition_equals_transform_route(dims):
    m1, m2, m4, m3 = dims
    rng = np.random.default_rng(7)
    X = rng.standard_normal((m1, m2, m3))
    Y = rng.standard_normal((m2, m4, m3))
    Z1 = O.tprod_btph(X, Y)   # Eq. 13, by definition
    Z2 = O.tprod(X, Y)        # Eq. 14, facewise in the transform domain
    assert np.abs(Z1 - Z2).max() <= 1e-12


def test_tproduct_single_slice_is_matrix_product():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, 3, 1))
    Y = rng.standard_normal((3, 5, 1))
    assert np.abs(O.tprod_btph(X, Y)[:, :, 0] - X[:, :, 0] @ Y[:, :, 0]).max() <= 1e-14
    assert np.abs(O.tprod(X, Y)[:, :, 0] - X[:, :, 0] @ Y[:, :, 0]).max() <= 1e-14


@pytest.mark.parametrize("m3", [1, 2, 5, 9])
def test_identity_tensor_is_the_unit(m3):
    # Definition 2: first slice I, other slices 0.  It must be the unit of Eq. 13.
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, 4, m3))
    I3 = np.zeros((3, 3, m3)); I3[:, :, 0] = np.eye(3)
    I4 = np.zeros((4, 4, m3)); I4[:, :, 0] = np.eye(4)
    assert np.abs(O.tprod_btph(I3, X) - X).max() <= 1e-13
    assert np.abs(O.tprod_btph(X, I4) - X).max() <= 1e-13
    assert np.abs(O.tprod(I3, X) - X).max() <= 1e-13
    assert np.abs(O.tprod(X, I4) - X).max() <= 1e-13


def test_tproduct_associative():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((3, 4, 5))
    B = rng.standard_normal((4, 2, 5))
    C = rng.standard_normal((2, 3, 5))
    lhs = O.tprod_btph(O.tprod_btph(A, B), C)
    rhs = O.tprod_btph(A, O.tprod_btph(B, C))
    assert np.abs(lhs - rhs).max() <= 1e-12
