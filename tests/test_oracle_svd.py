"""Pins of the oracle's SVD layer: the Jacobi SVD against LAPACK, the t-SVT
(Theorem 5, Algorithm 1) against its optimality certificate, a brute-force
perturbation test, library special cases and closed forms, and the t-SVD
(Theorem 4) against its defining properties.
"""
import numpy as np
import pytest
import scipy.fft

import oracle as O


def _mats():
    rng = np.random.default_rng(21)
    yield "gauss_30x20", rng.standard_normal((30, 20))
    yield "square_16", rng.standard_normal((16, 16))
    yield "col", rng.standard_normal((7, 1))
    yield "rank3_40x25", rng.standard_normal((40, 3)) @ rng.standard_normal((3, 25))
    g = rng.standard_normal((25, 12))
    q, _ = np.linalg.qr(g)
    yield "graded", q @ np.diag(10.0 ** -np.arange(12)) @ np.linalg.qr(rng.standard_normal((12, 12)))[0]
    yield "zeros", np.zeros((6, 4))
    yield "uniform_176x144", rng.random((176, 144))


@pytest.mark.parametrize("name,A", list(_mats()), ids=[n for n, _ in _mats()])
def test_jacobi_svd_vs_lapack(name, A):
    U, s, V, sweeps, conv = O.jacobi_svd(A)
    assert conv
    ref = np.linalg.svd(A, compute_uv=False)
    scale = max(ref[0], 1e-300)
    assert np.abs(s - ref).max() <= 1e-13 * scale
    assert (np.diff(s) <= 0).all()
    n = A.shape[1]
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-13
    nz = s > 1e-12 * scale
    Ur = U[:, nz]
    if nz.any():
        assert np.abs(Ur.T @ Ur - np.eye(nz.sum())).max() <= 1e-12
    if A.any():
        assert np.linalg.norm(U @ np.diag(s) @ V.T - A) <= 1e-14 * np.linalg.norm(A) * np.sqrt(n)


def _svt_library(A, tau):
    u, s, vt = np.linalg.svd(A, full_matrices=False)
    return (u * np.maximum(s - tau, 0.0)) @ vt


def _tsvt_library(Z, tau):
    # Algorithm 1's t-SVT assembled from library routines only (scipy DCT, LAPACK SVD)
    Zb = scipy.fft.dct(Z, type=2, norm="ortho", axis=2)
    Yb = np.stack([_svt_library(Zb[:, :, k], tau) for k in range(Z.shape[2])], axis=2)
    return scipy.fft.idct(Yb, type=2, norm="ortho", axis=2)


@pytest.mark.parametrize("shape,tau", [((6, 5, 4), 0.7), ((5, 8, 3), 1.5), ((12, 9, 7), 0.3),
                                        ((20, 25, 8), 2.0), ((9, 9, 1), 0.5)])
def test_tsvt_matches_library_route(shape, tau):
    rng = np.random.default_rng(31)
    Z = rng.standard_normal(shape)
    Y, tnn, info = O.tsvt(Z, tau, return_info=True)
    assert info["converged"]
    ref = _tsvt_library(Z, tau)
    assert np.linalg.norm(Y - ref) <= 1e-13 * np.linalg.norm(Z)
    # tnn_out = sum_k ||dct(Y)_k||_*  (no 1/n3)
    Yb = scipy.fft.dct(Y, type=2, norm="ortho", axis=2)
    nuc = sum(np.linalg.svd(Yb[:, :, k], compute_uv=False).sum() for k in range(shape[2]))
    assert abs(tnn - nuc) <= 1e-12 * max(1.0, nuc)


@pytest.mark.parametrize("shape,tau", [((6, 5, 4), 0.7), ((5, 8, 3), 1.5), ((10, 7, 6), 0.9)])
def test_tsvt_optimality_certificate(shape, tau):
    """Theorem 5: Y is the prox of tau * sum_k ||dct(.)_k||_*.  Per transformed
    slice, G = Zbar_k - Ybar_k must equal tau (U_r V_r^T + W) with U_r^T W = 0,
    W V_r = 0 and ||W||_2 <= 1 (the subdifferential of the nuclear norm)."""
    rng = np.random.default_rng(41)
    Z = rng.standard_normal(shape)
    Y = O.tsvt(Z, tau)
    Zb = scipy.fft.dct(Z, type=2, norm="ortho", axis=2)
    Yb = scipy.fft.dct(Y, type=2, norm="ortho", axis=2)
    for k in range(shape[2]):
        G = Zb[:, :, k] - Yb[:, :, k]
        u, s, vt = np.linalg.svd(Yb[:, :, k], full_matrices=False)
        r = int((s > 1e-10 * max(1.0, s[0] if s.size else 0)).sum())
        Ur, Vr = u[:, :r], vt[:r, :].T
        assert np.linalg.norm(G, 2) <= tau * (1 + 1e-12)
        if r:
            assert np.abs(Ur.T @ G @ Vr - tau * np.eye(r)).max() <= 1e-12 * max(1.0, tau)
            W = G - tau * Ur @ Vr.T
            assert np.abs(Ur.T @ W).max() <= 1e-12 * max(1.0, tau)
            assert np.abs(W @ Vr).max() <= 1e-12 * max(1.0, tau)


def test_tsvt_brute_force_perturbation():
    """f(Y) = tau sum_k ||dct(Y)_k||_* + 1/2 ||Y - Z||_F^2 is minimal at the
    oracle's Y: no random perturbation lowers it."""
    rng = np.random.default_rng(51)
    Z = rng.standard_normal((4, 3, 3))
    tau = 0.8

    def f(Y):
        Yb = scipy.fft.dct(Y, type=2, norm="ortho", axis=2)
        nuc = sum(np.linalg.svd(Yb[:, :, k], compute_uv=False).sum() for k in range(Y.shape[2]))
        return tau * nuc + 0.5 * np.sum((Y - Z) ** 2)

    Y = O.tsvt(Z, tau)
    f0 = f(Y)
    viol = 0
    for t in range(1000):
        d = rng.standard_normal(Z.shape) * (10.0 ** rng.uniform(-6, 0))
        if f(Y + d) < f0 - 1e-12:
            viol += 1
    assert viol == 0


def test_tsvt_special_cases():
    rng = np.random.default_rng(61)
    Z = rng.standard_normal((7, 5, 6))
    # tau = 0 returns the input
    assert np.abs(O.tsvt(Z, 0.0) - Z).max() <= 1e-13
    # tau above every singular value of every transformed slice returns 0
    Zb = scipy.fft.dct(Z, type=2, norm="ortho", axis=2)
    smax = max(np.linalg.svd(Zb[:, :, k], compute_uv=False)[0] for k in range(6))
    assert np.abs(O.tsvt(Z, smax * 1.0001)).max() == 0.0
    # n3 = 1 is the matrix SVT
    A = rng.standard_normal((8, 6))
    Y1 = O.tsvt(A[:, :, None], 0.9)[:, :, 0]
    assert np.abs(Y1 - _svt_library(A, 0.9)).max() <= 1e-13


def test_svt_rank1_closed_form():
    # A = s u v^T with unit u, v: SVT gives max(s - tau, 0) u v^T
    rng = np.random.default_rng(71)
    u = rng.standard_normal(9); u /= np.linalg.norm(u)
    v = rng.standard_normal(5); v /= np.linalg.norm(v)
    A = 3.0 * np.outer(u, v)
    Y, nuc = O.svt_matrix(A, 1.25)
    assert np.abs(Y - 1.75 * np.outer(u, v)).max() <= 1e-14
    assert abs(nuc - 1.75) <= 1e-14
    Y, nuc = O.svt_matrix(A.T, 1.25)   # wide input takes the transposed route
    assert np.abs(Y - 1.75 * np.outer(v, u)).max() <= 1e-14


@pytest.mark.parametrize("shape", [(6, 4, 5), (4, 6, 5), (5, 5, 1), (8, 3, 7)])
def test_tsvd_theorem4(shape):
    rng = np.random.default_rng(81)
    X = rng.standard_normal(shape)
    U, S, V = O.tsvd(X)
    m1, m2, m3 = shape
    r = min(m1, m2)
    Sf = O.fdiag(S, r)
    # every frontal slice of S is diagonal (Definition 4): the off-diagonal entries are exactly 0
    off = Sf.copy()
    for i in range(r):
        off[i, i, :] = 0.0
    assert not off.any()
    # X = U * S * V^T under the t-product of Eq. 13
    R = O.tprod_btph(O.tprod_btph(U, Sf), O.ttranspose(V))
    assert np.abs(R - X).max() <= 1e-13 * max(1.0, np.abs(X).max())
    # U^T * U = I and V^T * V = I (identity tensor of Definition 2)
    I = np.zeros((r, r, m3)); I[:, :, 0] = np.eye(r)
    assert np.abs(O.tprod_btph(O.ttranspose(U), U) - I).max() <= 1e-13
    assert np.abs(O.tprod_btph(O.ttranspose(V), V) - I).max() <= 1e-13
    # the singular values of L(X)_k are those of dct(X)_k divided by w_k
    L = O.tube_transform(X, scaled=True)
    w = O.dct_matrix(m3)[:, 0]
    Sh = O.tube_transform(S[:, None, :], scaled=True)[:, 0, :]
    for k in range(m3):
        ref = np.linalg.svd(L[:, :, k], compute_uv=False)
        assert np.abs(Sh[:, k] - ref).max() <= 1e-13 * max(1.0, ref[0])
        ref2 = np.linalg.svd(scipy.fft.dct(X, type=2, norm="ortho", axis=2)[:, :, k], compute_uv=False) / w[k]
        assert np.abs(Sh[:, k] - ref2).max() <= 1e-12 * max(1.0, ref2[0])
