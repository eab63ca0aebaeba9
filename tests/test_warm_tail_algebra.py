"""The algebra of the warm-started SVT's tail (no GPU): from converged
one-sided Jacobi columns S = A W (W orthogonal, S's columns orthogonal, the
column scales d folded in), R = S^T A gives both outputs the tail kernel
writes:

- the recovered right singular vectors, v_c = R[c, :]^T / |s_c|^2 (that is
  A^T u_c / sigma_c), orthonormal when S is converged;
- the SVT of Theorem 5 (the matrix form of one slice), Y = sum over sigma_c
  > tau of (1 - tau / sigma_c) / |s_c|^2 s_c R[c, :], equal to U (Sigma -
  tau)_+ V^T from an SVD.

A warm start from an orthogonal Q changes neither: S = (A Q) W' has the same
singular values and left vectors, and R is still S^T A."""
import numpy as np
import pytest


def _svt(A, tau):
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    return (U * np.maximum(s - tau, 0.0)) @ Vt


@pytest.mark.parametrize("m,n", [(30, 20), (25, 25), (40, 7)])
@pytest.mark.parametrize("warm", [False, True])
def test_tail_outputs_from_r(m, n, warm):
    rng = np.random.default_rng(m * 100 + n + warm)
    A = rng.standard_normal((m, n)) @ np.diag(np.logspace(0, -2, n))
    # converged columns: S = A W with W the right singular vectors, columns
    # permuted (a Jacobi run leaves them in any order); with a warm start the
    # iteration runs on A Q, and S = A Q (Q^T W)
    _, s, Vt = np.linalg.svd(A, full_matrices=False)
    perm = rng.permutation(n)
    W = Vt.T[:, perm]
    if warm:
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        S = (A @ Q) @ (Q.T @ W)
    else:
        S = A @ W
    R = S.T @ A
    n2 = (S * S).sum(0)
    sig = np.sqrt(n2)
    # recovered right vectors, by descending sigma
    order = np.argsort(-sig)
    Vrec = (R[order] / n2[order, None]).T
    assert np.abs(Vrec.T @ Vrec - np.eye(n)).max() <= 1e-10
    assert np.abs(np.abs(Vrec) - np.abs(Vt.T)).max() <= 1e-10
    # the rebuild from R: the SVT, for thresholds inside and outside the spectrum
    for tau in (0.0, 0.5 * s[n // 2], s[0] * 1.01):
        kept = sig > tau
        Y = (S[:, kept] * ((1.0 - tau / sig[kept]) / n2[kept])) @ R[kept]
        assert np.linalg.norm(Y - _svt(A, tau)) <= 1e-10 * max(np.linalg.norm(A), 1.0)


def test_tail_rebuild_detects_a_wrong_scale():
    # the coefficient is (1 - tau/sigma) / |s|^2: with / |s| instead the
    # rebuild is off (guards the formula the tail kernel uses)
    rng = np.random.default_rng(7)
    A = rng.standard_normal((20, 12))
    _, s, Vt = np.linalg.svd(A, full_matrices=False)
    S = A @ Vt.T * 3.0  # columns scaled: |s_c| = 3 sigma_c
    R = S.T @ A
    n2 = (S * S).sum(0)
    sig = np.sqrt(n2) / 3.0
    tau = s[4]
    kept = sig > tau
    good = (S[:, kept] * ((1.0 - tau / sig[kept]) / n2[kept])) @ R[kept]
    bad = (S[:, kept] * ((1.0 - tau / sig[kept]) / np.sqrt(n2[kept]))) @ R[kept]
    assert np.linalg.norm(good - _svt(A, tau)) <= 1e-10 * np.linalg.norm(A)
    assert np.linalg.norm(bad - _svt(A, tau)) > 1e-2 * np.linalg.norm(A)
