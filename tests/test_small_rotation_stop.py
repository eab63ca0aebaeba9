"""The small-rotation stop of the one-sided Jacobi kernels, as a property of
the iteration itself (no GPU): a sweep whose applied rotations all had
|gamma| / sqrt(alpha beta) <= theta and |t| <= theta, theta = sqrt(tol / 4n),
leaves every column pair within 2 tol of orthogonal, the level the plain
rule (no rotation above 2 tol in a sweep) accepts.

The iteration is a plain FP64 one-sided Hestenes Jacobi in cyclic order with
Rutishauser's rotation (the same update the kernels apply), run with an
artificially large tol so that the quadratic end of the convergence is
visible; the matrices include clusters of nearly equal singular values,
where rotation angles stay large while the off-diagonality is small."""
import numpy as np
import pytest


def _rotate(A, i, j):
    a, b = A[:, i], A[:, j]
    al, be, ga = a @ a, b @ b, a @ b
    zeta = (be - al) / (2.0 * ga)
    t = np.sign(zeta) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta)) if zeta != 0.0 else 1.0
    c = 1.0 / np.sqrt(1.0 + t * t)
    s = c * t
    A[:, i], A[:, j] = c * a - s * b, s * a + c * b
    return abs(t)


def _offdiag(A):
    n2 = (A * A).sum(0)
    G = np.abs(A.T @ A) / np.sqrt(np.outer(n2, n2))
    np.fill_diagonal(G, 0.0)
    return G.max()


def _matrix(rng, m, n, kind):
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    if kind == "spread":
        s = np.logspace(0, -3, n)
    elif kind == "clusters":  # groups of four singular values within 1e-6 of each other
        s = np.repeat(np.logspace(0, -2, n // 4), 4)[:n] * (1.0 + 1e-6 * rng.standard_normal(n))
    else:  # a near-identity start, as a warm start gives: small rotations from the first sweep
        s = np.linspace(1.0, 0.5, n)
        V = np.eye(n) + 1e-3 * rng.standard_normal((n, n))
    return (U * s) @ V.T


@pytest.mark.parametrize("kind", ["spread", "clusters", "warm"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_small_rotation_stop_leaves_pairs_within_two_tol(kind, seed):
    rng = np.random.default_rng(100 * seed + len(kind))
    m, n = 40, 24
    tol = 1e-9
    theta = np.sqrt(tol / (4.0 * n))
    A = _matrix(rng, m, n, kind)
    fired = False
    for sweep in range(40):
        big = 0
        small_only = True
        for i in range(n - 1):
            for j in range(i + 1, n):
                a, b = A[:, i], A[:, j]
                off = abs(a @ b) / np.sqrt((a @ a) * (b @ b))
                if off <= tol:
                    continue
                big += off > 2.0 * tol
                t = _rotate(A, i, j)
                if off > theta or t > theta:
                    small_only = False
        if small_only:  # the stop fires: every pair is already within 2 tol
            fired = True
            assert _offdiag(A) <= 2.0 * tol, (kind, seed, sweep, _offdiag(A))
            break
        if big == 0:
            break
    # the stop is the first of the two rules to fire whenever it fires; on
    # these matrices it fires in every case
    assert fired, (kind, seed)
