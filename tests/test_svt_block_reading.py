"""The property behind the Jacobi SVT's small-column sweeps (Theorem 5's SVT,
checked against the oracle's matrix SVT).

Let A = S V^T with V orthogonal and S = [S_H | S_Lo], where S_H's columns are
orthogonal to each other and to every column of S_Lo, and S_Lo's columns are
not orthogonal to each other.  If ||S_Lo||_F <= tau, then the SVT of A equals
the rebuild over S_H's columns with sigma > tau, sum (1 - tau/sigma_i)
/ |s_i|^2 s_i (s_i^T A), whatever S_Lo's inner structure.  If S_Lo carries a
singular value above tau, the same rebuild is wrong: the block cannot be left
unrotated.

And the zero-SVT certificate: when the Gershgorin bound on S^T S, computed in
FP32 with the kernel's rounding margins, is below tau^2, the oracle's SVT is
exactly zero; the bound never fires for a slice whose top singular value is
above tau."""
import numpy as np
import pytest

import oracle as O


def _case(rng, m, n, nh, lo_fro, tau):
    # S_H: nh orthogonal columns with norms spread around tau; S_Lo: the rest,
    # correlated columns in the orthogonal complement of S_H, Frobenius lo_fro
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    sig = tau * np.linspace(0.5, 6.0, nh)
    SH = Q[:, :nh] * sig
    base = Q[:, nh:nh + 3] @ rng.standard_normal((3, n - nh))  # rank 3: far from orthogonal
    base += 1e-3 * Q[:, nh:] @ rng.standard_normal((m - nh, n - nh))
    SLo = base * (lo_fro / np.linalg.norm(base))
    S = np.hstack([SH, SLo])
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return S, V, S @ V.T


def _rebuild(S, A, nh, tau):
    Y = np.zeros_like(A)
    for i in range(nh):
        s = S[:, i]
        n2 = s @ s
        sg = np.sqrt(n2)
        if sg > tau:
            Y += (1.0 - tau / sg) / n2 * np.outer(s, s @ A)
    return Y


@pytest.mark.parametrize("m,n,nh", [(40, 30, 5), (60, 60, 12), (25, 24, 1)])
@pytest.mark.parametrize("frac", [0.3, 0.9, 0.999])
def test_small_block_needs_no_rotation(m, n, nh, frac):
    rng = np.random.default_rng(m * 100 + n + int(frac * 1000))
    tau = 0.8
    S, V, A = _case(rng, m, n, nh, frac * tau, tau)
    # S_Lo is far from orthogonal (the premise of the shortcut)
    SLo = S[:, nh:]
    G = SLo.T @ SLo
    off = np.abs(G - np.diag(np.diag(G))).max() / np.diag(G).max()
    assert off > 1e-2
    Y, _ = O.svt_matrix(A, tau)
    Yb = _rebuild(S, A, nh, tau)
    assert np.linalg.norm(Yb - Y) <= 1e-12 * np.linalg.norm(A)


def test_large_block_must_be_rotated():
    # S_Lo with Frobenius norm 3 tau on three directions: its top singular
    # value is above tau, so leaving it out changes the SVT
    rng = np.random.default_rng(7)
    tau = 0.8
    S, V, A = _case(rng, 40, 30, 5, 3.0 * tau, tau)
    assert np.linalg.svd(S[:, 5:], compute_uv=False)[0] > tau
    Y, _ = O.svt_matrix(A, tau)
    Yb = _rebuild(S, A, 5, tau)
    assert np.linalg.norm(Yb - Y) > 1e-3 * np.linalg.norm(A)


def _gershgorin_fp32(S, tau):
    # the kernel's certificate, in FP32 like the FP32 kernel: row sums of
    # |S^T S| plus the rounding margins (m u |a_i| sum_j |a_j|, 2 n u)
    S32 = S.astype(np.float32)
    G = S32.T @ S32
    m, n = S.shape
    u = 2.0 ** -24
    nrm = np.linalg.norm(S, axis=0)
    rows = np.abs(G).astype(np.float64).sum(1) * (1 + 2 * n * u) + 2 * m * u * nrm * 1.01 * nrm.sum()
    return rows.max() <= (1 - 1e-4) * tau * tau


@pytest.mark.parametrize("s1", [0.2, 0.6, 0.9, 0.99, 1.01, 1.2])
@pytest.mark.parametrize("ortho", [0.0, 1e-4, 1e-2])
def test_zero_svt_certificate(s1, ortho):
    # S = U diag(sigma) W with W close to orthogonal (columns nearly
    # orthogonal after a Jacobi sweep or two); A = S V^T.  Where the bound
    # certifies, the oracle's SVT is exactly zero; it never certifies a slice
    # whose top singular value is above tau.
    rng = np.random.default_rng(int(s1 * 100) + int(ortho * 1e5))
    m, n, tau = 50, 40, 0.6
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    sig = s1 * tau * np.linspace(1.0, 0.1, n)
    W = np.eye(n) + ortho * rng.standard_normal((n, n))
    S = (U * sig) @ W
    S *= s1 * tau / np.linalg.svd(S, compute_uv=False)[0]  # top singular value exactly s1 tau
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = S @ V.T
    cert = _gershgorin_fp32(S, tau)
    Y, _ = O.svt_matrix(A, tau)
    if cert:
        assert np.abs(Y).max() == 0.0
    if s1 > 1.0:
        assert not cert
    if s1 <= 0.9 and ortho <= 1e-4:
        assert cert  # nearly orthogonal columns well below tau: the bound is tight enough


def _low_block_cert_fp32(S, tau, eps):
    # the kernel's low-block certificate (reading 22), in FP32 like the FP32
    # kernel: the low set is the columns below tau^2; row sums of |S_L^T S_L|
    # plus the rounding margins, accepted up to (tau + eps)^2
    S32 = S.astype(np.float32)
    nrm = np.linalg.norm(S, axis=0)
    L = nrm < tau
    SL = S32[:, L]
    G = SL.T @ SL
    m = S.shape[0]
    nl = int(L.sum())
    u = 2.0 ** -24
    rows = (np.abs(G).astype(np.float64).sum(1) * (1 + 2 * nl * u)
            + 2 * m * u * nrm[L] * 1.01 * nrm[L].sum())
    return rows.max() <= (tau + eps) ** 2, L


def _low_case(rng, m, n, nh, top, spread, tau):
    # S_H: nh orthogonal columns far above tau; S_L: the other columns,
    # orthogonal to S_H, with singular values from top * tau down, mixed by a
    # near-identity matrix so that its columns are not quite orthogonal
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    SH = Q[:, :nh] * (tau * np.geomspace(2000.0, 30.0, nh))
    nl = n - nh
    sl = tau * np.linspace(top, 0.1, nl)
    W = np.eye(nl) + spread * rng.standard_normal((nl, nl))
    SL = (Q[:, nh:nh + nl] * sl) @ W
    SL *= top * tau / np.linalg.svd(SL, compute_uv=False)[0]   # top low singular value exactly top * tau
    S = np.hstack([SH, SL])
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return S, S @ V.T


@pytest.mark.parametrize("top", [0.9, 0.99, 0.999, 1.02, 1.2])
@pytest.mark.parametrize("spread", [1e-5, 1e-3, 3e-2])
def test_low_block_certificate(top, spread):
    # soundness: where the certificate accepts, the rebuild over the columns
    # above tau is the oracle's SVT to within the allowance eps per low
    # singular value; a low set (columns below tau) whose block has a
    # singular value above tau + eps is never certified
    rng = np.random.default_rng(int(top * 1000) + int(spread * 1e5))
    m, n, nh, tau = 60, 48, 10, 0.5
    S, A = _low_case(rng, m, n, nh, top, spread, tau)
    Y, _ = O.svt_matrix(A, tau)
    eps = 1e-7 * np.linalg.norm(Y)
    cert, L = _low_block_cert_fp32(S, tau, eps)
    if cert:
        H = np.flatnonzero(~L)
        Yb = _rebuild(S[:, H], A, len(H), tau)
        assert np.linalg.norm(Yb - Y) <= np.sqrt(L.sum()) * eps + 1e-12 * np.linalg.norm(A)
    if np.linalg.svd(S[:, L], compute_uv=False)[0] > tau + 2 * eps:
        assert not cert
    if top <= 0.99 and spread <= 1e-5:
        assert cert  # nearly orthogonal and clear of tau: the bound is tight enough


def test_low_block_certificate_rejects_correlated_columns():
    # every low column below tau, but correlated so that the block has a
    # singular value above tau: the certificate must refuse, and leaving the
    # block out would indeed be wrong
    rng = np.random.default_rng(3)
    m, n, nh, tau = 60, 40, 6, 0.5
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    SH = Q[:, :nh] * (tau * np.geomspace(500.0, 40.0, nh))
    base = Q[:, nh:nh + 2] @ rng.standard_normal((2, n - nh))
    SL = base * (0.9 * tau / np.linalg.norm(base, axis=0))   # each column at 0.9 tau
    S = np.hstack([SH, SL])
    assert np.linalg.svd(SL, compute_uv=False)[0] > 1.5 * tau
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = S @ V.T
    Y, _ = O.svt_matrix(A, tau)
    cert, L = _low_block_cert_fp32(S, tau, 1e-7 * np.linalg.norm(Y))
    assert L.sum() == n - nh and not cert
    assert np.linalg.norm(_rebuild(S, A, nh, tau) - Y) > 1e-3 * np.linalg.norm(Y)
