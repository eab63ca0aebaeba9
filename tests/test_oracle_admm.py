"""Pins of the oracle's Algorithm 1 (ADMM for the completion model, Eq. 17):
bit-exact invariants, full observation, exact recovery of a low-tubal-rank
tensor, and the optimality certificate of the completion model at the limit.
"""
import numpy as np
import pytest
import scipy.fft

import oracle as O
from paper_1902_03070_gb300 import inputs


def _problem(n1, n2, n3, r, frac, seed):
    rng = np.random.default_rng(seed)
    A, F = inputs.lowrank_factors(n1, n2, n3, r, rng)
    T = O.tprod(A, F)
    mask = inputs.uniform_mask(T.shape, frac, np.random.default_rng(seed + 1))
    return T, inputs.fortran(T * mask), mask


def test_admm_invariants_bit_exact():
    T, B, mask = _problem(10, 12, 5, 2, 0.5, 1)
    for iters in (1, 2, 7):
        X, M, rep = O.admm(B, mask, beta0=1.0, rho=1.1, tol=-1.0, max_iter=iters)
        assert rep["iters"] == iters
        m = mask.astype(bool)
        # X_Omega = B_Omega and M_{Omega^c} = 0 hold exactly (from M = 0 at start)
        assert np.array_equal(X[m], B[m])
        assert not M[~m].any()


def test_admm_full_observation_one_iteration():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((6, 7, 4))
    mask = np.ones(B.shape, dtype=np.uint8)
    for iters in (1, 3):
        X, M, rep = O.admm(B, mask, beta0=1.0, rho=1.0, tol=-1.0, max_iter=iters)
        assert rep["iters"] == iters
        assert np.array_equal(X, B)
        # the multiplier collects beta (Y - B) every iteration
        assert M.any()


def test_admm_empty_observation_stays_zero():
    B = np.zeros((5, 4, 3))
    mask = np.zeros(B.shape, dtype=np.uint8)
    X, M, rep = O.admm(B, mask, beta0=1.0, rho=1.0, tol=1e-12, max_iter=5)
    assert rep["iters"] == 1 and rep["converged"] and not X.any() and not M.any()


def test_admm_fixed_beta_is_rho_one():
    T, B, mask = _problem(8, 8, 4, 2, 0.6, 3)
    _, _, rep = O.admm(B, mask, beta0=0.5, rho=1.0, tol=-1.0, max_iter=4)
    assert rep["beta_final"] == 0.5
    _, _, rep = O.admm(B, mask, beta0=0.5, rho=2.0, beta_max=3.0, tol=-1.0, max_iter=4)
    assert rep["beta_final"] == 3.0


@pytest.mark.slow
def test_admm_recovers_low_tubal_rank_and_certificate():
    T, B, mask = _problem(20, 18, 6, 2, 0.6, 4)
    # beta_max is kept moderate: at the last iterate the certificate holds up to
    # beta ||X - Y||, so beta times the final residual must stay small.
    X, M, rep = O.admm(B, mask, beta0=1e-2, rho=1.2, beta_max=1e3, tol=1e-12, max_iter=600, nthreads=4)
    assert rep["converged"]
    rel = np.linalg.norm(X - T) / np.linalg.norm(T)
    assert rel <= 1e-10
    # Optimality of Eq. 17 at the limit: -M (supported on Omega) is a subgradient of
    # sum_k ||dct(.)_k||_* at X.  Per transformed slice: U_r^T G V_r = I, ||G||_2 <= 1.
    Xb = scipy.fft.dct(X, type=2, norm="ortho", axis=2)
    Gb = scipy.fft.dct(-M, type=2, norm="ortho", axis=2)
    for k in range(X.shape[2]):
        u, s, vt = np.linalg.svd(Xb[:, :, k], full_matrices=False)
        r = int((s > 1e-6 * s[0]).sum())
        Ur, Vr = u[:, :r], vt[:r].T
        assert np.abs(Ur.T @ Gb[:, :, k] @ Vr - np.eye(r)).max() <= 1e-6
        assert np.linalg.norm(Gb[:, :, k], 2) <= 1 + 1e-6


def test_admm_resume_equals_one_run():
    # Algorithm 1 continued from the state (X, M, beta) after 3 iterations
    # gives, 2 iterations later, bit for bit the state of one 5-iteration run
    T, B, mask = _problem(9, 11, 6, 2, 0.4, 5)
    X5, M5, r5 = O.admm(B, mask, beta0=0.3, rho=1.3, tol=-1.0, max_iter=5)
    X3, M3, r3 = O.admm(B, mask, beta0=0.3, rho=1.3, tol=-1.0, max_iter=3)
    assert r3["beta_final"] == 0.3 * 1.3 * 1.3 * 1.3
    X, M, r = O.admm(B, mask, beta0=r3["beta_final"], rho=1.3, tol=-1.0, max_iter=2, X0=X3, M0=M3)
    assert r["iters"] == 2
    assert np.array_equal(X, X5) and np.array_equal(M, M5)
    assert r["beta_final"] == r5["beta_final"]
    # the state passed in is not modified
    X3b, M3b, _ = O.admm(B, mask, beta0=0.3, rho=1.3, tol=-1.0, max_iter=3)
    assert np.array_equal(X3, X3b) and np.array_equal(M3, M3b)
