"""GPU parity: thin DCT t-SVD (Theorem 4) and its inverse through the C ABI.
The singular tubes S are unique and compared with the oracle; U and V are
unique only up to signs, so they are checked through the theorem's
properties: X = U * S * V^T, U^T * U = V^T * V = I, S f-diagonal."""
import numpy as np
import pytest

import oracle as O
from gpu_common import dtype_of, torch_cuda
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with tnn.Context(0) as c:
        yield c


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("shape", [(6, 4, 5), (4, 6, 5), (48, 48, 16), (33, 70, 3), (9, 1, 2), (100, 60, 7)])
def test_tsvd_properties_and_tubes(ctx, prec, shape):
    from paper_1902_03070_gb300 import tnn
    n1, n2, n3 = shape
    r = min(n1, n2)
    rng = np.random.default_rng(n1 + 7 * n2 + 31 * n3)
    X = inputs.random_tensor(shape, rng)
    if prec != "fp64":
        X = X.astype(np.float32).astype(np.float64)
    dt = dtype_of(prec)
    U = tnn.fortran_empty((n1, r, n3), dt)
    S = tnn.fortran_empty((r, n3), dt)
    V = tnn.fortran_empty((n2, r, n3), dt)
    ctx.tsvd(tnn.to_fortran(X, dtype=dt), U, S, V, prec=prec)
    U, S, V = tnn.to_numpy(U).astype(np.float64), tnn.to_numpy(S).astype(np.float64), tnn.to_numpy(V).astype(np.float64)
    tol = 1e-12 if prec == "fp64" else 2e-5
    scale = np.abs(X).max()
    Sf = O.fdiag(S, r)
    R = O.tprod(O.tprod(U, Sf), O.ttranspose(V))
    assert np.abs(R - X).max() <= tol * scale * max(1, r / 8)
    I = np.zeros((r, r, n3)); I[:, :, 0] = np.eye(r)
    assert np.abs(O.tprod(O.ttranspose(U), U) - I).max() <= tol * max(1, r / 8)
    assert np.abs(O.tprod(O.ttranspose(V), V) - I).max() <= tol * max(1, r / 8)
    _, So, _ = O.tsvd(X)
    assert np.abs(S - So).max() <= tol * np.abs(So).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_tsvd_inverse_roundtrip(ctx, prec):
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(3)
    X = inputs.random_tensor((20, 14, 9), rng)
    dt = dtype_of(prec)
    Xd = tnn.to_fortran(X, dtype=dt)
    U = tnn.fortran_empty((20, 14, 9), dt)
    S = tnn.fortran_empty((14, 9), dt)
    V = tnn.fortran_empty((14, 14, 9), dt)
    ctx.tsvd(Xd, U, S, V, prec=prec)
    Xr = tnn.fortran_empty((20, 14, 9), dt)
    ctx.tsvd_inverse(U, S, V, Xr, prec=prec)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.linalg.norm(tnn.to_numpy(Xr) - X) <= tol * np.linalg.norm(X)
