"""GPU parity: tube transforms (dct / idct / L / L^-1) and the DCT t-product
(Eq. 13) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from gpu_common import dtype_of, torch_cuda
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(48, 48, 16), (7, 5, 31), (3, 1, 1), (1, 9, 2), (129, 3, 65), (144, 176, 100), (20, 30, 130)]
# three-part BF16 split: each value kept to about 24 significant bits and
# the products of order above two dropped: FP32 accuracy, as 3xTF32
TOL = {"fp64": 1e-13, "fp32": 2e-6, "tf32x3": 2e-6, "bf16split": 2e-6}


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with tnn.Context(0) as c:
        yield c


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16split"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("inverse,scaled", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_tdct3_matches_oracle(ctx, prec, shape, inverse, scaled):
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(sum(shape) + 10 * inverse + 100 * scaled)
    X = inputs.random_tensor(shape, rng)
    Xd = tnn.to_fortran(X, dtype=dtype_of(prec))
    Yd = tnn.fortran_empty(shape, dtype_of(prec))
    ctx.tdct3(Xd, Yd, inverse=inverse, scaled=scaled, prec=prec)
    ref = O.tube_transform(X.astype(np.float32).astype(np.float64) if prec != "fp64" else X,
                           inverse=bool(inverse), scaled=bool(scaled))
    Y = tnn.to_numpy(Yd).astype(np.float64)
    assert np.linalg.norm(Y - ref) <= TOL[prec] * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16split"])
@pytest.mark.parametrize("dims", [(4, 3, 5, 6), (48, 3, 48, 16), (1, 7, 2, 3), (70, 65, 66, 9)])
def test_tprod_matches_oracle(ctx, prec, dims):
    from paper_1902_03070_gb300 import tnn
    m1, m2, m4, m3 = dims
    rng = np.random.default_rng(m1 * m2 + m4)
    X = inputs.random_tensor((m1, m2, m3), rng)
    Y = inputs.random_tensor((m2, m4, m3), rng)
    if prec != "fp64":
        X = X.astype(np.float32).astype(np.float64)
        Y = Y.astype(np.float32).astype(np.float64)
    Z = tnn.fortran_empty((m1, m4, m3), dtype_of(prec))
    ctx.tprod(tnn.to_fortran(X, dtype=dtype_of(prec)), tnn.to_fortran(Y, dtype=dtype_of(prec)), Z, prec=prec)
    ref = O.tprod(X, Y)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.linalg.norm(tnn.to_numpy(Z) - ref) <= tol * np.linalg.norm(ref)


def test_tprod_host_buffers(ctx):
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(5)
    X = inputs.random_tensor((6, 4, 5), rng)
    Y = inputs.random_tensor((4, 3, 5), rng)
    Z = np.zeros((6, 3, 5), order="F")
    ctx.tprod(X, Y, Z, prec="fp64")
    assert np.linalg.norm(Z - O.tprod(X, Y)) <= 1e-12 * np.linalg.norm(Z)
