"""GPU parity at the sizes of the paper's Table 2 (U[0,1) tensors, the
distribution the paper leaves unstated read as MATLAB's rand): the chosen
t-SVT form (3xTF32 transforms, FP32 Jacobi; slices of 400 x 400 spread over
thread-block clusters) against the FP64 oracle, held to 1e-5 relative to the
oracle's Y, with the threshold at the median singular value of the
transformed slices."""
import numpy as np
import pytest

import oracle as O
from gpu_common import THREADS, log_err, rel_err, tau_at_quantile, torch_cuda
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with tnn.Context(0) as c:
        yield c


@pytest.mark.parametrize("shape", [(100, 100, 100), (100, 100, 400), (200, 200, 100), (400, 400, 100)])
def test_tsvt_table2_sizes(ctx, shape):
    from paper_1902_03070_gb300 import tnn
    torch = torch_cuda()
    Z = inputs.random_tensor(shape, np.random.default_rng(sum(shape)), "uniform")
    Z = Z.astype(np.float32).astype(np.float64)
    tau = tau_at_quantile(Z, 0.5)
    Zd = tnn.to_fortran(Z, dtype=torch.float32)
    Yd = tnn.fortran_empty(shape, torch.float32)
    ctx.tsvt(Zd, tau, Y=Yd, prec="tf32x3")
    Y = tnn.to_numpy(Yd).astype(np.float64)
    ref = O.tsvt(Z, tau, nthreads=THREADS)
    err = rel_err(Y, ref, Z)
    log_err("tsvt table2 %s" % (shape,), err_y=err, err_z=np.linalg.norm(Y - ref) / np.linalg.norm(Z))
    assert err <= 1e-5, err
