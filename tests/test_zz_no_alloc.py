"""tsvt_dct_static, the t-SVT entry point that allocates nothing, against
tsvt_dct.  It serves callers that cannot allocate device memory when they need
a t-SVT (a loop bound to a memory budget owned by another allocator, code that
must not create a context); its scratch is a static device array.  The test
calls it through the C ABI twice in a row, on different inputs, so that a
second call cannot lean on what the first one left in the shared scratch.
It runs last (the file name sorts after every other test file) and also
passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from gpu_common import dtype_of, torch_cuda
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_static_matches_tsvt_dct_two_calls(prec):
    torch = torch_cuda()
    from paper_1902_03070_gb300 import tnn
    L = tnn._lib
    dt = dtype_of(prec)
    rng = np.random.default_rng(99)
    with tnn.Context(0) as ctx:
        for call, shape in enumerate([(40, 30, 12), (25, 48, 7)]):
            Z = inputs.random_tensor(shape, rng)
            Zd = tnn.to_fortran(Z, dtype=dt)
            tau = 0.5 + call
            Yref = tnn.fortran_empty(shape, dt)
            ctx.tsvt(Zd, tau, Y=Yref, prec=prec)
            Y = tnn.fortran_empty(shape, dt)
            Y.fill_(float("nan"))
            stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            st = L.tsvt_dct_static(Zd.data_ptr(), tnn.Shape(*shape), tau, tnn.PRECISIONS[prec], Y.data_ptr(),
                                   stream)
            assert st == tnn.OK, tnn.status_string(st)
            torch.cuda.synchronize()
            a, b = tnn.to_numpy(Y).astype(np.float64), tnn.to_numpy(Yref).astype(np.float64)
            assert np.isfinite(a).all()
            assert np.linalg.norm(a - b) <= TOL[prec] * max(np.linalg.norm(b), 1e-300), call


def test_static_rejects_beyond_scratch_and_host_pointers():
    torch = torch_cuda()
    from paper_1902_03070_gb300 import tnn
    L = tnn._lib
    big = tnn.fortran_empty((128, 128, 300), torch.float32)   # 19.7 MB > 16 MiB of scratch
    st = L.tsvt_dct_static(big.data_ptr(), tnn.Shape(128, 128, 300), 1.0, tnn.PRECISIONS["fp32"], big.data_ptr(),
                           None)
    assert st == tnn.EINVAL
    host = np.zeros((4, 4, 4), order="F")
    st = L.tsvt_dct_static(host.ctypes.data, tnn.Shape(4, 4, 4), 1.0, tnn.PRECISIONS["fp64"], host.ctypes.data, None)
    assert st == tnn.EINVAL
