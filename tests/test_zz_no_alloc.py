"""tsvt_dct_static, the t-SVT entry point that allocates nothing, against
tsvt_dct.  It serves callers that cannot allocate device memory when they need
a t-SVT (a loop bound to a memory budget owned by another allocator, code that
must not create a context); its scratch is a static device array.  The test
calls it through the C ABI twice in a row for every precision, on different
inputs, so that a second call cannot lean on what the first one left in the
shared scratch, and checks that a call changes neither the device's free
memory nor torch's reserved memory.  It runs last (the file name sorts after
every other test file) and also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from gpu_common import dtype_of, torch_cuda
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "tf32x3": 1e-5, "bf16split": 1e-5}
SHAPES = [(40, 30, 12), (25, 48, 7)]


def _static(L, tnn, torch, Zd, shape, tau, prec, Y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.tsvt_dct_static(Zd.data_ptr(), tnn.Shape(*shape), tau, tnn.PRECISIONS[prec], Y.data_ptr(), stream)


@pytest.mark.parametrize("prec", ["fp32", "fp64", "tf32x3", "bf16split"])
def test_static_matches_tsvt_dct_two_calls(prec):
    torch = torch_cuda()
    from paper_1902_03070_gb300 import tnn
    L = tnn._lib
    dt = dtype_of(prec)
    rng = np.random.default_rng(99)
    with tnn.Context(0) as ctx:
        for call, shape in enumerate(SHAPES):
            Z = inputs.random_tensor(shape, rng)
            Zd = tnn.to_fortran(Z, dtype=dt)
            tau = 0.5 + call
            Yref = tnn.fortran_empty(shape, dt)
            ctx.tsvt(Zd, tau, Y=Yref, prec=prec)
            Y = tnn.fortran_empty(shape, dt)
            Y.fill_(float("nan"))
            st = _static(L, tnn, torch, Zd, shape, tau, prec, Y)
            assert st == tnn.OK, tnn.status_string(st)
            torch.cuda.synchronize()
            a, b = tnn.to_numpy(Y).astype(np.float64), tnn.to_numpy(Yref).astype(np.float64)
            assert np.isfinite(a).all()
            assert np.linalg.norm(a - b) <= TOL[prec] * max(np.linalg.norm(b), 1e-300), call


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_static_call_allocates_nothing(prec):
    torch = torch_cuda()
    from paper_1902_03070_gb300 import tnn
    L = tnn._lib
    dt = dtype_of(prec)
    shape = SHAPES[0]
    rng = np.random.default_rng(5)
    Zs = [tnn.to_fortran(inputs.random_tensor(shape, rng), dtype=dt) for _ in range(2)]
    Y = tnn.fortran_empty(shape, dt)
    # the first call loads the kernels (lazy module loading may take memory)
    assert _static(L, tnn, torch, Zs[0], shape, 0.7, prec, Y) == tnn.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    assert _static(L, tnn, torch, Zs[1], shape, 0.9, prec, Y) == tnn.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == res0


def test_static_reports_nonfinite():
    torch = torch_cuda()
    from paper_1902_03070_gb300 import tnn
    shape = (20, 16, 5)
    Z = inputs.random_tensor(shape, np.random.default_rng(3))
    Z[2, 3, 1] = np.inf
    Zd = tnn.to_fortran(Z, dtype=torch.float32)
    Y = tnn.fortran_empty(shape, torch.float32)
    assert _static(tnn._lib, tnn, torch, Zd, shape, 0.5, "fp32", Y) == tnn.ENONFINITE
    # the next call starts from cleared counters
    Z[2, 3, 1] = 0.0
    Zd = tnn.to_fortran(Z, dtype=torch.float32)
    assert _static(tnn._lib, tnn, torch, Zd, shape, 0.5, "fp32", Y) == tnn.OK


def test_static_rejects_beyond_scratch_and_foreign_pointers():
    torch = torch_cuda()
    from paper_1902_03070_gb300 import tnn
    L = tnn._lib
    big = tnn.fortran_empty((128, 128, 300), torch.float32)   # 19.7 MB > 16 MiB of scratch
    st = L.tsvt_dct_static(big.data_ptr(), tnn.Shape(128, 128, 300), 1.0, tnn.PRECISIONS["fp32"], big.data_ptr(),
                           None)
    assert st == tnn.EINVAL
    # sizes whose byte counts would wrap around size_t are rejected before anything is computed
    for shp in [(4, 4, 1 << 59), (1 << 40, 1 << 40, 1), (3, 1 << 62, 2)]:
        st = L.tsvt_dct_static(big.data_ptr(), tnn.Shape(*shp), 1.0, tnn.PRECISIONS["fp32"], big.data_ptr(), None)
        assert st == tnn.EINVAL, shp
    host = np.zeros((4, 4, 4), order="F")
    st = L.tsvt_dct_static(host.ctypes.data, tnn.Shape(4, 4, 4), 1.0, tnn.PRECISIONS["fp64"], host.ctypes.data, None)
    assert st == tnn.EINVAL
    if torch.cuda.device_count() >= 2:
        other = torch.zeros((4, 4, 4), dtype=torch.float64, device="cuda:1")
        st = L.tsvt_dct_static(other.data_ptr(), tnn.Shape(4, 4, 4), 1.0, tnn.PRECISIONS["fp64"], other.data_ptr(),
                               None)
        assert st == tnn.EINVAL
