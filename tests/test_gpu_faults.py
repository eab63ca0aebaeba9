"""Failure detection on the GPU without a GPU fault.

Each failure is made on purpose from the host side and must come back as a
status, with the context still usable afterwards:
  - a NaN in Z: the per-slice Jacobi SVT meets a non-finite singular value
    and tsvt_dct returns TNN_ENONFINITE;
  - a sweep cap of 1 (TNN_OPT_JACOBI_MAX_SWEEPS) on dense Gaussian slices:
    tsvt_dct returns TNN_ENOCONV and still writes Y (the shrinkage and rebuild
    of the columns as they are);
  - a poll limit of 0 for the tensor-core transforms' mbarrier waits
    (TNN_OPT_TC_WAIT_POLLS): every wait gives up at once, the kernels record
    the timeout, let their own copies in flight land (waiting with the default
    bound) and return, and tsvt_dct returns TNN_ECUDA.
Nothing here traps, faults or hangs the GPU: the timeout path waits for its
in-flight copies with the normal bound before the kernel exits."""
import ctypes

import numpy as np
import pytest

import oracle as O
from gpu_common import dtype_of, rel_err, tau_at_quantile, torch_cuda
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with tnn.Context(0) as c:
        yield c


def _raw_tsvt(ctx, Zd, Yd, tau, prec):
    """tsvt_dct through the C ABI with a tnn_out, so the call reports the
    Jacobi and transform status; returns (status, tnn_out)."""
    from paper_1902_03070_gb300 import tnn
    torch = torch_cuda()
    out = ctypes.c_double(0.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = tnn._lib.tsvt_dct(ctx._h, Zd.data_ptr(), tnn.Shape(*Zd.shape), float(tau), tnn.PRECISIONS[prec],
                           Yd.data_ptr(), ctypes.byref(out), stream)
    return st, out.value


def _parity_after(ctx, prec, seed):
    """A clean t-SVT on the same context still matches the oracle."""
    from paper_1902_03070_gb300 import tnn
    Z = inputs.random_tensor((24, 20, 6), np.random.default_rng(seed))
    tau = tau_at_quantile(Z, 0.4)
    Zd = tnn.to_fortran(Z, dtype=dtype_of(prec))
    Yd = tnn.fortran_empty(Z.shape, dtype_of(prec))
    st, _ = _raw_tsvt(ctx, Zd, Yd, tau, prec)
    assert st == tnn.OK, tnn.status_string(st)
    ref = O.tsvt(Z, tau)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert rel_err(tnn.to_numpy(Yd), ref, Z) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16split"])
def test_nan_input_reports_nonfinite(ctx, prec):
    from paper_1902_03070_gb300 import tnn
    Z = inputs.random_tensor((20, 16, 5), np.random.default_rng(7))
    Z[3, 4, 2] = np.nan
    Zd = tnn.to_fortran(Z, dtype=dtype_of(prec))
    Yd = tnn.fortran_empty(Z.shape, dtype_of(prec))
    st, _ = _raw_tsvt(ctx, Zd, Yd, 0.5, prec)
    assert st == tnn.ENONFINITE, tnn.status_string(st)
    assert "non-finite" in ctx.last_error()
    _parity_after(ctx, prec, 8)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_sweep_cap_reports_noconv_and_writes_y(ctx, prec):
    from paper_1902_03070_gb300 import tnn
    torch = torch_cuda()
    Z = inputs.random_tensor((48, 40, 4), np.random.default_rng(9))
    tau = tau_at_quantile(Z, 0.3)
    Zd = tnn.to_fortran(Z, dtype=dtype_of(prec))
    Yd = tnn.fortran_empty(Z.shape, dtype_of(prec))
    Yd.fill_(float("nan"))
    try:
        ctx.set_option(tnn.OPT_JACOBI_MAX_SWEEPS, 1)
        st, _ = _raw_tsvt(ctx, Zd, Yd, tau, prec)
        assert st == tnn.ENOCONV, tnn.status_string(st)
        assert "sweep cap" in ctx.last_error()
        torch.cuda.synchronize()
        y = tnn.to_numpy(Yd).astype(np.float64)
        assert np.isfinite(y).all()
        # one sweep leaves the columns far from orthogonal: Y is written but
        # is not the t-SVT yet
        ref = O.tsvt(Z, tau)
        assert 1e-4 < rel_err(y, ref, Z) < 1.0
        stats = ctx.last_jacobi_stats()
        assert stats["max_sweeps"] == 1 and stats["unconverged"] > 0
    finally:
        ctx.set_option(tnn.OPT_JACOBI_MAX_SWEEPS, 0)
    _parity_after(ctx, prec, 10)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16split"])
def test_tensor_core_wait_timeout_reports_error(ctx, prec):
    from paper_1902_03070_gb300 import tnn
    torch = torch_cuda()
    Z = inputs.random_tensor((32, 36, 40), np.random.default_rng(11))
    Zd = tnn.to_fortran(Z, dtype=torch.float32)
    Yd = tnn.fortran_empty(Z.shape, torch.float32)
    try:
        ctx.set_option(tnn.OPT_TC_WAIT_POLLS, 0)
        st, _ = _raw_tsvt(ctx, Zd, Yd, 0.5, prec)
        assert st == tnn.ECUDA, tnn.status_string(st)
        assert "timed out" in ctx.last_error()
    finally:
        ctx.set_option(tnn.OPT_TC_WAIT_POLLS, -1)
    # the flag was cleared by the call that reported it, and the device is fine
    assert torch.cuda.current_stream().query() in (True, False)
    torch.cuda.synchronize()
    _parity_after(ctx, prec, 12)


def test_options_reject_out_of_range(ctx):
    from paper_1902_03070_gb300 import tnn
    for opt, val in ((tnn.OPT_JACOBI_MAX_SWEEPS, -1), (tnn.OPT_JACOBI_MAX_SWEEPS, 1001),
                     (tnn.OPT_TC_WAIT_POLLS, 1 << 31), (tnn.OPT_JACOBI_SMALL_STOP, 2), (99, 0)):
        assert tnn._lib.tnn_set_option(ctx._h, opt, val) == tnn.EINVAL
