"""GPU test of the FMA-pipe microbenchmark (tnn_fma_peak), the roofline
denominator of the Jacobi kernels: plausible rates for each pipe, the packed
form at least as fast as the scalar one, invalid kinds refused."""
import pytest

from gpu_common import torch_cuda

pytestmark = pytest.mark.gpu


def test_fma_peaks():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    f32 = tnn.fma_peak("fp32")
    f32x2 = tnn.fma_peak("fp32x2")
    f64 = tnn.fma_peak("fp64")
    # 152 SMs x 128 FP32 lanes x 2 flop at 2.07 GHz is 80.5 TFLOP/s; allow clocks well below the maximum
    assert 20e12 < f32 < 200e12, f32
    assert f32x2 > 0.8 * f32, (f32, f32x2)
    assert 0.1e12 < f64 < f32, f64


def test_fma_peak_rejects_unknown_kind():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    import ctypes
    out = ctypes.c_double(0.0)
    assert tnn._lib.tnn_fma_peak(0, 3, ctypes.byref(out)) == tnn.EINVAL
    assert tnn._lib.tnn_fma_peak(0, 0, None) == tnn.EINVAL
