"""GPU parity: the DFT comparison path (tsvt_dft, the proximal operator of
tau * TNN-F, Definition 6) against the DFT oracle, and tsvt_dct_plain (the
DCT t-SVT on the same plain Jacobi kernel) against the DCT oracle.

FP64: ||Y - Y_oracle||_F <= 1e-12 ||Y_oracle||_F.  FP32: ||Y - Y_oracle||_F
<= max(1e-5, 2 sqrt(m n) u) ||Z||_F, u = 2^-24 (the bound of the other FP32
t-SVT tests: FP32 rounding of the input, and columns orthogonal to the
rotation threshold sqrt(m) u)."""
import numpy as np
import pytest

import oracle as O
from gpu_common import THREADS, dtype_of, log_err, rel_err, torch_cuda
from oracle import dft as D
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(48, 48, 16), (7, 5, 3), (5, 7, 3), (9, 1, 4), (1, 9, 4), (33, 65, 5), (40, 40, 1), (65, 33, 2),
          (130, 100, 7), (144, 176, 10)]
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with tnn.Context(0) as c:
        yield c


def _tau(Z, q, dft):
    # threshold at quantile q of the singular values of the transformed slices
    if dft:
        Zf = np.fft.fft(Z, axis=2)
        s = np.concatenate([np.linalg.svd(Zf[:, :, k], compute_uv=False) for k in range(Z.shape[2])])
    else:
        Zb = O.tube_transform(Z)
        s = np.concatenate([np.linalg.svd(Zb[:, :, k], compute_uv=False) for k in range(Z.shape[2])])
    return float(np.quantile(s, q))


def _bound(prec, shape, Z):
    if prec == "fp64":
        return None
    m, n = max(shape[:2]), min(shape[:2])
    return max(1e-5, 2.0 * np.sqrt(m * n) * U32) * np.linalg.norm(Z)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("q", [0.3, 0.8])
def test_tsvt_dft_matches_oracle(ctx, prec, shape, q):
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(shape[0] * 31 + shape[1] * 7 + shape[2])
    Z = inputs.random_tensor(shape, rng)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    tau = _tau(Z, q, True)
    Yd = tnn.fortran_empty(shape, dtype_of(prec))
    _, t_gpu = ctx.tsvt_dft(tnn.to_fortran(Z, dtype=dtype_of(prec)), tau, Y=Yd, prec=prec, want_tnn=True)
    Y = tnn.to_numpy(Yd).astype(np.float64)
    ref, t_ref = D.tsvt_dft(Z, tau, return_info=True)
    log_err("dft %s %s q=%s" % (prec, shape, q), err_y=rel_err(Y, ref, Z))
    if prec == "fp64":
        assert rel_err(Y, ref, Z) <= 1e-12
        assert abs(t_gpu - t_ref) <= 1e-12 * max(t_ref, 1e-300)
    else:
        assert np.linalg.norm(Y - ref) <= _bound(prec, shape, Z)
        # TNN-F is sqrt(n)-Lipschitz in Y (Frobenius): |nuc(A) - nuc(B)| <=
        # sqrt(rank) ||A - B||_F per DFT slice, and Parseval sums the slices
        # back to sqrt(n3) ||Y - Y'||_F, which the 1/n3 of Definition 6 offsets
        assert abs(t_gpu - t_ref) <= np.sqrt(min(shape[:2])) * _bound(prec, shape, Z)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_tsvt_dct_plain_matches_oracle(ctx, prec, shape):
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(shape[0] * 13 + shape[1] * 5 + shape[2])
    Z = inputs.random_tensor(shape, rng)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    tau = _tau(Z, 0.5, False)
    Yd = tnn.fortran_empty(shape, dtype_of(prec))
    _, t_gpu = ctx.tsvt_dct_plain(tnn.to_fortran(Z, dtype=dtype_of(prec)), tau, Y=Yd, prec=prec, want_tnn=True)
    Y = tnn.to_numpy(Yd).astype(np.float64)
    ref, t_ref, _ = O.tsvt(Z, tau, nthreads=THREADS, return_info=True)
    if prec == "fp64":
        assert rel_err(Y, ref, Z) <= 1e-12
        assert abs(t_gpu - t_ref) <= 1e-12 * t_ref
    else:
        assert np.linalg.norm(Y - ref) <= _bound(prec, shape, Z)


def test_tsvt_dft_video_shaped(ctx):
    """The 144 x 176 x 100 video-shaped tensor through the DFT path, FP32."""
    from paper_1902_03070_gb300 import tnn
    parts = inputs.config2_parts()
    T = inputs.config2_assemble(O.tprod(parts["A"], parts["F"]), parts)
    Z = T.astype(np.float32).astype(np.float64)
    tau = 0.5
    Yd = tnn.fortran_empty(Z.shape, dtype_of("fp32"))
    ctx.tsvt_dft(tnn.to_fortran(Z, dtype=dtype_of("fp32")), tau, Y=Yd, prec="fp32")
    Y = tnn.to_numpy(Yd).astype(np.float64)
    ref = D.tsvt_dft(Z, tau)
    err = rel_err(Y, ref, Z)
    log_err("dft video fp32", err_y=err)
    assert err <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tsvt_dft_special_cases(ctx, prec):
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(9)
    Z = inputs.random_tensor((12, 10, 6), rng)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    tol = 1e-13 if prec == "fp64" else 2e-6
    Zd = tnn.to_fortran(Z, dtype=dtype_of(prec))
    Y = tnn.to_numpy(ctx.tsvt_dft(Zd, 0.0, Y=tnn.fortran_empty(Z.shape, dtype_of(prec)), prec=prec))
    assert np.linalg.norm(Y - Z) <= tol * np.linalg.norm(Z)     # tau = 0: Y = Z
    big = 10 * np.abs(np.fft.fft(Z, axis=2)).sum()
    Y = tnn.to_numpy(ctx.tsvt_dft(Zd, big, Y=tnn.fortran_empty(Z.shape, dtype_of(prec)), prec=prec))
    assert not Y.any()                                          # above every singular value: zero
    ctx.tsvt_dft(Zd, 0.7, prec=prec)                            # in place
    ref = D.tsvt_dft(Z, 0.7)
    assert rel_err(tnn.to_numpy(Zd), ref, Z) <= (1e-12 if prec == "fp64" else 1e-5)
    with pytest.raises(tnn.TnnError):
        ctx.tsvt_dft(np.asfortranarray(Z.astype(np.float64 if prec == "fp64" else np.float32)), 0.5, prec=prec)


@pytest.mark.parametrize("n3", [1, 2, 3, 4])
def test_tsvt_dft_short_tubes(ctx, n3):
    # n3 = 1 is the matrix SVT; n3 = 2 has a real Nyquist slice
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(40 + n3)
    Z = inputs.random_tensor((9, 7, n3), rng)
    Yd = tnn.fortran_empty(Z.shape, dtype_of("fp64"))
    ctx.tsvt_dft(tnn.to_fortran(Z), 0.8, Y=Yd, prec="fp64")
    assert rel_err(tnn.to_numpy(Yd), D.tsvt_dft(Z, 0.8), Z) <= 1e-12
