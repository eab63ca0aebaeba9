"""GPU parity: t-SVT (Theorem 5, Algorithm 1) through the C ABI against the
FP64 oracle.

FP64 path: ||Y - Y_oracle||_F <= 1e-12 ||Y_oracle||_F (||Z||_F when the
oracle's Y is below 1e-6 ||Z||_F).

FP32 forms (CUDA-core, 3xTF32 and BF16-split transforms; FP32 Jacobi):
||Y - Y_oracle||_F <= 1e-5 ||Y_oracle||_F and <= 1e-5 ||Z||_F on every case
held by one CTA, the Gaussian stress cases with tau at the 80th-percentile
singular value (||Y|| about 0.13 ||Z||) included.  Gaussian slices spread
over thread-block clusters (several hundred rows and columns, dense spectra)
are held to 2 sqrt(m n) u ||Z|| (u = 2^-24): one-sided Jacobi leaves each
column pair orthogonal only to its threshold sqrt(m) u, and on such spectra
the rebuilt slice carries an error of that order."""
import numpy as np
import pytest
import scipy.fft

import oracle as O
from gpu_common import THREADS, dtype_of, log_err, rel_err, tau_at_quantile, torch_cuda
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "tf32x3": 1e-5,
       # three-part BF16 transforms: FP32 accuracy (the Jacobi stage is FP32
       # as in the other FP32 forms)
       "bf16split": 1e-5}

SHAPES = [
    (48, 48, 16),    # the 48 x 48 x 16 completion workload
    (7, 5, 3), (5, 7, 3),          # tall / wide (transposed orientation)
    (1, 9, 4), (9, 1, 4),          # single row / column
    (33, 65, 5), (65, 33, 2),      # ragged tails over several column blocks
    (130, 100, 3),                 # more rows than 4 x 32
    (40, 40, 1),                   # one slice: the matrix SVT
]


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with tnn.Context(0) as c:
        yield c


def _run(ctx, Z, tau, prec, want_tnn=False):
    from paper_1902_03070_gb300 import tnn
    Zd = tnn.to_fortran(Z, dtype=dtype_of(prec))
    Yd = tnn.fortran_empty(Z.shape, dtype_of(prec))
    out = ctx.tsvt(Zd, tau, Y=Yd, prec=prec, want_tnn=want_tnn)
    if want_tnn:
        return tnn.to_numpy(out[0]).astype(np.float64), out[1]
    return tnn.to_numpy(out).astype(np.float64)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16split"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("q", [0.3, 0.8])
def test_tsvt_matches_oracle(ctx, prec, shape, q):
    rng = np.random.default_rng(shape[0] * 1000 + shape[1] * 10 + shape[2])
    Z = inputs.random_tensor(shape, rng)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    tau = tau_at_quantile(Z, q)
    Y = _run(ctx, Z, tau, prec)
    ref = O.tsvt(Z, tau, nthreads=THREADS)
    err_y = rel_err(Y, ref, Z)
    log_err("tsvt %s %s q=%s" % (prec, shape, q), err_y=err_y, err_z=np.linalg.norm(Y - ref) / np.linalg.norm(Z))
    if prec == "fp64":
        assert err_y <= TOL["fp64"]
    else:
        err_z = np.linalg.norm(Y - ref) / np.linalg.norm(Z)
        assert err_z <= TOL[prec], (err_z, err_y)
        assert err_y <= TOL[prec], (err_z, err_y)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16split"])
def test_tsvt_low_rank_plus_noise(ctx, prec):
    # a 48 x 48 x 16 tubal-rank-3 tensor plus noise, threshold above the noise edge
    rng = np.random.default_rng(7)
    A, F = inputs.lowrank_factors(48, 48, 16, 3, rng)
    Z = O.tprod(A, F) + 1e-3 * rng.standard_normal((48, 48, 16))
    Z = np.asfortranarray(Z)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    tau = 0.05
    Y, tnn_gpu = _run(ctx, Z, tau, prec, want_tnn=True)
    ref, tnn_ref, _ = O.tsvt(Z, tau, nthreads=THREADS, return_info=True)
    log_err("tsvt lowrank %s" % prec, err_y=rel_err(Y, ref, Z))
    assert rel_err(Y, ref, Z) <= TOL[prec]
    assert abs(tnn_gpu - tnn_ref) <= (1e-12 if prec == "fp64" else 1e-5) * tnn_ref


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16split"])
def test_tsvt_video_shaped(ctx, prec):
    """The 144 x 176 x 100 video-shaped tensor at full size."""
    parts = inputs.config2_parts()
    T = inputs.config2_assemble(O.tprod(parts["A"], parts["F"]), parts)
    Z = T.astype(np.float32).astype(np.float64)
    for q in (0.5, 0.95):
        tau = tau_at_quantile(Z, q)
        Y = _run(ctx, Z, tau, prec)
        ref = O.tsvt(Z, tau, nthreads=THREADS)
        log_err("tsvt video %s q=%s" % (prec, q), err_y=rel_err(Y, ref, Z),
                ynorm_over_z=np.linalg.norm(ref) / np.linalg.norm(Z))
        assert rel_err(Y, ref, Z) <= TOL[prec], q


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16split"])
def test_tsvt_special_cases(ctx, prec):
    rng = np.random.default_rng(11)
    Z = inputs.random_tensor((20, 12, 6), rng)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    tol = {"fp64": 1e-13}.get(prec, 2e-6)
    # tau = 0: Y = Z
    Y = _run(ctx, Z, 0.0, prec)
    assert np.linalg.norm(Y - Z) <= tol * np.linalg.norm(Z)
    # tau above every singular value: Y = 0 exactly
    Zb = scipy.fft.dct(Z, type=2, norm="ortho", axis=2)
    smax = max(np.linalg.svd(Zb[:, :, k], compute_uv=False)[0] for k in range(6))
    Y = _run(ctx, Z, smax * 1.01, prec)
    assert not Y.any()
    # zero input: zero output
    Y = _run(ctx, np.zeros((9, 8, 3), order="F"), 0.1, prec)
    assert not Y.any()


def test_tsvt_in_place_and_host_buffers(ctx):
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(13)
    Z = inputs.random_tensor((30, 20, 7), rng)
    tau = tau_at_quantile(Z, 0.5)
    ref = O.tsvt(Z, tau)
    Zd = tnn.to_fortran(Z, dtype=dtype_of("fp64"))
    ctx.tsvt(Zd, tau, prec="fp64")           # Y is Z: in place
    assert rel_err(tnn.to_numpy(Zd), ref) <= 1e-12
    Zh = np.asfortranarray(Z.copy())
    Yh = np.zeros_like(Zh, order="F")
    ctx.tsvt(Zh, tau, Y=Yh, prec="fp64")     # host pointers, staged by the library
    assert rel_err(Yh, ref) <= 1e-12


def test_tsvt_invalid_arguments(ctx):
    from paper_1902_03070_gb300 import tnn
    Zd = tnn.fortran_empty((4, 4, 4), dtype_of("fp64"))
    with pytest.raises(tnn.TnnError) as e:
        ctx.tsvt(Zd, -1.0, prec="fp64")
    assert e.value.status == tnn.EINVAL
    with pytest.raises(tnn.TnnError) as e:
        ctx.tsvt(tnn.fortran_empty((600, 600, 1), dtype_of("fp32")), 1.0, prec="fp32")
    assert e.value.status == tnn.EINVAL


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16split"])
def test_tsvt_msi_shaped(ctx, prec):
    """The 512 x 512 x 31 multispectral-shaped tensor at full size (slices too
    large for one CTA's shared memory: each is spread over a cluster of 8)."""
    d = inputs.config3()
    Z = d["T"].astype(np.float32).astype(np.float64)
    for q in (0.9, 0.99):
        tau = tau_at_quantile(Z, q)
        Y = _run(ctx, Z, tau, prec)
        ref = O.tsvt(Z, tau, nthreads=THREADS)
        err = rel_err(Y, ref, Z)
        log_err("tsvt msi %s q=%s" % (prec, q), err_y=err, ynorm_over_z=np.linalg.norm(ref) / np.linalg.norm(Z))
        assert err <= TOL[prec], (q, err)


# slices larger than one CTA's shared memory: spread over clusters of 2, 4
# or 8 CTAs (tall, wide and ragged column counts).  Gaussian slices this
# large have dense spectra, and FP32 one-sided Jacobi leaves the columns
# orthogonal only to the rotation threshold sqrt(m) u (u = 2^-24) each, so
# the rebuilt slice carries an error of order sqrt(m n) u ||Z||: the FP32
# bound here is 2 sqrt(m n) u ||Z||_F.
U32 = 2.0 ** -24
CLUSTER_SHAPES = [("fp32", (300, 280, 3)), ("fp32", (150, 400, 2)), ("fp32", (512, 512, 2)),
                  ("fp32", (260, 250, 4)), ("fp64", (200, 150, 3)), ("fp64", (140, 250, 2)),
                  ("fp64", (400, 300, 2)), ("fp64", (512, 512, 2))]


@pytest.mark.parametrize("prec,shape", CLUSTER_SHAPES)
@pytest.mark.parametrize("q", [0.3, 0.8])
def test_tsvt_cluster_slices(ctx, prec, shape, q):
    rng = np.random.default_rng(shape[0] * 7 + shape[1] * 3 + shape[2])
    Z = inputs.random_tensor(shape, rng)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    tau = tau_at_quantile(Z, q)
    Y = _run(ctx, Z, tau, prec)
    st = ctx.last_jacobi_stats()
    assert st["unconverged"] == 0
    ref = O.tsvt(Z, tau, nthreads=THREADS)
    err_y = rel_err(Y, ref, Z)
    err_z = np.linalg.norm(Y - ref) / np.linalg.norm(Z)
    log_err("tsvt cluster %s %s q=%s" % (prec, shape, q), err_y=err_y, err_z=err_z)
    if prec == "fp64":
        assert err_y <= TOL["fp64"]
    else:
        m, n = max(shape[:2]), min(shape[:2])
        assert err_z <= 2.0 * np.sqrt(m * n) * U32, (err_z, err_y)
        if q <= 0.5:  # tau keeps most of the energy: within 1e-5 of Y as everywhere else
            assert err_y <= TOL[prec], (err_z, err_y)


@pytest.mark.parametrize("C", ["2", "4", "8"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tsvt_forced_cluster(ctx, monkeypatch, prec, C):
    # slices that fit one CTA, spread over a cluster anyway (a different but
    # equally cyclic pair ordering): same bounds against the oracle, and the
    # nuclear norm of the result agrees with the single-CTA kernel's
    rng = np.random.default_rng(21)
    shape = (176, 128, 6) if prec == "fp32" else (190, 64, 4)
    Z = inputs.random_tensor(shape, rng)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    tau = tau_at_quantile(Z, 0.5)
    Y1, t1 = _run(ctx, Z, tau, prec, want_tnn=True)
    monkeypatch.setenv("TNN_JACOBI_CLUSTER", C)
    Y2, t2 = _run(ctx, Z, tau, prec, want_tnn=True)
    assert ctx.last_jacobi_stats()["unconverged"] == 0
    monkeypatch.delenv("TNN_JACOBI_CLUSTER")
    ref = O.tsvt(Z, tau, nthreads=THREADS)
    if prec == "fp64":
        assert rel_err(Y2, ref, Z) <= TOL["fp64"]
        assert rel_err(Y1, ref, Z) <= TOL["fp64"]
    else:
        bound = 2.0 * np.sqrt(shape[0] * shape[1]) * U32 * np.linalg.norm(Z)
        assert np.linalg.norm(Y2 - ref) <= bound
        assert np.linalg.norm(Y1 - ref) <= bound
    assert abs(t1 - t2) <= (1e-12 if prec == "fp64" else 1e-5) * abs(t1)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tsvt_random_shape_sweep(ctx, prec):
    """Seeded random shapes across the variant, shared-memory, global-memory
    and cluster boundaries (m up to 512, either orientation, n3 up to 6),
    each against the oracle."""
    rng = np.random.default_rng(2026 if prec == "fp64" else 2027)
    for _ in range(14):
        n1 = int(rng.integers(1, 513))
        n2 = int(rng.integers(1, 513))
        n3 = int(rng.integers(1, 7))
        if n1 * n2 * n3 > 600_000:
            n3 = max(1, 600_000 // (n1 * n2))
        shape = (n1, n2, n3)
        Z = inputs.random_tensor(shape, rng)
        if prec != "fp64":
            Z = Z.astype(np.float32).astype(np.float64)
        tau = tau_at_quantile(Z, float(rng.uniform(0.1, 0.9)))
        Y = _run(ctx, Z, tau, prec)
        ref = O.tsvt(Z, tau, nthreads=THREADS)
        if prec == "fp64":
            assert rel_err(Y, ref, Z) <= TOL["fp64"], shape
        else:
            m, n = max(n1, n2), min(n1, n2)
            bound = max(1e-5, 2.0 * np.sqrt(m * n) * U32) * np.linalg.norm(Z)
            assert np.linalg.norm(Y - ref) <= bound, shape


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(120, 96, 2), (80, 130, 2)])
@pytest.mark.parametrize("f", [0.3, 0.8, 0.95, 1.2, 2.0])
def test_tsvt_dominant_plus_small_tail(ctx, prec, shape, f):
    # Each transformed slice is one singular value of 10 tau plus a Gaussian
    # tail of Frobenius norm f tau: the shape of the DC slice in the early
    # completion iterations.  Below f = 0.9 the tail's columns can be left
    # unrotated among themselves (their block's SVT is zero); around and above
    # it the kernel must fall back to full sweeps.  Either way the result is
    # the SVT.
    n1, n2, n3 = shape
    rng = np.random.default_rng(int(f * 100) + n1)
    tau = 0.7
    Zb = np.zeros(shape)
    for k in range(n3):
        u = rng.standard_normal(n1)
        v = rng.standard_normal(n2)
        N = rng.standard_normal((n1, n2))
        Zb[:, :, k] = 10 * tau * np.outer(u / np.linalg.norm(u), v / np.linalg.norm(v)) + f * tau * N / np.linalg.norm(N)
    Z = O.tube_transform(Zb, inverse=True)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    Y = _run(ctx, Z, tau, prec)
    ref = O.tsvt(Z, tau, nthreads=THREADS)
    err_y = rel_err(Y, ref, Z)
    err_z = np.linalg.norm(Y - ref) / np.linalg.norm(Z)
    log_err("tsvt tail %s %s f=%s" % (prec, shape, f), err_y=err_y, err_z=err_z)
    if prec == "fp64":
        assert err_y <= TOL["fp64"], err_y
    else:
        assert err_z <= TOL["fp32"], (err_z, err_y)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(176, 144, 2), (60, 90, 3)])
@pytest.mark.parametrize("s1", [0.3, 0.7, 0.97, 1.03, 1.3])
def test_tsvt_top_singular_value_near_tau(ctx, prec, shape, s1):
    # Transformed slices with Frobenius norm above tau (so the slice is not
    # skipped) and largest singular value s1 tau spread over all columns:
    # below tau the SVT is zero (the kernel may stop early on a Gershgorin
    # bound); just above it, that bound must not fire.
    n1, n2, n3 = shape
    rng = np.random.default_rng(int(s1 * 1000) + n1 + n3)
    tau = 0.5
    r = min(n1, n2)
    Zb = np.zeros(shape)
    for k in range(n3):
        U, _ = np.linalg.qr(rng.standard_normal((n1, r)))
        V, _ = np.linalg.qr(rng.standard_normal((n2, r)))
        sig = s1 * tau * np.linspace(1.0, 0.2, r)  # ||.||_F well above tau
        Zb[:, :, k] = (U * sig) @ V.T
    Z = O.tube_transform(Zb, inverse=True)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    Y = _run(ctx, Z, tau, prec)
    ref = O.tsvt(Z, tau, nthreads=THREADS)
    err_z = np.linalg.norm(Y - ref) / np.linalg.norm(Z)
    log_err("tsvt near-tau %s %s s1=%s" % (prec, shape, s1), err_z=err_z)
    if s1 < 1.0:
        assert np.count_nonzero(ref) == 0 or np.abs(ref).max() == 0.0
        assert np.abs(Y).max() == 0.0
    assert err_z <= (TOL["fp64"] if prec == "fp64" else TOL["fp32"]), err_z


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
@pytest.mark.parametrize("shape", [(48, 48, 16), (130, 100, 3), (33, 65, 5)])
def test_tsvt_fp64_angles(ctx, prec, shape):
    """TNN_OPT_JACOBI_FP64_ANGLES: the FP32 Jacobi with its rotation angles
    and convergence tests in FP64 meets the same gates as the FP32 form on the
    hardest cases of the suite (Gaussian slices, tau at the 80th-percentile
    singular value, ||Y|| about 0.13 ||Z||); both errors are logged, for the
    comparison of the two forms."""
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(shape[0] * 1000 + shape[1] * 10 + shape[2])
    Z = inputs.random_tensor(shape, rng).astype(np.float32).astype(np.float64)
    tau = tau_at_quantile(Z, 0.8)
    ref = O.tsvt(Z, tau, nthreads=THREADS)
    errs = {}
    try:
        for a64 in (0, 1):
            ctx.set_option(tnn.OPT_JACOBI_FP64_ANGLES, a64)
            Y = _run(ctx, Z, tau, prec)
            errs[a64] = (rel_err(Y, ref, Z), np.linalg.norm(Y - ref) / np.linalg.norm(Z))
    finally:
        ctx.set_option(tnn.OPT_JACOBI_FP64_ANGLES, 0)
    log_err("tsvt angles %s %s q=0.8" % (prec, shape), err_y_fp32_angles=errs[0][0], err_y_fp64_angles=errs[1][0],
            err_z_fp32_angles=errs[0][1], err_z_fp64_angles=errs[1][1])
    for a64 in (0, 1):
        assert errs[a64][1] <= TOL[prec], errs
        assert errs[a64][0] <= TOL[prec], errs


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_slice_stats_match_totals(ctx, prec):
    # the per-slice statistics add up to the launch totals, and each slice's
    # kept count is the oracle's count of singular values above tau
    rng = np.random.default_rng(5)
    shape = (60, 44, 7)
    Z = inputs.random_tensor(shape, rng)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    tau = tau_at_quantile(Z, 0.6)
    _run(ctx, Z, tau, prec)
    tot = ctx.last_jacobi_stats()
    per = ctx.last_slice_stats()
    assert len(per["sweeps"]) == shape[2]
    assert max(per["sweeps"]) == tot["max_sweeps"]
    assert sum(per["kept"]) == tot["kept"]
    assert sum(per["rotations"]) == tot["rotations"]
    Zbar = O.tube_transform(Z)
    for k in range(shape[2]):
        s = np.linalg.svd(Zbar[:, :, k], compute_uv=False)
        # a singular value within rounding of tau may fall either way
        sure = int((s > tau * (1 + 1e-5)).sum())
        maybe = int((s > tau * (1 - 1e-5)).sum())
        assert sure <= per["kept"][k] <= maybe


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("q", [0.3, 0.8])
def test_small_rotation_stop(ctx, prec, q):
    # the small-rotation stop (default on) against the plain stopping rule:
    # never more sweeps, and both within the same bounds of the oracle
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(31)
    shape = (120, 90, 5)
    Z = inputs.random_tensor(shape, rng)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    tau = tau_at_quantile(Z, q)
    ref = O.tsvt(Z, tau, nthreads=THREADS)
    out = {}
    try:
        for flag in (1, 0):
            ctx.set_option(tnn.OPT_JACOBI_SMALL_STOP, flag)
            Y = _run(ctx, Z, tau, prec)
            st = ctx.last_jacobi_stats()
            assert st["unconverged"] == 0
            out[flag] = (Y, sum(ctx.last_slice_stats()["sweeps"]))
    finally:
        ctx.set_option(tnn.OPT_JACOBI_SMALL_STOP, 1)
    assert out[1][1] <= out[0][1]
    for flag in (1, 0):
        err_y = rel_err(out[flag][0], ref, Z)
        log_err("tsvt small-stop=%d %s q=%s sweeps=%d" % (flag, prec, q, out[flag][1]), err_y=err_y)
        assert err_y <= TOL[prec]


def test_sweep_log(ctx):
    # the per-sweep log: one row per sweep run, and the last row of every
    # slice meets a stopping rule (no big rotation, or no wide one)
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(41)
    shape = (96, 72, 6)
    Z = inputs.random_tensor(shape, rng).astype(np.float32).astype(np.float64)
    tau = tau_at_quantile(Z, 0.3)
    try:
        ctx.set_option(tnn.OPT_JACOBI_SWEEP_LOG, 1)
        _run(ctx, Z, tau, "fp32")
        log = ctx.last_sweep_log()
    finally:
        ctx.set_option(tnn.OPT_JACOBI_SWEEP_LOG, 0)
    sweeps = ctx.last_slice_stats()["sweeps"]
    assert log.shape == (shape[2], 9, 8)
    for k in range(shape[2]):
        s = sweeps[k]
        assert 1 <= s <= 8
        last = log[k, s - 1]
        assert last[0] == 0 or last[1] == 0
        assert np.all(log[k, s:8] == 0)
        assert log[k, 0, 0] > 0  # a random slice is not orthogonal to begin with
        assert np.all(np.isfinite(log[k])) and np.all(log[k] >= 0)
        assert np.all(log[k, :s, 6] > 0)  # every sweep took time
        ph = log[k, 8]
        # (the parts are rounded to float one by one)
        assert ph[3] >= 0.999 * (ph[0] + ph[1] + ph[2]) > 0
        assert ph[1] >= 0.999 * (log[k, :s, 6].sum() + log[k, :s, 7].sum())
    _run(ctx, Z, tau, "fp32")
    with pytest.raises(tnn.TnnError):
        ctx.last_sweep_log()  # the launch after the option was cleared kept none
