"""GPU parity: Algorithm 1 (ADMM, Eq. 17) through the C ABI.
FP64: iterates match the oracle's, the invariants X_Omega = B_Omega and
M_{Omega^c} = 0 hold bit-exactly, a run split over several calls equals one
call bit-for-bit, and the 48 x 48 x 16 completion ends within 1e-4 of the
oracle's final error."""
import numpy as np
import pytest

import oracle as O
from gpu_common import THREADS, dtype_of, log_err, torch_cuda
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with tnn.Context(0) as c:
        yield c


def _small(seed=1, shape=(20, 18, 6), r=2, frac=0.5):
    rng = np.random.default_rng(seed)
    A, F = inputs.lowrank_factors(shape[0], shape[1], shape[2], r, rng)
    T = O.tprod(A, F)
    mask = inputs.uniform_mask(T.shape, frac, np.random.default_rng(seed + 1))
    return T, inputs.fortran(T * mask), mask


@pytest.mark.parametrize("iters", [1, 4, 12])
def test_admm_iterates_match_oracle_fp64(ctx, iters):
    from paper_1902_03070_gb300 import tnn
    T, B, mask = _small()
    prm = dict(beta0=0.05, rho=1.3, beta_max=1e6, tol=-1.0, max_iter=iters)
    Xo, Mo, rep_o = O.admm(B, mask, **prm)
    dt = dtype_of("fp64")
    Bd, md = tnn.to_fortran(B, dtype=dt), tnn.to_fortran(mask)
    Xd = tnn.fortran_empty(B.shape, dt)
    st, rep = ctx.complete(Bd, md, Xd, ctx.params(**prm), prec="fp64")
    assert rep["iters"] == iters == rep_o["iters"]
    X = tnn.to_numpy(Xd)
    assert np.linalg.norm(X - Xo) <= 1e-12 * np.linalg.norm(Xo)
    assert abs(rep["beta_final"] - rep_o["beta_final"]) <= 1e-15 * rep_o["beta_final"]
    m = mask.astype(bool)
    assert np.array_equal(X[m], B[m])


def test_admm_invariants_and_resume_bit_exact(ctx):
    from paper_1902_03070_gb300 import tnn
    torch = torch_cuda()
    T, B, mask = _small(seed=5)
    dt = dtype_of("fp64")
    prm = ctx.params(beta0=0.05, rho=1.2, beta_max=1e6, tol=-1.0, max_iter=100)
    Bd, md = tnn.to_fortran(B, dtype=dt), tnn.to_fortran(mask)

    def state():
        X = tnn.to_fortran(B * mask, dtype=dt)
        M = tnn.to_fortran(np.zeros(B.shape), dtype=dt)
        return X, M

    X1, M1 = state()
    b1, _ = ctx.admm_iterate(Bd, md, X1, M1, 0.05, 7, prm, prec="fp64")
    X2, M2 = state()
    b2, _ = ctx.admm_iterate(Bd, md, X2, M2, 0.05, 3, prm, prec="fp64")
    b2, _ = ctx.admm_iterate(Bd, md, X2, M2, b2, 4, prm, prec="fp64")
    assert b1 == b2
    assert torch.equal(X1, X2) and torch.equal(M1, M2)
    m = torch.from_numpy(mask.astype(bool).transpose(2, 1, 0).copy()).cuda().permute(2, 1, 0)
    assert torch.equal(X1[m], Bd[m])
    assert not M1[~m].any()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16split"])
def test_completion_48x48x16(ctx, prec):
    """Tubal rank 3, 40% observed, beta0 1e-4, rho 1.1, tol 1e-8, <= 300
    iterations.  This workload recovers the tensor to about 2e-8 in FP64;
    every FP32 form (the three-part BF16 split included) ends within 1e-4 of
    the oracle's final error."""
    from paper_1902_03070_gb300 import tnn
    d = inputs.config1(O.tprod)
    T, B, mask, prm = d["T"], d["B"], d["mask"], d["admm"]
    Xo, _, rep_o = O.admm(B, mask, nthreads=THREADS, **prm)
    err_o = np.linalg.norm(Xo - T) / np.linalg.norm(T)
    dt = dtype_of(prec)
    Xd = tnn.fortran_empty(B.shape, dt)
    st, rep = ctx.complete(tnn.to_fortran(B, dtype=dt), tnn.to_fortran(mask), Xd, ctx.params(**prm), prec=prec)
    err = np.linalg.norm(tnn.to_numpy(Xd) - T) / np.linalg.norm(T)
    assert abs(err - err_o) <= 1e-4, (err, err_o, rep, rep_o)
    if prec == "fp64":
        assert rep["iters"] == rep_o["iters"]
        assert np.linalg.norm(tnn.to_numpy(Xd) - Xo) <= 1e-9 * np.linalg.norm(Xo)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16split"])
def test_completion_video_shaped_matches_oracle_final_error(ctx, prec):
    """144 x 176 x 100 video-shaped completion, 20% observed, 200 iterations:
    the final relative error against the ground truth is within 1e-4 of the
    FP64 oracle's (stored by tests/golden/make_admm_golden.py, which calls
    only the oracle)."""
    import json
    import os
    from paper_1902_03070_gb300 import tnn
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "admm_video_144x176x100.json")
    gold = json.load(open(path))
    d = inputs.config2(O.tprod)
    T, B, mask, prm = d["T"], d["B"], d["mask"], d["admm"]
    dt = dtype_of(prec)
    Xd = tnn.fortran_empty(B.shape, dt)
    st, rep = ctx.complete(tnn.to_fortran(B, dtype=dt), tnn.to_fortran(mask), Xd, ctx.params(**prm), prec=prec)
    err = np.linalg.norm(tnn.to_numpy(Xd) - T) / np.linalg.norm(T)
    if prec == "fp64":
        assert rep["iters"] == gold["iters"]
    assert abs(err - gold["rel_err_vs_ground_truth"]) <= 1e-4, (err, gold)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16split"])
def test_completion_msi_window_matches_oracle_final_error(ctx, prec):
    """A 128 x 128 x 31 window of the multispectral-shaped workload (10%
    observed, 150 iterations): the final relative error against the ground
    truth is within 1e-4 of the FP64 oracle's (tests/golden/make_admm_golden.py)."""
    import json
    import os
    from paper_1902_03070_gb300 import tnn
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "admm_msi_128x128x31.json")
    gold = json.load(open(path))
    d = inputs.config3(n1=128, n2=128)
    T, B, mask, prm = d["T"], d["B"], d["mask"], d["admm"]
    dt = dtype_of(prec)
    Xd = tnn.fortran_empty(B.shape, dt)
    st, rep = ctx.complete(tnn.to_fortran(B, dtype=dt), tnn.to_fortran(mask), Xd, ctx.params(**prm), prec=prec)
    err = np.linalg.norm(tnn.to_numpy(Xd) - T) / np.linalg.norm(T)
    log_err("admm msi window %s" % prec, err=err, oracle=gold["rel_err_vs_ground_truth"])
    assert abs(err - gold["rel_err_vs_ground_truth"]) <= 1e-4, (err, gold)



@pytest.mark.parametrize("prec", ["tf32x3", "bf16split"])
def test_completion_msi_full_size_matches_oracle(ctx, prec):
    """The full 512 x 512 x 31 multispectral-shaped completion (10% observed,
    150 iterations; the oracle's run, stored by tests/golden/make_admm_golden.py
    msi512, took 46 minutes on 8 host cores): the final relative error against
    the ground truth is within 1e-4 of the oracle's, and the oracle's final X
    at 512 seeded positions is matched to 1e-3 of the RMS entry."""
    import json
    import os
    from paper_1902_03070_gb300 import tnn
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "admm_msi_512x512x31.json")
    gold = json.load(open(path))
    d = inputs.config3()
    T, B, mask, prm = d["T"], d["B"], d["mask"], d["admm"]
    Xd = tnn.fortran_empty(B.shape, dtype_of(prec))
    st, rep = ctx.complete(tnn.to_fortran(B, dtype=dtype_of(prec)), tnn.to_fortran(mask), Xd, ctx.params(**prm),
                           prec=prec)
    X = tnn.to_numpy(Xd).astype(np.float64)
    err = np.linalg.norm(X - T) / np.linalg.norm(T)
    idx = np.array(gold["sample_index"])
    xs = X.ravel(order="F")[idx]
    rms = gold["norm_x"] / np.sqrt(X.size)
    dev = np.sqrt(np.mean((xs - np.array(gold["sample_x"])) ** 2)) / rms
    log_err("admm msi full %s" % prec, err=err, oracle=gold["rel_err_vs_ground_truth"], sample_rms_dev=dev)
    assert rep["iters"] == gold["iters"]
    assert abs(err - gold["rel_err_vs_ground_truth"]) <= 1e-4, (err, gold["rel_err_vs_ground_truth"])
    assert dev <= 1e-3, dev


def _video_state(ctx, iters, warm):
    """The video-shaped completion (3xTF32 transforms) after `iters` warm-
    started iterations from its start: (d, Bd, md, X, M, beta)."""
    from paper_1902_03070_gb300 import tnn
    torch = torch_cuda()
    d = inputs.config2(O.tprod)
    B, mask = d["B"], d["mask"]
    Bd, md = tnn.to_fortran(B, dtype=torch.float32), tnn.to_fortran(mask)
    X = tnn.to_fortran(B * mask, dtype=torch.float32)
    M = tnn.to_fortran(np.zeros(B.shape), dtype=torch.float32)
    prm = ctx.params(**{**d["admm"], "tol": -1.0})
    beta, _ = ctx.admm_iterate(Bd, md, X, M, d["admm"]["beta0"], iters, prm, prec="tf32x3", warm=warm)
    return d, Bd, md, X, M, beta, prm


def test_admm_warm_start_one_iteration_matches_cold_and_oracle(ctx):
    """Warm start (the previous iteration's right singular vectors): from one
    late state of the video-shaped completion, one warm-started iteration,
    one cold iteration and one oracle iteration (FP64, same state) agree, the
    warm one with a fraction of the sweeps, and the kept Q are orthogonal."""
    from paper_1902_03070_gb300 import tnn
    torch = torch_cuda()
    shape = (144, 176, 100)
    warm = ctx.admm_warm_state(shape, "tf32x3")
    assert warm is not None
    d, Bd, md, X, M, beta, prm = _video_state(ctx, 150, warm)
    x0, m0 = tnn.to_numpy(X).astype(np.float64), tnn.to_numpy(M).astype(np.float64)
    # the kept Q (n x n per slice, then one flag per slice) are orthogonal
    n, n3 = 144, 100
    q = warm[: n3 * n * n * 4].view(torch.float32).reshape(n3, n, n).double()
    flags = warm[(n3 * n * n * 4 + 255) // 256 * 256:][: 4 * n3].view(torch.int32).cpu().numpy()
    assert flags.sum() == n3
    err = (q.transpose(1, 2) @ q - torch.eye(n, dtype=torch.float64, device=q.device)).abs().amax().item()
    assert err <= 5e-6, err
    Xw, Mw = X.clone(), M.clone()
    ctx.admm_iterate(Bd, md, Xw, Mw, beta, 1, prm, prec="tf32x3", warm=warm)
    sw_warm = ctx.last_jacobi_stats()["max_sweeps"]
    Xc, Mc = X.clone(), M.clone()
    ctx.admm_iterate(Bd, md, Xc, Mc, beta, 1, prm, prec="tf32x3")
    sw_cold = ctx.last_jacobi_stats()["max_sweeps"]
    Xo, _, _ = O.admm(d["B"], d["mask"], X0=x0, M0=m0, **{**d["admm"], "beta0": beta, "tol": -1.0,
                                                            "max_iter": 1}, nthreads=THREADS)
    xw, xc = tnn.to_numpy(Xw).astype(np.float64), tnn.to_numpy(Xc).astype(np.float64)
    dx = np.linalg.norm(Xo - x0)
    log_err("admm warm one iteration", warm_vs_cold=np.linalg.norm(xw - xc) / dx,
            warm_vs_oracle=np.linalg.norm(xw - Xo) / dx, cold_vs_oracle=np.linalg.norm(xc - Xo) / dx,
            sweeps_warm=sw_warm, sweeps_cold=sw_cold)
    # relative to the iteration's own change of X (the t-SVT's contribution)
    assert np.linalg.norm(xw - Xo) <= 1e-3 * dx + 1e-5 * np.linalg.norm(Xo)
    assert np.linalg.norm(xw - xc) <= 1e-3 * dx + 1e-5 * np.linalg.norm(Xo)
    assert sw_warm * 2 <= sw_cold, (sw_warm, sw_cold)


def test_admm_warm_start_resume_bit_exact(ctx):
    """With the warm-start buffer as part of the state, 40 + 40 iterations in
    two calls give bit for bit the 80 of one call."""
    from paper_1902_03070_gb300 import tnn
    torch = torch_cuda()
    shape = (144, 176, 100)
    w1 = ctx.admm_warm_state(shape, "tf32x3")
    w2 = ctx.admm_warm_state(shape, "tf32x3")
    _, Bd, md, X1, M1, b1, prm = _video_state(ctx, 80, w1)
    d, Bd, md, X2, M2, b2, prm = _video_state(ctx, 40, w2)
    b2, _ = ctx.admm_iterate(Bd, md, X2, M2, b2, 40, prm, prec="tf32x3", warm=w2)
    assert b1 == b2
    assert torch.equal(X1, X2) and torch.equal(M1, M2) and torch.equal(w1, w2)


def test_admm_warm_size_zero_where_unused():
    from paper_1902_03070_gb300 import tnn
    torch_cuda()
    assert tnn.Context.admm_warm_state((48, 48, 16), "fp64") is None        # FP64: cold
    assert tnn.Context.admm_warm_state((512, 512, 31), "bf16split") is None  # slices on clusters
    assert tnn.Context.admm_warm_state((48, 48, 16), "fp32") is not None


@pytest.mark.parametrize("shape", [(100, 70, 6), (70, 101, 5), (52, 52, 4)])
def test_warm_tail_ragged_shapes_match_oracle(ctx, shape):
    """The warm start with its offloaded SVT tail on shapes whose smaller
    side leaves a partial 48-column tile of the tail kernel, in both slice
    orientations, one of them with a leading dimension that is not a multiple
    of 4 (the tail's element-wise load and store paths): a whole FP32
    completion has the oracle's final error and the cold run's iterates."""
    from paper_1902_03070_gb300 import tnn
    torch = torch_cuda()
    T, B, mask = _small(seed=3, shape=shape, r=3, frac=0.5)
    prm = dict(beta0=1e-2, rho=1.15, beta_max=1e8, tol=-1.0, max_iter=60)
    Xo, _, _ = O.admm(B, mask, nthreads=THREADS, **prm)
    dt = dtype_of("fp32")
    Bd, md = tnn.to_fortran(B, dtype=dt), tnn.to_fortran(mask)
    assert ctx.admm_warm_state(shape, "fp32") is not None
    Xw = tnn.fortran_empty(B.shape, dt)
    ctx.profile(True)
    ctx.complete(Bd, md, Xw, ctx.params(**prm), prec="fp32")
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    assert "svt_tail" in prof and "warm" in prof  # the warm-started path with its tail ran
    Xc = tnn.fortran_empty(B.shape, dt)
    try:
        ctx.set_option(tnn.OPT_ADMM_WARM_START, 0)
        ctx.complete(Bd, md, Xc, ctx.params(**prm), prec="fp32")
    finally:
        ctx.set_option(tnn.OPT_ADMM_WARM_START, 1)
    xw, xc = tnn.to_numpy(Xw).astype(np.float64), tnn.to_numpy(Xc).astype(np.float64)
    nt = np.linalg.norm(T)
    ew, ec, eo = np.linalg.norm(xw - T) / nt, np.linalg.norm(xc - T) / nt, np.linalg.norm(Xo - T) / nt
    log_err("warm tail ragged %s" % (shape,), warm=ew, cold=ec, oracle=eo,
            warm_vs_oracle=np.linalg.norm(xw - Xo) / np.linalg.norm(Xo))
    assert abs(ew - eo) <= 1e-4 and abs(ec - eo) <= 1e-4, (ew, ec, eo)
    assert np.linalg.norm(xw - Xo) <= 1e-3 * np.linalg.norm(Xo)
    assert np.linalg.norm(xw - xc) <= 1e-3 * np.linalg.norm(Xo)
