"""GPU parity: the batched t-SVT plan (tnn_tsvt_batch_*) — many tensors of
different shapes through one launch sequence — against the FP64 oracle's
t-SVT (Theorem 5) of each tensor, and against the single-tensor entry point.

Tolerances are those of the single-tensor t-SVT: FP64 ||Y - Y_oracle||_F <=
1e-12 ||Y_oracle||_F; FP32 <= 1e-5 ||Y_oracle||_F and <= 1e-5 ||Z||_F on
every tensor (Gaussian slices and the low-rank-plus-noise batched workload)."""
import numpy as np
import pytest

import oracle as O
from gpu_common import THREADS, dtype_of, log_err, rel_err, tau_at_quantile, torch_cuda
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu

# uneven mix: several Jacobi variants, transposed slices, single rows and
# columns, one slice, ragged column blocks, repeated shapes (same group)
MIX = [(48, 48, 16), (7, 5, 3), (5, 7, 3), (1, 9, 4), (9, 1, 4), (33, 65, 5), (65, 33, 2),
       (130, 100, 3), (40, 40, 1), (48, 48, 7), (200, 90, 6), (96, 250, 2)]


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with tnn.Context(0) as c:
        yield c


def _mix(prec, seed=11, q=0.3):
    rng = np.random.default_rng(seed)
    Zs, taus = [], []
    for sh in MIX:
        Z = inputs.random_tensor(sh, rng)
        if prec != "fp64":
            Z = Z.astype(np.float32).astype(np.float64)
        Zs.append(Z)
        taus.append(tau_at_quantile(Z, q))
    return Zs, taus


def _device(Zs, prec):
    from paper_1902_03070_gb300 import tnn
    Zd = [tnn.to_fortran(Z, dtype=dtype_of(prec)) for Z in Zs]
    Yd = [tnn.fortran_empty(Z.shape, dtype_of(prec)) for Z in Zs]
    return Zd, Yd


def _host(Ys):
    from paper_1902_03070_gb300 import tnn
    return [tnn.to_numpy(Y).astype(np.float64) for Y in Ys]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_oracle(ctx, prec, graph):
    Zs, taus = _mix(prec)
    Zd, Yd = _device(Zs, prec)
    plan = ctx.tsvt_batch(Zd, taus, Yd, prec=prec, graph=graph)
    info = plan.info()
    assert info["slices"] == sum(s[2] for s in MIX)
    assert info["graph"] == int(graph)
    assert info["launches"] == (1 if graph else 2 + info["groups"])
    plan.run()
    st = plan.stats()
    assert st["unconverged"] == 0 and st["nonfinite"] == 0
    for Z, tau, Y in zip(Zs, taus, _host(Yd)):
        ref = O.tsvt(Z, tau, nthreads=THREADS)
        err = rel_err(Y, ref, Z)
        log_err("batch %s %s graph=%d" % (prec, Z.shape, graph), err_y=err)
        if prec == "fp64":
            assert err <= 1e-12, (Z.shape, err)
        else:
            assert np.linalg.norm(Y - ref) <= 1e-5 * np.linalg.norm(Z), (Z.shape, err)
            assert err <= 1e-5, (Z.shape, err)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_single_tensor_calls(ctx, prec):
    # same Jacobi variant per tensor as the single-tensor call; only the
    # transforms' summation order may differ
    Zs, taus = _mix(prec, seed=12)
    Zd, Yd = _device(Zs, prec)
    plan = ctx.tsvt_batch(Zd, taus, Yd, prec=prec, graph=True)
    plan.run()
    got = _host(Yd)
    for Z, Zt, tau, Y in zip(Zs, Zd, taus, got):
        from paper_1902_03070_gb300 import tnn
        Y1 = tnn.to_numpy(ctx.tsvt(Zt, tau, Y=tnn.fortran_empty(Z.shape, dtype_of(prec)), prec=prec))
        tol = 1e-13 if prec == "fp64" else 2e-6
        assert np.linalg.norm(Y - Y1) <= tol * np.linalg.norm(Z), Z.shape


def test_batch_graph_replay_is_deterministic(ctx):
    torch = torch_cuda()
    Zs, taus = _mix("fp32", seed=13)
    Zd, Yd = _device(Zs, "fp32")
    plan = ctx.tsvt_batch(Zd, taus, Yd, prec="fp32", graph=True)
    plan.run()
    first = [y.clone() for y in Yd]
    for y in Yd:
        y.zero_()
    plan.run()
    plan.run()
    torch.cuda.synchronize()
    for a, b in zip(first, Yd):
        assert torch.equal(a, b)
    # the graph reads the inputs' current contents (thresholds stay those
    # the plan was created with)
    for z in Zd:
        z.mul_(2.0)
    plan.run()
    for Z, tau, Y in zip(Zs, taus, _host(Yd)):
        ref = O.tsvt(2 * Z, tau, nthreads=THREADS)
        assert np.linalg.norm(Y - ref) <= 1e-5 * np.linalg.norm(2 * Z)


def test_batch_in_place(ctx):
    torch = torch_cuda()
    Zs, taus = _mix("fp64", seed=14)
    Zd, Yd = _device(Zs, "fp64")
    ref_plan = ctx.tsvt_batch(Zd, taus, Yd, prec="fp64", graph=False)
    ref_plan.run()
    plan = ctx.tsvt_batch(Zd, taus, None, prec="fp64", graph=True)  # Y aliases Z
    # creating the plan writes no item buffer
    for Z, z in zip(Zs, _host(Zd)):
        assert np.array_equal(Z, z)
    plan.run()
    torch.cuda.synchronize()
    for a, b in zip(Yd, Zd):
        assert torch.equal(a, b)


def test_batch_threshold_extremes(ctx):
    rng = np.random.default_rng(15)
    Zs = [inputs.random_tensor(s, rng) for s in [(20, 30, 4), (30, 20, 5), (17, 17, 3)]]
    big = [10 * np.linalg.norm(Z) for Z in Zs]
    Zd, Yd = _device(Zs, "fp64")
    plan = ctx.tsvt_batch(Zd, [0.0, big[1], 0.0], Yd, prec="fp64")
    plan.run()
    Y = _host(Yd)
    assert rel_err(Y[0], Zs[0]) <= 1e-12  # tau = 0: identity
    assert np.count_nonzero(Y[1]) == 0     # tau above every singular value: zero
    assert rel_err(Y[2], Zs[2]) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_autotuned(ctx, prec):
    Zs, taus = _mix(prec, seed=16)
    Zd, Yd = _device(Zs, prec)
    plan = ctx.tsvt_batch(Zd, taus, Yd, prec=prec, graph=True, autotune=True)
    for g in plan.groups():
        assert g["L"] * g["R"] >= g["m"]
    plan.run()
    assert plan.stats()["unconverged"] == 0
    for Z, tau, Y in zip(Zs, taus, _host(Yd)):
        ref = O.tsvt(Z, tau, nthreads=THREADS)
        err = rel_err(Y, ref, Z)
        if prec == "fp64":
            assert err <= 1e-12, (Z.shape, err)
        else:
            assert np.linalg.norm(Y - ref) <= 1e-5 * np.linalg.norm(Z), (Z.shape, err)
            assert err <= 1e-5, (Z.shape, err)


def test_batch_rejects_bad_input(ctx):
    torch = torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with pytest.raises(ValueError):
        ctx.tsvt_batch([], [], prec="fp32")
    Zh = np.asfortranarray(np.zeros((4, 4, 2), dtype=np.float32))
    with pytest.raises(tnn.TnnError):
        ctx.tsvt_batch([Zh], [0.1], [Zh], prec="fp32")  # host memory
    Zd = tnn.fortran_empty((4, 4, 2), torch.float32)
    with pytest.raises(tnn.TnnError):
        ctx.tsvt_batch([Zd], [-1.0], prec="fp32")
    Zbig = tnn.fortran_empty((600, 4, 1), torch.float32)
    with pytest.raises(tnn.TnnError):
        ctx.tsvt_batch([Zbig], [0.1], prec="fp32")


def test_batch_64_uneven_tensors_full_size(ctx):
    """The 64-tensor batched workload (n1, n2 in [32, 256], n3 in [8, 64],
    tubal rank 2-12 plus N(0, 1e-3) noise, per-tensor threshold), FP32 in
    one captured graph with autotuned variants, every tensor against the
    oracle."""
    torch = torch_cuda()
    Zs = inputs.config4(O.tprod)
    taus = [inputs.config4_tau(Z.shape[0], Z.shape[1]) for Z in Zs]
    Zs32 = [Z.astype(np.float32).astype(np.float64) for Z in Zs]
    Zd, Yd = _device(Zs32, "fp32")
    plan = ctx.tsvt_batch(Zd, taus, Yd, prec="fp32", graph=True, autotune=True)
    assert plan.info()["slices"] == sum(Z.shape[2] for Z in Zs)
    plan.run()
    torch.cuda.synchronize()
    assert plan.stats()["unconverged"] == 0
    worst = 0.0
    for Z, tau, Y in zip(Zs32, taus, _host(Yd)):
        ref = O.tsvt(Z, tau, nthreads=THREADS)
        err = rel_err(Y, ref, Z)
        worst = max(worst, err)
        assert err <= 1e-5, (Z.shape, err)
    log_err("batch c4", worst=worst)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_edge_shapes(ctx, prec):
    # single tensor; 1 x 1 x 1; one slice; one row / column; identical shapes
    shapes = [(1, 1, 1), (1, 7, 3), (7, 1, 2), (5, 5, 1), (16, 16, 4), (16, 16, 4)]
    rng = np.random.default_rng(31)
    Zs = [inputs.random_tensor(s, rng) for s in shapes]
    if prec != "fp64":
        Zs = [Z.astype(np.float32).astype(np.float64) for Z in Zs]
    taus = [0.1, 0.5, 0.5, 1.0, 2.0, 0.0]
    for one in (False, True):
        sel = [0] if one else list(range(len(Zs)))
        Zd, Yd = _device([Zs[i] for i in sel], prec)
        plan = ctx.tsvt_batch(Zd, [taus[i] for i in sel], Yd, prec=prec, graph=True)
        plan.run()
        for i, Y in zip(sel, _host(Yd)):
            ref = O.tsvt(Zs[i], taus[i])
            tol = 1e-12 if prec == "fp64" else 1e-5
            assert np.linalg.norm(Y - ref) <= tol * max(np.linalg.norm(Zs[i]), 1e-300), shapes[i]
        plan.close()
