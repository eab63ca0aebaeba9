"""GPU tests of the batched ADMM plan (tnn_admm_batch_*): Algorithm 1 for
many completion problems of different shapes in one launch sequence per
iteration gives every job exactly the iterates of tnn_complete run on it
alone (CUDA-core transforms), bit for bit, with and without graph replay."""
import numpy as np
import pytest

import oracle as O
from gpu_common import dtype_of, torch_cuda
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(48, 48, 16), (33, 17, 5), (20, 64, 7), (1, 9, 4), (64, 64, 31), (300, 280, 2), (9, 9, 1)]


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with tnn.Context(0) as c:
        # the reference runs: tnn_complete without the warm start, the
        # iterates the batched and served paths reproduce bit for bit
        c.set_option(tnn.OPT_ADMM_WARM_START, 0)
        yield c


def _jobs(seed):
    rng = np.random.default_rng(seed)
    jobs = []
    for sh in SHAPES:
        A, F = inputs.lowrank_factors(sh[0], sh[1], sh[2], 2, rng)
        T = O.tprod(A, F)
        mask = inputs.uniform_mask(sh, 0.35, rng)
        jobs.append((T, inputs.fortran(T * mask), mask))
    return jobs


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("graph", [True, False])
def test_batched_admm_equals_separate_runs(ctx, prec, graph):
    torch = torch_cuda()
    from paper_1902_03070_gb300 import tnn
    dt = dtype_of(prec)
    prm = dict(beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-8, max_iter=60)
    jobs = _jobs(3)
    Bs = [tnn.to_fortran(B, dtype=dt) for _, B, _ in jobs]
    ms = [tnn.to_fortran(m) for _, _, m in jobs]
    Xs = [tnn.fortran_empty(B.shape, dt) for _, B, _ in jobs]
    Ms = [tnn.fortran_empty(B.shape, dt) for _, B, _ in jobs]
    plan = ctx.admm_batch(Bs, ms, Xs, Ms, ctx.params(**prm), prec=prec, graph=graph)
    plan.run()
    assert plan.sync() == 0
    for i, (T, B, mask) in enumerate(jobs):
        st, rep = plan.report(i)
        Xa = tnn.fortran_empty(B.shape, dt)
        st_a, rep_a = ctx.complete(Bs[i], ms[i], Xa, ctx.params(**prm), prec=prec)
        assert rep["iters"] == rep_a["iters"], (SHAPES[i], rep, rep_a)
        assert rep["converged"] == rep_a["converged"]
        assert torch.equal(Xs[i], Xa), SHAPES[i]
    # reset and run again: the same result
    X0 = [x.clone() for x in Xs]
    plan.reset()
    plan.run()
    for a, b in zip(X0, Xs):
        assert torch.equal(a, b)
    plan.close()


def test_batched_admm_stepwise_and_invalid(ctx):
    torch = torch_cuda()
    from paper_1902_03070_gb300 import tnn
    jobs = _jobs(4)[:3]
    dt = dtype_of("fp32")
    prm = dict(beta0=1e-3, rho=1.2, beta_max=1e8, tol=1e-6, max_iter=25)
    Bs = [tnn.to_fortran(B, dtype=dt) for _, B, _ in jobs]
    ms = [tnn.to_fortran(m) for _, _, m in jobs]
    Xs = [tnn.fortran_empty(B.shape, dt) for _, B, _ in jobs]
    Ms = [tnn.fortran_empty(B.shape, dt) for _, B, _ in jobs]
    plan = ctx.admm_batch(Bs, ms, Xs, Ms, ctx.params(**prm), prec="fp32")
    for _ in range(30):          # more steps than max_iter: stopped jobs are skipped
        plan.step(1)
    assert plan.sync() == 0
    for i in range(len(jobs)):
        _, rep = plan.report(i)
        assert 1 <= rep["iters"] <= 25
        Xa = tnn.fortran_empty(jobs[i][1].shape, dt)
        ctx.complete(Bs[i], ms[i], Xa, ctx.params(**prm), prec="fp32")
        assert torch.equal(Xs[i], Xa)
    plan.close()
    Bh = np.asfortranarray(jobs[0][1].astype(np.float32))
    with pytest.raises(tnn.TnnError):
        ctx.admm_batch([Bh], [ms[0]], [Xs[0]], [Ms[0]], ctx.params(**prm), prec="fp32")
