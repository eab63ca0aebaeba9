"""GPU tests of the completion server (tnn_server_*): a job's result is the
same, bit for bit, whether it runs alone through tnn_complete or in a mix of
concurrent jobs of other shapes and precisions, with each job's own kernels or
with batched iterations for the FP32 and FP64 jobs; admission keeps the
device footprint under the cap; invalid jobs are refused at submission."""
import time

import numpy as np
import pytest

import oracle as O
from gpu_common import dtype_of, torch_cuda
from paper_1902_03070_gb300 import inputs

pytestmark = pytest.mark.gpu

# (shape, precision, observed fraction, iteration cap): the 48 x 48 x 16
# FP64 workload, small FP32 / 3xTF32 / BF16-split tensors, and slices large
# enough for the cluster Jacobi kernel
MIX = [((48, 48, 16), "fp64", 0.4, 60), ((64, 80, 12), "fp32", 0.3, 40), ((40, 50, 20), "tf32x3", 0.25, 50),
       ((64, 64, 31), "bf16split", 0.2, 30), ((300, 280, 3), "fp32", 0.3, 8), ((33, 17, 5), "fp64", 0.5, 70)]


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with tnn.Context(0) as c:
        # the reference runs: tnn_complete without the warm start, the
        # iterates the batched and served paths reproduce bit for bit
        c.set_option(tnn.OPT_ADMM_WARM_START, 0)
        yield c


def _jobs(seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for shape, prec, frac, iters in MIX:
        n1, n2, n3 = shape
        A, F = inputs.lowrank_factors(n1, n2, n3, 3, rng)
        T = O.tprod(A, F)
        mask = inputs.uniform_mask(shape, frac, rng)
        B = inputs.fortran(T * mask)
        out.append(dict(shape=shape, prec=prec, B=B, mask=mask,
                        prm=dict(beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-8, max_iter=iters)))
    return out


def _alone(ctx, job, batch_kernels=False):
    """The job through tnn_complete, warm-started exactly when the server
    warm-starts it (FP32 precisions on the job's own kernels; not an FP32
    job that a batching server puts on the batched kernels)."""
    from paper_1902_03070_gb300 import tnn
    dt = dtype_of(job["prec"])
    Xd = tnn.fortran_empty(job["shape"], dt)
    warm = not (batch_kernels and job["prec"] == "fp32")
    ctx.set_option(tnn.OPT_ADMM_WARM_START, 1 if warm else 0)
    try:
        st, rep = ctx.complete(tnn.to_fortran(job["B"], dtype=dt), tnn.to_fortran(job["mask"]), Xd,
                               ctx.params(**job["prm"]), prec=job["prec"])
    finally:
        ctx.set_option(tnn.OPT_ADMM_WARM_START, 0)
    return tnn.to_numpy(Xd), rep


def _run_server(server, jobs, device_inputs, stagger=0.0):
    from paper_1902_03070_gb300 import tnn
    ids = []
    for i, job in enumerate(jobs):
        dt = dtype_of(job["prec"])
        if device_inputs and i % 2 == 0:
            B, mask = tnn.to_fortran(job["B"], dtype=dt), tnn.to_fortran(job["mask"])
        else:
            B = np.asfortranarray(job["B"].astype(np.float64 if job["prec"] == "fp64" else np.float32))
            mask = np.asfortranarray(job["mask"])
        ids.append(server.submit(B, mask, tnn.Context.params(**job["prm"]), prec=job["prec"]))
        server.step()
        if stagger:
            time.sleep(stagger)
    results = {}
    t_end = time.time() + 120
    while len(results) < len(ids):
        server.step()
        for jid in ids:
            if jid not in results and server.state(jid) >= 2:
                results[jid] = server.take(jid)
        assert time.time() < t_end, server.stats()
    return [results[j] for j in ids]


@pytest.mark.parametrize("batch_kernels", [False, True])
def test_alone_equals_in_mix(ctx, batch_kernels):
    from paper_1902_03070_gb300 import tnn
    jobs = _jobs()
    alone = [_alone(ctx, j, batch_kernels) for j in jobs]
    with tnn.Server(streams=4, chunk=3, batch_kernels=batch_kernels) as sv:
        mixed = _run_server(sv, jobs, device_inputs=True, stagger=0.002)
        st = sv.stats()
    assert st["queued"] == 0 and st["running"] == 0
    for job, (Xa, ra), (status, Xm, rm, times) in zip(jobs, alone, mixed):
        assert status in (tnn.OK, tnn.ENOCONV), (job["shape"], status)
        assert rm["iters"] == ra["iters"], (job["shape"], rm, ra)
        assert np.array_equal(Xa, Xm), job["shape"]
        assert times[0] <= times[1] <= times[2]


def test_admission_respects_the_footprint_cap(ctx):
    from paper_1902_03070_gb300 import tnn
    jobs = _jobs(seed=6)[:4]
    alone = [_alone(ctx, j) for j in jobs]
    # room for about two of these jobs at a time
    sizes = []
    for j in jobs:
        n = int(np.prod(j["shape"]))
        e = 8 if j["prec"] == "fp64" else 4
        sizes.append(5 * n * e + n)
    cap = int(sorted(sizes)[-1] + sorted(sizes)[-2] + (8 << 20))
    with tnn.Server(hbm_cap_bytes=cap, streams=2, chunk=4) as sv:
        mixed = _run_server(sv, jobs, device_inputs=False)
        st = sv.stats()
    assert 0 < st["peak_bytes"] <= cap
    assert st["completed"] == len(jobs)
    for (Xa, ra), (status, Xm, rm, times) in zip(alone, mixed):
        assert np.array_equal(Xa, Xm)


def test_max_active_serialises_jobs(ctx):
    from paper_1902_03070_gb300 import tnn
    jobs = _jobs(seed=7)[:3]
    with tnn.Server(max_active=1, streams=2, chunk=8) as sv:
        res = _run_server(sv, jobs, device_inputs=False)
    spans = sorted((r[3][1], r[3][2]) for r in res)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1 - 1e-9  # the next job is admitted only after the previous one finished


def test_server_rejects_invalid_jobs(ctx):
    torch = torch_cuda()
    from paper_1902_03070_gb300 import tnn
    with tnn.Server(hbm_cap_bytes=1 << 20) as sv:
        B = np.asfortranarray(np.zeros((200, 200, 4), dtype=np.float32))
        mask = np.asfortranarray(np.ones((200, 200, 4), dtype=np.uint8))
        with pytest.raises(tnn.TnnError):
            sv.submit(B, mask, tnn.Context.params(), prec="fp32")  # never fits 1 MiB
        Bs = np.asfortranarray(np.zeros((8, 8, 2), dtype=np.float32))
        ms = np.asfortranarray(np.ones((8, 8, 2), dtype=np.uint8))
        bad = tnn.Context.params()
        bad.beta0 = -1.0
        with pytest.raises(tnn.TnnError):
            sv.submit(Bs, ms, bad, prec="fp32")
        jid = sv.submit(Bs, ms, tnn.Context.params(max_iter=5), prec="fp32")
        while sv.state(jid) < 2:
            sv.step()
        status, X, rep, t = sv.take(jid)
        assert rep["iters"] <= 5
        with pytest.raises(KeyError):
            sv.take(jid)  # already taken


def test_shortest_first_admission_order(ctx):
    from paper_1902_03070_gb300 import tnn
    jobs = _jobs(seed=8)[:4]
    work = [j["prm"]["max_iter"] * j["shape"][2] * max(j["shape"][:2]) * min(j["shape"][:2]) ** 2 for j in jobs]
    with tnn.Server(max_active=1, streams=1, chunk=16, policy=tnn.Server.SHORTEST_FIRST) as sv:
        ids = []
        for j in jobs:  # all queued before the first scheduling pass
            dt = np.float64 if j["prec"] == "fp64" else np.float32
            ids.append(sv.submit(np.asfortranarray(j["B"].astype(dt)), np.asfortranarray(j["mask"]),
                                 tnn.Context.params(**j["prm"]), prec=j["prec"]))
        t_end = time.time() + 120
        admitted = {}
        while len(admitted) < len(ids):
            sv.step()
            for jid in ids:
                if jid not in admitted and sv.state(jid) >= 2:
                    admitted[jid] = sv.take(jid)[3][1]
            assert time.time() < t_end
    order = sorted(range(len(ids)), key=lambda i: admitted[ids[i]])
    assert order == sorted(range(len(ids)), key=lambda i: work[i])


def test_server_zero_iterations_and_full_observation(ctx):
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(12)
    T = inputs.random_tensor((10, 8, 3), rng)
    full = np.asfortranarray(np.ones(T.shape, dtype=np.uint8))
    with tnn.Server(streams=2) as sv:
        j0 = sv.submit(np.asfortranarray(T), full, tnn.Context.params(max_iter=0), prec="fp64")
        j1 = sv.submit(np.asfortranarray(T), full, tnn.Context.params(max_iter=20), prec="fp64")
        t_end = time.time() + 60
        while sv.state(j0) < 2 or sv.state(j1) < 2:
            sv.step()
            assert time.time() < t_end
        st0, X0, r0, _ = sv.take(j0)
        st1, X1, r1, _ = sv.take(j1)
    assert r0["iters"] == 0 and np.array_equal(X0, T)   # X = B on the mask, nothing run
    assert np.array_equal(X1, T)                        # everything observed: X stays B


def test_batched_jobs_join_and_leave(ctx):
    """Many FP32 and FP64 jobs of uneven shapes (several Jacobi plans, one
    cluster-sized) with uneven iteration caps and two Jacobi sweep caps, so
    that the batch is rebuilt as jobs join and leave: every job's result
    equals its run alone."""
    from paper_1902_03070_gb300 import tnn
    rng = np.random.default_rng(31)
    shapes = [(32, 40, 8), (96, 64, 16), (50, 120, 9), (256, 200, 4), (40, 40, 33), (70, 30, 12), (129, 65, 5),
              (300, 260, 2)]
    jobs = []
    for i, shape in enumerate(shapes * 2):
        n1, n2, n3 = shape
        A, F = inputs.lowrank_factors(n1, n2, n3, 2 + i % 5, rng)
        T = O.tprod(A, F)
        mask = inputs.uniform_mask(shape, float(rng.uniform(0.2, 0.5)), rng)
        prm = dict(beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-6, max_iter=int(rng.integers(5, 40)))
        if i % 7 == 3:
            prm["jacobi_max_sweeps"] = 6
        jobs.append(dict(shape=shape, prec="fp64" if i % 3 == 0 else "fp32", B=inputs.fortran(T * mask), mask=mask,
                         prm=prm))
    alone = [_alone(ctx, j, batch_kernels=True) for j in jobs]
    with tnn.Server(streams=2, chunk=4, batch_kernels=True) as sv:
        mixed = _run_server(sv, jobs, device_inputs=True, stagger=0.001)
        st = sv.stats()
    assert st["running"] == 0 and st["completed"] == len(jobs)
    for job, (Xa, ra), (status, Xm, rm, times) in zip(jobs, alone, mixed):
        assert status in (tnn.OK, tnn.ENOCONV), (job["shape"], status)
        assert rm["iters"] == ra["iters"], (job["shape"], rm, ra)
        assert np.array_equal(Xa, Xm), job["shape"]
