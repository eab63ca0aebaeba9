"""Serving workload and driver for the completion server (tnn.Server).

A seeded Poisson stream of completion jobs (mean rate `rate` jobs/s) whose
shapes are drawn uniformly from four classes:

  video48  - the 48 x 48 x 16 tubal-rank-3 tensor, FP64, at most 300 iterations
  video    - the 144 x 176 x 100 video-shaped tensor, 3xTF32 transforms, 200
  msi      - the 512 x 512 x 31 multispectral-shaped tensor, BF16-split
             transforms, 150
  batch    - a tensor of the uneven-batch range (n1, n2 in [32, 256],
             n3 in [8, 64], tubal rank 2-12), FP32, 200

Every job samples its own observed fraction ~ U[0.1, 0.5] and mask, and
stops at tol = 1e-5.  The driver submits each job at its arrival time, steps
the server, takes results as they finish and reports per-job latency
(arrival to finish), p50/p99 overall and per class, jobs/s and the peak
admitted device footprint.

    python -m paper_1902_03070_gb300.serve --jobs 48 --rate 200
"""
import argparse
import json
import time

import numpy as np

CLASSES = ["video48", "video", "msi", "batch"]
PREC = {"video48": "fp64", "video": "tf32x3", "msi": "bf16split", "batch": "fp32"}
ITERS = {"video48": 300, "video": 200, "msi": 150, "batch": 200}


def library_tprod(ctx):
    """The DCT t-product (Eq. 13) through the library, FP64, for building the
    low-rank workload tensors."""
    import torch

    from . import tnn

    def tp(A, F):
        Ad = tnn.to_fortran(A, dtype=torch.float64)
        Fd = tnn.to_fortran(F, dtype=torch.float64)
        Z = tnn.fortran_empty((A.shape[0], F.shape[1], A.shape[2]), torch.float64)
        ctx.tprod(Ad, Fd, Z, prec="fp64")
        return tnn.to_numpy(Z)
    return tp


def make_stream(n_jobs, rate, seed=1902_03075, tprod=None, n_batch_shapes=8):
    """Arrival times, classes and inputs of the job stream (host arrays).
    `tprod` builds the low-rank tensors (the DCT t-product)."""
    from . import inputs
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_jobs)
    arrivals = np.cumsum(gaps) - gaps[0]
    kinds = rng.integers(0, len(CLASSES), size=n_jobs)
    base = {}
    if (kinds == 0).any():
        base["video48"] = [inputs.config1(tprod)["T"]]
    if (kinds == 1).any():
        base["video"] = [inputs.config2(tprod)["T"]]
    if (kinds == 2).any():
        base["msi"] = [inputs.config3()["T"]]
    if (kinds == 3).any():
        base["batch"] = inputs.config4(tprod, count=n_batch_shapes)
    jobs = []
    for i in range(n_jobs):
        cls = CLASSES[kinds[i]]
        pool = base[cls]
        T = pool[int(rng.integers(0, len(pool)))]
        frac = float(rng.uniform(0.1, 0.5))
        mask = inputs.uniform_mask(T.shape, frac, rng)
        dt = np.float64 if PREC[cls] == "fp64" else np.float32
        B = np.asfortranarray((T * mask).astype(dt))
        jobs.append(dict(arrival=float(arrivals[i]), cls=cls, prec=PREC[cls], B=B, mask=np.asfortranarray(mask),
                         shape=T.shape, observed=frac,
                         params=dict(beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-5, max_iter=ITERS[cls])))
    return jobs


def run(jobs, hbm_cap_bytes=150e9, streams=8, chunk=8, max_active=0, policy=0, device=0, timeout_s=600.0,
        batch_kernels=False):
    """Drive a server through the stream; returns per-job records and a summary.
    `batch_kernels`: FP32 and FP64 jobs share one launch sequence per iteration."""
    from . import tnn
    recs = [None] * len(jobs)
    with tnn.Server(hbm_cap_bytes=int(hbm_cap_bytes), streams=streams, chunk=chunk, max_active=max_active,
                    policy=policy, device=device, batch_kernels=batch_kernels) as sv:
        t0 = time.perf_counter()
        pending = {}
        nxt = 0
        while nxt < len(jobs) or pending:
            now = time.perf_counter() - t0
            while nxt < len(jobs) and jobs[nxt]["arrival"] <= now:
                j = jobs[nxt]
                jid = sv.submit(j["B"], j["mask"], tnn.Context.params(**j["params"]), prec=j["prec"])
                pending[jid] = (nxt, time.perf_counter() - t0)
                nxt += 1
            sv.step()
            for jid in list(pending):
                if sv.state(jid) >= 2:
                    i, t_sub = pending.pop(jid)
                    st, _, rep, times = sv.take(jid)
                    t_done = time.perf_counter() - t0
                    recs[i] = dict(cls=jobs[i]["cls"], arrival=jobs[i]["arrival"], submitted=t_sub, done=t_done,
                                   latency=t_done - jobs[i]["arrival"], queued_s=times[1] - times[0],
                                   status=int(st), iters=rep["iters"], converged=rep["converged"])
            if time.perf_counter() - t0 > timeout_s:
                raise RuntimeError("serving run exceeded %.0f s" % timeout_s)
            if not pending and nxt < len(jobs):
                time.sleep(max(0.0, min(0.001, jobs[nxt]["arrival"] - (time.perf_counter() - t0))))
        stats = sv.stats()
    lat = np.array([r["latency"] for r in recs])
    span = max(r["done"] for r in recs) - min(r["arrival"] for r in recs)
    summary = {"jobs": len(recs), "jobs_per_s": len(recs) / span, "span_s": span,
               "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
               "peak_device_bytes": stats["peak_bytes"],
               "failed": sum(1 for r in recs if r["status"] not in (tnn.OK, tnn.ENOCONV)),
               "per_class": {}}
    for c in CLASSES:
        lc = np.array([r["latency"] for r in recs if r["cls"] == c])
        if len(lc):
            summary["per_class"][c] = {"jobs": int(len(lc)), "p50_s": float(np.percentile(lc, 50)),
                                       "p99_s": float(np.percentile(lc, 99)),
                                       "mean_iters": float(np.mean([r["iters"] for r in recs if r["cls"] == c]))}
    return recs, summary


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--jobs", type=int, default=48)
    p.add_argument("--rate", type=float, default=200.0)
    p.add_argument("--streams", type=int, default=8)
    p.add_argument("--chunk", type=int, default=8)
    p.add_argument("--hbm-cap-gb", type=float, default=150.0)
    p.add_argument("--max-active", type=int, default=0)
    p.add_argument("--policy", choices=["fifo", "shortest"], default="fifo")
    p.add_argument("--seed", type=int, default=1902_03075)
    p.add_argument("--batch-kernels", action="store_true")
    a = p.parse_args()
    from . import tnn
    with tnn.Context(0) as ctx:
        jobs = make_stream(a.jobs, a.rate, seed=a.seed, tprod=library_tprod(ctx))
    _, summary = run(jobs, hbm_cap_bytes=a.hbm_cap_gb * 1e9, streams=a.streams, chunk=a.chunk,
                     max_active=a.max_active, policy=1 if a.policy == "shortest" else 0,
                     batch_kernels=a.batch_kernels)
    summary.update({"rate": a.rate, "streams": a.streams, "chunk": a.chunk, "hbm_cap_gb": a.hbm_cap_gb,
                    "max_active": a.max_active, "policy": a.policy, "batch_kernels": a.batch_kernels})
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
