"""Write the oracle's end-to-end completion results used by the GPU tests.

Calls only oracle/ (and the seeded input generators).  It runs Algorithm 1
in FP64 and stores the final relative error against the ground truth, the
iteration count and the last residuals, for
  - the video-shaped 144 x 176 x 100 workload (tubal-rank-10 core built by
    the oracle's t-product, drift, noise, 20% observed, beta0 1e-4, rho 1.1,
    beta_max 1e10, tol 1e-8, 200 iterations), and
  - a 128 x 128 x 31 window of the multispectral-shaped workload (5 smooth
    spectral signatures times smoothed abundance maps, 10% observed, the same
    beta schedule, 150 iterations): the full 512 x 512 x 31 run takes the
    oracle hours.

    python tests/golden/make_admm_golden.py [threads] [video|msi]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1902_03070_gb300 import inputs  # noqa: E402


WORKLOADS = {
    "video": ("admm_video_144x176x100.json", lambda: inputs.config2(O.tprod),
              "video-shaped 144x176x100, 20% observed, beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-8, "
              "max_iter=200 (seeded inputs of paper_1902_03070_gb300.inputs.config2)"),
    "msi": ("admm_msi_128x128x31.json", lambda: inputs.config3(n1=128, n2=128),
            "multispectral-shaped window 128x128x31, 10% observed, beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-8, "
            "max_iter=150 (seeded inputs of paper_1902_03070_gb300.inputs.config3(n1=128, n2=128))"),
    "msi512": ("admm_msi_512x512x31.json", lambda: inputs.config3(),
               "multispectral-shaped 512x512x31, 10% observed, beta0=1e-4, rho=1.1, beta_max=1e10, tol=1e-8, "
               "max_iter=150 (seeded inputs of paper_1902_03070_gb300.inputs.config3())"),
}


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else len(os.sched_getaffinity(0))
    names = sys.argv[2:] or ["video", "msi"]
    for name in names:
        fname, make, desc = WORKLOADS[name]
        d = make()
        t0 = time.time()
        X, M, rep = O.admm(d["B"], d["mask"], nthreads=threads, **d["admm"])
        err = float(np.linalg.norm(X - d["T"]) / np.linalg.norm(d["T"]))
        out = {"workload": desc,
               "rel_err_vs_ground_truth": err, "iters": rep["iters"], "rel_change": rep["rel_change"],
               "primal_res": rep["primal_res"], "beta_final": rep["beta_final"], "converged": rep["converged"],
               "oracle_seconds": time.time() - t0, "threads": threads}
        if name == "msi512":
            # the oracle's final X at seeded positions, for an elementwise check
            # of sampled outputs of the full-size run
            idx = np.sort(np.random.default_rng(1902_03070).choice(X.size, size=512, replace=False))
            out["sample_index"] = [int(i) for i in idx]
            out["sample_x"] = [float(v) for v in X.ravel(order="F")[idx]]
            out["norm_x"] = float(np.linalg.norm(X))
        with open(os.path.join(HERE, fname), "w") as f:
            json.dump(out, f, indent=1)
        print(json.dumps(out))


if __name__ == "__main__":
    main()
