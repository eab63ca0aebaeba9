"""The Jacobi launch planner on the host (tnn_jacobi_plan_info, no device):
every plan covers its slice (rows L R >= m, columns nb K >= n, an even block
count), fits the CTA limits (at most 1024 threads, 227 KB of shared memory),
sends only large slices to thread-block clusters, and the limits and
invalid arguments are refused."""
import numpy as np
import pytest

SMEM_MAX = 227 * 1024


@pytest.fixture(scope="module")
def tnn():
    from paper_1902_03070_gb300 import tnn as t
    return t


def _check(plan, n1, n2, prec):
    m, n = max(n1, n2), min(n1, n2)
    elem = 8 if prec == "fp64" else 4
    L, R, K, nb, W = plan["L"], plan["R"], plan["K"], plan["nb"], plan["W"]
    C = plan["cluster"]
    assert L in (8, 16, 32) and L * R >= m
    assert nb % 2 == 0 and nb * K >= n
    assert 1 <= W <= 32
    assert plan["smem_bytes"] <= SMEM_MAX
    if C > 1:
        assert C in (2, 4, 8, 16) and nb % (4 * C) == 0 and plan["in_smem"] == 1
        # only slices whose working copy is large go to clusters (one CTA holds
        # a copy of up to about 200 KB next to its other shared arrays)
        assert (L * R + (2 if elem == 4 else 1)) * n * elem > 100 * 1024
    if plan["in_smem"]:
        assert plan["work_bytes"] == 0
    else:
        assert plan["work_bytes"] > 0


def test_workload_plans(tnn):
    p = tnn.jacobi_plan_info((144, 176, 100), "fp32")
    _check(p, 144, 176, "fp32")
    assert p["cluster"] == 1 and p["in_smem"] == 1 and (p["L"], p["R"], p["K"]) == (16, 12, 4)
    p = tnn.jacobi_plan_info((512, 512, 31), "bf16split")
    _check(p, 512, 512, "bf16split")
    assert p["cluster"] >= 2
    p = tnn.jacobi_plan_info((48, 48, 16), "fp64")
    _check(p, 48, 48, "fp64")
    assert p["in_smem"] == 1 and p["cluster"] == 1


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_random_shapes(tnn, prec):
    rng = np.random.default_rng(5 if prec == "fp32" else 6)
    for _ in range(300):
        n1, n2 = (int(x) for x in rng.integers(1, 513, size=2))
        n3 = int(rng.integers(1, 65))
        p = tnn.jacobi_plan_info((n1, n2, n3), prec)
        _check(p, n1, n2, prec)
        assert tnn.jacobi_plan_info((n2, n1, n3), prec) == p  # orientation does not change the plan


def test_limits_refused(tnn):
    for shape in ((513, 10, 2), (10, 513, 2), (0, 5, 5), (5, 0, 5), (5, 5, 0), (-1, 4, 4)):
        with pytest.raises(tnn.TnnError):
            tnn.jacobi_plan_info(shape, "fp32")
    import ctypes
    out = (ctypes.c_int64 * 9)()
    assert tnn._lib.tnn_jacobi_plan_info(tnn.Shape(4, 4, 4), 7, out) == tnn.EINVAL
    assert tnn._lib.tnn_jacobi_plan_info(tnn.Shape(4, 4, 4), 1, None) == tnn.EINVAL


def test_server_footprint(tnn):
    # B, X, M and the transformed tensor (elem bytes each) plus the mask, at
    # least; the Jacobi scratch only when the slices are not in shared memory;
    # for a warm-started job also its warm-start state (tnn_admm_warm_size)
    # and the scratch of its start columns (one L R x nb K working copy per
    # slice, the slice oriented with its rows the longer side) and of the
    # offloaded SVT tail's record
    import ctypes
    for shape, prec in (((144, 176, 100), "tf32x3"), ((48, 48, 16), "fp64"), ((512, 512, 31), "bf16split"),
                        ((300, 20, 7), "fp32")):
        N = int(np.prod(shape))
        elem = 8 if prec == "fp64" else 4
        fp = tnn.server_footprint(shape, prec)
        plan = tnn.jacobi_plan_info(shape, prec)
        wb = ctypes.c_size_t(0)
        assert tnn._lib.tnn_admm_warm_size(tnn.Shape(*shape), tnn.PRECISIONS[prec], ctypes.byref(wb)) == tnn.OK
        warm = wb.value
        if warm:
            warm += shape[2] * plan["L"] * plan["R"] * plan["nb"] * plan["K"] * elem + 4 * shape[2]
            # the offloaded SVT tail's per-slice record: 4 (nb K) + 4 words
            warm += shape[2] * 4 * (4 * plan["nb"] * plan["K"] + 4)
        # warm-started: the video-shaped FP32 job; not FP64, not slices on clusters or over 256 rows
        assert (warm > 0) == (shape == (144, 176, 100))
        assert fp >= 4 * N * elem + N + plan["work_bytes"] + warm
        assert fp <= 4 * N * elem + N + plan["work_bytes"] + warm + 64 * 1024 + 64 * shape[2] + 16 * N // 32
    assert tnn.server_footprint((64, 64, 8), "fp32") < tnn.server_footprint((64, 64, 16), "fp32")
    for shape in ((513, 4, 4), (0, 4, 4)):
        with pytest.raises(tnn.TnnError):
            tnn.server_footprint(shape, "fp32")
