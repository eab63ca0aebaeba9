"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2):
every rank reports the slowest rank's time, and the whole-job rate counts
the units of all ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://")
    env = bench.dist_env()
    slowest = bench.max_over_ranks(100.0 + 50.0 * rank, ws, dist, "cpu")  # rank 1 took 150 ms
    rate = bench.job_rate(env[0], 100, 10, slowest)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, env, slowest, rate))


def test_max_over_ranks_and_job_rate_with_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, slowest, rate in out:
        assert env[0] == 2 and env[1] == rank
        assert slowest == 150.0
        assert abs(rate - 2 * 100 * 10 / 0.150) < 1e-6


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, None, "cpu") == 12.5
    assert abs(bench.job_rate(1, 100, 197, 400.0) - 100 * 197 / 0.4) < 1e-9


def test_timed_window_is_the_jobs_last_iterations():
    sys.path.insert(0, ROOT)
    import bench
    # the driver's --steps 20 --warmup 5: prefix 0-174 untimed, warm-up 175-179, timed 180-199
    assert bench.window(20, 5) == {"start": 180, "prefix": 175, "warm_in": 5, "warm_extra": 0}
    # the whole job timed: the warm-up runs on a throw-away copy
    assert bench.window(200, 5) == {"start": 0, "prefix": 0, "warm_in": 0, "warm_extra": 5}
    assert bench.window(197, 5) == {"start": 3, "prefix": 0, "warm_in": 3, "warm_extra": 2}
    for K in (1, 7, 20, 199, 200):
        for W in (0, 3, 5, 250):
            w = bench.window(K, W)
            assert w["prefix"] + w["warm_in"] == w["start"] == bench.JOB_ITERS - K
            assert w["warm_in"] + w["warm_extra"] == W and min(w.values()) >= 0
