"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
replica of the workload (seeded by its rank), the job timed by its slowest
rank, and the whole-job SD-steps/s summed over ranks."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.dist_max(1.0 + rank, world)  # rank 1 is the slower
        bench.dist_barrier(world)
        w = bench.make_workload("icmw_2d", seed=rank)
        out.put((rank, t, w.n_sd, w.cfg["seed"], float(np.asarray(w.rhod).sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, n0, s0, rho0), (r1, t1, n1, s1, rho1) = res
    assert t0 == t1 == 2.0  # both ranks see the slowest rank's time
    assert n0 == n1 and rho0 == rho1  # same workload shape and fields
    assert (s0, s1) == (0, 1)  # each rank its own replica
    # the whole job: both replicas' SD-steps over the slowest rank's time
    assert bench.whole_job_value(n0, 10, 2, t0) == pytest.approx(2 * n0 * 10 / 2.0)


def test_single_rank_needs_no_process_group():
    assert bench.dist_max(3.5, 1) == 3.5
    bench.dist_barrier(1)
    assert bench.whole_job_value(360000, 20, 1, 0.5) == pytest.approx(360000 * 20 / 0.5)
