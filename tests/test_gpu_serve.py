"""Continuous-batching server: each request's result is the same served
alone and in a mix of overlapping requests; admission respects the device
memory budget; latency percentiles are reported beside throughput."""
import numpy as np
import pytest

import workloads
from paper_1310_1905_gb300.serve import Request, Server, poisson_requests

pytestmark = pytest.mark.gpu


def rhod_fn(m, t):
    return float(workloads.hydrostatic_rhod(np.array([m["z0"] + m["w"] * t]), 289.0, 7.5e-3, 101500.0)[0])


def requests(n, seed, rate=400.0, steps=(20, 60)):
    ms = workloads.ensemble_members(n, seed=seed, n_min=500, n_max=40000)
    return poisson_requests(ms, rate, steps, seed=seed, rhod_fn=rhod_fn)


def clone(r: Request, arrival=None) -> Request:
    return Request(rid=r.rid, member=dict(r.member), steps=r.steps,
                   arrival=r.arrival if arrival is None else arrival, rhod_of_t=r.rhod_of_t)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_result_same_alone_and_in_the_mix(precision):
    mix = requests(10, seed=3)
    target = mix[4]
    s_mix = Server(mem_budget_bytes=int(400e6), precision=precision)
    s_mix.run([clone(r) for r in mix])
    got_mix = {r.rid: r.result for r in s_mix.finished}[target.rid]
    s_mix.close()
    s_alone = Server(mem_budget_bytes=int(400e6), precision=precision)
    s_alone.run([clone(target, arrival=0.0)])
    got_alone = s_alone.finished[0].result
    s_alone.close()
    assert got_mix == got_alone  # bit-identical diagnostics
    assert got_alone["liquid"] >= 0.0 and got_alone["rv"] > 0.0


def test_admission_by_device_memory_and_latency_report():
    """The arena is sized by what the ensemble actually reserves
    (sdm_ens_memory): its reservation fits the budget, and requests wait
    for room."""
    reqs = requests(16, seed=5, rate=2000.0, steps=(10, 30))
    budget_sd = max(r.member["n_sd"] for r in reqs) * 2
    budget = budget_sd * 130
    srv = Server(mem_budget_bytes=budget, precision="mixed")
    assert srv.reserved_bytes <= budget and srv.max_sd >= max(r.member["n_sd"] for r in reqs)
    assert 100 < srv.bytes_per_sd < 140
    stats = srv.run(reqs)
    assert stats["served"] == 16
    assert srv.peak_resident_sd <= srv.max_sd
    assert stats["mean_queue_wait_s"] > 0.0  # some requests had to wait for room
    assert 0.0 < stats["p50_latency_s"] <= stats["p99_latency_s"]
    assert stats["sd_steps"] == sum(r.member["n_sd"] * r.steps for r in reqs)
    srv.close()
