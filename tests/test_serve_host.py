"""The serving loop's host logic (paper_1310_1905_gb300/serve.py) on the CPU,
over a stand-in for the batched ensemble that records what the server asks
of it: admission in arrival order within the arena's super-droplet budget
and member count, first come first served (a request that does not fit
holds back the ones behind it), retirement after each request's own step
count with its diagnostics, each parcel's rho_d from its own clock, and a
captured graph only while membership stays the same."""
import numpy as np
import pytest

import paper_1310_1905_gb300.serve as serve

BYTES_PER_SD, FIXED = 120, 1_000_000


class FakeEnsemble:
    """Holds members' sizes and counts steps; device work is not simulated."""
    log = []

    def __init__(self, max_sd, max_members, **kw):
        self.max_sd, self.max_members = max_sd, max_members
        self.members, self.next_id, self.graph = {}, 0, None
        self.steps = []
        FakeEnsemble.log.append(self)

    def memory(self):
        return dict(device_bytes=FIXED + BYTES_PER_SD * self.max_sd)

    def add(self, m):
        assert sum(self.members.values()) + m["n_sd"] <= self.max_sd
        assert len(self.members) < self.max_members
        mid = self.next_id
        self.next_id += 1
        self.members[mid] = m["n_sd"]
        return mid

    def remove(self, mid):
        del self.members[mid]

    def use_graph(self, on):
        self.graph = on

    def step(self, opts, rhod=None):
        self.steps.append(dict(members=dict(self.members), rhod=dict(rhod or {}), graph=self.graph))

    def wait(self):
        pass

    def fields(self, mids):
        return np.array([289.0]), np.array([7.5e-3])

    def moments(self, mids, wet, rmin, rmax, k):
        return np.array([1.0e8])

    def attr(self, mid, k, n):
        return np.zeros(n)

    def close(self):
        pass


@pytest.fixture()
def fake(monkeypatch):
    FakeEnsemble.log.clear()
    monkeypatch.setattr(serve, "Ensemble", FakeEnsemble)
    return FakeEnsemble


def req(rid, n_sd, steps, arrival, rhod=None):
    return serve.Request(rid=rid, member=dict(n_sd=n_sd), steps=steps, arrival=arrival, rhod_of_t=rhod)


def test_capacity_comes_from_the_probe_reservations(fake):
    cap, per_sd, fixed = serve.arena_capacity(FIXED + BYTES_PER_SD * 50_000, max_members=8)
    assert per_sd == BYTES_PER_SD and fixed == FIXED and cap == 50_000


def test_admission_budget_order_and_retirement(fake):
    s = serve.Server(FIXED + BYTES_PER_SD * 10_000, max_members=4)
    assert s.max_sd == 10_000 and s.reserved_bytes <= s.budget
    # 6000 + 3000 fit; 5000 does not and holds back the 500 behind it
    for r in (req(0, 6000, 2, 0.0), req(1, 3000, 3, 0.0), req(2, 5000, 1, 0.0), req(3, 500, 1, 0.0)):
        s.submit(r)
    assert s.step(0.0)
    e = s.ens
    assert sorted(e.steps[-1]["members"].values()) == [3000, 6000]
    assert s.step(1.0)  # step 1 done; nothing else fits, step 2 of the same two
    assert not s.finished and sorted(e.steps[-1]["members"].values()) == [3000, 6000]
    assert s.step(2.0)  # request 0 has run its two steps and retires; 3000 + 5000 fit now, and 500 too
    assert {r.rid for r in s.finished} == {0}
    assert sorted(e.steps[-1]["members"].values()) == [500, 3000, 5000]
    while s.step(2.0):
        assert sum(e.steps[-1]["members"].values()) <= 10_000
    s.close()
    assert sorted(r.rid for r in s.finished) == [0, 1, 2, 3]
    for r in s.finished:
        assert r.admitted >= r.arrival and r.done >= r.admitted
        assert r.result["liquid"] > 0 and r.result["th"] == 289.0
    assert s.peak_resident_sd <= 10_000
    # every member took exactly its own step count
    counts = {}
    for st in e.steps:
        for mid in st["members"]:
            counts[mid] = counts.get(mid, 0) + 1
    assert sorted(counts.values()) == sorted(r.steps for r in s.finished)


def test_member_limit_and_future_arrivals(fake):
    s = serve.Server(FIXED + BYTES_PER_SD * 100_000, max_members=2)
    for r in (req(0, 100, 3, 0.0), req(1, 100, 3, 0.0), req(2, 100, 1, 0.0), req(3, 100, 1, 5.0)):
        s.submit(r)
    s.step(0.0)
    assert len(s.ens.steps[-1]["members"]) == 2  # the member table is full
    s.step(1.0)
    s.step(2.0)
    s.step(3.0)  # the first two retire here; request 2 joins, request 3 has not arrived
    assert len(s.resident) == 1 and s.resident[0].rid == 2
    s.close()


def test_parcels_take_rho_d_from_their_own_clock_and_graphs_follow_membership(fake):
    s = serve.Server(FIXED + BYTES_PER_SD * 100_000, max_members=8)
    a = req(0, 100, 4, 0.0, rhod=lambda t: 1.0 - 0.01 * t)
    b = req(1, 100, 4, 0.0)
    c = req(2, 100, 2, 1.5, rhod=lambda t: 2.0 - 0.1 * t)
    for r in (a, b, c):
        s.submit(r)
    for t in (0.0, 1.0, 2.0, 3.0, 4.0, 5.0):
        s.step(t)
    s.close()
    steps = s.ens.steps
    # parcel a: rho_d at its own times 1, 2, 3, 4; parcel c joined later, from its own t = 1
    ra = [st["rhod"][a._mid] for st in steps if a._mid in st["rhod"]]
    assert ra == pytest.approx([0.99, 0.98, 0.97, 0.96])
    rc = [st["rhod"][c._mid] for st in steps if c._mid in st["rhod"]]
    assert rc == pytest.approx([1.9, 1.8])
    assert b._mid not in steps[0]["rhod"]  # boxes keep their rho_d
    # a graph only where the previous step had the same members
    for prev, cur in zip(steps, steps[1:]):
        assert cur["graph"] == (set(prev["members"]) == set(cur["members"]))
    assert steps[0]["graph"] is False


def test_requests_larger_than_the_arena_are_refused(fake):
    s = serve.Server(FIXED + BYTES_PER_SD * 5_000, max_members=4)
    with pytest.raises(ValueError):
        s.submit(req(0, 6_000, 1, 0.0))
    s.close()
