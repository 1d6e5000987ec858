"""Continuous-batching server for parcel and box simulations.

Requests (a 0D member and a step count) arrive at any time.  The server
keeps one batched step (sdm_ens_step, a captured graph while membership is
unchanged) in flight: while it runs on the GPU the host polls arrivals,
queues them and prepares the next step's rho_d; when it completes, the
members that have done their steps are retired with their diagnostics, the
waiting requests are admitted in arrival order while the arena has room for
their super-droplets, and the next step is launched.  Requests that arrive
while a step runs join at the next boundary, so their work overlaps with
that of the requests already on the GPU.

Admission is by device memory: the arena's capacity comes from what the
ensemble actually reserves (sdm_ens_memory), measured on two small probe
arenas (bytes per super-droplet and the fixed part) and checked on the real
one against the budget.

Each member keeps its own seed, step count and clock (a parcel's rho_d
follows its own elapsed time), so a request's result does not depend on what
else is being served.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from .ensemble import Ensemble


@dataclasses.dataclass
class Request:
    rid: int
    member: dict            # ensemble member dict (n_sd, dV, th, rv, rhod, modes, seed)
    steps: int
    arrival: float          # seconds on the server clock
    rhod_of_t: object = None  # callable t -> rho_d (parcels), None for boxes
    admitted: float = -1.0
    done: float = -1.0
    result: dict | None = None
    _mid: int = -1
    _t: int = 0


def diagnostics(ens: Ensemble, mid: int) -> dict:
    th, rv = ens.fields([mid])
    m0 = ens.moments([mid], True, 1e-6, 25e-6, 0)[0]
    m1 = ens.moments([mid], True, 1e-6, 25e-6, 1)[0]
    m3 = ens.moments([mid], True, 1e-6, 1.0, 3)[0]
    return dict(th=float(th[0]), rv=float(rv[0]), cloud_conc=float(m0),
                cloud_mean_radius=float(m1 / m0) if m0 > 0 else 0.0,
                liquid=float(4.0 / 3.0 * np.pi * 1000.0 * m3))


def arena_capacity(budget_bytes: int, max_members: int, **ens_kw) -> tuple[int, float, float]:
    """The most super-droplets an arena may hold within budget_bytes: the
    reservation of two probe arenas (2^16 and 2^17 super-droplets, the same
    member capacity) gives the bytes per super-droplet and the fixed part."""
    sizes = (1 << 16, 1 << 17)
    got = []
    for n in sizes:
        e = Ensemble(max_sd=n, max_members=max_members, **ens_kw)
        got.append(e.memory()["device_bytes"])
        e.close()
    per_sd = (got[1] - got[0]) / (sizes[1] - sizes[0])
    fixed = got[0] - per_sd * sizes[0]
    return int((budget_bytes - fixed) // per_sd), per_sd, fixed


class Server:
    """Serves requests on one GPU with a fixed device-memory budget."""

    def __init__(self, mem_budget_bytes: int, max_members: int = 512, precision: str = "mixed",
                 opts: dict | None = None, dt: float = 1.0, graph: bool = True, keep_state: bool = False):
        kw = dict(dt=dt, precision=precision)
        cap, self.bytes_per_sd, self.fixed_bytes = arena_capacity(mem_budget_bytes, max_members, **kw)
        if cap < 1024:
            raise ValueError("the memory budget holds fewer than 1024 super-droplets")
        for _ in range(8):  # the arena's own reservation must fit the budget
            self.ens = Ensemble(max_sd=cap, max_members=max_members, **kw)
            self.reserved_bytes = self.ens.memory()["device_bytes"]
            if self.reserved_bytes <= mem_budget_bytes:
                break
            self.ens.close()
            cap = int(cap * 0.99)
        else:
            raise RuntimeError("no arena fits the memory budget")
        self.max_sd = cap
        self.budget = mem_budget_bytes
        self.max_members = max_members
        self.opts = opts or dict(adve=0, sedi=0, cond=1, coal=1, RH_max=44.0, sstp_cond=10, sstp_coal=10)
        self.graph = graph
        self.keep_state = keep_state  # copy each finished member's super-droplets into its result
        self.queue: collections.deque[Request] = collections.deque()
        self.resident: list[Request] = []
        self.finished: list[Request] = []
        self.resident_sd = 0
        self.peak_resident_sd = 0
        self.sd_steps = 0
        self.steps = 0
        self.in_flight = False
        self._membership_changed = True

    def submit(self, req: Request):
        if req.member["n_sd"] > self.max_sd:
            raise ValueError("request larger than the whole device budget")
        self.queue.append(req)

    def _admit(self, now: float):
        while self.queue and self.queue[0].arrival <= now:
            r = self.queue[0]
            if self.resident_sd + r.member["n_sd"] > self.max_sd or len(self.resident) >= self.max_members:
                break  # wait for room (requests are served in order)
            self.queue.popleft()
            r._mid = self.ens.add(r.member)
            r.admitted = now
            self.resident.append(r)
            self.resident_sd += r.member["n_sd"]
            self.peak_resident_sd = max(self.peak_resident_sd, self.resident_sd)
            self._membership_changed = True

    def _complete(self, now: float):
        """Wait for the step in flight; advance its members' clocks and
        retire those that have done their steps."""
        self.ens.wait()
        self.in_flight = False
        keep = []
        for r in self.resident:
            r._t += 1
            if r._t >= r.steps:
                r.result = diagnostics(self.ens, r._mid)
                if self.keep_state:
                    n = r.member["n_sd"]
                    r.result["state"] = {k: self.ens.attr(r._mid, k, n) for k in ("N", "rw2", "rd3", "kappa")}
                self.ens.remove(r._mid)
                self.resident_sd -= r.member["n_sd"]
                r.done = now
                self.finished.append(r)
                self._membership_changed = True
            else:
                keep.append(r)
        self.resident = keep

    def step(self, now: float, clock=None) -> bool:
        """One server iteration: finish the step in flight (if any), retire,
        admit, launch the next step without waiting for it.  False when
        nothing is resident or in flight."""
        if self.in_flight:
            self._complete(clock() if clock else now)
            now = clock() if clock else now
        self._admit(now)
        if not self.resident:
            return False
        rhod = {}
        for r in self.resident:
            if r.rhod_of_t is not None:
                rhod[r._mid] = float(r.rhod_of_t(r._t + 1.0))
        # a captured graph pays off only while membership stays the same
        self.ens.use_graph(self.graph and not self._membership_changed)
        self._membership_changed = False
        self.ens.step(self.opts, rhod=rhod)
        self.in_flight = True
        self.steps += 1
        self.sd_steps += self.resident_sd
        return True

    def run(self, requests: list[Request], clock=time.perf_counter, max_wall: float = 1800.0) -> dict:
        """Serve ``requests`` (arrival times relative to the start) until all
        are done; returns latency and throughput statistics.  Between the
        launch of a step and its completion the host takes the arrivals."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = clock()
        now = lambda: clock() - t0  # noqa: E731
        k = 0
        while (k < len(pending) or self.queue or self.resident or self.in_flight) and now() < max_wall:
            while k < len(pending) and pending[k].arrival <= now():
                self.submit(pending[k])
                k += 1
            if not self.step(now(), now):
                if k < len(pending):  # idle until the next arrival
                    time.sleep(max(0.0, min(0.01, pending[k].arrival - now())))
        if self.in_flight:
            self._complete(now())
        wall = now()
        lat = np.array([r.done - r.arrival for r in self.finished]) if self.finished else np.zeros(1)
        wait = np.array([r.admitted - r.arrival for r in self.finished]) if self.finished else np.zeros(1)
        return dict(served=len(self.finished), wall_s=wall, sd_steps=self.sd_steps,
                    sd_steps_per_s=self.sd_steps / wall if wall > 0 else 0.0, steps=self.steps,
                    p50_latency_s=float(np.percentile(lat, 50)), p99_latency_s=float(np.percentile(lat, 99)),
                    mean_queue_wait_s=float(wait.mean()), peak_resident_sd=self.peak_resident_sd,
                    arena_sd=self.max_sd, arena_bytes=self.reserved_bytes, bytes_per_sd=self.bytes_per_sd)

    def close(self):
        if self.in_flight:
            self.ens.wait()
            self.in_flight = False
        self.ens.close()


def poisson_requests(members: list[dict], rate_per_s: float, steps_range=(300, 1800), seed: int = 0,
                     rhod_fn=None) -> list[Request]:
    """Requests with Poisson arrivals at ``rate_per_s``; step counts uniform
    in ``steps_range``; ``rhod_fn(member, t)`` gives parcels their rho_d."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i, m in enumerate(members):
        t += rng.exponential(1.0 / rate_per_s)
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        f = None
        if rhod_fn is not None and m.get("w", 0.0) > 0.0:
            f = (lambda mm: (lambda tt: rhod_fn(mm, tt)))(m)
        mem = {k: v for k, v in m.items() if k not in ("w", "z0")}
        out.append(Request(rid=i, member=mem, steps=steps, arrival=t, rhod_of_t=f))
    return out
