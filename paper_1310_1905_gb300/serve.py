"""Continuous-batching server for parcel and box simulations.

Requests (a 0D member and a step count) arrive at any time.  At every step
boundary the server admits waiting requests in arrival order while the
device arena has room for their super-droplets, advances every resident
member with one batched step (sdm_ens_step), and retires the members that
have done their steps, returning their diagnostics.  Requests that arrive
while a step runs wait in the queue and join at the next boundary, so their
work overlaps with that of the requests already on the GPU.

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

BYTES_PER_SD = 120  # arena bytes per resident super-droplet (state, sort and scratch)


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


class Server:
    """Serves requests on one GPU with a fixed device-memory budget."""

    def __init__(self, mem_budget_bytes: int, max_members: int = 512, precision: str = "mixed",
                 opts: dict | None = None, dt: float = 1.0, graph: bool = True, keep_state: bool = False):
        self.max_sd = max(1024, int(mem_budget_bytes // BYTES_PER_SD))
        self.ens = Ensemble(dt=dt, precision=precision, max_sd=self.max_sd, max_members=max_members)
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
        self._retired_last = False

    def submit(self, req: Request):
        if req.member["n_sd"] > self.max_sd:
            raise ValueError("request larger than the whole device budget")
        self.queue.append(req)

    def _admit(self, now: float) -> bool:
        changed = False
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
            changed = True
        return changed

    def step(self, now: float) -> bool:
        """One server iteration at time ``now``; False when idle."""
        changed = self._admit(now)
        if not self.resident:
            return False
        rhod = {}
        for r in self.resident:
            if r.rhod_of_t is not None:
                rhod[r._mid] = float(r.rhod_of_t(r._t + 1.0))
        # a captured graph pays off only while membership stays the same
        self.ens.use_graph(self.graph and not changed and not self._retired_last)
        self.ens.step(self.opts, rhod=rhod)
        self.ens.wait()
        self.steps += 1
        self.sd_steps += self.resident_sd
        keep = []
        self._retired_last = False
        for r in self.resident:
            r._t += 1
            if r._t >= r.steps:
                self._retired_last = True
                r.result = diagnostics(self.ens, r._mid)
                if self.keep_state:
                    n = r.member["n_sd"]
                    r.result["state"] = {k: self.ens.attr(r._mid, k, n) for k in ("N", "rw2", "rd3", "kappa")}
                self.ens.remove(r._mid)
                self.resident_sd -= r.member["n_sd"]
                self.finished.append(r)
            else:
                keep.append(r)
        self.resident = keep
        return True

    def run(self, requests: list[Request], clock=time.perf_counter, max_wall: float = 600.0) -> dict:
        """Serve ``requests`` (arrival times relative to the start) until all
        are done; returns latency and throughput statistics."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = clock()
        k = 0
        while (k < len(pending) or self.queue or self.resident) and clock() - t0 < max_wall:
            now = clock() - t0
            while k < len(pending) and pending[k].arrival <= now:
                self.submit(pending[k])
                k += 1
            if not self.step(now):
                if k < len(pending):  # idle until the next arrival
                    time.sleep(max(0.0, min(0.01, pending[k].arrival - (clock() - t0))))
                continue
            tnow = clock() - t0
            for r in self.finished:
                if r.done < 0:
                    r.done = tnow
        wall = clock() - t0
        lat = np.array([r.done - r.arrival for r in self.finished]) if self.finished else np.zeros(1)
        wait = np.array([r.admitted - r.arrival for r in self.finished]) if self.finished else np.zeros(1)
        return dict(served=len(self.finished), wall_s=wall, sd_steps=self.sd_steps,
                    sd_steps_per_s=self.sd_steps / wall if wall > 0 else 0.0, steps=self.steps,
                    p50_latency_s=float(np.percentile(lat, 50)), p99_latency_s=float(np.percentile(lat, 99)),
                    mean_queue_wait_s=float(wait.mean()))

    def close(self):
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
