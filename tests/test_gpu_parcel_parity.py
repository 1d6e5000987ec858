"""Batched and served forms against the oracle (FP64 mode): multiplicities
bit-exact, radii and the parcel's theta and r_v within 1e-12, or, for a
parcel that crosses cloud base, within the oracle's own spread when its
theta moves, after every step, by as many ulps as the GPU's T and rho_vs
differ from the oracle's (measured; near activation the growth rate is a
small difference of nearly equal vapour densities, and the root moves by
more than 1e-12 for a few ulps of the ambient state; the two sides' rounding
differs at every step, not only at the start), and nearly all within the
spread of that difference at the start alone.

- parcel members (the parcel framework of Sec. 5.2.1) rising through cloud
  base in a mix with a box, 30 steps with rho_d changing every step, against
  the oracle's parcel mode (a new rho_d sets dV = m_d / rho_d);
- one request served through the continuous-batching Server among other
  requests, against the oracle's parcel run of the same member;
- a member of 1e5 super-droplets, whose condensation spans many tiles and
  whose pairing goes through the radix-sorted path the small members do not
  reach;
- the Long (1974) kernel in ensemble members whose drops sit where the
  efficiency is neither its floor nor one.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import theta_ulps
from paper_1310_1905_gb300 import sdm
from paper_1310_1905_gb300.ensemble import Ensemble
from paper_1310_1905_gb300.serve import Request, Server

pytestmark = pytest.mark.gpu

ALL0D = dict(adve=0, sedi=0, cond=1, coal=1, sstp_cond=10, sstp_coal=10)


def rhod_at(z):
    return float(workloads.hydrostatic_rhod(np.array([z]), 289.0, 7.5e-3, 101500.0)[0])


def oracle_of(m, kernel="geometric"):
    """The oracle's 0D run of an ensemble member (volume dV kept as dx)."""
    cfg = dict(nx=0, ny=0, nz=0, dx=m["dV"], dy=1.0, dz=1.0, dt=1.0, sd_conc=m["n_sd"], kernel=kernel,
               init_dist=m.get("init_dist", "lognormal"), modes=m.get("modes", []), seed=m["seed"], physics=1,
               exp_mean_volume=m.get("exp_mean_volume", 0.0), exp_n0=m.get("exp_n0", 0.0))
    o = oracle.Oracle(cfg)
    o.init(np.array([m["th"]]), np.array([m["rv"]]), np.array([m["rhod"]]))
    return o


def gpu_ulps(m):
    """theta ulps matching the GPU's T and rho_vs at the member's initial
    state: a one-cell context on the same inputs (the ensemble's condensation
    calls the same thermodynamics routine as sdm_diag_ambient)."""
    o = oracle_of(m)
    p = sdm.Particles(o.cfg, np.array([m["th"]]), np.array([m["rv"]]), np.array([m["rhod"]]))
    k = theta_ulps(p.diag_ambient("T")[0], p.diag_ambient("rho_vs")[0], m["th"], m["rv"], m["rhod"])
    p.close()
    return k


def spread_of(m, run, ulps, kernel="geometric", every_step=False):
    """The oracle's run (run(o, after) advances it, calling after() after
    every step) from the member's initial state, and with theta moved by
    ulps ulps: at the start (both signs), or (every_step) after every step
    (both signs, and four random-sign sequences).  The base run and the
    largest move of r_w^2, theta and r_v."""
    base = oracle_of(m, kernel)
    run(base, lambda: None)
    ref = base.state.sorted_by_uid().rw2
    sp, sth, srv = np.zeros_like(ref), 0.0, 0.0
    cases = [(np.inf, None), (-np.inf, None)] + ([(None, k) for k in range(4)] if every_step else [])
    for d, seed in cases:
        o = oracle_of(m, kernel)
        rng = np.random.default_rng(seed)

        def nudge(o=o, d=d, rng=rng):
            dd = d if d is not None else (np.inf if rng.uniform() < 0.5 else -np.inf)
            for _ in range(ulps):
                o.th[0] = np.nextafter(o.th[0], dd)

        if not every_step:
            nudge()
        run(o, nudge if every_step else (lambda: None))
        sp = np.maximum(sp, np.abs(o.state.sorted_by_uid().rw2 - ref))
        sth, srv = max(sth, abs(o.th[0] - base.th[0])), max(srv, abs(o.rv[0] - base.rv[0]))
    return base, sp, sth, srv


def check_envelopes(got, m, run, ulps, label, kernel="geometric"):
    """got within the per-step spread everywhere and within the start spread
    for all but 2 % of the droplets; returns the oracle's base run and the
    fraction of droplets beyond 1e-12."""
    o, sp, sth, srv = spread_of(m, run, ulps, kernel, every_step=True)
    wide = check_member(got, m, o, sp, sth, srv, label=label)
    _, sp0, _, _ = spread_of(m, run, ulps, kernel)
    r = o.state.sorted_by_uid()
    outside = (np.abs(got["rw2"] - r.rw2) > np.maximum(1e-12 * r.rw2, sp0)).mean()
    print(f"{label}: {outside * 100:.2f} % beyond the start-perturbation spread")
    assert outside <= 0.02
    return o, wide


def check_member(got, m, o, spread=None, sth=0.0, srv=0.0, label=""):
    """got: N, rw2, rd3, kappa (id order) and th, rv of a GPU member."""
    r = o.state.sorted_by_uid()
    assert np.array_equal(got["N"], r.N), label
    for k in ("rd3", "kappa"):
        np.testing.assert_allclose(got[k], getattr(r, k), rtol=1e-12, atol=0, err_msg=k)
    tol = 1e-12 * r.rw2 if spread is None else np.maximum(1e-12 * r.rw2, spread)
    err = np.abs(got["rw2"] - r.rw2)
    assert (err <= tol).all(), f"{label}: rw2 {(err > tol).sum()} of {err.size} outside; worst rel " \
                               f"{np.max(err / r.rw2):.3e}"
    assert abs(got["th"] - o.th[0]) <= max(1e-12 * o.th[0], sth)
    assert abs(got["rv"] - o.rv[0]) <= max(1e-12 * o.rv[0], srv)
    wide = (err > 1e-12 * r.rw2).mean()
    print(f"{label}: worst rel {np.max(err / r.rw2):.2e}, {wide * 100:.1f} % beyond 1e-12")
    return wide


def member_state(ens, mid, n):
    th, rv = ens.fields([mid])
    out = {k: ens.attr(mid, k, n) for k in ("N", "rw2", "rd3", "kappa")}
    out.update(th=th[0], rv=rv[0])
    return out


def parcel_member(n_sd, seed, z0=750.0, rv=7.5e-3, modes=None):
    return dict(n_sd=n_sd, dV=1.0, th=289.0, rv=rv, rhod=rhod_at(z0), seed=seed,
                modes=modes or workloads.AEROSOL_BIMODAL[:1])


def test_parcel_members_match_oracle_parcel_mode():
    # two parcels (2 and 4 m/s from 750 m: through cloud base, about 790 m,
    # within the run), a supersaturated box whose drops grow and collide, and
    # a box of equal-multiplicity drops (exponential volumes, mean radius
    # 12 um) whose collisions leave zeros: they are recycled at the beginning
    # of the next step, before its condensation
    mv = 4.0 / 3.0 * np.pi * (12e-6) ** 3
    ms = [parcel_member(1500, 41), parcel_member(700, 42, modes=workloads.AEROSOL_BIMODAL),
          dict(parcel_member(900, 43, rv=1.2e-2), dV=1e6),
          dict(n_sd=600, dV=1e6, th=289.0, rv=8.5e-3, rhod=rhod_at(750.0), seed=44, init_dist="exponential",
               exp_mean_volume=mv, exp_n0=1e8)]
    w = [2.0, 4.0, 0.0, 0.0]
    ens = Ensemble(max_sd=1 << 14, max_members=4)
    ids = [ens.add(m) for m in ms]
    for k in range(1, 31):
        rh = {ids[q]: rhod_at(750.0 + w[q] * k) for q in range(len(ms)) if w[q] > 0}
        ens.step(ALL0D, rhod=rh)
        ens.wait()
    orcs = []
    for q, m in enumerate(ms):
        def run(o, after, q=q):
            for k in range(1, 31):
                o.parcel_step(ALL0D, rhod_at(750.0 + w[q] * k) if w[q] > 0 else None)
                after()
        ulps = gpu_ulps(m)
        o, wide = check_envelopes(member_state(ens, ids[q], m["n_sd"]), m, run, ulps,
                                  label=f"member {q} ({ulps} theta ulps)")
        assert wide < 0.25
        orcs.append(o)
    assert orcs[1].rhod[0] < ms[1]["rhod"] * 0.99  # the parcel rose and expanded
    assert abs(orcs[1].rv[0] - 7.5e-3) > 1e-5        # and condensed
    assert orcs[3].stats.n_recycled > 10
    st = ens.stats()
    assert st["n_coll"] > 0 and st["n_coll"] == sum(o.stats.n_coll for o in orcs)
    assert st["n_recycled"] == sum(o.stats.n_recycled for o in orcs)


def test_served_request_matches_oracle():
    def rhod_fn(m, t):
        return rhod_at(m["z0"] + m["w"] * t)

    ms = workloads.ensemble_members(6, seed=9, n_min=300, n_max=3000, parcel_fraction=1.0)
    reqs = []
    for i, m in enumerate(ms):
        f = (lambda mm: (lambda tt: rhod_fn(mm, tt)))(m)
        mem = {k: v for k, v in m.items() if k not in ("w", "z0")}
        reqs.append(Request(rid=i, member=mem, steps=25 + 3 * i, arrival=0.002 * i, rhod_of_t=f))
    srv = Server(mem_budget_bytes=int(50e6), precision="fp64", keep_state=True)
    stats = srv.run(reqs)
    srv.close()
    assert stats["served"] == len(reqs)
    target = reqs[3]
    got = {r.rid: r.result for r in srv.finished}[target.rid]
    m = target.member

    def run(o, after):
        for k in range(1, target.steps + 1):
            o.parcel_step(ALL0D, rhod_fn(ms[3], float(k)))
            after()

    ulps = gpu_ulps(m)
    o, wide = check_envelopes(dict(got["state"], th=got["th"], rv=got["rv"]), m, run, ulps,
                              label=f"served request ({ulps} theta ulps)")
    assert wide < 0.25
    if wide == 0.0:
        np.testing.assert_allclose(got["liquid"], 4.0 / 3.0 * np.pi * 1000.0 * o.moments(True, 1e-6, 1.0, 3)[0],
                                   rtol=1e-12)
        np.testing.assert_allclose(got["cloud_conc"], o.moments(True, 1e-6, 25e-6, 0)[0], rtol=1e-12)


def test_large_member_matches_oracle():
    m = dict(n_sd=100_000, dV=1e6, th=289.0, rv=9.0e-3, rhod=rhod_at(1200.0), seed=21,
             modes=workloads.AEROSOL_BIMODAL[:1])
    ens = Ensemble(max_sd=1 << 17, max_members=2)
    small = ens.add(parcel_member(500, 22))
    mid = ens.add(m)
    o = oracle_of(m)
    for _ in range(3):
        ens.step(ALL0D)
        ens.wait()
        o.parcel_step(ALL0D, None)
    check_member(member_state(ens, mid, m["n_sd"]), m, o, label="1e5-SD member")
    assert o.stats.n_coll > 0
    assert ens.attr(small, "N", 500).min() >= 1


def test_long_kernel_ensemble_members_match_oracle():
    """Drops of 3-50 um (exponential volumes, mean radius 12 um): the
    efficiency 4.5e8 R^2 (1 - 3e-6/r) is between its floor and one for most
    pairs."""
    mv = 4.0 / 3.0 * np.pi * (12e-6) ** 3
    ms = [dict(n_sd=n, dV=1e6, th=289.0, rv=7.5e-3, rhod=1.0, seed=s, init_dist="exponential",
               exp_mean_volume=mv, exp_n0=5e8) for n, s in ((2000, 51), (300, 52))]
    ens = Ensemble(kernel="long", max_sd=1 << 13, max_members=4)
    ids = [ens.add(m) for m in ms]
    orcs = [oracle_of(m, kernel="long") for m in ms]
    r = np.sqrt(orcs[0].state.rw2)
    assert ((r > 3e-6) & (r < 50e-6)).mean() > 0.8
    opts = dict(adve=0, sedi=0, cond=0, coal=1, sstp_cond=1, sstp_coal=5)
    for _ in range(30):
        ens.step(opts)
        ens.wait()
        for o in orcs:
            o.parcel_step(opts, None)
    for mid, m, o in zip(ids, ms, orcs):
        check_member(member_state(ens, mid, m["n_sd"]), m, o, label="Long kernel member")
    assert sum(o.stats.n_coll for o in orcs) > 10
