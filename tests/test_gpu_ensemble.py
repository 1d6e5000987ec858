"""Batched ensembles of 0D members (sdm_ens_* through the C ABI): each
member matches the same box run as a single context and as the oracle,
is bit-identical alone and in a mix, under graph replay, and across the
repacking that follows a removal."""
import math

import numpy as np
import pytest

import oracle
import workloads
from paper_1310_1905_gb300 import sdm
from paper_1310_1905_gb300.ensemble import Ensemble

pytestmark = pytest.mark.gpu

ALL0D = dict(adve=0, sedi=0, cond=1, coal=1, sstp_cond=10, sstp_coal=10)
RHOD = float(workloads.hydrostatic_rhod(np.array([1200.0]), 289.0, 7.5e-3, 101500.0)[0])


def member(n_sd, seed, dV=1e6, rv=8.0e-3, modes=None):
    return dict(n_sd=n_sd, dV=dV, th=289.0, rv=rv, rhod=RHOD, seed=seed,
                modes=modes or workloads.AEROSOL_BIMODAL[:1])


def box_cfg(m):
    side = round(m["dV"] ** (1.0 / 3.0))
    assert side ** 3 == m["dV"]
    return dict(nx=0, ny=0, nz=0, dx=float(side), dy=float(side), dz=float(side), dt=1.0, sd_conc=m["n_sd"],
                kernel="geometric", init_dist="lognormal", modes=m["modes"], seed=m["seed"], physics=1)


def state(ens, mid, n):
    return {k: ens.attr(mid, k, n) for k in ("N", "rw2", "rd3", "kappa")}


def test_member_matches_single_context_and_oracle():
    ms = [member(300, 1), member(2000, 2, dV=8.0, rv=7.8e-3), member(5000, 3, dV=1.0)]
    ens = Ensemble(max_sd=1 << 16, max_members=8)
    ids = [ens.add(m) for m in ms]
    singles, oracles = [], []
    for m in ms:
        cfg = box_cfg(m)
        f = lambda v: np.array([v])
        singles.append(sdm.Particles(cfg, f(m["th"]), f(m["rv"]), f(m["rhod"])))
        o = oracle.Oracle(cfg)
        o.init(f(m["th"]), f(m["rv"]), f(m["rhod"]))
        oracles.append(o)
    th = [np.array([m["th"]]) for m in ms]
    rv = [np.array([m["rv"]]) for m in ms]
    for _ in range(6):
        ens.step(ALL0D)
        ens.wait()
        for k, (p, o) in enumerate(zip(singles, oracles)):
            p.step_sync(ALL0D, th[k], rv[k])
            p.step_async(ALL0D)
            p.wait()
            o.step_sync(ALL0D)
            o.step_async(ALL0D)
    e_th, e_rv = ens.fields(ids)
    for k, m in enumerate(ms):
        g = state(ens, ids[k], m["n_sd"])
        s = singles[k].state()
        r = oracles[k].state.sorted_by_uid()
        assert np.array_equal(g["N"], s["N"]) and np.array_equal(g["N"], r.N)
        np.testing.assert_allclose(g["rw2"], s["rw2"], rtol=1e-12)
        np.testing.assert_allclose(g["rw2"], r.rw2, rtol=1e-12)
        np.testing.assert_allclose([e_th[k], e_rv[k]], [oracles[k].th[0], oracles[k].rv[0]], rtol=1e-12)
    assert abs(e_rv[0] - 8.0e-3) > 1e-6  # condensation did something


def test_golovin_members_bit_exact_vs_oracle():
    w = workloads.golovin_box(seed=4)
    m = dict(n_sd=8192, dV=1e6, th=300.0, rv=0.01, rhod=1.0, seed=4, init_dist="exponential",
             exp_mean_volume=w.cfg["exp_mean_volume"], exp_n0=w.cfg["exp_n0"])
    ens = Ensemble(kernel="golovin", golovin_b=1500.0, max_sd=1 << 15, max_members=4)
    mid = ens.add(m)
    o = oracle.Oracle(w.cfg)
    o.init(w.th, w.rv, w.rhod)
    opts = dict(adve=0, sedi=0, cond=0, coal=1, sstp_cond=1, sstp_coal=1)
    for _ in range(300):
        ens.step(opts)
        ens.wait()
        o.step_async(opts)
    r = o.state.sorted_by_uid()
    assert np.array_equal(ens.attr(mid, "N", 8192), r.N)
    np.testing.assert_allclose(ens.attr(mid, "rw2", 8192), r.rw2, rtol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_alone_and_in_the_mix_bit_identical(precision):
    x = member(3000, 11)
    others = [member(n, s) for n, s in ((200, 1), (70000, 2), (9000, 3), (1500, 4))]
    alone = Ensemble(precision=precision, max_sd=1 << 17, max_members=8)
    a = alone.add(x)
    mix = Ensemble(precision=precision, max_sd=1 << 17, max_members=8)
    ids = [mix.add(m) for m in others[:2]]
    b = mix.add(x)
    ids += [mix.add(m) for m in others[2:]]
    for _ in range(5):
        for e in (alone, mix):
            e.step(ALL0D)
            e.wait()
    sa, sb = state(alone, a, 3000), state(mix, b, 3000)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(alone.fields([a])[1], mix.fields([b])[1])


def test_graph_replay_and_repacking():
    ms = [member(n, s) for n, s in ((4000, 5), (300, 6), (12000, 7), (800, 8))]
    ref = Ensemble(max_sd=1 << 16, max_members=8)
    rid = [ref.add(m) for m in ms]
    g = Ensemble(max_sd=1 << 16, max_members=8)
    gid = [g.add(m) for m in ms]
    g.use_graph(True)
    for step in range(6):
        if step == 3:  # retire one member: the others are repacked and carry on
            ref.remove(rid[1])
            g.remove(gid[1])
        for e in (ref, g):
            e.step(ALL0D)
            e.wait()
    # the same member in a third ensemble that never held member 1
    solo = Ensemble(max_sd=1 << 16, max_members=8)
    sid = solo.add(ms[2])
    for _ in range(6):
        solo.step(ALL0D)
        solo.wait()
    for k in (0, 2, 3):
        assert np.array_equal(state(ref, rid[k], ms[k]["n_sd"])["rw2"], state(g, gid[k], ms[k]["n_sd"])["rw2"])
    assert np.array_equal(state(g, gid[2], 12000)["N"], state(solo, sid, 12000)["N"])
    assert ref.members()[0] == [rid[0], rid[2], rid[3]]


def test_large_member_conserves_liquid_and_counts():
    ens = Ensemble(precision="mixed", max_sd=1 << 21, max_members=4)
    mid = ens.add(member(1_000_000, 21, rv=9.0e-3))
    n = 1_000_000
    for _ in range(3):
        ens.step(ALL0D)
        ens.wait()
    r3_0 = (ens.attr(mid, "N", n).astype(float) * ens.attr(mid, "rw2", n) ** 1.5).sum()
    N0 = ens.attr(mid, "N", n).astype(np.int64).sum()
    ens.step(dict(ALL0D, cond=0))
    ens.wait()
    N1 = ens.attr(mid, "N", n).astype(np.int64)
    r3_1 = (N1.astype(float) * ens.attr(mid, "rw2", n) ** 1.5).sum()
    assert r3_1 == pytest.approx(r3_0, rel=1e-11)
    assert (N1 >= 0).all() and N1.sum() <= N0
    st = ens.stats()
    assert st["n_pairs"] > 0


def test_parcel_keeps_dry_air_mass():
    ens = Ensemble(max_sd=1 << 15, max_members=4)
    mid = ens.add(member(2000, 31))
    z = np.arange(1, 6) * 2.0  # 2 m/s updraft, 1 s steps
    rh = workloads.hydrostatic_rhod(1200.0 + z, 289.0, 7.5e-3, 101500.0)
    m0 = ens.moments([mid], False, 0.0, 1.0, 0)[0]   # dry particles per kg of dry air
    for r in rh:
        ens.step(ALL0D, rhod={mid: float(r)})
        ens.wait()
    m1 = ens.moments([mid], False, 0.0, 1.0, 0)[0]
    # coalescence of haze is negligible here: the number per unit dry-air mass stays
    assert m1 == pytest.approx(m0, rel=1e-3)
    th, rv = ens.fields([mid])
    assert rv[0] < 8.0e-3  # the rising parcel condenses


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_keeps_state_and_picks_a_launchable_shape(precision):
    """The autotuner times condensation tile/block shapes on the resident
    state: it must leave that state and the counters as they were, skip the
    block sizes the kernel's register count rules out, and leave the
    ensemble stepping as before (two ensembles, one tuned, stay within the
    rounding of a different tile split)."""
    ms = [member(n, s) for n, s in ((30000, 21), (700, 22), (120000, 23))]
    tuned, plain = (Ensemble(precision=precision, max_sd=1 << 18, max_members=4) for _ in range(2))
    tid = [tuned.add(m) for m in ms]
    pid = [plain.add(m) for m in ms]
    for e in (tuned, plain):
        e.step(ALL0D)
        e.wait()
    before = [state(tuned, i, m["n_sd"]) for i, m in zip(tid, ms)]
    stats_before = tuned.stats()
    tile, threads, pair_threads = tuned.autotune(ALL0D)
    assert tile in (128, 256, 512, 1024, 2048) and threads in (128, 256, 512)
    assert pair_threads in (64, 128, 256, 512)
    after = [state(tuned, i, m["n_sd"]) for i, m in zip(tid, ms)]
    for b, a in zip(before, after):
        for k in b:
            assert np.array_equal(b[k], a[k]), k
    assert tuned.stats() == stats_before
    for _ in range(3):
        for e in (tuned, plain):
            e.step(ALL0D)
            e.wait()
    for i, j, m in zip(tid, pid, ms):
        a, b = state(tuned, i, m["n_sd"]), state(plain, j, m["n_sd"])
        assert np.isfinite(a["rw2"]).all()
        if precision == "fp64":  # FP32 accept decisions may flip under rounding changes
            assert np.array_equal(a["N"], b["N"])
            # another tile split rounds the member sums differently; activating
            # droplets amplify that (up to ~1e-11 per ulp of the ambient state)
            np.testing.assert_allclose(a["rw2"], b["rw2"], rtol=1e-9)


def test_full_size_ensemble_members_same_alone():
    """The benchmarked ensemble itself (256 ragged members, N_sd log-uniform
    in [1e3, 1e6], about 3.4e7 super-droplets, mixed precision, graph
    replay): after two steps with the parcels' rho_d, sampled members are bit
    for bit what they are when stepped alone."""
    members = workloads.ensemble_members(256, seed=0)
    opts = dict(adve=0, sedi=0, cond=1, coal=1, RH_max=44.0, sstp_cond=10, sstp_coal=10)
    n_sd = sum(m["n_sd"] for m in members)
    ens = Ensemble(precision="mixed", max_sd=n_sd + 1024, max_members=len(members))
    ids = [ens.add(m) for m in members]
    ens.use_graph(True)
    for t in (1.0, 2.0):
        r = workloads.parcel_rhod(members, t)
        ens.step(opts, rhod={ids[k]: v for k, v in r.items()})
        ens.wait()
    rng = np.random.default_rng(0)
    picks = [int(np.argmax([m["n_sd"] for m in members]))] + rng.choice(len(members), 3, replace=False).tolist()
    for k in picks:
        m = members[k]
        alone = Ensemble(precision="mixed", max_sd=m["n_sd"], max_members=1)
        a = alone.add(m)
        for t in (1.0, 2.0):
            r = workloads.parcel_rhod([m], t)
            alone.step(opts, rhod={a: r[0]} if 0 in r else None)
            alone.wait()
        for name in ("N", "rw2", "rd3", "kappa"):
            assert np.array_equal(ens.attr(ids[k], name, m["n_sd"]), alone.attr(a, name, m["n_sd"])), (k, name)
        assert np.array_equal(ens.fields([ids[k]])[1], alone.fields([a])[1])
        alone.close()
    ens.close()
