"""The device side of the x-slab decomposition (sdm_step_transport,
sdm_export_leavers, sdm_import, sdm_step_coalesce; x_open contexts) on one
GPU: two slab contexts hold the two halves of a 2D domain and exchange
their leavers every step, routed by global position the way
decomp.exchange routes them (decomp.slab_of, periodic in x).

Checked: the split step gives sdm_step_async's results bit for bit; every
leaver arrives on the slab that owns its position with N, r_w^2, r_d^3,
kappa, z and its id bit-identical and x moved by one slab width (a periodic
wrap rounds it like any wrap); no live id is duplicated; after the import
every super-droplet is counted in the cell of its position; the exchange
itself conserves sum N r^3."""
import numpy as np
import pytest

import workloads
from gpu_helpers import gpu_particles
from paper_1310_1905_gb300 import decomp, sdm

pytestmark = pytest.mark.gpu

ALL = dict(adve=1, sedi=1, cond=1, coal=1, sstp_cond=10, sstp_coal=10)


def test_split_step_is_step_async():
    w = workloads.icmw_2d(nx=8, nz=16, sd_conc=16, seed=4, dz=93.75)
    a, b = gpu_particles(w), gpu_particles(w)
    tha, rva, thb, rvb = w.th.copy(), w.rv.copy(), w.th.copy(), w.rv.copy()
    for _ in range(6):
        a.step_sync(ALL, tha, rva)
        a.step_async(ALL)
        a.wait()
        b.step_sync(ALL, thb, rvb)
        b.step_transport(ALL)
        b.step_coalesce(ALL)
        b.wait()
    sa, sb = a.state(), b.state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(tha, thb) and np.array_equal(rva, rvb)
    assert a.stats() == b.stats()


def slab(w, i0, i1):
    """The columns [i0, i1) of workload w as an x_open context's inputs."""
    cfg = dict(w.cfg, nx=i1 - i0, x_open=1)
    f = lambda a: np.ascontiguousarray(a[i0:i1])  # noqa: E731
    return cfg, f(w.th), f(w.rv), f(w.rhod), np.ascontiguousarray(w.rhoCx[i0:i1 + 1]), f(w.rhoCz)


def two_slabs(seed=5):
    w = workloads.icmw_2d(nx=12, nz=20, sd_conc=16, seed=seed, dz=75.0)
    nxs = 6
    parts, fields = [], []
    for r in range(2):
        cfg, th, rv, rhod, cx, cz = slab(w, r * nxs, (r + 1) * nxs)
        # 256 reserved slots: room for a step's net inflow from the other slab
        p = sdm.Particles(dict(cfg, seed=10 + r, sd_reserve=256), th, rv, rhod, cx, None, cz)
        p.set_attr("uid", p.attr("uid") + r * p.n_sd)  # ids unique over the domain
        parts.append(p)
        fields.append([th.copy(), rv.copy()])
    return w, nxs * w.cfg["dx"], parts, fields


def route(out, width):
    """Leavers of slab r (local x outside [0, width)) to the other slab's
    local coordinates, checked against decomp.slab_of on the global,
    periodic position: one slab width across (below width on arrival)."""
    X = 2 * width
    inbox = [None, None]
    for r, o in enumerate(out):
        assert (o["N"] > 0).all() and ((o["x"] < 0) | (o["x"] >= width)).all()
        xg = o["x"] + r * width
        xg = np.where(xg < 0, xg + X, np.where(xg >= X, xg - X, xg))
        assert (decomp.slab_of(xg, X, 2) == 1 - r).all()
        xl = np.where(o["x"] < 0, o["x"] + width, o["x"] - width)
        xl = np.minimum(xl, np.nextafter(width, 0.0))
        assert np.allclose(xl, xg - (1 - r) * width, rtol=0, atol=4 * np.spacing(X))
        inbox[1 - r] = dict(o, x=xl)
    return inbox


def test_two_slabs_exchange_their_leavers_every_step():
    """The sharded step: transport, export, exchange, import, coalescence."""
    w, width, parts, fields = two_slabs()
    n_tot = sum(p.n_sd for p in parts)
    moved = 0
    for step in range(12):
        for r, p in enumerate(parts):
            p.step_sync(ALL, *fields[r])
            p.step_transport(ALL)
        inbox = route([p.export_leavers() for p in parts], width)
        for r, p in enumerate(parts):
            p.import_(inbox[r])
            moved += len(inbox[r]["N"])
        for p in parts:
            p.step_coalesce(ALL)
            p.wait()
    assert moved > 20
    # none lost or duplicated: live ids unique over both slabs and unmarked;
    # the slots a leaver emptied carry the mark of a slot kept for arrivals
    uids = np.concatenate([p.attr("uid").astype(np.int64) for p in parts])
    Ns = np.concatenate([p.attr("N") for p in parts])
    live = uids[Ns > 0]
    assert len(uids) == n_tot and len(np.unique(live)) == len(live)
    assert (live < 2 ** 31).all() and ((uids >= 2 ** 31) <= (Ns == 0)).all()
    dx, dz, nz = w.cfg["dx"], w.cfg["dz"], w.cfg["nz"]
    for p in parts:
        x, z, N = p.attr("x"), p.attr("z"), p.attr("N")
        live = N > 0
        assert ((x[live] >= 0) & (x[live] < width)).all()
        i = np.floor(x[live] / dx).astype(int)
        k = np.clip(np.floor(z[live] / dz).astype(int), 0, nz - 1)
        want = np.bincount(i * nz + k, minlength=p.n_cells).astype(float)
        np.testing.assert_array_equal(p.diag_sd_conc(), want)
        assert np.isfinite(p.attr("rw2")).all()


def test_exchange_moves_attributes_exactly():
    """Between steps (after sdm_wait): the leavers a step left outside the
    slabs go across and arrive with every attribute bit-identical, in free
    slots; the exchange conserves sum N r^3."""
    w, width, parts, fields = two_slabs(seed=7)
    for _ in range(3):
        for r, p in enumerate(parts):
            p.step_sync(ALL, *fields[r])
            p.step_async(ALL)
            p.wait()
        liquid0 = sum((p.attr("N").astype(float) * p.attr("rw2") ** 1.5).sum() for p in parts)
        inbox = route([p.export_leavers() for p in parts], width)
        for r, p in enumerate(parts):
            p.import_(inbox[r])
        liquid1 = sum((p.attr("N").astype(float) * p.attr("rw2") ** 1.5).sum() for p in parts)
        assert liquid1 == pytest.approx(liquid0, rel=1e-14)
        for r, p in enumerate(parts):
            blk = inbox[r]
            uid = p.attr("uid").astype(np.int64)
            pos = {int(u): i for i, u in enumerate(uid)}
            idx = np.array([pos[int(u)] for u in blk["uid"]], dtype=np.int64)
            for k in ("N", "rw2", "rd3", "kappa", "x", "z"):
                assert np.array_equal(p.attr(k)[idx], blk[k]), k
            x = p.attr("x")[p.attr("N") > 0]
            assert ((x >= 0) & (x < width)).all()


def test_export_and_import_refuse_what_they_cannot_do():
    w = workloads.icmw_2d(nx=4, nz=8, sd_conc=8, seed=6, dz=187.5)
    periodic = gpu_particles(w)
    with pytest.raises(sdm.SdmError) as e:
        periodic.export_leavers()
    assert e.value.status == 1  # SDM_EINVAL: not an x_open context
    cfg, th, rv, rhod, cx, cz = slab(w, 0, 4)
    p = sdm.Particles(cfg, th, rv, rhod, cx, None, cz)
    one = {k: v[:1] for k, v in dict(N=np.array([5], np.uint64), uid=np.array([999], np.uint32),
                                      rw2=np.array([1e-12]), rd3=np.array([1e-21]), kappa=np.array([0.6]),
                                      x=np.array([10.0]), z=np.array([100.0])).items()}
    with pytest.raises(sdm.SdmError) as e:  # no free slot: every super-droplet has N > 0
        p.import_(one)
    assert e.value.status == 2
    with pytest.raises(sdm.SdmError) as e:  # a position outside the slab
        p.import_(dict(one, x=np.array([-1.0])))
    assert e.value.status == 1
    with pytest.raises(sdm.SdmError) as e:
        p.step_coalesce(ALL)
    assert e.value.status == 6  # SDM_ESTATE: no transport pending
