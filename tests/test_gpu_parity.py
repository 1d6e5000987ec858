"""Parity of the CUDA library (through its C ABI) with the CPU oracle on the
same seeded inputs: element by element, multiplicities bit-exact, radii,
mixing ratios and moments within 1e-12 relative (FP64)."""
import numpy as np
import pytest

import workloads
from gpu_helpers import (RTOL, assert_close, compare_states, gpu_particles, oracle_sim, oracle_state, pair,
                         present_dims)
from paper_1310_1905_gb300 import sdm

pytestmark = pytest.mark.gpu

COND_ONLY = dict(adve=0, sedi=0, cond=1, coal=0, sstp_cond=10, sstp_coal=10)
COAL_ONLY = dict(adve=0, sedi=0, cond=0, coal=1, sstp_cond=10, sstp_coal=10)
MOVE_ONLY = dict(adve=1, sedi=1, cond=0, coal=0, sstp_cond=10, sstp_coal=10)
ALL = dict(adve=1, sedi=1, cond=1, coal=1, sstp_cond=10, sstp_coal=10)


def small_2d(seed=0, nx=9, nz=13, sd=20):
    # several warps' worth of cells, a ragged count per cell, supersaturated top
    return workloads.icmw_2d(nx=nx, nz=nz, sd_conc=sd, seed=seed, dz=115.0)


@pytest.mark.parametrize("seed", [0, 1])
def test_init_matches_oracle(seed):
    w = small_2d(seed)
    p = gpu_particles(w)
    o = oracle_sim(w)
    compare_states(p.state(), oracle_state(o, present_dims(w.cfg)), nreal=o.nreal)


def test_init_large_multiplicities_3d():
    # 150 m cubes: multiplicities ~1e14, where an ulp of the FP64 value is
    # ~0.03 and ties to the rounding boundary really occur
    w = workloads.updraft_3d(nx=4, ny=3, nz=9, sd_conc=10, seed=8, dx=150.0)
    p = gpu_particles(w)
    o = oracle_sim(w)
    compare_states(p.state(), oracle_state(o, present_dims(w.cfg)), nreal=o.nreal)


def test_init_golovin_box():
    w = workloads.golovin_box(seed=5)
    p = gpu_particles(w)
    o = oracle_sim(w)
    compare_states(p.state(), oracle_state(o, ()))


@pytest.mark.parametrize("solver", ["fast", "bisect"])
def test_condensation_matches_oracle(solver):
    w = small_2d(3)
    w.cfg["cond_solver"] = solver
    p, o = pair(w)
    th, rv = w.th.copy(), w.rv.copy()
    for _ in range(4):
        p.step_sync(COND_ONLY, th, rv)
        o.step_sync(COND_ONLY)
        assert_close("theta", th.ravel(), o.th)
        assert_close("r_v", rv.ravel(), o.rv)
    compare_states(p.state(), oracle_state(o, present_dims(w.cfg)))
    assert np.abs(o.rv - w.rv.ravel()).max() > 1e-6  # something condensed


def test_condensation_several_roots():
    """A 25 nm haze droplet (r_d = 13 nm, kappa 0.61) at S = 1.0088, just
    below its critical supersaturation, with dt' = 0.1 s: over the bracket of
    eq. rw2_implicit the residual changes sign three times (near 2.0e-15,
    2.7e-14 and 5.0e-14 m^2).  The bisection ends at the first; a solver
    that polishes from wherever FP32 stops deciding ends at the third.  The
    droplet and the ambient state are one the 2D case reaches in its first
    substep (level z = 810 m)."""
    w = workloads.icmw_2d(nx=2, nz=2, sd_conc=3, seed=1, dt=0.1)
    w.th[...] = 289.0
    w.rv[...] = 7.5e-3
    w.rhod[...] = 1.1275719998589389
    for solver in ("fast", "bisect"):
        w.cfg["cond_solver"] = solver
        p, o = pair(w)
        n = len(o.state.N)
        vals = dict(rw2=6.5206016327642645e-16, rd3=2.3321073379471742e-24, kappa=0.61)
        for k, v in vals.items():
            sdm.sdm_set_attr(p.ctx, k, np.full(n, v))
            getattr(o.state, k)[:] = v
        sdm.sdm_set_attr(p.ctx, "N", np.full(n, 12609913, np.uint64))
        o.state.N[:] = 12609913
        th, rv = w.th.copy(), w.rv.copy()
        one = dict(COND_ONLY, sstp_cond=1, sstp_coal=1)
        p.step_sync(one, th, rv)
        o.step_sync(one)
        r = oracle_state(o, present_dims(w.cfg))
        assert 1.9e-15 < r["rw2"][0] < 2.1e-15, r["rw2"][0]  # the first root
        compare_states(p.state(), r)
        assert_close("r_v", rv.ravel(), o.rv)


def test_condensation_bare_maxwell_mason():
    w = workloads.icmw_2d(nx=5, nz=11, sd_conc=12, seed=4, dz=130.0, physics=0)
    p, o = pair(w)
    th, rv = w.th.copy(), w.rv.copy()
    for _ in range(3):
        p.step_sync(COND_ONLY, th, rv)
        o.step_sync(COND_ONLY)
    assert_close("theta", th.ravel(), o.th)
    assert_close("r_v", rv.ravel(), o.rv)
    compare_states(p.state(), oracle_state(o, present_dims(w.cfg)))


def test_transport_matches_oracle():
    w = small_2d(5)
    p, o = pair(w)
    for _ in range(6):
        p.step_async(MOVE_ONLY)
        rain_g = p.wait()
        o.step_async(MOVE_ONLY, w.rhoCx, None, w.rhoCz)
    compare_states(p.state(), oracle_state(o, present_dims(w.cfg)))
    assert rain_g == pytest.approx(o.stats.rainfall, rel=1e-12, abs=0.0)


def test_coalescence_golovin_box_full_run():
    """Config: Golovin box, 8192 super-droplets, 1 s steps, 3600 s."""
    w = workloads.golovin_box(seed=2)
    p, o = pair(w)
    for t in range(1, 3601):
        p.step_async(w.opts)
        p.wait()
        o.step_async(w.opts)
        if t in (1, 10, 100, 1200, 3600):
            compare_states(p.state(), oracle_state(o, ()))
    st = p.stats()
    assert st["n_coll"] == o.stats.n_coll
    assert st["n_recycled"] == o.stats.n_recycled
    assert st["n_pgt1"] == o.stats.n_pgt1


def test_coalescence_geometric_2d():
    w = small_2d(6, sd=40)
    p, o = pair(w)
    # grow big drops first so that collisions happen: condense for a while
    th, rv = w.th.copy(), w.rv.copy()
    for _ in range(3):
        p.step_sync(COND_ONLY, th, rv)
        o.step_sync(COND_ONLY)
    for _ in range(5):
        p.step_async(COAL_ONLY)
        p.wait()
        o.step_async(COAL_ONLY)
    compare_states(p.state(), oracle_state(o, present_dims(w.cfg)))
    assert p.stats()["n_pairs"] == o.stats.n_pairs


def test_full_steps_2d():
    w = small_2d(7)
    p, o = pair(w)
    th, rv = w.th.copy(), w.rv.copy()
    for _ in range(8):
        p.step_sync(ALL, th, rv)
        p.step_async(ALL)
        p.wait()
        o.step_sync(ALL)
        o.step_async(ALL, w.rhoCx, None, w.rhoCz)
    assert_close("theta", th.ravel(), o.th)
    assert_close("r_v", rv.ravel(), o.rv)
    compare_states(p.state(), oracle_state(o, present_dims(w.cfg)))
    st = p.stats()
    assert st["n_coll"] == o.stats.n_coll and st["n_pairs"] == o.stats.n_pairs


def test_full_steps_3d_small():
    w = workloads.updraft_3d(nx=4, ny=3, nz=9, sd_conc=10, seed=8, dx=150.0)
    p, o = pair(w)
    th, rv = w.th.copy(), w.rv.copy()
    for _ in range(6):
        p.step_sync(ALL, th, rv)
        p.step_async(ALL)
        p.wait()
        o.step_sync(ALL)
        o.step_async(ALL, w.rhoCx.ravel(), w.rhoCy.ravel(), w.rhoCz.ravel())
    assert_close("theta", th.ravel(), o.th)
    assert_close("r_v", rv.ravel(), o.rv)
    compare_states(p.state(), oracle_state(o, present_dims(w.cfg)))


@pytest.mark.parametrize("zero_fraction", [0.2, 0.8])
def test_recycling_matches_oracle(zero_fraction):
    """Zeros take donors in (N descending, id ascending) order.  With a fifth
    of the multiplicities zeroed the donors are selected (radix select on N,
    then on the id among ties); with four fifths every donor is taken."""
    w = small_2d(9)
    p, o = pair(w)
    # zero out a pseudo-random share of the multiplicities on both sides
    g = p.state()
    rng = np.random.default_rng(0)
    zero_ids = set(rng.choice(len(g["uid"]), size=int(len(g["uid"]) * zero_fraction), replace=False).tolist())
    uid_store = p.attr("uid")
    N_store = p.attr("N")
    N_store[[i for i, u in enumerate(uid_store) if int(u) in zero_ids]] = 0
    sdm.sdm_set_attr(p.ctx, "N", N_store)
    o.state.N[[i for i, u in enumerate(o.state.uid) if int(u) in zero_ids]] = 0
    opts = dict(COAL_ONLY, coal=0)
    p.step_async(opts)
    p.wait()  # first wait learns about the zeros
    o.step_async(opts)
    p.step_async(opts)
    p.wait()
    o.step_async(opts)
    compare_states(p.state(), oracle_state(o, present_dims(w.cfg)))
    assert p.stats()["n_recycled"] == o.stats.n_recycled > 0


def test_recycling_select_with_ties():
    """More donors than one block sorts (18 000 super-droplets), a fifth of
    them zeroed, and the multiplicities forced onto three values, so that the
    donors at the threshold are picked by id: the radix select on N and then
    on the id must reproduce the oracle's (N descending, id ascending) order."""
    w = small_2d(12, nx=30, nz=30, sd=20)
    p, o = pair(w)
    uid_store = p.attr("uid").astype(np.int64)
    N_by_uid = 1000 + (np.arange(len(uid_store)) * 7919) % 3  # 1000, 1001, 1002
    rng = np.random.default_rng(3)
    zero = rng.choice(len(uid_store), size=len(uid_store) // 5, replace=False)
    N_by_uid[zero] = 0
    sdm.sdm_set_attr(p.ctx, "N", N_by_uid[uid_store].astype(np.uint64))
    o.state.N[:] = N_by_uid[o.state.uid.astype(np.int64)]
    opts = dict(COAL_ONLY, coal=0)
    for _ in range(2):
        p.step_async(opts)
        p.wait()  # the first wait learns about the zeros
        o.step_async(opts)
    compare_states(p.state(), oracle_state(o, present_dims(w.cfg)))
    assert p.stats()["n_recycled"] == o.stats.n_recycled == len(zero)


def test_diagnostics_match_oracle():
    w = small_2d(10)
    p, o = pair(w)
    th, rv = w.th.copy(), w.rv.copy()
    p.step_sync(COND_ONLY, th, rv)
    o.step_sync(COND_ONLY)
    for wet, rmin, rmax in ((True, 0.0, 1.0), (True, 0.5e-6, 25e-6), (False, 1e-8, 1e-6)):
        for k in range(4):
            assert_close(f"M{k}", p.diag_moments(wet, rmin, rmax, k), o.moments(wet, rmin, rmax, k),
                         atol=1e-300)
    assert np.array_equal(p.diag_sd_conc(), o.sd_conc())


def test_device_resident_fields_and_strides():
    torch = pytest.importorskip("torch")
    w = small_2d(11)
    p, o = pair(w)
    # fields on the device, transposed storage (strides (1, nx))
    th = torch.tensor(w.th.T.copy(), dtype=torch.float64, device="cuda").t()
    rv = torch.tensor(w.rv.T.copy(), dtype=torch.float64, device="cuda").t()
    assert th.stride() == (1, w.th.shape[0])
    p.step_sync(COND_ONLY, th, rv)
    o.step_sync(COND_ONLY)
    torch.cuda.synchronize()
    assert_close("theta", th.cpu().numpy().ravel(), o.th)
    assert_close("r_v", rv.cpu().numpy().ravel(), o.rv)


def test_status_codes():
    w = small_2d(12)
    p = gpu_particles(w)
    th, rv = w.th.copy(), w.rv.copy()
    p.step_async(ALL)
    with pytest.raises(sdm.SdmError) as e:
        p.step_sync(ALL, th, rv)          # step_sync before wait
    assert e.value.status == 6
    p.wait()
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_diag_mom(p.ctx, 2)        # diag_mom before diag_rng
    assert e.value.status == 6
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_init(w.cfg, w.th, w.rv, w.rhod, backend="openmp")
    assert e.value.status == 1
    bad = dict(w.cfg, sd_conc=0)
    with pytest.raises(sdm.SdmError):
        sdm.sdm_init(bad, w.th, w.rv, w.rhod)


def test_spectrum_matches_oracle():
    """Binned spectrum (one pass over all bins) against the oracle's, after
    some condensation; log-spaced bins, a single bin, and bins that leave
    part of the spectrum out.  Also into device memory, and the moments of
    diag_mom are left as they were."""
    w = small_2d(13)
    p, o = pair(w)
    th, rv = w.th.copy(), w.rv.copy()
    for _ in range(2):
        p.step_sync(COND_ONLY, th, rv)
        o.step_sync(COND_ONLY)
    m3 = p.diag_moments(True, 0.0, 1.0, 3)
    for wet in (True, False):
        for edges in (np.geomspace(1e-9, 1e-3, 41), np.array([1e-9, 1.0]), np.geomspace(3e-8, 2e-6, 7)):
            for k in range(4):
                assert_close(f"spectrum wet={wet} k={k} bins={len(edges) - 1}", p.diag_spectrum(wet, edges, k),
                             o.spectrum(wet, edges, k), atol=1e-300)
    assert np.array_equal(sdm.sdm_outbuf(p.ctx), m3)
    torch = pytest.importorskip("torch")
    edges = np.geomspace(1e-9, 1e-3, 65)
    out = torch.empty((64, p.n_cells), dtype=torch.float64, device="cuda")
    sdm.sdm_diag_spectrum(p.ctx, True, edges, 3, out)
    torch.cuda.synchronize()
    assert_close("spectrum on device", out.cpu().numpy(), o.spectrum(True, edges, 3), atol=1e-300)
    for bad in (np.array([1e-6, 1e-6]), np.array([1e-6, 1e-7]), np.geomspace(1e-9, 1e-3, 258),
                np.array([-1e-6, 1e-6])):
        with pytest.raises(sdm.SdmError) as e:
            p.diag_spectrum(True, bad, 0)
        assert e.value.status == 1
