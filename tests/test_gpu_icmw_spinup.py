"""The 2D kinematic case run as the paper runs it (Sec. 2.2): a spin-up
with coalescence and sedimentation off and drop growth capped at RH = 1.05,
then the main run with every process on, theta and r_v transported by the
eddy and relaxed to their initial level means before every step; against
the oracle doing the same sequence on a reduced domain (the same 1.5 km
eddy on 12 x 40 cells).  Multiplicities bit-exact; radii within 1e-12 or
within the oracle's own spread when its theta moves, after every Eulerian
step, by as many ulps as the GPU's T and rho_vs differ from the oracle's
(measured at the start): over a long transported run the two sides'
rounding differs at every step, and near activation that moves a root by
more than 1e-12.  Then the
dry and wet spectra of the ten regions (Sec. 5.4) from sdm_diag_spectrum
against the oracle's binning."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import RTOL, gpu_particles, start_from_oracle_multiplicities, theta_ulps
from paper_1310_1905_gb300 import icmw

pytestmark = pytest.mark.gpu

SPINUP, MAIN = 60, 30


def oracle_run(w, ulps=None, direction=np.inf, every_step=False, seed=None):
    """The oracle's spin-up + main run; with ulps, theta moved by that many
    ulps per cell at the start, or (every_step) after every Eulerian step,
    towards direction, or (seed) in a random direction per cell and step."""
    o = oracle.Oracle(w.cfg, omp=True)
    o.init(w.th, w.rv, w.rhod)
    th0, rv0 = w.th.mean(axis=0), w.rv.mean(axis=0)
    rng = np.random.default_rng(seed)

    def nudge():
        dirs = rng.choice([np.inf, -np.inf], len(o.th)) if seed is not None else np.full(len(o.th), direction)
        for c in range(len(o.th)):
            for _ in range(int(ulps[c])):
                o.th[c] = np.nextafter(o.th[c], dirs[c])

    if ulps is not None and not every_step:
        nudge()
    for n in range(SPINUP + MAIN):
        opts = icmw.SPINUP_OPTS if n < SPINUP else icmw.MAIN_OPTS
        o.euler_step(w.rhoCx, None, w.rhoCz, th0, rv0)
        if ulps is not None and every_step:
            nudge()
        o.step_sync(opts)
        o.step_async(opts, w.rhoCx, None, w.rhoCz)
    return o


def spread(w, ref, ulps, every_step):
    """The largest move of the oracle's r_w^2 under the perturbations: both
    one-sided directions, and (every_step) four random-sign patterns."""
    runs = [dict(direction=np.inf), dict(direction=-np.inf)]
    if every_step:
        runs += [dict(seed=k) for k in range(4)]
    out = np.zeros_like(ref)
    for kw in runs:
        s = oracle_run(w, ulps, every_step=every_step, **kw).state.sorted_by_uid()
        out = np.maximum(out, np.abs(s.rw2 - ref))
    return out


def test_spinup_then_main_run_matches_oracle():
    w = workloads.icmw_2d(nx=12, nz=40, sd_conc=16, seed=2, dz=37.5)
    p = gpu_particles(w)
    base = oracle_run(w)
    # the measured difference of the two sides' T and rho_vs, in theta ulps
    Tg, rg = p.diag_ambient("T"), p.diag_ambient("rho_vs")
    th, rv, rhod = (np.ascontiguousarray(a).ravel() for a in (w.th, w.rv, w.rhod))
    ulps = np.array([theta_ulps(Tg[c], rg[c], th[c], rv[c], rhod[c]) for c in range(len(th))])
    ref_init = oracle.Oracle(w.cfg)
    ref_init.init(w.th, w.rv, w.rhod)
    start_from_oracle_multiplicities(p, ref_init)
    th_g, rv_g = w.th.copy(), w.rv.copy()
    icmw.run(p, w, th_g, rv_g, SPINUP, MAIN)
    g = p.state()
    r = base.state.sorted_by_uid()
    assert np.array_equal(g["N"], r.N)
    err = np.abs(g["rw2"] - r.rw2)
    # every droplet within the envelope of the oracle's spread when the
    # measured difference enters at every step (one-sided drifts and random
    # signs of that many ulps per step), and nearly all within its spread
    # under the measured difference at the start
    env = np.maximum(RTOL * r.rw2, spread(w, r.rw2, ulps, True))
    assert (err <= env).all(), f"{(err > env).sum()} of {err.size} outside; worst rel {np.max(err / r.rw2):.3e}"
    start = np.maximum(RTOL * r.rw2, spread(w, r.rw2, ulps, False))
    outside = (err > start).mean()
    beyond = (err > RTOL * r.rw2).mean()
    print(f"spin-up + main: theta ulps median {np.median(ulps):.0f}, max {ulps.max()}; worst rel "
          f"{np.max(err / r.rw2):.2e}; {beyond * 100:.2f} % beyond 1e-12, {outside * 100:.2f} % beyond the "
          f"start-perturbation spread")
    assert outside < 0.02
    assert base.stats.n_coll > 0 and np.abs(rv_g.ravel() - w.rv.ravel()).max() > 1e-5
    # the spectra of the ten regions against the oracle's binning of its own state
    nx, nz = w.cfg["nx"], w.cfg["nz"]
    sp = icmw.spectra(p, nx, nz)
    for wet, edges, key in ((False, icmw.DRY_EDGES, "dry"), (True, icmw.WET_EDGES, "wet")):
        ref = base.spectrum(wet, edges, 0)
        for name, (i, k) in icmw.locations(nx, nz).items():
            want = ref[:, icmw.region_cells(i, k, nz)].mean(axis=1)
            np.testing.assert_allclose(sp[name][key], want, rtol=1e-9, atol=1e-300, err_msg=f"{key} {name}")
            assert want.sum() > 0
