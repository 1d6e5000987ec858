"""Mixed FP32/FP64 mode against the FP64 oracle.  FP32 accept/reject
decisions can flip, so the mode is judged by moment statistics, with the
error stated per diagnostic: cloud-droplet concentration, mean cloud-droplet
radius, rain-water mixing ratio (ensemble of seeds), liquid water."""
import math

import numpy as np
import pytest

import workloads
from gpu_helpers import oracle_sim, start_from_oracle_multiplicities
from paper_1310_1905_gb300 import sdm

pytestmark = pytest.mark.gpu

ALL = dict(adve=1, sedi=1, cond=1, coal=1, sstp_cond=10, sstp_coal=10)
RHO_W = 1000.0


def diagnostics(get_mom, rhod, dV=None):
    """Domain means: cloud (0.5-25 um) number per kg, mean radius; rain
    (> 25 um) and total liquid mixing ratios."""
    m0c = get_mom(True, 0.5e-6, 25e-6, 0)
    m1c = get_mom(True, 0.5e-6, 25e-6, 1)
    m3r = get_mom(True, 25e-6, 1.0, 3)
    m3 = get_mom(True, 0.5e-6, 1.0, 3)
    conc = m0c.mean()
    rmean = m1c.sum() / max(m0c.sum(), 1e-300)
    rain = 4.0 / 3.0 * math.pi * RHO_W * m3r.mean()
    lwc = 4.0 / 3.0 * math.pi * RHO_W * m3.mean()
    return dict(conc=conc, rmean=rmean, rain=rain, lwc=lwc)


def run_pair(seed, steps):
    w = workloads.icmw_2d(nx=8, nz=30, sd_conc=32, seed=seed, dz=50.0)
    p = sdm.Particles(w.cfg, w.th, w.rv, w.rhod, w.rhoCx, None, w.rhoCz, precision="mixed")
    o = oracle_sim(w)
    start_from_oracle_multiplicities(p, o)
    th, rv = w.th.copy(), w.rv.copy()
    for _ in range(steps):
        p.step_sync(ALL, th, rv)
        p.step_async(ALL)
        p.wait()
        o.step_sync(ALL)
        o.step_async(ALL, w.rhoCx, None, w.rhoCz)
    dg = diagnostics(lambda wet, a, b, k: p.diag_moments(wet, a, b, k), w.rhod)
    do = diagnostics(lambda wet, a, b, k: o.moments(wet, a, b, k), w.rhod)
    return dg, do, rv.ravel(), o.rv


def test_mixed_precision_diagnostics_2d():
    dg, do, rv_g, rv_o = run_pair(seed=3, steps=12)
    err = {k: abs(dg[k] - do[k]) / max(abs(do[k]), 1e-30) for k in ("conc", "rmean", "lwc")}
    print("mixed vs FP64 oracle, relative errors:", err)
    assert do["conc"] > 0 and do["lwc"] > 0
    assert err["conc"] < 5e-3
    assert err["rmean"] < 5e-3
    assert err["lwc"] < 5e-3
    np.testing.assert_allclose(rv_g, rv_o, rtol=1e-4)


def test_mixed_precision_golovin_statistics():
    """Mixed-mode coalescence against the analytic Golovin number moment
    (ensemble of 4 seeds), the same bar the FP64 oracle meets."""
    B, N0, VBAR, DV = 1500.0, 2.0 ** 23, 4.0 / 3.0 * math.pi * (30.531e-6) ** 3, 1e6
    opts = dict(adve=0, sedi=0, cond=0, coal=1, sstp_coal=1, sstp_cond=1)
    m0 = {600: [], 1200: []}
    for seed in range(4):
        w = workloads.golovin_box(seed=seed)
        p = sdm.Particles(w.cfg, w.th, w.rv, w.rhod, precision="mixed")
        for t in range(1, 1201):
            p.step_async(opts)
            p.wait()
            if t in m0:
                m0[t].append(p.attr("N").astype(float).sum() / DV)
        p.close()
    for t, v in m0.items():
        assert np.mean(v) == pytest.approx(N0 * math.exp(-B * N0 * VBAR * t), rel=0.04)


def test_mixed_precision_long_kernel_statistics():
    """Mixed-mode coalescence with the Long (1974) efficiency (FP32 R, r and
    3e-6/r) against the FP64 oracle: a box of drops with exponential volumes
    (mean radius 12 um, 3-50 um for most), 600 s, 4 seeds.  The mean number
    concentration (drops 5 % over the run, seed spread 0.4 %) must agree
    within 1 %, the second volume moment (grows 20 %, spread 1.2 %) within
    5 %, the liquid volume within 1e-9."""
    mv = 4.0 / 3.0 * math.pi * (12e-6) ** 3
    opts = dict(adve=0, sedi=0, cond=0, coal=1, sstp_cond=1, sstp_coal=5)
    got, ref = [], []
    for seed in range(4):
        cfg = dict(nx=0, ny=0, nz=0, dx=100.0, dy=100.0, dz=100.0, dt=1.0, sd_conc=2048, kernel="long",
                   init_dist="exponential", exp_mean_volume=mv, exp_n0=1e8, modes=[], seed=seed, physics=1)
        one = np.ones(1)
        p = sdm.Particles(cfg, 289.0 * one, 7.5e-3 * one, one, precision="mixed")
        o = oracle_sim(workloads.Workload("long_box", cfg, 289.0 * one, 7.5e-3 * one, one, None, None, None,
                                          opts, 600))
        for _ in range(600):
            p.step_async(opts)
            p.wait()
            o.step_async(opts)
        for out, N, rw2 in ((got, p.attr("N"), p.attr("rw2")), (ref, o.state.N, o.state.rw2)):
            V = 4.0 / 3.0 * math.pi * rw2 ** 1.5
            out.append((N.astype(float).sum(), (N * V * V).sum(), (N * V).sum()))
        p.close()
    g, r = np.mean(got, axis=0), np.mean(ref, axis=0)
    assert r[0] < 0.97 * 1e8 * 1e6  # collisions took place
    assert g[0] == pytest.approx(r[0], rel=1e-2)
    assert g[1] == pytest.approx(r[1], rel=5e-2)
    assert g[2] == pytest.approx(r[2], rel=1e-9)
