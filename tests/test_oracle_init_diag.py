"""Pins of the oracle's initialisation (paper Sec. 5.1.6) and diagnostics
(Sec. 5.2.1): sampled spectra against their analytic integrals, the
multiplicity >= 1 criterion at the ends of the radius range, Koehler
equilibrium of the initial wet radii, and moments against brute-force sums."""
import math

import numpy as np
import pytest
from scipy.stats import kstest

import oracle
import workloads

R_D = 287.0
RHO_STP = 101325.0 / (R_D * 293.15)


def test_golovin_init_exponential_volumes():
    w = workloads.golovin_box(seed=3)
    o = oracle.Oracle(w.cfg)
    s = o.init(w.th, w.rv, w.rhod)
    assert s.n == 8192
    assert (s.N == 1024 * 10 ** 6).all()          # n0 dV / N_sd exactly
    V = 4.0 / 3.0 * math.pi * s.rw2 ** 1.5
    Vbar = w.cfg["exp_mean_volume"]
    assert V.mean() == pytest.approx(Vbar, rel=4.5 / math.sqrt(8192))
    assert kstest(V / Vbar, "expon").pvalue > 1e-4
    assert sorted(s.uid.tolist()) == list(range(8192))


def lognormal_n(lnr, modes):
    return sum(m["n_stp"] / (math.sqrt(2 * math.pi) * math.log(m["sigma"]))
               * np.exp(-0.5 * ((lnr - math.log(m["rm"])) / math.log(m["sigma"])) ** 2) for m in modes)


def test_rd_range_multiplicity_criterion():
    w = workloads.icmw_2d(nx=4, nz=4, sd_conc=64)
    o = oracle.Oracle(w.cfg)
    lo, hi = o.rd_range(0)
    dV = 20.0 * 20.0 * 1.0
    dl = (hi - lo) / 64
    f = lambda l: lognormal_n(l, w.cfg["modes"]) * dl * dV
    # the range is a fixed point of 8 narrowing passes: equality to 1e-9
    assert f(lo) >= 1.0 - 1e-9 and f(hi) >= 1.0 - 1e-9
    assert f(lo - 1e-3) < 1.0 and f(hi + 1e-3) < 1.0
    assert math.exp(lo) < 0.01e-6 and math.exp(hi) > 1e-6


def test_lognormal_init_represents_spectrum():
    w = workloads.icmw_2d(nx=16, nz=16, sd_conc=64, seed=4)
    o = oracle.Oracle(w.cfg)
    s = o.init(w.th, w.rv, w.rhod)
    lo, hi = o.rd_range(0)
    assert s.n == 16 * 16 * 64
    assert (s.N >= 1).all()
    lnr = np.log(np.cbrt(s.rd3))
    # dry radii uniform in ln r over [lo, hi]
    assert kstest((lnr - lo) / (hi - lo), "uniform").pvalue > 1e-4
    # concentration at STP: total over all super-droplets vs the integral
    k = np.floor(s.z / 20.0).astype(int)
    i = np.floor(s.x / 20.0).astype(int)
    rhod = w.rhod.ravel()[i * 16 + k]
    n_stp = (s.N / (20.0 * 20.0 * 1.0) * RHO_STP / rhod).sum() / (16 * 16)
    grid = np.linspace(lo, hi, 20001)
    integral = np.trapezoid(lognormal_n(grid, w.cfg["modes"]), grid)
    assert n_stp == pytest.approx(integral, rel=0.03)
    assert integral == pytest.approx(100e6, rel=0.01)


def test_initial_wet_radii_in_equilibrium():
    w = workloads.icmw_2d(nx=2, nz=75, sd_conc=8, seed=5)
    o = oracle.Oracle(w.cfg)
    s = o.init(w.th, w.rv, w.rhod)
    k = np.floor(s.z / 20.0).astype(int)
    i = np.floor(s.x / 20.0).astype(int)
    sat = 0
    for q in range(s.n):
        c = i[q] * 75 + k[q]
        t = oracle.thermo(w.th.ravel()[c], w.rv.ravel()[c], w.rhod.ravel()[c])
        RH = t.rho_v / t.rho_vs
        if RH >= 1.0:
            RH, sat = 0.95, sat + 1
        r = math.sqrt(s.rw2[q])
        S = (r ** 3 - s.rd3[q]) / (r ** 3 - s.rd3[q] * (1 - 0.61)) * math.exp(2 * 0.072 / (461.5 * t.T * 1000 * r))
        assert S == pytest.approx(RH, rel=1e-9)
    assert 0 < sat < s.n  # the upper part of the domain starts supersaturated


def test_moments_brute_force():
    w = workloads.icmw_2d(nx=3, nz=5, sd_conc=16, seed=6)
    o = oracle.Oracle(w.cfg)
    s = o.init(w.th, w.rv, w.rhod)
    s.rw2[::3] *= 1e4  # spread the wet radii
    dV = 400.0
    for wet in (True, False):
        for (rmin, rmax) in ((0.0, 1.0), (1e-8, 1e-6), (5e-8, 2e-5)):
            for k in range(4):
                got = o.moments(wet, rmin, rmax, k)
                ref = np.zeros(15)
                for q in range(s.n):
                    r = math.sqrt(s.rw2[q]) if wet else s.rd3[q] ** (1.0 / 3.0)
                    if rmin <= r <= rmax:
                        c = int(s.x[q] // 20.0) * 5 + int(s.z[q] // 20.0)
                        ref[c] += float(s.N[q]) * r ** k
                ref /= w.rhod.ravel() * dV
                np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-300)
    conc = o.sd_conc()
    assert conc.sum() == s.n and (conc == 16).all()


def test_spectrum_matches_weighted_histogram():
    """Binned spectrum: per cell, the bin of each radius from numpy's
    digitize (half-open [e_b, e_b+1)) and bincount sums of N r^k (numpy's
    weighted histogram differences cumulative sums, which loses digits),
    divided by rho_d dV; a radius that
    sits on an inner edge counts in the bin above it; the k = 0 spectrum
    over bins that cover every radius sums to the concentration."""
    w = workloads.icmw_2d(nx=3, nz=5, sd_conc=16, seed=7)
    o = oracle.Oracle(w.cfg)
    s = o.init(w.th, w.rv, w.rhod)
    s.rw2[::3] *= 1e4
    dV = 400.0
    edges = np.geomspace(1e-9, 1e-3, 25)
    s.rw2[5] = edges[7] ** 2  # exactly on an edge (sqrt of a square is exact)
    cells = (s.x // 20.0).astype(int) * 5 + (s.z // 20.0).astype(int)
    for wet in (True, False):
        r = np.sqrt(s.rw2) if wet else np.cbrt(s.rd3)
        for k in (0, 1, 3):
            got = o.spectrum(wet, edges, k)
            assert got.shape == (24, 15)
            b = np.digitize(r, edges) - 1
            for c in range(15):
                sel = (cells == c) & (b >= 0) & (b < 24)
                h = np.bincount(b[sel], weights=s.N[sel].astype(float) * r[sel] ** k, minlength=24)
                np.testing.assert_allclose(got[:, c], h / (w.rhod.ravel()[c] * dV), rtol=1e-12, atol=1e-300)
    got = o.spectrum(True, edges, 0)
    assert got[7, cells[5]] > 0 and got[7, cells[5]] >= s.N[5] / (w.rhod.ravel()[cells[5]] * dV)
    np.testing.assert_allclose(got.sum(axis=0), o.moments(True, 0.0, 1.0, 0), rtol=1e-12)
