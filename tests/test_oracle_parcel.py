"""Pins of the oracle's parcel mode (the parcel framework of Sec. 5.2.1,
no spatial dimension): a new rho_d given for a step sets the volume to the
parcel's dry-air mass over it (reading 20), and the step begins with
recycling (Sec. 5.1.4), then condensation, then coalescence.

What fixes it, independently of the oracle's own code:
- the dry-air mass rho_d dV stays m_d through every rho_d change;
- the number of particles per unit dry-air mass stays put without
  coalescence (the moment (rho_d dV)^-1 sum N);
- total water r_v + r_l, r_l = 4/3 pi rho_w sum N r^3 / m_d, is conserved to
  rounding while rho_d changes: eq. rhov_update takes dV rho_d, which is m_d
  only if the volume follows rho_d (a volume left at its initial value
  breaks this by the density ratio);
- a rising parcel's liquid water approaches, from below, the saturation
  adjustment of its total water at the final rho_d, computed here by
  integrating d theta / d r_v = -theta l_v / (c_pd T) (Sec. 3, Appendix A)
  with scipy to r_v = r_vs;
- with rho_d constant and no zero multiplicities, a parcel step is the
  box's step_sync + step_async bit for bit.
"""
import numpy as np
import pytest

import oracle
import workloads

scipy = pytest.importorskip("scipy")
from scipy.integrate import solve_ivp  # noqa: E402
from scipy.optimize import brentq  # noqa: E402

COND = dict(adve=0, sedi=0, cond=1, coal=0, sstp_cond=10, sstp_coal=10)
ALL0D = dict(adve=0, sedi=0, cond=1, coal=1, sstp_cond=10, sstp_coal=10)


def rhod_at(z):
    return float(workloads.hydrostatic_rhod(np.array([z]), 289.0, 7.5e-3, 101500.0)[0])


def parcel(n_sd=256, seed=7, z0=600.0, dV=1.0, modes=None, rv=7.5e-3):
    cfg = dict(nx=0, ny=0, nz=0, dx=dV, dy=1.0, dz=1.0, dt=1.0, sd_conc=n_sd, kernel="geometric",
               init_dist="lognormal", modes=modes or workloads.AEROSOL_BIMODAL[:1], seed=seed, physics=1)
    o = oracle.Oracle(cfg)
    o.init(np.array([289.0]), np.array([rv]), np.array([rhod_at(z0)]))
    return o


def liquid(o):
    s = o.state
    return 4.0 / 3.0 * np.pi * 1000.0 * float((s.N.astype(float) * s.rw2 ** 1.5).sum()) / o.m_d


def test_dry_air_mass_and_number_per_mass_kept():
    o = parcel()
    n0 = o.moments(False, 0.0, 1.0, 0)[0]
    for k in range(1, 41):
        o.parcel_step(COND, rhod_at(600.0 + 3.0 * k))
        assert o.volume * o.rhod[0] == pytest.approx(o.m_d, rel=2e-16)
        assert o.moments(False, 0.0, 1.0, 0)[0] == pytest.approx(n0, rel=1e-14)
    assert o.volume > 1.0  # the parcel expanded


def test_total_water_conserved_through_rho_d_changes():
    o = parcel()
    rt0 = o.rv[0] + liquid(o)
    for k in range(1, 201):
        o.parcel_step(COND, rhod_at(600.0 + 2.0 * k))
    assert liquid(o) > 1e-4  # cloud formed: the feedback carried real mass
    assert o.rv[0] + liquid(o) == pytest.approx(rt0, rel=1e-13)


# Appendix A and the list of symbols, restated for the adjustment
RD, RV, CPD, CPV, CL, LV0, T0, PVS0, P1000 = 287.0, 461.5, 1005.0, 1850.0, 4218.0, 2.5e6, 273.16, 611.73, 1e5


def _T(th, rhod):
    return (th * (rhod * RD / P1000) ** (RD / CPD)) ** (CPD / (CPD - RD))


def _rvs(T, rhod):
    a, b = (LV0 + (CL - CPV) * T0) / RV, (CL - CPV) / RV
    return PVS0 * np.exp(a * (1.0 / T0 - 1.0 / T) - b * np.log(T / T0)) / (RV * T) / rhod


def _adjusted_liquid(th0, rt, rhod):
    def dth(rv, y):
        T = _T(y[0], rhod)
        return [-y[0] * (LV0 + (CPV - CL) * (T - T0)) / (CPD * T)]

    def resid(rv):
        th = solve_ivp(dth, (rt, rv), [th0], rtol=1e-12, atol=1e-12).y[0, -1]
        return rv - _rvs(_T(th, rhod), rhod)

    return rt - brentq(resid, 0.5 * rt, rt, xtol=1e-16)


def test_rising_parcel_approaches_saturation_adjustment_from_below():
    o = parcel()
    th0, rt = o.th[0], o.rv[0] + liquid(o)
    for k in range(1, 301):  # 2 m/s for 300 s: from 600 m to 1200 m, through cloud base
        o.parcel_step(COND, rhod_at(600.0 + 2.0 * k))
    adj = _adjusted_liquid(th0, rt, o.rhod[0])
    assert adj > 3e-4
    assert 0.95 * adj < liquid(o) < adj  # supersaturated: some vapour not yet condensed


def test_constant_rho_d_parcel_step_is_the_box_step():
    # supersaturated (r_v = 12 g/kg at 600 m): the droplets grow to ~20 um and collide
    a, b = (parcel(n_sd=512, seed=3, dV=1e6, rv=1.2e-2) for _ in range(2))
    for _ in range(20):
        a.parcel_step(ALL0D, None)
        b.step_sync(ALL0D)
        b.step_async(ALL0D)
    assert a.stats.n_recycled == 0 and (a.state.N > 0).all()  # no zero to recycle in either order
    sa, sb = a.state.sorted_by_uid(), b.state.sorted_by_uid()
    assert a.stats.n_coll > 0
    for f in ("N", "rw2", "rd3", "kappa"):
        assert np.array_equal(getattr(sa, f), getattr(sb, f)), f
    assert a.th[0] == b.th[0] and a.rv[0] == b.rv[0]
