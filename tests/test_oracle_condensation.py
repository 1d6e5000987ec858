"""Pins of the oracle's phase-change step (paper Sec. 5.1.3, Appendix A)
against results fixed outside the oracle:

* theta/T/p: the definition theta = T (p1000/p_d)^(R_d/c_pd) inverted back;
* saturation vapour pressure: numerical integration of Clausius-Clapeyron
  with the paper's l_v(T), and textbook values;
* growth rate: the Rogers & Yau (1989, eq. 7.17-7.18) textbook arrangement
  r dr/dt = (S - S_eq) / (F_k + F_d) of the Maxwell-Mason equation;
* terminal velocity: Stokes' law at small radii, Gunn & Kinzer (1949)
  measured fall speeds for mm-size drops;
* Koehler equilibrium: an independent root finder (scipy brentq) on the
  kappa-Koehler equilibrium condition;
* the implicit solve: the Euler special case of the ill-posed bracket, the
  equation residual at the returned root;
* per-cell total water and the theta update of eq. (rhov_update).
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import brentq

import oracle
import workloads
from oracle_helpers import box_cfg, condense, make_state

R_D, R_V, C_PD, C_PV, C_L, LV0, T0 = 287.0, 461.5, 1005.0, 1850.0, 4218.0, 2.5e6, 273.16
RHO_W, SIGMA_W = 1000.0, 0.072

RHOD_1KM = float(workloads.hydrostatic_rhod(np.array([1000.0]), 289.0, 7.5e-3, 101500.0)[0])


def test_temperature_inverts_theta_definition():
    for th, rv, rhod in [(289.0, 7.5e-3, RHOD_1KM), (300.0, 0.012, 1.15), (270.0, 1e-3, 0.7)]:
        t = oracle.thermo(th, rv, rhod)
        pd = rhod * R_D * t.T
        assert t.T * (1e5 / pd) ** (R_D / C_PD) == pytest.approx(th, rel=1e-13)
        assert t.p == pytest.approx(pd + rv * rhod * R_V * t.T, rel=1e-13)


def test_saturation_vapour_pressure():
    def lv(T):
        return LV0 + (C_PV - C_L) * (T - T0)
    for T_target in (250.0, 273.16, 283.0, 293.15, 303.0):
        # find theta giving this T at rho_d = 1 with the oracle's own T(theta)
        rhod = 1.0
        th = T_target * (1e5 / (rhod * R_D * T_target)) ** (R_D / C_PD)
        t = oracle.thermo(th, 0.0, rhod)
        assert t.T == pytest.approx(T_target, rel=1e-12)
        pvs = t.rho_vs * R_V * t.T
        integral, _ = quad(lambda T: lv(T) / (R_V * T * T), T0, t.T, epsabs=0, epsrel=1e-13)
        assert pvs == pytest.approx(611.73 * math.exp(integral), rel=1e-11)
    # textbook magnitudes (e.g. Rogers & Yau Table 2.1): 611 Pa at 0 C, 2339 Pa at 20 C
    t20 = oracle.thermo(293.15 * (1e5 / (R_D * 293.15)) ** (R_D / C_PD), 0.0, 1.0)
    assert t20.rho_vs * R_V * t20.T == pytest.approx(2339.0, rel=0.01)


def test_growth_rate_matches_rogers_yau_arrangement():
    t = oracle.thermo(289.0, 7.5e-3, RHOD_1KM)
    for r, rd, kappa in [(20e-6, 0.05e-6, 0.61), (1e-6, 0.1e-6, 0.61), (0.3e-6, 0.1e-6, 1.2)]:
        x = r * r
        rd3 = rd ** 3
        g = oracle.growth(x, rd3, kappa, t, physics=0)
        # Rogers & Yau: r dr/dt = (S - S_eq) / (F_k + F_d) with
        # F_k = (L/(R_v T) - 1) L rho_w / (K T),  F_d = rho_w R_v T / (D e_s)
        es = t.rho_vs * R_V * t.T
        Fk = (t.lv / (R_V * t.T) - 1.0) * t.lv * RHO_W / (2.4e-2 * t.T)
        Fd = RHO_W * R_V * t.T / (2.26e-5 * es)
        S = t.rho_v / t.rho_vs
        a_w = (r ** 3 - rd3) / (r ** 3 - rd3 * (1 - kappa))
        S_eq = a_w * math.exp(2 * SIGMA_W / (R_V * t.T * RHO_W * r))
        assert g == pytest.approx(2 * (S - S_eq) / (Fk + Fd), rel=1e-12)


def test_rh_limit_caps_vapour_used_for_growth():
    t = oracle.thermo(289.0, 9e-3, RHOD_1KM, RH_max=1.01)
    assert t.rho_v / t.rho_vs > 1.05
    assert t.rho_v_eff == pytest.approx(1.01 * t.rho_vs, rel=1e-15)


def test_terminal_velocity_limits():
    t = oracle.thermo(293.15 * (1e5 / (R_D * 293.15)) ** (R_D / C_PD), 0.0, 101325.0 / (R_D * 293.15))
    # Stokes' law for small drops: v = 2 (rho_w - rho_a) g r^2 / (9 mu)
    for r in (0.5e-6, 2e-6, 5e-6):
        v_stokes = 2 * (RHO_W - t.rho_a) * 9.81 * r * r / (9 * t.mu)
        # Khvorostyanov-Curry's delta0^2 C0 = 23.97 (not 24) and the first inertial
        # correction set the allowed departure
        assert oracle.vterm(r * r, t) == pytest.approx(v_stokes, rel=2e-3 + 3e-3 * (r / 1e-6) ** 1.5)
    # Gunn & Kinzer (1949) at 1013 hPa, 20 C: D = 0.2, 1, 2 mm
    for D, v_gk in [(0.2e-3, 0.72), (1e-3, 4.03), (2e-3, 6.49)]:
        assert oracle.vterm((D / 2) ** 2, t) == pytest.approx(v_gk, rel=0.12)


def test_corrections_slow_small_and_ventilate_large_drops():
    t = oracle.thermo(289.0, 7.5e-3, RHOD_1KM)
    small = oracle.growth(0.2e-6 ** 2, 0.01e-6 ** 3, 0.61, t, 1) / oracle.growth(0.2e-6 ** 2, 0.01e-6 ** 3, 0.61, t, 0)
    large = oracle.growth(300e-6 ** 2, 0.1e-6 ** 3, 0.61, t, 1) / oracle.growth(300e-6 ** 2, 0.1e-6 ** 3, 0.61, t, 0)
    assert 0.2 < small < 1.0       # gas-kinetic (transition regime) limitation
    assert 1.5 < large < 10.0      # ventilation of a falling drizzle drop
    # limits: Re -> 0 and Kn -> 0 leave the bare Maxwell-Mason rate
    mid = oracle.growth(8e-6 ** 2, 0.05e-6 ** 3, 0.61, t, 1) / oracle.growth(8e-6 ** 2, 0.05e-6 ** 3, 0.61, t, 0)
    assert mid == pytest.approx(1.0, abs=0.03)


@pytest.mark.parametrize("RH", [0.5, 0.8, 0.95, 0.999])
@pytest.mark.parametrize("rd", [0.01e-6, 0.05e-6, 0.3e-6])
def test_koehler_equilibrium_root(RH, rd):
    T, kappa = 285.0, 0.61
    rd3 = rd ** 3
    A = 2 * SIGMA_W / (R_V * T * RHO_W)

    def S(r):
        return (r ** 3 - rd3) / (r ** 3 - rd3 * (1 - kappa)) * math.exp(A / r)
    # left branch: below the Koehler maximum
    rgrid = np.exp(np.linspace(math.log(rd * 1.0000001), math.log(rd * 1e4), 20000))
    r_crit = rgrid[np.argmax([S(r) for r in rgrid])]
    r_ref = brentq(lambda r: S(r) - RH, rd * (1 + 1e-12), r_crit, xtol=1e-22, rtol=1e-15)
    x = oracle.equilibrium_rw2(rd3, kappa, RH, T)
    assert math.sqrt(x) == pytest.approx(r_ref, rel=1e-12)


def _solve_case(x0, rd3, kappa, th, rv, rhod, dtp, physics):
    t = oracle.thermo(th, rv, rhod)
    x1, st = oracle.solve_rw2(x0, rd3, kappa, t, dtp, physics)
    g0 = oracle.growth(x0, rd3, kappa, t, physics)
    return t, x1, st, g0


def test_implicit_solve_residual_and_bracket():
    rng = np.random.default_rng(3)
    n_bis = 0
    for _ in range(300):
        rd = math.exp(rng.uniform(math.log(0.01e-6), math.log(0.5e-6)))
        r = rd * math.exp(rng.uniform(0.01, 6.0))
        rv = rng.uniform(5e-3, 9e-3)
        t, x1, st, g0 = _solve_case(r * r, rd ** 3, 0.61, 289.0, rv, RHOD_1KM, 0.1, 1)
        a = max(rd ** 2, r * r + min(0.2 * g0, 0.0))
        b = r * r + max(0.2 * g0, 0.0)
        assert a <= x1 <= b
        if st.n_euler == 0:
            n_bis += 1
            # x1 solves x = x0 + dt' g(x) to the bisection's resolution
            f = x1 - r * r - 0.1 * oracle.growth(x1, rd ** 3, 0.61, t, 1)
            slope = 1.0 + 0.1 * abs(g0) / max(b - a, 1e-300)
            assert abs(f) <= 64 * 2.0 ** -52 * b * max(slope, 1.0)
    assert n_bis > 100


def test_ill_posed_bracket_returns_euler_step():
    # search for inputs where f keeps its sign over [a, b]; there the paper's
    # procedure reduces to the explicit Euler step x0 + dt' g(x0)
    rng = np.random.default_rng(5)
    found = 0
    for _ in range(4000):
        rd = math.exp(rng.uniform(math.log(0.01e-6), math.log(0.2e-6)))
        r = rd * math.exp(rng.uniform(0.3, 4.0))
        rv = rng.uniform(7.5e-3, 1.2e-2)
        t, x1, st, g0 = _solve_case(r * r, rd ** 3, 0.61, 289.0, rv, RHOD_1KM, 1.0, 1)
        if st.n_euler and g0 != 0.0 and r * r + 2.0 * g0 > rd * rd:
            found += 1
            assert x1 == pytest.approx(r * r + 1.0 * g0, rel=1e-15)
    assert found >= 5


def test_condensation_conserves_total_water_and_updates_theta():
    w = workloads.icmw_2d(nx=4, nz=75, sd_conc=16, seed=2)
    o = oracle.Oracle(w.cfg)
    o.init(w.th, w.rv, w.rhod)
    s = o.state
    dV = w.cfg["dx"] * w.cfg["dy"] * w.cfg["dz"]

    def per_cell_liquid(state):
        k = np.floor(state.z / w.cfg["dz"]).astype(int).clip(0, 74)
        i = np.floor(state.x / w.cfg["dx"]).astype(int).clip(0, 3)
        c = i * 75 + k
        return np.bincount(c, weights=state.N.astype(float) * state.rw2 ** 1.5, minlength=o.n_cells)

    th0, rv0 = o.th.copy(), o.rv.copy()
    L0 = per_cell_liquid(s)
    condense(w.cfg, s, o.th, o.rv, o.rhod, sstp=1)
    L1 = per_cell_liquid(s)
    total0 = rv0 + 4 * math.pi * RHO_W / (3 * o.rhod * dV) * L0
    total1 = o.rv + 4 * math.pi * RHO_W / (3 * o.rhod * dV) * L1
    np.testing.assert_allclose(total1, total0, rtol=1e-13)
    assert np.abs(o.rv - rv0).max() > 1e-6  # something condensed
    # theta moves by dr_v * dtheta/dr_v with -theta l_v / (c_pd T) at the start
    for c in range(o.n_cells):
        t = oracle.thermo(th0[c], rv0[c], o.rhod[c])
        dth = (o.rv[c] - rv0[c]) * (-th0[c] * t.lv / (C_PD * t.T))
        assert o.th[c] - th0[c] == pytest.approx(dth, rel=1e-9, abs=1e-15)
    # several substeps: still conserved
    condense(w.cfg, s, o.th, o.rv, o.rhod, sstp=10)
    L2 = per_cell_liquid(s)
    total2 = o.rv + 4 * math.pi * RHO_W / (3 * o.rhod * dV) * L2
    np.testing.assert_allclose(total2, total0, rtol=1e-13)


def test_parabolic_growth_of_a_large_drop():
    # one 25 um drop with a negligible solute in a huge cell (no feedback)
    cfg = box_cfg(n_sd=1, dV=1e12, dt=1.0)
    cfg.update(kernel="geometric", physics=0)
    rd = 1e-9
    s = make_state([1], np.array([(25e-6) ** 2]), rd3=np.array([rd ** 3]), kappa=np.array([0.61]))
    th, rv, rhod = np.array([289.0]), np.array([9.0e-3]), np.array([RHOD_1KM])
    t = oracle.thermo(289.0, 9.0e-3, RHOD_1KM)
    x0 = s.rw2[0]
    for _ in range(20):
        condense(cfg, s, th, rv, rhod, sstp=10)
    es = t.rho_vs * R_V * t.T
    Fk = (t.lv / (R_V * t.T) - 1.0) * t.lv * RHO_W / (2.4e-2 * t.T)
    Fd = RHO_W * R_V * t.T / (2.26e-5 * es)
    S = t.rho_v / t.rho_vs
    # r^2 grows linearly at 2 (S - 1) / (F_k + F_d) (Kelvin term ~1e-4 of S - 1)
    assert (s.rw2[0] - x0) / 20.0 == pytest.approx(2 * (S - 1) / (Fk + Fd), rel=2e-3)
