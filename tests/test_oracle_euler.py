"""Pins of the oracle's Eulerian stand-in (the kinematic framework's transport
of theta and r_v, Sec. 2.1-2.2: first-order donor cell in flux form) and of
the relaxation of the horizontal means (Sec. 2.2), against results fixed by
the scheme's definition and by conservation:

* uniform flow in a periodic row: Courant 1 shifts the field by exactly one
  cell (either way), Courant 1/2 gives the textbook upwind average;
* the ICMW eddy (divergence free in the rho_d-weighted sense): a constant
  field stays constant, sum rho_d psi dV is conserved, no new extrema;
* relaxation: the level mean approaches the profile by dt/tau with
  tau = 300 s exp(z / 200 m), deviations from the mean are untouched.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def row_cfg(nx, dx=10.0, dt=1.0):
    return dict(nx=nx, ny=0, nz=0, dx=dx, dy=1.0, dz=1.0, dt=dt, sd_conc=1, kernel="geometric", modes=[],
                seed=0, physics=1)


@pytest.mark.parametrize("C", [1.0, -1.0])
def test_courant_one_shifts_by_one_cell(C):
    nx = 12
    rng = np.random.default_rng(1)
    psi = rng.uniform(280, 300, nx)
    rhod = np.full(nx, 1.2)
    rhoCx = np.full(nx + 1, 1.2 * C)
    out = oracle.upwind(row_cfg(nx), psi, rhod, rhoCx)
    np.testing.assert_allclose(out, np.roll(psi, 1 if C > 0 else -1), rtol=1e-15)


def test_courant_half_is_the_upwind_average():
    nx = 9
    psi = np.arange(nx, dtype=float) ** 2
    rhod = np.full(nx, 0.8)
    out = oracle.upwind(row_cfg(nx), psi, rhod, np.full(nx + 1, 0.8 * 0.5))
    np.testing.assert_allclose(out, 0.5 * psi + 0.5 * np.roll(psi, 1), rtol=1e-15)


def test_icmw_eddy_constant_conservation_and_bounds():
    w = workloads.icmw_2d(nx=15, nz=15, sd_conc=1, seed=0, dx=100.0, dz=100.0)
    rhod = w.rhod.ravel()
    # a constant field stays constant: the flow is divergence free
    const = oracle.upwind(w.cfg, np.full(rhod.size, 289.0), rhod, w.rhoCx, None, w.rhoCz)
    np.testing.assert_allclose(const, 289.0, rtol=1e-13)
    # a lumpy field: total rho_d psi conserved, no value outside the old range
    rng = np.random.default_rng(3)
    psi = rng.uniform(7e-3, 8e-3, rhod.size)
    start = psi.copy()
    tot0 = (rhod * psi).sum()
    for _ in range(20):
        new = oracle.upwind(w.cfg, psi, rhod, w.rhoCx, None, w.rhoCz)
        assert new.min() >= psi.min() * (1 - 1e-14) and new.max() <= psi.max() * (1 + 1e-14)
        psi = new
    assert (rhod * psi).sum() == pytest.approx(tot0, rel=1e-13)
    assert np.abs(psi - start).max() > 1e-5  # it moved


def test_relaxation_of_level_means():
    nx, nz, dz, dt = 6, 5, 20.0, 1.0
    cfg = dict(nx=nx, ny=0, nz=nz, dx=20.0, dy=1.0, dz=dz, dt=dt, sd_conc=1, kernel="geometric", modes=[],
               seed=0, physics=1)
    rng = np.random.default_rng(2)
    psi = rng.uniform(288, 292, (nx, nz))
    psi0 = np.full(nz, 289.0)
    psi0[2] = psi[:, 2].mean()  # this level is already at its profile
    out = oracle.relax(cfg, psi, psi0).reshape(nx, nz)
    for k in range(nz):
        tau = 300.0 * math.exp((k + 0.5) * dz / 200.0)
        m0, m1 = psi[:, k].mean(), out[:, k].mean()
        assert m1 - psi0[k] == pytest.approx((m0 - psi0[k]) * (1 - dt / tau), rel=1e-9, abs=1e-12)
        np.testing.assert_allclose(out[:, k] - m1, psi[:, k] - m0, atol=1e-12)
    np.testing.assert_allclose(out[:, 2], psi[:, 2], rtol=1e-15)
