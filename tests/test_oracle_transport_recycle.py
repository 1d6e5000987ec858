"""Pins of the oracle's particle transport (paper Sec. 5.1.2 eqs. adv_implicit,
adv_c, adv_w; Sec. 5.1.5) and recycling (Sec. 5.1.4): exact translation in a
uniform flow, the residual of the implicit equation in a linear flow,
periodic wrap, exits with rainfall, and a hand-worked recycling example."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle_helpers import make_state, recycle, transport

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def slab_cfg(nx, nz, dx=20.0, dz=20.0, dt=1.0):
    return dict(nx=nx, ny=0, nz=nz, dx=dx, dy=1.0, dz=dz, dt=dt, sd_conc=1, kernel="geometric",
                init_dist="lognormal", modes=[dict(rm=1e-7, sigma=1.5, n_stp=1e8, kappa=0.6)],
                seed=0, physics=1)


def fields(nx, nz, rhod=1.1):
    f = lambda v: np.full(nx * nz, v, np.float64)
    return f(289.0), f(7e-3), f(rhod)


def test_uniform_courant_translates_exactly():
    nx, nz = 8, 6
    cfg = slab_cfg(nx, nz)
    th, rv, rhod = fields(nx, nz)
    Cx, Cz = 0.23, -0.11
    rhoCx = np.full((nx + 1) * nz, Cx * 1.1)
    rhoCz = np.full(nx * (nz + 1), Cz * 1.1)
    rng = np.random.default_rng(0)
    x0 = rng.uniform(0, nx * 20.0, 50)
    z0 = rng.uniform(30.0, nz * 20.0 - 30.0, 50)
    s = make_state(np.ones(50), np.full(50, 1e-12), x=x0, z=z0)
    transport(cfg, s, th, rv, rhod, rhoCx=rhoCx, rhoCz=rhoCz, sedi=0)
    np.testing.assert_allclose(s.z, z0 + 20.0 * Cz, rtol=1e-13)
    np.testing.assert_allclose(s.x, np.mod(x0 + 20.0 * Cx, nx * 20.0), rtol=1e-13)


def test_linear_courant_solves_backward_euler():
    # C varies from edge to edge; the new position must satisfy
    # x' = x + dx C(x') with C linear between the edges of the old cell
    nx, nz = 10, 1
    cfg = slab_cfg(nx, nz)
    th, rv, rhod = fields(nx, nz, rhod=1.0)
    Cedge = np.linspace(0.05, 0.4, nx + 1)
    Cedge[-1] = Cedge[0]  # periodic: first and last edge coincide
    rhoCx = Cedge.copy()
    rng = np.random.default_rng(1)
    x0 = rng.uniform(0, 9 * 20.0, 200)
    s = make_state(np.ones(200), np.full(200, 1e-12), x=x0, z=np.full(200, 10.0))
    transport(cfg, s, th, rv, rhod, rhoCx=rhoCx, rhoCz=np.zeros(nx * 2), sedi=0)
    i = np.floor(x0 / 20.0)
    Cl, Cr = Cedge[i.astype(int)], Cedge[i.astype(int) + 1]
    xn = s.x + np.where(s.x < x0, nx * 20.0, 0.0)  # undo the wrap
    omega = xn / 20.0 - i
    resid = xn - x0 - 20.0 * ((1 - omega) * Cl + omega * Cr)
    assert np.abs(resid).max() < 1e-11


def test_periodic_wrap_and_exits():
    nx, nz = 4, 3
    cfg = slab_cfg(nx, nz)
    th, rv, rhod = fields(nx, nz)
    rhoCx = np.full((nx + 1) * nz, 0.5 * 1.1)
    rhoCz = np.zeros(nx * (nz + 1))
    s = make_state([3, 5], np.array([1e-12, (1e-3) ** 2]), x=np.array([79.0, 10.0]), z=np.array([30.0, 2.0]))
    st = transport(cfg, s, th, rv, rhod, rhoCx=rhoCx, rhoCz=rhoCz, sedi=1)
    # first: 79 + 10 wraps to 9, falls negligibly
    assert s.x[0] == pytest.approx(9.0, abs=1e-12)
    assert s.N[0] == 3
    # second: 1 mm drop falls > 2 m in 1 s and leaves through the bottom
    assert s.N[1] == 0 and s.z[1] == 0.0
    assert st.rainfall == pytest.approx(5 * 4.0 / 3.0 * math.pi * 1000.0 * 1e-9, rel=1e-14)


def test_sedimentation_is_explicit_euler():
    """z' = z - v_t dt with v_t fixed at the step start: the displacement is
    exactly proportional to dt (a fall speed re-evaluated along the way, or
    an implicit step, would not be), and for a 5 um droplet it is Stokes'
    fall speed 2/9 (rho_w - rho_a) g r^2 / mu with the textbook viscosity of
    air at 10 C, 1.76e-5 Pa s (the cell is at about 283 K)."""
    nx, nz = 1, 50
    th, rv, rhod = fields(nx, nz)
    r = np.array([5e-6, 50e-6, 400e-6])
    dz = {}
    for dt in (1.0, 2.5):
        cfg = dict(slab_cfg(nx, nz), dt=dt)
        s = make_state([1, 1, 1], r * r, z=np.array([600.0, 600.0, 600.0]))
        transport(cfg, s, th, rv, rhod, adve=0, sedi=1)
        dz[dt] = 600.0 - s.z
    assert (dz[1.0] > 0).all()
    # z - v dt is rounded at the magnitude of z: a few ulps of 600 m
    np.testing.assert_allclose(dz[2.5], 2.5 * dz[1.0], rtol=1e-13, atol=4 * np.spacing(600.0))
    stokes = 2.0 / 9.0 * (1000.0 - 1.1) * 9.81 * r[0] ** 2 / 1.76e-5
    assert dz[1.0][0] == pytest.approx(stokes, rel=0.03)


def test_recycling_golden():
    g = json.load(open(os.path.join(GOLDEN, "recycle_small.json")))
    b = g["before"]
    s = make_state(b["N"], np.array(b["rw2"]), uid=b["uid"], x=np.array(b["x"]))
    # shuffle the storage order: recycling must depend on ids only
    perm = np.array([5, 2, 7, 0, 3, 6, 1, 4])
    s2 = make_state(np.array(b["N"])[perm], np.array(b["rw2"])[perm], uid=np.array(b["uid"])[perm],
                    x=np.array(b["x"])[perm])
    for st in (s, s2):
        recycle(st)
        o = np.argsort(st.uid)
        assert st.N[o].tolist() == g["after"]["N"]
        assert st.rw2[o].tolist() == g["after"]["rw2"]
        assert st.x[o].tolist() == g["after"]["x"]


def test_recycling_conserves_droplets_and_skips_singletons():
    s = make_state([0, 1, 1, 0, 3], np.arange(1, 6) * 1.0)
    recycle(s)
    assert s.N.tolist() == [1, 1, 1, 0, 2]  # only one donor with N >= 2
