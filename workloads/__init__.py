"""Seeded synthetic workloads for the super-droplet hot path.

Each generator returns a :class:`Workload`: a plain domain description (the
dict both the CUDA binding and the oracle turn into their own option
structs), the Eulerian input fields theta, r_v, rho_d on cell centres, the
rho_d * Courant fields on the Arakawa-C cell edges, the per-step process
options and the step count.

This module holds only the *set-up* of the paper's test cases (Sec. 2.1-2.2:
hydrostatic profile, single-eddy stream function) and of the box / 3D /
ensemble stand-ins; none of the microphysics.  Random perturbations come from
numpy's seeded generator.  The super-droplets themselves are drawn by the
library and by the oracle from their own counter-based generators.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# set-up constants (dry-air and vapour gas constants, c_pd, gravity, p1000);
# the same values as the readings used by the library and the oracle
_R_D, _R_V, _C_PD, _G, _P1000 = 287.0, 461.5, 1005.0, 9.81, 1.0e5

# bimodal ammonium-sulphate aerosol with the radii of the measured workloads
AEROSOL_BIMODAL = [
    dict(rm=0.04e-6, sigma=1.4, n_stp=60e6, kappa=0.61),
    dict(rm=0.15e-6, sigma=1.6, n_stp=40e6, kappa=0.61),
]
# the same modes with the paper's mode *diameters* halved (Sec. 2.2 prints
# d = 2 r = 0.04 and 0.15 um)
AEROSOL_BIMODAL_PAPER = [dict(m, rm=m["rm"] / 2) for m in AEROSOL_BIMODAL]

OPTS_DEFAULT = dict(adve=1, sedi=1, cond=1, coal=1, RH_max=44.0, sstp_cond=10, sstp_coal=10)


@dataclasses.dataclass
class Workload:
    name: str
    cfg: dict
    th: np.ndarray
    rv: np.ndarray
    rhod: np.ndarray
    rhoCx: np.ndarray | None
    rhoCy: np.ndarray | None
    rhoCz: np.ndarray | None
    opts: dict
    n_steps: int

    @property
    def n_cells(self) -> int:
        return int(self.th.size)

    @property
    def n_sd(self) -> int:
        groups = 1 if self.cfg.get("init_dist") == "exponential" else len({m["kappa"] for m in self.cfg["modes"]})
        return self.n_cells * self.cfg["sd_conc"] * groups


def hydrostatic_rhod(z: np.ndarray, theta: float, rv: float, p0: float) -> np.ndarray:
    """Dry-air density of a hydrostatic column with constant dry potential
    temperature ``theta`` (defined with the dry-air pressure) and constant
    vapour mixing ratio ``rv``; ``p0`` is the total pressure at z = 0.

    With p = p_d (1 + r_v R_v/R_d) and rho = rho_d (1 + r_v), hydrostatic
    balance makes p_d^(R_d/c_pd) linear in z."""
    k = _R_D / _C_PD
    f = 1.0 + rv * _R_V / _R_D
    pd0 = p0 / f
    pdk = pd0 ** k - k * _G * (1.0 + rv) * _P1000 ** k * z / (f * _R_D * theta)
    pd = pdk ** (1.0 / k)
    T = theta * (pd / _P1000) ** k
    return pd / (_R_D * T)


def golovin_box(seed: int = 0, n_sd: int = 2 ** 13, n_steps: int = 3600) -> Workload:
    """Box-model coalescence test (Shima et al. 2009 set-up): one cell of
    1e6 m^3, Golovin kernel b = 1500 s^-1, exponential-in-volume initial
    spectrum with mean radius 30.531 um and n0 = 2^23 m^-3, dt = 1 s."""
    rbar = 30.531e-6
    cfg = dict(nx=0, ny=0, nz=0, dx=100.0, dy=100.0, dz=100.0, dt=1.0, sd_conc=n_sd,
               kernel="golovin", golovin_b=1500.0, init_dist="exponential",
               exp_mean_volume=4.0 / 3.0 * math.pi * rbar ** 3, exp_n0=2.0 ** 23,
               modes=[], seed=seed, physics=1)
    one = np.ones(1)
    opts = dict(adve=0, sedi=0, cond=0, coal=1, RH_max=44.0, sstp_cond=1, sstp_coal=1)
    return Workload("golovin_box", cfg, 300.0 * one, 0.01 * one, 1.0 * one, None, None, None, opts, n_steps)


def icmw_2d(nx: int = 75, nz: int = 75, sd_conc: int = 64, seed: int = 0, n_steps: int = 3600,
            dx: float = 20.0, dz: float = 20.0, dt: float = 1.0, w_max: float = 0.6,
            modes=None, physics: int = 1) -> Workload:
    """2D prescribed-flow kinematic case (8th ICMW case 1, Sec. 2.2):
    single-eddy stream function psi = -w_max X/pi sin(pi z/Z) cos(2 pi x/X),
    theta = theta_l = 289 K and r_v = r_t = 7.5 g/kg at all heights, hydrostatic
    rho_d with 1015 hPa at the ground.  rho_d u = -d psi/dz and
    rho_d w = d psi/dx are differenced from psi at cell corners, so the
    discrete rho_d-weighted flow is divergence free."""
    X, Z = nx * dx, nz * dz
    zc = (np.arange(nz) + 0.5) * dz
    rhod1 = hydrostatic_rhod(zc, 289.0, 7.5e-3, 101500.0)
    rhod = np.repeat(rhod1[None, :], nx, axis=0)
    th = np.full((nx, nz), 289.0)
    rv = np.full((nx, nz), 7.5e-3)

    def psi(x, z):
        return -w_max * X / math.pi * np.sin(math.pi * z / Z) * np.cos(2 * math.pi * x / X)

    xe = np.arange(nx + 1) * dx
    ze = np.arange(nz + 1) * dz
    # rho_d u on x-edges (nx+1, nz): minus the z-difference of psi at corners
    rhou = -(psi(xe[:, None], ze[None, 1:]) - psi(xe[:, None], ze[None, :-1])) / dz
    # rho_d w on z-edges (nx, nz+1): the x-difference of psi at corners
    rhow = (psi(xe[None, 1:].T, ze[None, :]) - psi(xe[None, :-1].T, ze[None, :])) / dx
    rhoCx = rhou * dt / dx
    rhoCz = rhow * dt / dz
    cfg = dict(nx=nx, ny=0, nz=nz, dx=dx, dy=1.0, dz=dz, dt=dt, sd_conc=sd_conc,
               kernel="geometric", golovin_b=0.0, init_dist="lognormal",
               exp_mean_volume=0.0, exp_n0=0.0, modes=list(modes or AEROSOL_BIMODAL),
               seed=seed, physics=physics)
    return Workload("icmw_2d", cfg, th, rv, rhod, np.ascontiguousarray(rhoCx), None,
                    np.ascontiguousarray(rhoCz), dict(OPTS_DEFAULT), n_steps)


def updraft_3d(nx: int = 128, ny: int = 128, nz: int = 128, sd_conc: int = 32, seed: int = 0,
               n_steps: int = 600, dx: float = 20.0, dt: float = 1.0, w: float = 1.0,
               physics: int = 1) -> Workload:
    """Large 3D-shaped kinematic domain: 20 m cubes, theta = 289 K,
    r_v = 7.5 g/kg, hydrostatic rho_d; rho_d * w = rho_d(0) * w * (1 + 0.1 xi)
    constant along each column, xi ~ U(-1, 1) per column from ``seed``;
    no horizontal flow; periodic in x and y, outflow through the top."""
    zc = (np.arange(nz) + 0.5) * dx
    rhod1 = hydrostatic_rhod(zc, 289.0, 7.5e-3, 101500.0)
    rhod = np.broadcast_to(rhod1[None, None, :], (nx, ny, nz)).copy()
    th = np.full((nx, ny, nz), 289.0)
    rv = np.full((nx, ny, nz), 7.5e-3)
    rng = np.random.default_rng(seed)
    xi = rng.uniform(-1.0, 1.0, size=(nx, ny))
    rho0 = float(hydrostatic_rhod(np.array([0.0]), 289.0, 7.5e-3, 101500.0)[0])
    flux = rho0 * w * (1.0 + 0.1 * xi)
    rhoCz = np.repeat((flux * dt / dx)[:, :, None], nz + 1, axis=2)
    rhoCx = np.zeros((nx + 1, ny, nz))
    rhoCy = np.zeros((nx, ny + 1, nz))
    cfg = dict(nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, dz=dx, dt=dt, sd_conc=sd_conc,
               kernel="geometric", golovin_b=0.0, init_dist="lognormal",
               exp_mean_volume=0.0, exp_n0=0.0, modes=list(AEROSOL_BIMODAL),
               seed=seed, physics=physics)
    return Workload("updraft_3d", cfg, th, rv, rhod, rhoCx, rhoCy, np.ascontiguousarray(rhoCz),
                    dict(OPTS_DEFAULT), n_steps)


def ensemble_members(n_members: int = 256, seed: int = 0, n_min: float = 1e3, n_max: float = 1e6,
                     parcel_fraction: float = 0.5) -> list[dict]:
    """Ragged ensemble of 0D members: N_sd log-uniform in [n_min, n_max];
    one or two lognormal modes sharing one kappa, with log-uniform mode radius
    (0.02-0.1 um) and concentration (50-500 cm^-3), sigma in [1.3, 1.8],
    kappa in [0.2, 1.2]; boxes and adiabatic parcels (updraft w in
    [0.1, 5] m/s from 600 m in the 2D case's hydrostatic column).  Each member
    is a dict for the ensemble binding plus 'w' and 'z0' for parcels."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_members):
        n_sd = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        kappa = float(rng.uniform(0.2, 1.2))
        modes = []
        for _ in range(int(rng.integers(1, 3))):
            modes.append(dict(rm=float(math.exp(rng.uniform(math.log(0.02e-6), math.log(0.1e-6)))),
                              sigma=float(rng.uniform(1.3, 1.8)),
                              n_stp=float(math.exp(rng.uniform(math.log(50e6), math.log(500e6)))), kappa=kappa))
        parcel = bool(rng.uniform() < parcel_fraction)
        z0 = 600.0
        rhod0 = float(hydrostatic_rhod(np.array([z0]), 289.0, 7.5e-3, 101500.0)[0])
        out.append(dict(n_sd=n_sd, dV=1.0, th=289.0, rv=7.5e-3, rhod=rhod0, modes=modes,
                        seed=int(seed) * 100003 + k, w=float(rng.uniform(0.1, 5.0)) if parcel else 0.0, z0=z0))
    return out


def parcel_rhod(members: list[dict], t: float) -> dict:
    """rho_d at time t of every parcel member (index -> value), rising at w
    from z0 through the 2D case's hydrostatic column."""
    out = {}
    for k, m in enumerate(members):
        if m.get("w", 0.0) > 0.0:
            out[k] = float(hydrostatic_rhod(np.array([m["z0"] + m["w"] * t]), 289.0, 7.5e-3, 101500.0)[0])
    return out
