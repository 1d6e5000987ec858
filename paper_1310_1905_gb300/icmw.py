"""The 2D kinematic cloud case run the way the paper runs it (Sec. 2.2):
a two-hour spin-up with precipitation formation and drop sedimentation off
and the supersaturation used in drop growth capped at RH = 1.05, then the
main run with every process on; the Eulerian fields theta and r_v are
transported by the prescribed eddy and their level means relaxed to the
initial profile before every step.  Then the dry and wet size spectra in
ten 3x3-cell regions along the cloud's pathway (Sec. 5.4).

Host orchestration only: every step runs in the CUDA library
(sdm_euler_step, sdm_step_sync, sdm_step_async, sdm_diag_spectrum).

    python -m paper_1310_1905_gb300.icmw [--spinup 7200] [--main 1800]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

SPINUP_OPTS = dict(adve=1, sedi=0, cond=1, coal=0, RH_max=1.05, sstp_cond=10, sstp_coal=10)
MAIN_OPTS = dict(adve=1, sedi=1, cond=1, coal=1, RH_max=44.0, sstp_cond=10, sstp_coal=10)

# Bins of the spectra (Sec. 5.4): dry, 40 log-spaced bins from 1 nm to
# 10 um; wet, 25 log-spaced bins from 1 nm to 100 um.
DRY_EDGES = np.geomspace(1e-9, 10e-6, 41)
WET_EDGES = np.geomspace(1e-9, 100e-6, 26)


def locations(nx: int, nz: int) -> dict:
    """Centres (i, k) of the ten 3x3-cell regions, as fractions of the
    domain along the pathway the paper describes: the updraught axis at
    x = X/4 below, across and above cloud base (i, g, e, c), near cloud top
    (a), above the downdraught (b), the downdraught at the altitude of (c)
    (d) and on its way down (f, h, j)."""
    frac = dict(i=(0.25, 0.33), g=(0.25, 0.50), e=(0.25, 0.55), c=(0.25, 0.60), a=(0.37, 0.93),
                b=(0.75, 0.93), d=(0.63, 0.60), f=(0.75, 0.50), h=(0.75, 0.33), j=(0.75, 0.13))
    return {k: (min(nx - 2, max(1, int(fx * nx))), min(nz - 2, max(1, int(fz * nz)))) for k, (fx, fz) in frac.items()}


def region_cells(i: int, k: int, nz: int) -> list[int]:
    return [(i + di) * nz + (k + dk) for di in (-1, 0, 1) for dk in (-1, 0, 1)]


def run(p, w, th, rv, spinup: int, main: int, on_step=None):
    """Advance the context p (set up from workload w, fields th, rv) by
    spinup + main steps; on_step(n, phase) after each."""
    th0, rv0 = w.th.mean(axis=0), w.rv.mean(axis=0)
    for n in range(spinup + main):
        opts = SPINUP_OPTS if n < spinup else MAIN_OPTS
        p.euler_step(th, rv, w.rhoCx, w.rhoCy, w.rhoCz, th0, rv0)
        p.step_sync(opts, th, rv)
        p.step_async(opts)
        p.wait()
        if on_step:
            on_step(n, "spinup" if n < spinup else "main")


def spectra(p, nx: int, nz: int) -> dict:
    """Number per unit dry-air mass [kg^-1] per bin (the k = 0 moment of
    sdm_diag_spectrum), dry and wet, averaged over each region's 9 cells."""
    dry = p.diag_spectrum(False, DRY_EDGES, 0)
    wet = p.diag_spectrum(True, WET_EDGES, 0)
    out = {}
    for name, (i, k) in locations(nx, nz).items():
        cells = region_cells(i, k, nz)
        out[name] = dict(centre_cell=(i, k), dry=dry[:, cells].mean(axis=1), wet=wet[:, cells].mean(axis=1))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--spinup", type=int, default=7200)
    ap.add_argument("--main", type=int, default=1800)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--json", default=None, help="also write the spectra here")
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads
    from . import sdm

    w = workloads.icmw_2d(seed=args.seed)
    th, rv = w.th.copy(), w.rv.copy()
    p = sdm.Particles(w.cfg, th, rv, w.rhod, w.rhoCx, None, w.rhoCz)
    lwc = []

    def probe(n, phase):
        if (n + 1) % 600 == 0:
            m3 = p.diag_moments(True, 0.5e-6, 1.0, 3)
            lwc.append((n + 1, phase, float(4.0 / 3.0 * math.pi * 1000.0 * m3.mean())))

    run(p, w, th, rv, args.spinup, args.main, probe)
    sp = spectra(p, w.cfg["nx"], w.cfg["nz"])
    print(f"ICMW 2D case: {args.spinup} s spin-up (coal = sedi = 0, RH_max = 1.05) + {args.main} s main run, "
          f"{p.n_sd} super-droplets; domain-mean liquid water [kg/kg] every 600 s:")
    for n, phase, v in lwc:
        print(f"  t = {n:5d} s ({phase}): {v:.4e}")
    print("region  centre(i,k)  wet spectrum: total [1/mg], modal radius [um]; dry: total [1/mg], modal [um]")
    wm = np.sqrt(WET_EDGES[1:] * WET_EDGES[:-1])
    dm = np.sqrt(DRY_EDGES[1:] * DRY_EDGES[:-1])
    for name in "abcdefghij":
        s = sp[name]
        print(f"  ({name})  {s['centre_cell']}  {s['wet'].sum() / 1e6:8.2f}  {wm[np.argmax(s['wet'])] * 1e6:8.3f}   "
              f"{s['dry'].sum() / 1e6:8.2f}  {dm[np.argmax(s['dry'])] * 1e6:8.4f}")
    if args.json:
        with open(args.json, "w") as f:
            json.dump(dict(spinup=args.spinup, main=args.main, lwc=lwc, dry_edges=DRY_EDGES.tolist(),
                           wet_edges=WET_EDGES.tolist(),
                           regions={k: dict(centre_cell=v["centre_cell"], dry=v["dry"].tolist(), wet=v["wet"].tolist())
                                    for k, v in sp.items()}), f)
    p.close()


if __name__ == "__main__":
    main()
