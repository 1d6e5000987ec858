"""Per-diagnostic errors of the mixed FP32/FP64 mode on the full 2D
kinematic case (75 x 75 cells, 64 super-droplets per cell).

theta and r_v are transported by the eddy and relaxed to their initial level
means every step (the library's Eulerian stand-in, sdm_euler_step).
The same seeded runs go through the FP64 mode (whose multiplicities match
the oracle bit for bit and whose radii match it to 1e-12, the parity tests'
bar) and the mixed mode.  FP32 accept/reject decisions can flip, so the two
are compared as statistics over seeds: at each output time the domain-mean
diagnostics of each mode are averaged over the seeds, and the difference of
the means is set against its standard error from the seed-to-seed spread.

Diagnostics (domain means of the moments of Sec. 5.2.1):
  cloud droplet concentration, wet radius 0.5-25 um  [1/mg of dry air]
  mean wet radius of those droplets                   [um]
  rain water mixing ratio, wet radius > 25 um         [g/kg]
  liquid water mixing ratio, wet radius > 0.5 um      [g/kg]
and the accumulated surface rainfall [kg].

  python -m paper_1310_1905_gb300.precision_report [--seeds 4] [--minutes 60] [--every 15]
"""
from __future__ import annotations

import argparse
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

RHO_W = 1000.0
NAMES = ("conc", "rmean", "rain", "lwc", "rainfall")
UNITS = dict(conc="1/mg", rmean="um", rain="g/kg", lwc="g/kg", rainfall="kg")


def diagnostics(p, rainfall: float) -> dict:
    m0c = p.diag_moments(True, 0.5e-6, 25e-6, 0)
    m1c = p.diag_moments(True, 0.5e-6, 25e-6, 1)
    m3r = p.diag_moments(True, 25e-6, 1.0, 3)
    m3 = p.diag_moments(True, 0.5e-6, 1.0, 3)
    return dict(conc=m0c.mean() * 1e-6,
                rmean=m1c.sum() / max(m0c.sum(), 1e-300) * 1e6,
                rain=4.0 / 3.0 * math.pi * RHO_W * m3r.mean() * 1e3,
                lwc=4.0 / 3.0 * math.pi * RHO_W * m3.mean() * 1e3,
                rainfall=rainfall)


def run(seed: int, precision: str, steps: int, every: int) -> dict:
    import torch

    import workloads
    from paper_1310_1905_gb300 import sdm

    w = workloads.icmw_2d(seed=seed)
    dev = lambda a: None if a is None else torch.tensor(a, dtype=torch.float64, device="cuda")
    th, rv = dev(w.th), dev(w.rv)
    Cx, Cz = dev(w.rhoCx), dev(w.rhoCz)
    th0, rv0 = w.th.mean(axis=0), w.rv.mean(axis=0)
    p = sdm.Particles(w.cfg, th, rv, dev(w.rhod), Cx, None, Cz, precision=precision)
    out = {}
    rain = 0.0
    for t in range(1, steps + 1):
        p.euler_step(th, rv, Cx, None, Cz, th0, rv0)  # the kinematic framework's Eulerian component
        p.step_sync(w.opts, th, rv)
        p.step_async(w.opts)
        rain = p.wait()
        if t % every == 0:
            out[t] = diagnostics(p, rain)
    p.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=4)
    ap.add_argument("--minutes", type=float, default=60.0)
    ap.add_argument("--every", type=float, default=15.0, help="output interval [min]")
    a = ap.parse_args()
    steps, every = int(a.minutes * 60), int(a.every * 60)
    res = {m: [run(s, m, steps, every) for s in range(a.seeds)] for m in ("fp64", "mixed")}
    print(f"2D kinematic case, 360 000 super-droplets, {a.seeds} seeds; mean over seeds (standard deviation); "
          f"z = (mixed - fp64) / standard error of that difference")
    print()
    print("| t [s] | diagnostic | FP64 | mixed | rel. difference | z |")
    print("|---|---|---|---|---|---|")
    for t in sorted(res["fp64"][0]):
        for n in NAMES:
            f = np.array([r[t][n] for r in res["fp64"]])
            m = np.array([r[t][n] for r in res["mixed"]])
            se = math.sqrt((f.var(ddof=1) + m.var(ddof=1)) / len(f)) if len(f) > 1 else float("nan")
            d = m.mean() - f.mean()
            rel = d / f.mean() if f.mean() != 0 else float("nan")
            z = d / se if se > 0 else float("nan")
            print(f"| {t} | {n} [{UNITS[n]}] | {f.mean():.6g} ({f.std(ddof=1):.2g}) | "
                  f"{m.mean():.6g} ({m.std(ddof=1):.2g}) | {rel:+.2e} | {z:+.2f} |")


if __name__ == "__main__":
    main()
