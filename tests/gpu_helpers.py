"""Shared driving code for the GPU parity tests: run a workload through the
C ABI (binding in paper_1310_1905_gb300.sdm) and through the oracle on the
same seeded inputs, and compare the results."""
import numpy as np

import oracle
from paper_1310_1905_gb300 import sdm

RTOL = 1e-12  # FP64 parity bar for radii, mixing ratios, moments


def gpu_particles(w, precision="fp64"):
    return sdm.Particles(w.cfg, w.th, w.rv, w.rhod, w.rhoCx, w.rhoCy, w.rhoCz, precision=precision)


def oracle_sim(w):
    o = oracle.Oracle(w.cfg)
    o.init(w.th, w.rv, w.rhod)
    return o


def oracle_state(o, present=("x", "z")):
    s = o.state.sorted_by_uid()
    out = {"uid": s.uid, "N": s.N, "rw2": s.rw2, "rd3": s.rd3, "kappa": s.kappa}
    for d in present:
        out[d] = getattr(s, d)
    return out


def present_dims(cfg):
    return tuple(d for d, n in (("x", "nx"), ("y", "ny"), ("z", "nz")) if cfg.get(n, 0) > 0)


def assert_close(name, got, ref, rtol=RTOL, atol=0.0):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    assert got.shape == ref.shape, name
    err = np.abs(got - ref)
    tol = rtol * np.abs(ref) + atol
    bad = err > tol
    if bad.any():
        i = int(np.argmax(err / np.maximum(tol, 1e-300)))
        raise AssertionError(f"{name}: {bad.sum()} of {bad.size} differ; worst at {i}: "
                             f"got {got[i]!r} ref {ref[i]!r} rel {err[i] / max(abs(ref[i]), 1e-300):.3e}")


def compare_states(g, r, rtol=RTOL, exact_N=True):
    assert np.array_equal(g["uid"], r["uid"].astype(g["uid"].dtype))
    if exact_N:
        bad = np.nonzero(g["N"] != r["N"])[0]
        assert bad.size == 0, f"multiplicities differ for {bad.size} super-droplets, first ids {g['uid'][bad[:5]]}: " \
                              f"gpu {g['N'][bad[:5]]} oracle {r['N'][bad[:5]]}"
    for k in ("rw2", "rd3", "kappa"):
        assert_close(k, g[k], r[k], rtol)
    for d in ("x", "y", "z"):
        if d in g:
            assert_close(d, g[d], r[d], rtol, atol=1e-9)
