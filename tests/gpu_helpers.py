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


def pair(w, precision="fp64"):
    """GPU particles and oracle on the same inputs, same initial integers."""
    p, o = gpu_particles(w, precision), oracle_sim(w)
    start_from_oracle_multiplicities(p, o)
    return p, o


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


def start_from_oracle_multiplicities(p, o):
    """Initial multiplicities are floor(v + 1/2) of an FP64 value v computed
    with exp() on both sides; where v lies within a few ulps of a half-integer
    the two sides may round differently (checked by the init tests).  The
    dynamics tests therefore start the GPU from the oracle's integers."""
    uid = p.attr("uid").astype(np.int64)
    order = np.argsort(o.state.uid)
    N_by_uid = o.state.N[order]
    sdm.sdm_set_attr(p.ctx, "N", N_by_uid[uid])


def rounding_ambiguous(v):
    """True where floor(v + 1/2) may flip under a few ulps of v."""
    v = np.asarray(v, np.float64)
    return np.abs(v - np.floor(v) - 0.5) <= 16 * np.spacing(v)


def compare_states(g, r, rtol=RTOL, exact_N=True, nreal=None):
    assert np.array_equal(g["uid"], r["uid"].astype(g["uid"].dtype))
    if exact_N:
        bad = np.nonzero(g["N"] != r["N"])[0]
        if nreal is not None and bad.size:
            # an init comparison: only rounding-ambiguous values may differ, by one
            assert rounding_ambiguous(nreal[bad]).all(), "a multiplicity differs away from a rounding tie"
            assert (np.abs(g["N"][bad].astype(np.int64) - r["N"][bad].astype(np.int64)) == 1).all()
            bad = bad[:0]
        assert bad.size == 0, f"multiplicities differ for {bad.size} super-droplets, first ids {g['uid'][bad[:5]]}: " \
                              f"gpu {g['N'][bad[:5]]} oracle {r['N'][bad[:5]]}"
    for k in ("rw2", "rd3", "kappa"):
        assert_close(k, g[k], r[k], rtol)
    for d in ("x", "y", "z"):
        if d in g:
            assert_close(d, g[d], r[d], rtol, atol=1e-9)


R_D, R_V, C_PD = 287.0, 461.5, 1005.0


def theta_ulps(T_gpu, rho_vs_gpu, th, rv, rhod):
    """The change of theta, in ulps of theta, that moves the oracle's T and
    rho_vs as far as they differ from the GPU's (d ln T / d ln theta =
    c_pd / (c_pd - R_d), d ln rho_vs / d ln T = l_v / (R_v T) - 1): the
    input perturbation under which the oracle's own spread measures what the
    two math libraries' rounding of exp, pow and log can move a result."""
    t = oracle.thermo(th, rv, rhod)
    dT = abs(T_gpu / t.T - 1.0)
    drho = abs(rho_vs_gpu / t.rho_vs - 1.0)
    eth = (C_PD - R_D) / C_PD * max(dT, drho / (t.lv / (R_V * t.T) - 1.0))
    return max(1, int(np.ceil(eth / (np.spacing(th) / th))))
