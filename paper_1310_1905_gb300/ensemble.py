"""ctypes binding of the batched-ensemble part of the C ABI (sdm_ens_*,
include/sdm.h): argument marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np

from .sdm import (ATTR, INIT, KERNEL, PRECISION, SOLVER, SdmError, load, make_opts, sdm_lognormal,
                  sdm_stats)

SYMBOLS = ["sdm_ens_create", "sdm_ens_destroy", "sdm_ens_last_error", "sdm_ens_add", "sdm_ens_remove",
           "sdm_ens_members", "sdm_ens_step", "sdm_ens_wait", "sdm_ens_moments", "sdm_ens_fields",
           "sdm_ens_get_attr", "sdm_ens_use_graph", "sdm_ens_autotune", "sdm_ens_stats", "sdm_ens_memory"]


class sdm_member(C.Structure):
    _fields_ = [("n_sd", C.c_int64), ("dV", C.c_double), ("th", C.c_double), ("rv", C.c_double),
                ("rhod", C.c_double), ("init_dist", C.c_int), ("n_modes", C.c_int),
                ("modes", sdm_lognormal * 4), ("exp_mean_volume", C.c_double), ("exp_n0", C.c_double),
                ("seed", C.c_uint64)]


class sdm_ens_opts(C.Structure):
    _fields_ = [("dt", C.c_double), ("kernel", C.c_int), ("golovin_b", C.c_double), ("physics", C.c_int),
                ("precision", C.c_int), ("cond_solver", C.c_int), ("max_sd", C.c_int64),
                ("max_members", C.c_int32)]


_DECLARED = False


def _lib():
    global _DECLARED
    L = load()
    if not _DECLARED:
        P, V, I32, I64, D = C.POINTER, C.c_void_p, C.c_int32, C.c_int64, C.c_double
        e = C.c_void_p
        L.sdm_ens_create.argtypes = [P(sdm_ens_opts), V, P(e)]
        L.sdm_ens_destroy.argtypes = [e]
        L.sdm_ens_last_error.argtypes = [e]
        L.sdm_ens_last_error.restype = C.c_char_p
        L.sdm_ens_add.argtypes = [e, P(sdm_member), P(I32)]
        L.sdm_ens_remove.argtypes = [e, I32]
        L.sdm_ens_members.argtypes = [e, P(I32), I32, P(I32), P(I64)]
        L.sdm_ens_step.argtypes = [e, V, P(I32), P(D), I32]
        L.sdm_ens_wait.argtypes = [e, D]
        L.sdm_ens_moments.argtypes = [e, C.c_int, D, D, C.c_int, P(I32), P(D), I32]
        L.sdm_ens_fields.argtypes = [e, P(I32), P(D), P(D), I32]
        L.sdm_ens_get_attr.argtypes = [e, I32, C.c_int, V, I64]
        L.sdm_ens_use_graph.argtypes = [e, C.c_int]
        L.sdm_ens_autotune.argtypes = [e, V, P(C.c_int), P(C.c_int), P(C.c_int)]
        L.sdm_ens_stats.argtypes = [e, P(sdm_stats)]
        L.sdm_ens_memory.argtypes = [e, P(C.c_size_t), P(I64), P(I32)]
        for s in SYMBOLS:
            if s != "sdm_ens_last_error":
                getattr(L, s).restype = C.c_int
        _DECLARED = True
    return L


def make_member(m: dict) -> sdm_member:
    s = sdm_member()
    s.n_sd = int(m["n_sd"])
    s.dV = m["dV"]
    s.th, s.rv, s.rhod = m["th"], m["rv"], m["rhod"]
    s.init_dist = INIT[m.get("init_dist", "lognormal")]
    modes = m.get("modes", [])
    s.n_modes = len(modes)
    for i, md in enumerate(modes):
        s.modes[i] = sdm_lognormal(md["rm"], md["sigma"], md["n_stp"], md["kappa"])
    s.exp_mean_volume = m.get("exp_mean_volume", 0.0)
    s.exp_n0 = m.get("exp_n0", 0.0)
    s.seed = m.get("seed", 0)
    return s


class Ensemble:
    """A batch of 0D members advanced together (sdm_ens_* of the C ABI)."""

    def __init__(self, dt=1.0, kernel="geometric", golovin_b=0.0, physics=1, precision="fp64",
                 cond_solver="fast", max_sd=1 << 20, max_members=256, stream=None):
        L = _lib()
        o = sdm_ens_opts(dt, KERNEL[kernel], golovin_b, physics, PRECISION[precision], SOLVER[cond_solver],
                         int(max_sd), int(max_members))
        self.h = C.c_void_p()
        st = L.sdm_ens_create(C.byref(o), C.c_void_p(stream or 0), C.byref(self.h))
        if st != 0:
            raise SdmError(st, (L.sdm_last_error(None) or b"").decode())

    def _check(self, st):
        if st != 0:
            raise SdmError(st, (_lib().sdm_ens_last_error(self.h) or b"").decode())

    def add(self, member: dict) -> int:
        mid = C.c_int32()
        m = make_member(member)
        self._check(_lib().sdm_ens_add(self.h, C.byref(m), C.byref(mid)))
        return mid.value

    def remove(self, mid: int):
        self._check(_lib().sdm_ens_remove(self.h, mid))

    def members(self):
        n, nsd = C.c_int32(), C.c_int64()
        self._check(_lib().sdm_ens_members(self.h, None, 0, C.byref(n), C.byref(nsd)))
        ids = (C.c_int32 * max(1, n.value))()
        self._check(_lib().sdm_ens_members(self.h, ids, n.value, C.byref(n), C.byref(nsd)))
        return list(ids)[:n.value], nsd.value

    def step(self, opts: dict, rhod: dict | None = None):
        o = make_opts(opts)
        if rhod:
            ids = (C.c_int32 * len(rhod))(*rhod.keys())
            vals = (C.c_double * len(rhod))(*rhod.values())
            self._check(_lib().sdm_ens_step(self.h, C.byref(o), ids, vals, len(rhod)))
        else:
            self._check(_lib().sdm_ens_step(self.h, C.byref(o), None, None, 0))

    def wait(self, timeout_s=-1.0):
        self._check(_lib().sdm_ens_wait(self.h, timeout_s))

    def moments(self, ids, wet: bool, r_min: float, r_max: float, k: int) -> np.ndarray:
        ids = list(ids)
        a = (C.c_int32 * max(1, len(ids)))(*ids)
        out = (C.c_double * max(1, len(ids)))()
        self._check(_lib().sdm_ens_moments(self.h, int(wet), r_min, r_max, k, a, out, len(ids)))
        return np.array(out[:len(ids)])

    def fields(self, ids):
        ids = list(ids)
        a = (C.c_int32 * max(1, len(ids)))(*ids)
        th = (C.c_double * max(1, len(ids)))()
        rv = (C.c_double * max(1, len(ids)))()
        self._check(_lib().sdm_ens_fields(self.h, a, th, rv, len(ids)))
        return np.array(th[:len(ids)]), np.array(rv[:len(ids)])

    def attr(self, mid: int, name: str, n: int) -> np.ndarray:
        out = np.empty(n, {"N": np.uint64, "uid": np.uint32}.get(name, np.float64))
        self._check(_lib().sdm_ens_get_attr(self.h, mid, ATTR[name], out.ctypes.data, n))
        return out

    def use_graph(self, on=True):
        self._check(_lib().sdm_ens_use_graph(self.h, int(on)))

    def autotune(self, opts: dict):
        """Tune and return (condensation tile, its block size, the pair
        kernel's block size)."""
        o = make_opts(opts)
        t, th, pt = C.c_int(), C.c_int(), C.c_int()
        self._check(_lib().sdm_ens_autotune(self.h, C.byref(o), C.byref(t), C.byref(th), C.byref(pt)))
        return t.value, th.value, pt.value

    def stats(self) -> dict:
        s = sdm_stats()
        self._check(_lib().sdm_ens_stats(self.h, C.byref(s)))
        return s.as_dict()

    def memory(self) -> dict:
        """Device bytes the arena reserved, and its capacities."""
        b, n, m = C.c_size_t(), C.c_int64(), C.c_int32()
        self._check(_lib().sdm_ens_memory(self.h, C.byref(b), C.byref(n), C.byref(m)))
        return dict(device_bytes=b.value, cap_sd=n.value, cap_members=m.value)

    def close(self):
        if self.h:
            _lib().sdm_ens_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
