"""CPU oracle for the super-droplet hot path (libcloudph++ 0.2, Sec. 5).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` / reference
legs may import this package.  It wraps the plain serial C99 oracle in
``sdm_oracle.c`` (double precision, ``-ffp-contract=off``) with ctypes and
numpy; it shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_SRC = [os.path.join(_HERE, f) for f in ("sdm_oracle.c", "philox.c")]
_lock = threading.Lock()
_libs: dict = {}

MAX_MODES = 8


def _build_one(so: str, extra: list, force: bool) -> str:
    newest = max(os.path.getmtime(p) for p in _SRC + [os.path.join(_HERE, "sdm_oracle.h")])
    if not force and os.path.exists(so) and os.path.getmtime(so) >= newest:
        return so
    tmp = so + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"] + extra + ["-o", tmp] + _SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def build(force: bool = False, omp: bool | None = None) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2,
    serial) and its cell-parallel timing build ``liboracle_omp.so`` (the
    same source with -fopenmp).  ``omp`` None builds both and returns the
    serial one's path."""
    os.makedirs(_BUILD, exist_ok=True)
    if omp is None:
        _build_one(_SO_OMP, ["-fopenmp"], force)
        return _build_one(_SO, [], force)
    return _build_one(_SO_OMP, ["-fopenmp"], force) if omp else _build_one(_SO, [], force)


class Mode(C.Structure):
    _fields_ = [("rm", C.c_double), ("sigma", C.c_double), ("n_stp", C.c_double), ("kappa", C.c_double)]


class Domain(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("dt", C.c_double),
        ("sd_conc", C.c_int), ("kernel", C.c_int), ("golovin_b", C.c_double),
        ("init_dist", C.c_int), ("exp_mean_volume", C.c_double), ("exp_n0", C.c_double),
        ("n_modes", C.c_int), ("modes", Mode * MAX_MODES),
        ("seed", C.c_uint64), ("physics", C.c_int),
    ]


class Opts(C.Structure):
    _fields_ = [
        ("adve", C.c_int), ("sedi", C.c_int), ("cond", C.c_int), ("coal", C.c_int),
        ("RH_max", C.c_double), ("sstp_cond", C.c_int), ("sstp_coal", C.c_int),
        ("coal_multi", C.c_int), ("coal_adapt", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("n_pairs", C.c_uint64), ("n_coll", C.c_uint64), ("n_pgt1", C.c_uint64),
        ("n_recycled", C.c_uint64), ("n_euler", C.c_uint64), ("n_bisect", C.c_uint64),
        ("max_p", C.c_double), ("rainfall", C.c_double), ("n_coal_substeps", C.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SDs(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("uid", C.POINTER(C.c_uint64)), ("N", C.POINTER(C.c_uint64)),
        ("rw2", C.POINTER(C.c_double)), ("rd3", C.POINTER(C.c_double)), ("kappa", C.POINTER(C.c_double)),
        ("x", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)), ("z", C.POINTER(C.c_double)),
    ]


class Thermo(C.Structure):
    _fields_ = [(k, C.c_double) for k in (
        "th", "rv", "rhod", "T", "p", "lv", "rho_v", "rho_vs", "rho_v_eff", "dth_drv", "A", "Dterm",
        "rho_a", "mu", "nu", "lambda_D", "lambda_K", "Sc", "Pr", "cX")]


_P = C.POINTER
_D = C.c_double


def lib(omp: bool = False):
    """The serial oracle (default) or its cell-parallel OpenMP build."""
    with _lock:
        if omp not in _libs:
            L = C.CDLL(build(omp=omp))
            L.orc_threads.argtypes = [C.c_int]; L.orc_threads.restype = C.c_int
            L.orc_philox4x64_10.argtypes = [_P(C.c_uint64), _P(C.c_uint64), _P(C.c_uint64)]
            L.orc_u01.argtypes = [C.c_uint64]; L.orc_u01.restype = _D
            L.orc_n_cells.argtypes = [_P(Domain)]; L.orc_n_cells.restype = C.c_int64
            L.orc_n_groups.argtypes = [_P(Domain)]; L.orc_n_groups.restype = C.c_int
            L.orc_cell_of.argtypes = [_P(Domain), _D, _D, _D]; L.orc_cell_of.restype = C.c_int64
            L.orc_thermo_eval.argtypes = [_D, _D, _D, _D, _P(Thermo)]
            L.orc_reynolds.argtypes = [_D, _P(Thermo)]; L.orc_reynolds.restype = _D
            L.orc_vterm.argtypes = [_D, _P(Thermo)]; L.orc_vterm.restype = _D
            L.orc_growth.argtypes = [_D, _D, _D, _P(Thermo), C.c_int]; L.orc_growth.restype = _D
            L.orc_solve_rw2.argtypes = [_D, _D, _D, _P(Thermo), _D, C.c_int, _P(Stats)]
            L.orc_solve_rw2.restype = _D
            L.orc_solve_batch.argtypes = [C.c_int64, _P(_D), _P(_D), _P(_D), _P(C.c_int64), _P(_D), _P(_D),
                                          _P(_D), _D, _D, C.c_int, _P(_D)]
            L.orc_equilibrium_rw2.argtypes = [_D, _D, _D, _D]; L.orc_equilibrium_rw2.restype = _D
            L.orc_rd_range.argtypes = [_P(Domain), C.c_int, _P(_D), _P(_D)]; L.orc_rd_range.restype = C.c_int
            L.orc_init_cells.argtypes = [_P(Domain), _P(_D), _P(_D), _P(_D), C.c_int64, _P(C.c_int64), _P(SDs)]
            L.orc_init_cells.restype = C.c_int
            L.orc_init_cells_nreal.argtypes = [_P(Domain), _P(_D), _P(_D), _P(_D), C.c_int64, _P(C.c_int64),
                                               _P(SDs), _P(_D)]
            L.orc_init_cells_nreal.restype = C.c_int
            L.orc_condense.argtypes = [_P(Domain), _P(Opts), _P(SDs), _P(_D), _P(_D), _P(_D), _P(Stats)]
            L.orc_recycle.argtypes = [_P(SDs), _P(Stats)]
            L.orc_advect.argtypes = [_P(Domain), _P(SDs), _P(_D), _P(_D), _P(_D), _P(_D)]
            L.orc_transport.argtypes = [_P(Domain), _P(Opts), _P(SDs), _P(_D), _P(_D), _P(_D),
                                        _P(_D), _P(_D), _P(_D), _P(Stats)]
            L.orc_coalesce.argtypes = [_P(Domain), _P(Opts), _P(SDs), _P(_D), _P(_D), _P(_D), C.c_uint64, _P(Stats)]
            L.orc_step_sync.argtypes = [_P(Domain), _P(Opts), _P(SDs), _P(_D), _P(_D), _P(_D), _P(Stats)]
            L.orc_step_async.argtypes = [_P(Domain), _P(Opts), _P(SDs), _P(_D), _P(_D), _P(_D),
                                         _P(_D), _P(_D), _P(_D), C.c_uint64, _P(Stats)]
            L.orc_parcel_step.argtypes = [_P(Domain), _P(Opts), _P(SDs), _P(_D), _P(_D), _P(_D), _D, _D,
                                          C.c_uint64, _P(Stats)]
            L.orc_moments.argtypes = [_P(Domain), _P(SDs), _P(_D), C.c_int, _D, _D, C.c_int, _P(_D)]
            L.orc_spectrum.argtypes = [_P(Domain), _P(SDs), _P(_D), C.c_int, _P(_D), C.c_int, C.c_int, _P(_D)]
            L.orc_sd_conc.argtypes = [_P(Domain), _P(SDs), _P(_D)]
            L.orc_upwind.argtypes = [_P(Domain), _P(_D), _P(_D), _P(_D), _P(_D), _P(_D)]
            L.orc_relax.argtypes = [_P(Domain), _P(_D), _P(_D), _D, _D]
            _libs[omp] = L
    return _libs[omp]


def threads(n: int = 0, omp: bool = True) -> int:
    """Threads the OpenMP build uses (n > 0 sets them); 1 for the serial one."""
    return int(lib(omp).orc_threads(int(n)))


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P(_D))


# ---------------------------------------------------------------------------
def philox(ctr, key):
    """Philox4x64-10 of one 256-bit counter under one 128-bit key."""
    c = (C.c_uint64 * 4)(*[int(v) for v in ctr])
    k = (C.c_uint64 * 2)(*[int(v) for v in key])
    o = (C.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(v) for v in o]


def u01(v):
    return lib().orc_u01(C.c_uint64(int(v)))


def make_domain(cfg: dict) -> Domain:
    """Build the oracle's domain struct from a plain workload dict."""
    d = Domain()
    d.nx, d.ny, d.nz = cfg.get("nx", 0), cfg.get("ny", 0), cfg.get("nz", 0)
    d.dx, d.dy, d.dz = cfg.get("dx", 1.0), cfg.get("dy", 1.0), cfg.get("dz", 1.0)
    d.dt = cfg.get("dt", 1.0)
    d.sd_conc = cfg.get("sd_conc", 64)
    d.kernel = {"geometric": 0, "golovin": 1, "long": 2}[cfg.get("kernel", "geometric")]
    d.golovin_b = cfg.get("golovin_b", 0.0)
    d.init_dist = {"lognormal": 0, "exponential": 1}[cfg.get("init_dist", "lognormal")]
    d.exp_mean_volume = cfg.get("exp_mean_volume", 0.0)
    d.exp_n0 = cfg.get("exp_n0", 0.0)
    modes = cfg.get("modes", [])
    d.n_modes = len(modes)
    for i, m in enumerate(modes):
        d.modes[i] = Mode(m["rm"], m["sigma"], m["n_stp"], m["kappa"])
    d.seed = cfg.get("seed", 0)
    d.physics = cfg.get("physics", 1)
    return d


def make_opts(o: dict | None = None) -> Opts:
    o = o or {}
    return Opts(o.get("adve", 1), o.get("sedi", 1), o.get("cond", 1), o.get("coal", 1),
                o.get("RH_max", 44.0), o.get("sstp_cond", 10), o.get("sstp_coal", 10),
                o.get("coal_multi", 0), o.get("coal_adapt", 0))


def thermo(th, rv, rhod, RH_max=44.0) -> Thermo:
    t = Thermo()
    lib().orc_thermo_eval(th, rv, rhod, RH_max, C.byref(t))
    return t


class State:
    """Super-droplet arrays held as numpy (structure of arrays)."""

    FIELDS = ("uid", "N", "rw2", "rd3", "kappa", "x", "y", "z")

    def __init__(self, n: int):
        self.uid = np.zeros(n, np.uint64)
        self.N = np.zeros(n, np.uint64)
        for f in ("rw2", "rd3", "kappa", "x", "y", "z"):
            setattr(self, f, np.zeros(n, np.float64))
        self._n = n

    @property
    def n(self):
        return self._n

    def copy(self) -> "State":
        s = State(self._n)
        for f in self.FIELDS:
            getattr(s, f)[:] = getattr(self, f)
        return s

    def subset(self, mask) -> "State":
        idx = np.nonzero(mask)[0]
        s = State(len(idx))
        for f in self.FIELDS:
            getattr(s, f)[:] = getattr(self, f)[idx]
        return s

    def struct(self) -> SDs:
        s = SDs()
        s.n = self._n
        s.uid = self.uid.ctypes.data_as(_P(C.c_uint64))
        s.N = self.N.ctypes.data_as(_P(C.c_uint64))
        for f in ("rw2", "rd3", "kappa", "x", "y", "z"):
            setattr(s, f, getattr(self, f).ctypes.data_as(_P(_D)))
        return s

    def sorted_by_uid(self) -> "State":
        o = np.argsort(self.uid, kind="stable")
        s = State(self._n)
        for f in self.FIELDS:
            getattr(s, f)[:] = getattr(self, f)[o]
        return s


class Oracle:
    """One simulated domain advanced by the oracle, following the paper's
    calling sequence (Sec. 5.2.2): init, then step_sync / step_async pairs."""

    def __init__(self, cfg: dict, omp: bool = False):
        self.cfg = dict(cfg)
        self.dom = make_domain(cfg)
        self._L = L = lib(omp)
        self.n_cells = int(L.orc_n_cells(C.byref(self.dom)))
        self.n_groups = int(L.orc_n_groups(C.byref(self.dom)))
        self.step_index = 0
        self.stats = Stats()
        self.state: State | None = None

    def rd_range(self, group=0):
        lo, hi = _D(), _D()
        rc = self._L.orc_rd_range(C.byref(self.dom), group, C.byref(lo), C.byref(hi))
        if rc != 0:
            raise RuntimeError(f"orc_rd_range failed ({rc})")
        return lo.value, hi.value

    def init_cells(self, th, rv, rhod, cells, with_nreal=False):
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        n = len(cells) * self.n_groups * self.dom.sd_conc
        st = State(n)
        s = st.struct()
        nreal = np.zeros(n) if with_nreal else None
        rc = self._L.orc_init_cells_nreal(C.byref(self.dom), _dp(np.ascontiguousarray(th, np.float64).ravel()),
                                        _dp(np.ascontiguousarray(rv, np.float64).ravel()),
                                        _dp(np.ascontiguousarray(rhod, np.float64).ravel()), len(cells),
                                        cells.ctypes.data_as(_P(C.c_int64)), C.byref(s), _dp(nreal))
        if rc != 0:
            raise RuntimeError(f"orc_init_cells failed ({rc})")
        return (st, nreal) if with_nreal else st

    def init(self, th, rv, rhod):
        self.th = np.array(th, np.float64).ravel().copy()
        self.rv = np.array(rv, np.float64).ravel().copy()
        self.rhod = np.array(rhod, np.float64).ravel().copy()
        self.state, self.nreal = self.init_cells(self.th, self.rv, self.rhod, np.arange(self.n_cells),
                                                 with_nreal=True)
        # dry-air mass of a parcel (no spatial dimension), kept through rho_d changes
        self.m_d = float(self.rhod[0]) * (self.dom.dx * self.dom.dy * self.dom.dz)
        return self.state

    def step_sync(self, opts: dict | None = None):
        o = make_opts(opts)
        s = self.state.struct()
        self._L.orc_step_sync(C.byref(self.dom), C.byref(o), C.byref(s), _dp(self.th), _dp(self.rv),
                            _dp(self.rhod), C.byref(self.stats))

    def step_async(self, opts: dict | None = None, rhoCx=None, rhoCy=None, rhoCz=None):
        o = make_opts(opts)
        s = self.state.struct()
        self._L.orc_step_async(C.byref(self.dom), C.byref(o), C.byref(s), _dp(self.th), _dp(self.rv),
                             _dp(self.rhod), _dp(rhoCx), _dp(rhoCy), _dp(rhoCz),
                             self.step_index, C.byref(self.stats))
        self.step_index += 1

    def parcel_step(self, opts: dict | None = None, rhod: float | None = None):
        """One timestep of a parcel or box (no spatial dimension): a new
        rho_d (if given) sets the volume to the dry-air mass over it, then
        recycling, condensation and coalescence."""
        o = make_opts(opts)
        s = self.state.struct()
        self._L.orc_parcel_step(C.byref(self.dom), C.byref(o), C.byref(s), _dp(self.th), _dp(self.rv),
                                _dp(self.rhod), self.m_d, float(rhod) if rhod else 0.0, self.step_index,
                                C.byref(self.stats))
        self.step_index += 1

    @property
    def volume(self) -> float:
        return self.dom.dx * self.dom.dy * self.dom.dz

    def moments(self, wet: bool, r_min: float, r_max: float, k: int):
        out = np.zeros(self.n_cells)
        s = self.state.struct()
        self._L.orc_moments(C.byref(self.dom), C.byref(s), _dp(self.rhod), int(wet), r_min, r_max, k, _dp(out))
        return out

    def spectrum(self, wet: bool, edges, k: int):
        """Moment k in each radius bin [edges[b], edges[b+1]): (n_bins, n_cells)."""
        edges = np.ascontiguousarray(edges, np.float64)
        nb = len(edges) - 1
        out = np.zeros(nb * self.n_cells)
        s = self.state.struct()
        self._L.orc_spectrum(C.byref(self.dom), C.byref(s), _dp(self.rhod), int(wet), _dp(edges), nb, k, _dp(out))
        return out.reshape(nb, self.n_cells)

    def euler_step(self, rhoCx=None, rhoCy=None, rhoCz=None, th0=None, rv0=None, tau_rlx=300.0, z_rlx=200.0):
        """The Eulerian component on theta and r_v: a donor-cell step, then
        (with th0, rv0 profiles) the relaxation of the horizontal means."""
        self.th = upwind(self.cfg, self.th, self.rhod, rhoCx, rhoCy, rhoCz)
        self.rv = upwind(self.cfg, self.rv, self.rhod, rhoCx, rhoCy, rhoCz)
        if th0 is not None:
            self.th = relax(self.cfg, self.th, th0, tau_rlx, z_rlx)
            self.rv = relax(self.cfg, self.rv, rv0, tau_rlx, z_rlx)

    def sd_conc(self):
        out = np.zeros(self.n_cells)
        s = self.state.struct()
        self._L.orc_sd_conc(C.byref(self.dom), C.byref(s), _dp(out))
        return out


def _field(a):
    return None if a is None else np.ascontiguousarray(a, np.float64).ravel()


def upwind(cfg: dict, psi, rhod, rhoCx=None, rhoCy=None, rhoCz=None):
    """One donor-cell step of the cell field psi (a new flat array)."""
    dom = make_domain(cfg)
    out = np.ascontiguousarray(psi, np.float64).ravel().copy()
    lib().orc_upwind(C.byref(dom), _dp(out), _dp(_field(rhod)), _dp(_field(rhoCx)), _dp(_field(rhoCy)),
                     _dp(_field(rhoCz)))
    return out


def relax(cfg: dict, psi, psi0, tau_rlx=300.0, z_rlx=200.0):
    """Relaxation of the horizontal means toward psi0 (nz values), one step."""
    dom = make_domain(cfg)
    out = np.ascontiguousarray(psi, np.float64).ravel().copy()
    lib().orc_relax(C.byref(dom), _dp(out), _dp(np.ascontiguousarray(psi0, np.float64)), tau_rlx, z_rlx)
    return out


def solve_rw2(x0, rd3, kappa, t: Thermo, dtp, physics=1):
    st = Stats()
    x = lib().orc_solve_rw2(x0, rd3, kappa, C.byref(t), dtp, physics, C.byref(st))
    return x, st


def growth(x, rd3, kappa, t: Thermo, physics=1):
    return lib().orc_growth(x, rd3, kappa, C.byref(t), physics)


def vterm(rw2, t: Thermo):
    return lib().orc_vterm(rw2, C.byref(t))


def reynolds(rw2, t: Thermo):
    return lib().orc_reynolds(rw2, C.byref(t))


def equilibrium_rw2(rd3, kappa, RH, T):
    return lib().orc_equilibrium_rw2(rd3, kappa, RH, T)


def solve_batch(x0, rd3, kappa, cell, th, rv, rhod, dtp, RH_max=44.0, physics=1, omp=True):
    """x1 of one condensation substep for each listed super-droplet in its
    cell's state (no feedback): the oracle's bisection, solve by solve."""
    x0, rd3, kappa = (np.ascontiguousarray(a, np.float64) for a in (x0, rd3, kappa))
    cell = np.ascontiguousarray(cell, np.int64)
    th, rv, rhod = (np.ascontiguousarray(a, np.float64).ravel() for a in (th, rv, rhod))
    out = np.empty_like(x0)
    lib(omp).orc_solve_batch(len(x0), _dp(x0), _dp(rd3), _dp(kappa), cell.ctypes.data_as(_P(C.c_int64)),
                             _dp(th), _dp(rv), _dp(rhod), RH_max, dtp, physics, _dp(out))
    return out
