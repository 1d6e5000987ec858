"""ctypes binding of the C ABI declared in ``include/sdm.h``.

Argument marshalling only: numpy arrays (host) and torch CUDA tensors
(device) become ``sdm_arr`` descriptors, option dicts become the C structs,
status codes become exceptions.  Every computation runs in the CUDA library
``_build/libsdm.so``; if it cannot be loaded this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None


class SdmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


STATUS = {0: "SDM_OK", 1: "SDM_EINVAL", 2: "SDM_ENOMEM", 3: "SDM_ECUDA", 4: "SDM_ETIMEOUT",
          5: "SDM_ENUMERIC", 6: "SDM_ESTATE", 7: "SDM_ENOTSUP"}
KERNEL = {"geometric": 0, "golovin": 1, "long": 2}
INIT = {"lognormal": 0, "exponential": 1}
PRECISION = {"fp64": 0, "mixed": 1}
BACKEND = {"serial": 0, "openmp": 1, "cuda": 2}
SOLVER = {"bisect": 0, "fast": 1}
COND_LAYOUT = {"auto": 0, "fused": 1, "staged": 2}
ATTR = {"N": 0, "rw2": 1, "rd3": 2, "kappa": 3, "x": 4, "y": 5, "z": 6, "uid": 7}
ATTR_DTYPE = {"N": np.uint64, "uid": np.uint32}


class sdm_arr(C.Structure):
    _fields_ = [("data_zero", C.c_void_p), ("strides", C.POINTER(C.c_int64)), ("on_device", C.c_int)]


class sdm_lognormal(C.Structure):
    _fields_ = [("rm", C.c_double), ("sigma", C.c_double), ("n_stp", C.c_double), ("kappa", C.c_double)]


class sdm_opts_init(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("dt", C.c_double),
        ("sd_conc", C.c_int), ("kernel", C.c_int), ("golovin_b", C.c_double),
        ("init_dist", C.c_int), ("exp_mean_volume", C.c_double), ("exp_n0", C.c_double),
        ("n_modes", C.c_int), ("modes", C.POINTER(sdm_lognormal)),
        ("seed", C.c_uint64), ("physics", C.c_int), ("precision", C.c_int), ("backend", C.c_int),
        ("cond_solver", C.c_int), ("x_open", C.c_int), ("cond_layout", C.c_int), ("sd_reserve", C.c_int64),
    ]


class sdm_sd_block(C.Structure):
    _fields_ = [("N", C.c_void_p), ("uid", C.c_void_p), ("rw2", C.c_void_p), ("rd3", C.c_void_p),
                ("kappa", C.c_void_p), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("on_device", C.c_int)]


class sdm_opts(C.Structure):
    _fields_ = [("adve", C.c_int), ("sedi", C.c_int), ("cond", C.c_int), ("coal", C.c_int),
                ("RH_max", C.c_double), ("sstp_cond", C.c_int), ("sstp_coal", C.c_int),
                ("coal_multi", C.c_int), ("coal_adapt", C.c_int)]


class sdm_euler_opts(C.Structure):
    _fields_ = [("advect", C.c_int), ("relax", C.c_int), ("tau_rlx", C.c_double), ("z_rlx", C.c_double),
                ("th0", C.POINTER(C.c_double)), ("rv0", C.POINTER(C.c_double))]


class sdm_stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("n_pairs", "n_coll", "n_pgt1", "n_recycled", "n_euler",
                                          "n_fallback", "n_steps", "n_zero")] + \
               [("max_p", C.c_double), ("rainfall", C.c_double), ("n_coal_substeps", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sdm_timing(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("cond_ms", "recycle_ms", "move_ms", "sort_ms", "coal_ms",
                                          "diag_ms", "copy_ms")] + \
               [(k, C.c_uint64) for k in ("cond_launches", "coal_launches", "launches")] + \
               [("euler_ms", C.c_double), ("euler_launches", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SYMBOLS = ["sdm_init", "sdm_destroy", "sdm_last_error", "sdm_step_sync", "sdm_step_async", "sdm_wait",
           "sdm_euler_step",
           "sdm_diag_rng", "sdm_diag_mom", "sdm_diag_sd_conc", "sdm_diag_ambient", "sdm_diag_spectrum", "sdm_outbuf", "sdm_sizes", "sdm_get_attr",
           "sdm_set_attr", "sdm_get_fields", "sdm_get_step", "sdm_set_step", "sdm_get_stats",
           "sdm_timing_enable", "sdm_get_timing", "sdm_cell_sort", "sdm_cell_sort_noalloc", "sdm_probe_device",
           "sdm_step_transport", "sdm_step_coalesce", "sdm_export_leavers", "sdm_import"]


class sdm_device_peaks(C.Structure):
    _fields_ = [("n_sm", C.c_int), ("blocks", C.c_int), ("fp64_tflops_burst", C.c_double),
                ("fp64_tflops_sustained", C.c_double), ("sustained_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load ``libsdm.so`` (building it first if needed) and declare the ABI."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libsdm.so is missing: run paper_1310_1905_gb300.build.build()")
    L = C.CDLL(_build.LIB)
    P, V, I64, D = C.POINTER, C.c_void_p, C.c_int64, C.c_double
    ctx = C.c_void_p
    L.sdm_last_error.argtypes = [ctx]; L.sdm_last_error.restype = C.c_char_p
    L.sdm_init.argtypes = [P(sdm_opts_init), sdm_arr, sdm_arr, sdm_arr, sdm_arr, sdm_arr, sdm_arr, V, P(ctx)]
    L.sdm_destroy.argtypes = [ctx]
    L.sdm_step_sync.argtypes = [ctx, P(sdm_opts), sdm_arr, sdm_arr, sdm_arr, sdm_arr, sdm_arr, sdm_arr]
    L.sdm_euler_step.argtypes = [ctx, P(sdm_euler_opts), sdm_arr, sdm_arr, sdm_arr, sdm_arr, sdm_arr]
    L.sdm_step_async.argtypes = [ctx, P(sdm_opts)]
    L.sdm_wait.argtypes = [ctx, D, P(D)]
    L.sdm_diag_rng.argtypes = [ctx, C.c_int, D, D]
    L.sdm_diag_mom.argtypes = [ctx, C.c_int]
    L.sdm_diag_sd_conc.argtypes = [ctx]
    L.sdm_diag_ambient.argtypes = [ctx, C.c_int]
    L.sdm_outbuf.argtypes = [ctx, V, C.c_int]
    L.sdm_diag_spectrum.argtypes = [ctx, C.c_int, P(C.c_double), C.c_int, C.c_int, V, C.c_int]
    L.sdm_sizes.argtypes = [ctx, P(I64), P(I64)]
    L.sdm_get_attr.argtypes = [ctx, C.c_int, V, I64]
    L.sdm_set_attr.argtypes = [ctx, C.c_int, V, I64]
    L.sdm_get_fields.argtypes = [ctx, V, V]
    L.sdm_get_step.argtypes = [ctx, P(C.c_uint64)]
    L.sdm_set_step.argtypes = [ctx, C.c_uint64]
    L.sdm_get_stats.argtypes = [ctx, P(sdm_stats)]
    L.sdm_timing_enable.argtypes = [ctx, C.c_int]
    L.sdm_get_timing.argtypes = [ctx, P(sdm_timing), C.c_int]
    L.sdm_cell_sort.argtypes = [V, I64, C.c_int32, V, V, V]
    L.sdm_cell_sort_noalloc.argtypes = [V, I64, C.c_int32, V, V, V]
    L.sdm_probe_device.argtypes = [D, P(sdm_device_peaks)]
    L.sdm_step_transport.argtypes = [ctx, P(sdm_opts)]
    L.sdm_step_coalesce.argtypes = [ctx, P(sdm_opts)]
    L.sdm_export_leavers.argtypes = [ctx, sdm_sd_block, I64, P(I64)]
    L.sdm_import.argtypes = [ctx, sdm_sd_block, I64]
    for s in SYMBOLS:
        if s != "sdm_last_error":
            getattr(L, s).restype = C.c_int
    _LIB = L
    return L


# ---------------------------------------------------------------- marshalling
class _Arr:
    """Keeps the strides buffer alive next to the descriptor."""

    def __init__(self, a):
        self.keep = a
        if a is None:
            self.c = sdm_arr(None, None, 0)
            return
        if isinstance(a, np.ndarray):
            assert a.dtype == np.float64, "fields are float64"
            st = [s // 8 for s in a.strides] if a.ndim else []
            self.strides = (C.c_int64 * max(1, len(st)))(*st) if st else None
            self.c = sdm_arr(a.ctypes.data, self.strides, 0)
        else:  # torch tensor on the GPU
            import torch
            assert a.dtype == torch.float64 and a.is_cuda, "device fields are float64 CUDA tensors"
            st = list(a.stride())
            self.strides = (C.c_int64 * max(1, len(st)))(*st) if st else None
            self.c = sdm_arr(a.data_ptr(), self.strides, 1)


def make_opts_init(cfg: dict, precision: str = "fp64", backend: str = "cuda"):
    o = sdm_opts_init()
    o.nx, o.ny, o.nz = cfg.get("nx", 0), cfg.get("ny", 0), cfg.get("nz", 0)
    o.dx, o.dy, o.dz, o.dt = cfg.get("dx", 1.0), cfg.get("dy", 1.0), cfg.get("dz", 1.0), cfg.get("dt", 1.0)
    o.sd_conc = cfg.get("sd_conc", 64)
    o.kernel = KERNEL[cfg.get("kernel", "geometric")]
    o.golovin_b = cfg.get("golovin_b", 0.0)
    o.init_dist = INIT[cfg.get("init_dist", "lognormal")]
    o.exp_mean_volume = cfg.get("exp_mean_volume", 0.0)
    o.exp_n0 = cfg.get("exp_n0", 0.0)
    modes = cfg.get("modes", [])
    arr = (sdm_lognormal * max(1, len(modes)))(*[sdm_lognormal(m["rm"], m["sigma"], m["n_stp"], m["kappa"])
                                                 for m in modes])
    o.n_modes = len(modes)
    o.modes = C.cast(arr, C.POINTER(sdm_lognormal))
    o.seed = cfg.get("seed", 0)
    o.physics = cfg.get("physics", 1)
    o.precision = PRECISION[precision]
    o.backend = BACKEND[backend]
    o.cond_solver = SOLVER[cfg.get("cond_solver", "fast")]
    o.x_open = int(cfg.get("x_open", 0))
    o.cond_layout = COND_LAYOUT[cfg.get("cond_layout", "auto")]
    o.sd_reserve = int(cfg.get("sd_reserve", 0))
    return o, arr


def make_opts(d: dict | None = None) -> sdm_opts:
    d = d or {}
    return sdm_opts(d.get("adve", 1), d.get("sedi", 1), d.get("cond", 1), d.get("coal", 1),
                    d.get("RH_max", 44.0), d.get("sstp_cond", 10), d.get("sstp_coal", 10),
                    d.get("coal_multi", 0), d.get("coal_adapt", 0))


def _check(L, ctx, status):
    if status != 0:
        msg = L.sdm_last_error(ctx)
        raise SdmError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------- same names as the ABI
def sdm_init(cfg: dict, th, rv, rhod, rhoCx=None, rhoCy=None, rhoCz=None, stream=None,
             precision="fp64", backend="cuda"):
    L = load()
    o, keep = make_opts_init(cfg, precision, backend)
    args = [_Arr(a) for a in (th, rv, rhod, rhoCx, rhoCy, rhoCz)]
    ctx = C.c_void_p()
    st = L.sdm_init(C.byref(o), *[a.c for a in args], C.c_void_p(stream or 0), C.byref(ctx))
    _check(L, None, st)
    return ctx


def sdm_destroy(ctx):
    load().sdm_destroy(ctx)


def sdm_step_sync(ctx, opts: dict, th, rv, rhoCx=None, rhoCy=None, rhoCz=None, rhod=None):
    L = load()
    o = make_opts(opts)
    args = [_Arr(a) for a in (th, rv, rhoCx, rhoCy, rhoCz, rhod)]
    _check(L, ctx, L.sdm_step_sync(ctx, C.byref(o), *[a.c for a in args]))


def sdm_euler_step(ctx, th, rv, rhoCx=None, rhoCy=None, rhoCz=None, th0=None, rv0=None, advect=True,
                   tau_rlx=300.0, z_rlx=200.0):
    """The kinematic framework's Eulerian step on theta and r_v (in place):
    donor-cell transport, then (with th0, rv0 level profiles) relaxation of
    the horizontal means."""
    L = load()
    relax = th0 is not None
    p0 = np.ascontiguousarray(th0 if relax else [0.0], np.float64)
    p1 = np.ascontiguousarray(rv0 if relax else [0.0], np.float64)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    o = sdm_euler_opts(int(advect), int(relax), tau_rlx, z_rlx, dp(p0), dp(p1))
    args = [_Arr(a) for a in (th, rv, rhoCx, rhoCy, rhoCz)]
    _check(L, ctx, L.sdm_euler_step(ctx, C.byref(o), *[a.c for a in args]))


def sdm_step_async(ctx, opts: dict):
    L = load()
    o = make_opts(opts)
    _check(L, ctx, L.sdm_step_async(ctx, C.byref(o)))


def sdm_step_transport(ctx, opts: dict):
    L = load()
    o = make_opts(opts)
    _check(L, ctx, L.sdm_step_transport(ctx, C.byref(o)))


def sdm_step_coalesce(ctx, opts: dict):
    L = load()
    o = make_opts(opts)
    _check(L, ctx, L.sdm_step_coalesce(ctx, C.byref(o)))


BLOCK_FIELDS = (("N", np.uint64), ("uid", np.uint32), ("rw2", np.float64), ("rd3", np.float64),
                ("kappa", np.float64), ("x", np.float64), ("y", np.float64), ("z", np.float64))


def _block(arrays: dict) -> sdm_sd_block:
    b = sdm_sd_block()
    for name, _ in BLOCK_FIELDS:
        a = arrays.get(name)
        setattr(b, name, None if a is None else a.ctypes.data)
    b.on_device = 0
    return b


def sdm_export_leavers(ctx, cap: int) -> dict:
    """The leavers of an x_open context (x outside its domain), host arrays."""
    L = load()
    cap = max(1, int(cap))
    arrays = {name: np.zeros(cap, dt) for name, dt in BLOCK_FIELDS}
    n = C.c_int64()
    _check(L, ctx, L.sdm_export_leavers(ctx, _block(arrays), cap, C.byref(n)))
    return {k: v[:n.value].copy() for k, v in arrays.items()}


def sdm_import(ctx, arrays: dict):
    """Put super-droplets (host arrays as sdm_export_leavers returns them)
    into free slots."""
    L = load()
    n = len(arrays["N"])
    conv = {name: np.ascontiguousarray(arrays[name], dt) if name in arrays else np.zeros(n, dt)
            for name, dt in BLOCK_FIELDS}
    _check(L, ctx, L.sdm_import(ctx, _block(conv), n))


def sdm_wait(ctx, timeout_s: float = -1.0) -> float:
    L = load()
    r = C.c_double()
    _check(L, ctx, L.sdm_wait(ctx, timeout_s, C.byref(r)))
    return r.value


def sdm_diag_rng(ctx, wet: bool, r_min: float, r_max: float):
    L = load()
    _check(L, ctx, L.sdm_diag_rng(ctx, int(wet), r_min, r_max))


def sdm_diag_mom(ctx, k: int):
    L = load()
    _check(L, ctx, L.sdm_diag_mom(ctx, k))


AMBIENT = {"T": 0, "p": 1, "rho_vs": 2, "RH": 3}


def sdm_diag_ambient(ctx, what: str):
    L = load()
    _check(L, ctx, L.sdm_diag_ambient(ctx, AMBIENT[what]))


def sdm_diag_sd_conc(ctx):
    L = load()
    _check(L, ctx, L.sdm_diag_sd_conc(ctx))


def sdm_sizes(ctx):
    L = load()
    n, nc = C.c_int64(), C.c_int64()
    _check(L, ctx, L.sdm_sizes(ctx, C.byref(n), C.byref(nc)))
    return n.value, nc.value


def sdm_outbuf(ctx, out=None):
    """Copy the output buffer into ``out`` (numpy host array or torch CUDA
    tensor of n_cells float64); returns it."""
    L = load()
    if out is None:
        out = np.empty(sdm_sizes(ctx)[1], np.float64)
    if isinstance(out, np.ndarray):
        _check(L, ctx, L.sdm_outbuf(ctx, out.ctypes.data, 0))
    else:
        _check(L, ctx, L.sdm_outbuf(ctx, out.data_ptr(), 1))
    return out


def sdm_diag_spectrum(ctx, wet: bool, edges, k: int, out=None):
    """Moment k per cell in every radius bin [edges[b], edges[b+1]) into
    ``out`` (numpy host array or torch CUDA tensor of (n_bins, n_cells)
    float64); returns it."""
    L = load()
    e = np.ascontiguousarray(edges, np.float64)
    nb = len(e) - 1
    if out is None:
        out = np.empty((nb, sdm_sizes(ctx)[1]), np.float64)
    ep = e.ctypes.data_as(C.POINTER(C.c_double))
    if isinstance(out, np.ndarray):
        assert out.flags.c_contiguous and out.dtype == np.float64 and out.size == nb * sdm_sizes(ctx)[1]
        _check(L, ctx, L.sdm_diag_spectrum(ctx, int(wet), ep, nb, k, out.ctypes.data, 0))
    else:
        assert out.is_contiguous() and out.numel() == nb * sdm_sizes(ctx)[1]
        _check(L, ctx, L.sdm_diag_spectrum(ctx, int(wet), ep, nb, k, out.data_ptr(), 1))
    return out


def sdm_get_attr(ctx, name: str) -> np.ndarray:
    L = load()
    n, _ = sdm_sizes(ctx)
    out = np.empty(n, ATTR_DTYPE.get(name, np.float64))
    _check(L, ctx, L.sdm_get_attr(ctx, ATTR[name], out.ctypes.data, n))
    return out


def sdm_set_attr(ctx, name: str, values):
    L = load()
    n, _ = sdm_sizes(ctx)
    a = np.ascontiguousarray(values, dtype=ATTR_DTYPE.get(name, np.float64))
    _check(L, ctx, L.sdm_set_attr(ctx, ATTR[name], a.ctypes.data, n))


def sdm_get_fields(ctx):
    L = load()
    _, nc = sdm_sizes(ctx)
    th, rv = np.empty(nc), np.empty(nc)
    _check(L, ctx, L.sdm_get_fields(ctx, th.ctypes.data, rv.ctypes.data))
    return th, rv


def sdm_get_step(ctx) -> int:
    L = load()
    s = C.c_uint64()
    _check(L, ctx, L.sdm_get_step(ctx, C.byref(s)))
    return s.value


def sdm_set_step(ctx, step: int):
    L = load()
    _check(L, ctx, L.sdm_set_step(ctx, step))


def sdm_get_stats(ctx) -> dict:
    L = load()
    s = sdm_stats()
    _check(L, ctx, L.sdm_get_stats(ctx, C.byref(s)))
    return s.as_dict()


def sdm_timing_enable(ctx, on: bool = True):
    L = load()
    _check(L, ctx, L.sdm_timing_enable(ctx, int(on)))


def sdm_get_timing(ctx, reset: bool = False) -> dict:
    L = load()
    t = sdm_timing()
    _check(L, ctx, L.sdm_get_timing(ctx, C.byref(t), int(reset)))
    return t.as_dict()


def sdm_cell_sort(cell, n_cells: int, perm, offsets, stream=None):
    """Counting sort of particles by cell on device tensors (32-bit):
    ``cell`` (n), ``perm`` (n, out), ``offsets`` (n_cells + 1, out)."""
    L = load()
    st = L.sdm_cell_sort(C.c_void_p(cell.data_ptr()), cell.numel(), n_cells, C.c_void_p(perm.data_ptr()),
                         C.c_void_p(offsets.data_ptr()), C.c_void_p(stream or 0))
    if st != 0:
        raise SdmError(st, "sdm_cell_sort failed")


def sdm_cell_sort_noalloc(cell, n_cells: int, perm, offsets, stream=None):
    """The allocation-free variant (fixed device scratch, enqueue only)."""
    L = load()
    st = L.sdm_cell_sort_noalloc(C.c_void_p(cell.data_ptr()), cell.numel(), n_cells,
                                 C.c_void_p(perm.data_ptr()), C.c_void_p(offsets.data_ptr()),
                                 C.c_void_p(stream or 0))
    if st != 0:
        msg = L.sdm_last_error(None)
        raise SdmError(st, msg.decode() if msg else "")


def sdm_probe_device(sustain_s: float = 2.0) -> dict:
    """SM count and measured FP64 FMA throughput of the current device."""
    L = load()
    out = sdm_device_peaks()
    st = L.sdm_probe_device(float(sustain_s), C.byref(out))
    if st != 0:
        msg = L.sdm_last_error(None)
        raise SdmError(st, msg.decode() if msg else "sdm_probe_device failed")
    return out.as_dict()


# ---------------------------------------------------------------- object wrapper
class Particles:
    """The paper's particles_t (Sec. 5.2.1) over the C ABI."""

    def __init__(self, cfg: dict, th, rv, rhod, rhoCx=None, rhoCy=None, rhoCz=None, stream=None,
                 precision="fp64"):
        self.cfg = dict(cfg)
        self.ctx = sdm_init(cfg, th, rv, rhod, rhoCx, rhoCy, rhoCz, stream, precision)
        self.n_sd, self.n_cells = sdm_sizes(self.ctx)

    def step_sync(self, opts, th, rv, rhoCx=None, rhoCy=None, rhoCz=None, rhod=None):
        sdm_step_sync(self.ctx, opts, th, rv, rhoCx, rhoCy, rhoCz, rhod)

    def step_async(self, opts):
        sdm_step_async(self.ctx, opts)

    def step_transport(self, opts):
        sdm_step_transport(self.ctx, opts)

    def step_coalesce(self, opts):
        sdm_step_coalesce(self.ctx, opts)

    def export_leavers(self, cap=None):
        return sdm_export_leavers(self.ctx, self.n_sd if cap is None else cap)

    def import_(self, arrays: dict):
        sdm_import(self.ctx, arrays)

    def euler_step(self, th, rv, rhoCx=None, rhoCy=None, rhoCz=None, th0=None, rv0=None, advect=True):
        sdm_euler_step(self.ctx, th, rv, rhoCx, rhoCy, rhoCz, th0, rv0, advect)

    def wait(self, timeout_s=-1.0):
        return sdm_wait(self.ctx, timeout_s)

    def diag_moments(self, wet: bool, r_min: float, r_max: float, k: int):
        sdm_diag_rng(self.ctx, wet, r_min, r_max)
        sdm_diag_mom(self.ctx, k)
        return sdm_outbuf(self.ctx)

    def diag_ambient(self, what: str):
        """T, p, rho_vs or RH per cell, as the condensation solve sees them."""
        sdm_diag_ambient(self.ctx, what)
        return sdm_outbuf(self.ctx)

    def diag_sd_conc(self):
        sdm_diag_sd_conc(self.ctx)
        return sdm_outbuf(self.ctx)

    def diag_spectrum(self, wet: bool, edges, k: int):
        return sdm_diag_spectrum(self.ctx, wet, edges, k)

    def attr(self, name):
        return sdm_get_attr(self.ctx, name)

    def set_attr(self, name, values):
        """Overwrite one attribute (storage order, as attr() returns it)."""
        sdm_set_attr(self.ctx, name, values)

    def state(self) -> dict:
        """All attributes of present dimensions, ordered by super-droplet id."""
        uid = self.attr("uid")
        o = np.argsort(uid, kind="stable")
        out = {"uid": uid[o].astype(np.uint64)}
        names = ["N", "rw2", "rd3", "kappa"] + [d for d, n in (("x", "nx"), ("y", "ny"), ("z", "nz"))
                                                  if self.cfg.get(n, 0) > 0]
        for nm in names:
            out[nm] = self.attr(nm)[o]
        return out

    def fields(self):
        return sdm_get_fields(self.ctx)

    def stats(self):
        return sdm_get_stats(self.ctx)

    def close(self):
        if self.ctx:
            sdm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
