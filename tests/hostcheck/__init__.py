"""Host build of the CUDA library's condensation solvers for CPU tests
(test infrastructure: compiled with nvcc from the library's own source,
run on the CPU, never loaded by the library)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
SRC = os.path.join(HERE, "solver_host.cu")
SO = os.path.join(HERE, "_build", "libsolver_host.so")
_lib = None


def build() -> str:
    csrc = os.path.join(ROOT, "paper_1310_1905_gb300", "csrc")
    deps = [SRC, os.path.join(csrc, "k_cond.cu"), os.path.join(csrc, "sdm_internal.cuh"),
            os.path.join(ROOT, "include", "sdm.h")]
    if os.path.exists(SO) and os.path.getmtime(SO) >= max(os.path.getmtime(d) for d in deps):
        return SO
    os.makedirs(os.path.dirname(SO), exist_ok=True)
    from paper_1310_1905_gb300.build import nvcc
    tmp = SO + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "--expt-relaxed-constexpr",
           "-gencode", "arch=compute_103a,code=sm_103a", "-I", os.path.join(ROOT, "include"), "-o", tmp, SRC]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, SO)
    return SO


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P, D, I64 = C.POINTER, C.c_double, C.c_int64
        L.hc_solve.argtypes = [I64, P(D), P(D), P(D), P(I64), P(D), P(D), P(D), D, D, C.c_int, C.c_int, P(D), P(I64)]
        L.hc_growth.argtypes = [I64, P(D), P(D), P(D), P(I64), P(D), P(D), P(D), D, C.c_int, P(C.c_float),
                                P(C.c_float), P(D)]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _prep(*arrs):
    return [np.ascontiguousarray(a, np.float64).ravel() for a in arrs]


def solve(x0, rd3, kappa, cell, th, rv, rhod, dtp, solver=1, RH_max=44.0, physics=1):
    x0, rd3, kappa, th, rv, rhod = _prep(x0, rd3, kappa, th, rv, rhod)
    cell = np.ascontiguousarray(cell, np.int64)
    out = np.empty_like(x0)
    cnt = np.zeros(4, np.int64)
    lib().hc_solve(len(x0), _d(x0), _d(rd3), _d(kappa), cell.ctypes.data_as(C.POINTER(C.c_int64)), _d(th), _d(rv),
                   _d(rhod), RH_max, dtp, physics, solver, _d(out), cnt.ctypes.data_as(C.POINTER(C.c_int64)))
    return out, dict(euler=int(cnt[0]), fallback=int(cnt[1]), evals=int(cnt[2]), certified=int(cnt[3]))


def staged_stats(x0, rd3, kappa, cell, th, rv, rhod, dtp, RH_max=44.0, physics=1):
    """Start classes (polish, Euler, tiny, exact) and deferred bracket ends of
    the staged sequence."""
    x0, rd3, kappa, th, rv, rhod = _prep(x0, rd3, kappa, th, rv, rhod)
    cell = np.ascontiguousarray(cell, np.int64)
    out = np.zeros(5, np.int64)
    L = lib()
    L.hc_staged_stats.argtypes = [C.c_int64] + [C.POINTER(C.c_double)] * 3 + [C.POINTER(C.c_int64)] + \
        [C.POINTER(C.c_double)] * 3 + [C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int64)]
    L.hc_staged_stats(len(x0), _d(x0), _d(rd3), _d(kappa), cell.ctypes.data_as(C.POINTER(C.c_int64)), _d(th), _d(rv),
                      _d(rhod), RH_max, dtp, physics, out.ctypes.data_as(C.POINTER(C.c_int64)))
    return dict(polish=int(out[0]), euler=int(out[1]), tiny=int(out[2]), exact=int(out[3]), deferred_ends=int(out[4]))


def growth(x, rd3, kappa, cell, th, rv, rhod, RH_max=44.0, physics=1):
    x, rd3, kappa, th, rv, rhod = _prep(x, rd3, kappa, th, rv, rhod)
    cell = np.ascontiguousarray(cell, np.int64)
    g32, e32 = np.empty(len(x), np.float32), np.empty(len(x), np.float32)
    g64 = np.empty_like(x)
    F = C.POINTER(C.c_float)
    lib().hc_growth(len(x), _d(x), _d(rd3), _d(kappa), cell.ctypes.data_as(C.POINTER(C.c_int64)), _d(th), _d(rv),
                    _d(rhod), RH_max, physics, g32.ctypes.data_as(F), e32.ctypes.data_as(F), _d(g64))
    return g32, e32, g64
