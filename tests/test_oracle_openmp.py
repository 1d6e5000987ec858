"""The oracle's cell-parallel timing build (the same C source compiled with
-fopenmp, the paper's OpenMP back-end of Sec. 6) gives the serial oracle's
results bit for bit: cells are independent within condensation and
coalescence, and each cell's counters are merged after the cell."""
import numpy as np

import oracle
import workloads


def _run(w, omp, steps):
    o = oracle.Oracle(w.cfg, omp=omp)
    o.init(w.th, w.rv, w.rhod)
    for _ in range(steps):
        o.step_sync(w.opts)
        o.step_async(w.opts, w.rhoCx, w.rhoCy, w.rhoCz)
    return o


def test_openmp_build_uses_threads():
    assert oracle.threads(0, omp=False) == 1
    assert oracle.threads(0, omp=True) >= 1


def test_openmp_build_matches_serial_bit_for_bit():
    oracle.threads(4, omp=True)
    for w in (workloads.icmw_2d(nx=6, nz=12, sd_conc=16, seed=3, dz=120.0),
              workloads.updraft_3d(nx=2, ny=2, nz=16, sd_conc=16, seed=5)):
        a, b = _run(w, False, 3), _run(w, True, 3)
        sa, sb = a.state.sorted_by_uid(), b.state.sorted_by_uid()
        for f in oracle.State.FIELDS:
            assert np.array_equal(getattr(sa, f), getattr(sb, f)), f
        assert np.array_equal(a.th, b.th) and np.array_equal(a.rv, b.rv)
        da, db = a.stats.as_dict(), b.stats.as_dict()
        assert da == db


def test_openmp_build_golovin_box_matches_serial():
    w = workloads.golovin_box(seed=2, n_sd=512)
    a, b = _run(w, False, 20), _run(w, True, 20)
    assert np.array_equal(a.state.sorted_by_uid().N, b.state.sorted_by_uid().N)
    assert np.array_equal(a.state.sorted_by_uid().rw2, b.state.sorted_by_uid().rw2)
