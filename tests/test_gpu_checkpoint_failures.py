"""Checkpoint / resume and the failure reports of the C ABI, on the GPU:

* a run restored from a checkpoint (every attribute, the step counter,
  theta and r_v) into a fresh context continues bit for bit like the
  uninterrupted run;
* a bounded wait on work still in flight returns SDM_ETIMEOUT and leaves the
  work running; the next unbounded wait completes it;
* a non-finite radius reaching the condensation kernel is reported as
  SDM_ENUMERIC (a device flag read on the host; no trap).
"""
import numpy as np
import pytest

import workloads
from gpu_helpers import gpu_particles
from paper_1310_1905_gb300 import sdm

pytestmark = pytest.mark.gpu

ALL = dict(adve=1, sedi=1, cond=1, coal=1, sstp_cond=10, sstp_coal=10)
ATTRS = ("uid", "N", "rw2", "rd3", "kappa", "x", "z")


def run(p, th, rv, w, steps):
    for _ in range(steps):
        p.step_sync(ALL, th, rv)
        p.step_async(ALL)
        p.wait()


def test_checkpoint_resume_bit_identical():
    w = workloads.icmw_2d(nx=9, nz=13, sd_conc=20, seed=14, dz=115.0)
    p = gpu_particles(w)
    th, rv = w.th.copy(), w.rv.copy()
    run(p, th, rv, w, 4)
    snap = {k: p.attr(k).copy() for k in ATTRS}
    step = sdm.sdm_get_step(p.ctx)
    th_s, rv_s = th.copy(), rv.copy()
    run(p, th, rv, w, 5)
    # a fresh context of the same set-up, restored (positions first, so that
    # a regroup between the calls would show)
    q = gpu_particles(w)
    for k in ("x", "z", "uid", "N", "rw2", "rd3", "kappa"):
        sdm.sdm_set_attr(q.ctx, k, snap[k])
    sdm.sdm_set_step(q.ctx, step)
    run(q, th_s, rv_s, w, 5)
    assert np.array_equal(th, th_s) and np.array_equal(rv, rv_s)
    a, b = p.state(), q.state()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert p.stats()["n_coll"] > 0


def test_bounded_wait_times_out_then_completes():
    w = workloads.updraft_3d(nx=32, ny=32, nz=32, seed=2)
    p = gpu_particles(w)
    th, rv = np.ascontiguousarray(w.th).copy(), np.ascontiguousarray(w.rv).copy()
    p.step_sync(ALL, th, rv)
    p.step_async(ALL)  # about 20 ms of device work
    with pytest.raises(sdm.SdmError) as e:
        p.wait(0.0)
    assert e.value.status == 4  # SDM_ETIMEOUT
    p.wait()  # unbounded: completes
    assert sdm.sdm_get_step(p.ctx) == 1
    p.step_sync(ALL, th, rv)  # the context is usable afterwards


def test_non_finite_radius_reported():
    w = workloads.icmw_2d(nx=4, nz=5, sd_conc=8, seed=3)
    p = gpu_particles(w)
    rw2 = p.attr("rw2")
    rw2[7] = np.nan
    sdm.sdm_set_attr(p.ctx, "rw2", rw2)
    th, rv = w.th.copy(), w.rv.copy()
    with pytest.raises(sdm.SdmError) as e:
        p.step_sync(dict(ALL, adve=0, sedi=0, coal=0), th, rv)
    assert e.value.status == 5  # SDM_ENUMERIC


def test_injected_allocation_failure_reports_enomem(monkeypatch):
    """SDM_FAIL_ALLOC=k makes the k-th device allocation of sdm_init fail on
    the host: the call returns SDM_ENOMEM, frees what it had taken, and a
    later init succeeds."""
    torch = pytest.importorskip("torch")
    w = workloads.icmw_2d(nx=4, nz=5, sd_conc=8, seed=3)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 3, 9, 17, 25):
        monkeypatch.setenv("SDM_FAIL_ALLOC", str(k))
        with pytest.raises(sdm.SdmError) as e:
            gpu_particles(w)
        assert e.value.status == 2  # SDM_ENOMEM
    monkeypatch.delenv("SDM_FAIL_ALLOC")
    p = gpu_particles(w)
    th, rv = w.th.copy(), w.rv.copy()
    p.step_sync(ALL, th, rv)
    p.close()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)  # nothing left behind
