"""The kinematic framework's Eulerian stand-in on the GPU (sdm_euler_step:
donor-cell transport of theta and r_v, relaxation of the level means)
against the oracle's: fields within 1e-12 relative, alone and coupled with
the particle step over several steps, from host and from device arrays."""
import numpy as np
import pytest

import workloads
from gpu_helpers import assert_close, compare_states, oracle_state, pair
from paper_1310_1905_gb300 import sdm

pytestmark = pytest.mark.gpu

ALL = dict(adve=1, sedi=1, cond=1, coal=1, sstp_cond=10, sstp_coal=10)


def small(seed):
    # 100 m cells: the eddy's Courant numbers reach ~0.1, so the fields move
    return workloads.icmw_2d(nx=9, nz=13, sd_conc=12, seed=seed, dx=100.0, dz=100.0)


def profiles(w):
    return w.th.mean(axis=0), w.rv.mean(axis=0)


def test_euler_step_matches_oracle():
    w = small(1)
    p, o = pair(w)
    th0, rv0 = profiles(w)
    th, rv = w.th.copy(), w.rv.copy()
    rng = np.random.default_rng(0)
    th += rng.uniform(-0.5, 0.5, th.shape)  # something to transport and to relax
    rv *= rng.uniform(0.95, 1.05, rv.shape)
    o.th, o.rv = th.ravel().copy(), rv.ravel().copy()
    for _ in range(15):
        p.euler_step(th, rv, w.rhoCx, None, w.rhoCz, th0, rv0)
        o.euler_step(w.rhoCx, None, w.rhoCz, th0, rv0)
    assert_close("theta", th.ravel(), o.th)
    assert_close("r_v", rv.ravel(), o.rv)
    assert np.abs(o.th - w.th.ravel()).max() > 1e-3


def test_euler_coupled_with_particles_device_fields():
    torch = pytest.importorskip("torch")
    w = small(2)
    p, o = pair(w)
    th0, rv0 = profiles(w)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    th, rv = dev(w.th), dev(w.rv)
    Cx, Cz = dev(w.rhoCx), dev(w.rhoCz)
    for _ in range(5):
        p.euler_step(th, rv, Cx, None, Cz, th0, rv0)
        p.step_sync(ALL, th, rv)
        p.step_async(ALL)
        p.wait()
        o.euler_step(w.rhoCx, None, w.rhoCz, th0, rv0)
        o.step_sync(ALL)
        o.step_async(ALL, w.rhoCx, None, w.rhoCz)
    torch.cuda.synchronize()
    assert_close("theta", th.cpu().numpy().ravel(), o.th)
    assert_close("r_v", rv.cpu().numpy().ravel(), o.rv)
    compare_states(p.state(), oracle_state(o, ("x", "z")))


def test_euler_step_rejects_relaxation_without_profiles():
    w = small(3)
    p, _ = pair(w)
    th, rv = w.th.copy(), w.rv.copy()
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_euler_step(p.ctx, th, rv, w.rhoCx, None, w.rhoCz, th0=np.zeros(13), rv0=np.zeros(13), tau_rlx=0.0)
    assert e.value.status == 1


def test_euler_step_full_size_2d():
    """The full 75 x 75 case, in the launch configuration the bench uses
    (device fields): 30 Eulerian steps against the oracle's, every cell."""
    torch = pytest.importorskip("torch")
    import oracle
    w = workloads.icmw_2d()
    th0, rv0 = profiles(w)
    p = sdm.Particles(w.cfg, w.th, w.rv, w.rhod, w.rhoCx, None, w.rhoCz)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(5)
    th_h = w.th + rng.uniform(-0.3, 0.3, w.th.shape)
    rv_h = w.rv * rng.uniform(0.97, 1.03, w.rv.shape)
    th, rv, Cx, Cz = dev(th_h), dev(rv_h), dev(w.rhoCx), dev(w.rhoCz)
    th_o, rv_o = th_h.ravel().copy(), rv_h.ravel().copy()
    for _ in range(30):
        p.euler_step(th, rv, Cx, None, Cz, th0, rv0)
        th_o = oracle.relax(w.cfg, oracle.upwind(w.cfg, th_o, w.rhod, w.rhoCx, None, w.rhoCz), th0)
        rv_o = oracle.relax(w.cfg, oracle.upwind(w.cfg, rv_o, w.rhod, w.rhoCx, None, w.rhoCz), rv0)
    torch.cuda.synchronize()
    assert_close("theta", th.cpu().numpy().ravel(), th_o)
    assert_close("r_v", rv.cpu().numpy().ravel(), rv_o)
    p.close()
