"""Parity of the Long (1974) collection kernel (the geometric kernel times a
closed-form efficiency; the paper tabulates its efficiencies, Sec. 5.1.4)
between the CUDA library and the oracle: multiplicities bit-exact, radii
within 1e-12, on the warp path (cells of up to 128 super-droplets) and the
block path (larger cells), after condensation has grown droplets into the
range where the efficiency is neither the floor nor one."""
import numpy as np
import pytest

import workloads
from gpu_helpers import compare_states, oracle_state, pair, present_dims

pytestmark = pytest.mark.gpu

COND_ONLY = dict(adve=0, sedi=0, cond=1, coal=0, sstp_cond=10, sstp_coal=10)
COAL_ONLY = dict(adve=0, sedi=0, cond=0, coal=1, sstp_cond=10, sstp_coal=10)


def grown(kernel, sd, seed=6):
    w = workloads.icmw_2d(nx=9, nz=13, sd_conc=sd, seed=seed, dz=115.0)
    w.cfg["kernel"] = kernel
    p, o = pair(w)
    th, rv = w.th.copy(), w.rv.copy()
    for _ in range(3):
        p.step_sync(COND_ONLY, th, rv)
        o.step_sync(COND_ONLY)
    return w, p, o


@pytest.mark.parametrize("sd", [40, 200])
def test_long_kernel_matches_oracle(sd):
    w, p, o = grown("long", sd)
    # the upper cells are supersaturated: about half the drops are above
    # 3 um, so many pairs take the efficiency formula 4.5e8 R^2 (1 - 3e-6/r)
    # rather than its floor (r <= 3 um) or the cap (R >= 50 um)
    r = np.sqrt(o.state.rw2)
    assert ((r > 3e-6) & (r < 50e-6)).mean() > 0.3
    for _ in range(5):
        p.step_async(COAL_ONLY)
        p.wait()
        o.step_async(COAL_ONLY)
    compare_states(p.state(), oracle_state(o, present_dims(w.cfg)))
    st = p.stats()
    assert st["n_pairs"] == o.stats.n_pairs and st["n_coll"] == o.stats.n_coll
    assert st["max_p"] == pytest.approx(o.stats.max_p, rel=1e-12)


def test_efficiency_lowers_the_collision_probability():
    """Same state, same draws: E <= 1 scales every P_ij down, so the largest
    P of the step is lower than the geometric kernel's and no more pairs
    collide."""
    out = {}
    for kernel in ("geometric", "long"):
        _, p, o = grown(kernel, 40)
        p.step_async(COAL_ONLY)
        p.wait()
        out[kernel] = p.stats()
        p.close()
    assert out["long"]["max_p"] < out["geometric"]["max_p"]
    assert out["long"]["n_coll"] <= out["geometric"]["n_coll"]
