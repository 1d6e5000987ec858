"""Parity of adaptive coalescence substeps (coal_adapt > 0: per cell,
max(sstp_coal, ceil(P_bound)) substeps from an upper bound of P_ij at the
start of the step) between the CUDA library and the oracle: multiplicities
bit-exact, radii within 1e-12, the substep counts equal, on the warp path
and the block path, with the Golovin and the geometric kernel, alone and
with multiple coalescence."""
import numpy as np
import pytest

import workloads
from gpu_helpers import compare_states, oracle_state, pair
from paper_1310_1905_gb300 import sdm

pytestmark = pytest.mark.gpu

ADAPT = dict(adve=0, sedi=0, cond=0, coal=1, sstp_cond=1, sstp_coal=1, coal_adapt=400)


def long_step_box(n_sd, seed, dt, kernel):
    w = workloads.golovin_box(seed=seed, n_sd=n_sd)
    w.cfg["dt"] = dt
    w.cfg["kernel"] = kernel
    return w


@pytest.mark.parametrize("n_sd,kernel,dt,steps,multi", [(100, "golovin", 300.0, 6, 0), (100, "geometric", 300.0, 6, 0),
                                                        (60, "geometric", 300.0, 6, 1),
                                                        (8192, "golovin", 100.0, 6, 0),
                                                        (8192, "geometric", 200.0, 4, 1)])
def test_adaptive_substeps_match_oracle(n_sd, kernel, dt, steps, multi):
    w = long_step_box(n_sd, 5, dt, kernel)
    opts = dict(ADAPT, coal_multi=multi)
    p, o = pair(w)
    for _ in range(steps):
        p.step_async(opts)
        p.wait()
        o.step_async(opts)
    compare_states(p.state(), oracle_state(o, ()))
    st = p.stats()
    assert st["n_coal_substeps"] == o.stats.n_coal_substeps > steps  # the bound raised the count
    assert st["n_coll"] == o.stats.n_coll and st["n_pairs"] == o.stats.n_pairs
    assert st["n_pgt1"] == o.stats.n_pgt1


def test_adaptive_substeps_2d_cells():
    """Many cells of a 2D domain, each with its own count: every twentieth
    super-droplet is given a drizzle-size radius (30-60 um, seeded), so that
    the bound exceeds the fixed count in some cells and not in others."""
    w = workloads.icmw_2d(nx=9, nz=13, sd_conc=20, seed=6, dz=115.0)
    p, o = pair(w)
    rng = np.random.default_rng(4)
    uid_o = o.state.uid.astype(np.int64)
    n = len(uid_o)
    big = np.zeros(n, bool)
    big[::20] = True
    r_by_uid = np.where(big, rng.uniform(30e-6, 60e-6, size=n), 0.0)
    rw2_by_uid = np.where(big, r_by_uid ** 2, 0.0)
    o_order = np.argsort(uid_o)
    rw2_o = o.state.rw2.copy()
    rw2_o[o_order[big]] = rw2_by_uid[big]
    o.state.rw2[:] = rw2_o
    uid_g = p.attr("uid").astype(np.int64)
    rw2_g = p.attr("rw2")
    sel = big[uid_g]
    rw2_g[sel] = rw2_by_uid[uid_g[sel]]
    sdm.sdm_set_attr(p.ctx, "rw2", rw2_g)
    opts = dict(adve=0, sedi=0, cond=0, coal=1, sstp_cond=10, sstp_coal=2, coal_adapt=200)
    for _ in range(3):
        p.step_async(opts)
        p.wait()
        o.step_async(opts)
    compare_states(p.state(), oracle_state(o, ("x", "z")))
    n_cells = 9 * 13
    assert p.stats()["n_coal_substeps"] == o.stats.n_coal_substeps
    assert 3 * 2 * n_cells < o.stats.n_coal_substeps < 3 * 200 * n_cells  # varies from cell to cell


def test_adaptive_rejected_by_ensembles_and_negative():
    from paper_1310_1905_gb300.ensemble import Ensemble
    ens = Ensemble(max_sd=1 << 10, max_members=2)
    with pytest.raises(sdm.SdmError):
        ens.step(dict(ADAPT))
    ens.close()
    w = long_step_box(64, 1, 1.0, "golovin")
    p, _ = pair(w)
    with pytest.raises(sdm.SdmError) as e:
        p.step_async(dict(ADAPT, coal_adapt=-1))
    assert e.value.status == 1
