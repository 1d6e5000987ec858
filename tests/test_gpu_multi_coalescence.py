"""Parity of multiple coalescence (coal_multi = 1: floor(P) or floor(P) + 1
events for a pair with P_ij > 1, the treatment Sec. 5.1.4 plans) between the
CUDA library and the oracle: multiplicities bit-exact, radii within 1e-12,
on the warp path (cells of up to 128 super-droplets), the block path
(8192) and the batched ensemble."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import compare_states, oracle_state, pair
from paper_1310_1905_gb300.ensemble import Ensemble

pytestmark = pytest.mark.gpu

MULTI = dict(adve=0, sedi=0, cond=0, coal=1, sstp_cond=1, sstp_coal=1, coal_multi=1)


def long_step_box(n_sd, seed, dt):
    """Golovin box with a long timestep: P_ij ~ 3e-3 dt at the start and far
    above 1 once large drops form."""
    w = workloads.golovin_box(seed=seed, n_sd=n_sd)
    w.cfg["dt"] = dt
    return w


@pytest.mark.parametrize("n_sd,dt,steps", [(24, 400.0, 12), (100, 300.0, 12), (8192, 100.0, 18)])
def test_multiple_coalescence_matches_oracle(n_sd, dt, steps):
    w = long_step_box(n_sd, seed=3, dt=dt)
    p, o = pair(w)
    for t in range(steps):
        p.step_async(MULTI)
        p.wait()
        o.step_async(MULTI)
        if t % 4 == 3:
            compare_states(p.state(), oracle_state(o, ()))
    st = p.stats()
    assert st["n_pgt1"] == o.stats.n_pgt1 > 0
    assert st["n_coll"] == o.stats.n_coll
    assert st["n_recycled"] == o.stats.n_recycled
    assert st["max_p"] == pytest.approx(o.stats.max_p, rel=1e-12)


def test_multiple_coalescence_changes_the_result():
    """The option is live: with P > 1 present, the one-event and the
    multiple-event runs part ways, and the multiple one loses more
    droplets."""
    w = long_step_box(100, seed=4, dt=300.0)
    out = []
    for multi in (0, 1):
        p, _ = pair(w)
        for _ in range(6):
            p.step_async(dict(MULTI, coal_multi=multi))
            p.wait()
        out.append(p.state()["N"].astype(np.float64).sum())
        assert p.stats()["n_pgt1"] > 0
        p.close()
    assert out[1] < out[0]


def test_ensemble_multiple_coalescence_matches_oracle():
    """Two Golovin members in one ensemble.  At most n_sd / 2 zeros appear
    per step (one substep), within what the ensemble recycles per member and
    step (64), so the recycling matches the oracle's too."""
    ens = Ensemble(dt=300.0, kernel="golovin", golovin_b=1500.0, max_sd=1 << 10, max_members=4)
    runs = []
    for n_sd, seed in ((128, 6), (100, 7)):
        w = long_step_box(n_sd, seed=seed, dt=300.0)
        m = dict(n_sd=n_sd, dV=1e6, th=300.0, rv=0.01, rhod=1.0, seed=seed, init_dist="exponential",
                 exp_mean_volume=w.cfg["exp_mean_volume"], exp_n0=w.cfg["exp_n0"])
        o = oracle.Oracle(w.cfg)
        o.init(w.th, w.rv, w.rhod)
        runs.append((ens.add(m), n_sd, o))
    for _ in range(15):
        ens.step(MULTI)
        ens.wait()
        for _, _, o in runs:
            o.step_async(MULTI)
    for mid, n_sd, o in runs:
        r = o.state.sorted_by_uid()
        assert o.stats.n_pgt1 > 0
        assert np.array_equal(ens.attr(mid, "N", n_sd), r.N)
        np.testing.assert_allclose(ens.attr(mid, "rw2", n_sd), r.rw2, rtol=1e-12)
        np.testing.assert_allclose(ens.attr(mid, "rd3", n_sd), r.rd3, rtol=1e-12)
    assert ens.stats()["n_pgt1"] == sum(o.stats.n_pgt1 for _, _, o in runs)
    ens.close()
