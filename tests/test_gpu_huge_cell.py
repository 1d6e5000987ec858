"""A grid cell above the block path's 8192 super-droplets (paper Sec. 5.1.4:
pairing within a cell, whatever its population): a context whose initial
cells are that large reserves global-memory scratch, and the block path
sorts and pairs such a cell there.  Against the oracle: multiplicities bit
exact, radii within 1e-12, the Golovin box with 20 000 and with 2^15 + 3
super-droplets (a ragged power-of-two padding), and the geometric kernel
with multiple coalescence."""
import numpy as np
import pytest

import workloads
from gpu_helpers import compare_states, oracle_state, pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_sd", [20000, 2 ** 15 + 3])
def test_huge_golovin_cell_matches_oracle(n_sd):
    w = workloads.golovin_box(seed=9, n_sd=n_sd)
    p, o = pair(w)
    for t in range(1, 41):
        p.step_async(w.opts)
        p.wait()
        o.step_async(w.opts)
        if t in (1, 40):
            compare_states(p.state(), oracle_state(o, ()))
    st = p.stats()
    assert st["n_coll"] == o.stats.n_coll > 0
    assert st["n_pairs"] == o.stats.n_pairs


def test_huge_geometric_cell_with_multiple_coalescence():
    w = workloads.golovin_box(seed=4, n_sd=12000)
    w.cfg["kernel"] = "geometric"
    opts = dict(w.opts, coal_multi=1, sstp_coal=2)
    p, o = pair(w)
    for _ in range(20):
        p.step_async(opts)
        p.wait()
        o.step_async(opts)
    compare_states(p.state(), oracle_state(o, ()))
    assert p.stats()["n_coll"] == o.stats.n_coll > 0
