"""Pins of the oracle's third collection kernel, the geometric kernel times
the hydrostatic collection efficiency of Long (1974) (a formula standing in
for the tabulated efficiencies the paper cites, Sec. 5.1.4): with the
largest P of a two-droplet cell as the probe, the ratio to the geometric
kernel is E itself, which is 1 where the larger drop has R >= 50 um, the
floor 1e-3 where the smaller has r <= 3 um, 1 where the formula exceeds 1,
and 4.5e8 R^2 (1 - 3e-6 / r) (SI) in between; where every drop is above
50 um the two kernels give the same run bit for bit."""
import numpy as np
import pytest

from oracle_helpers import box_cfg, coalesce, make_state


def max_p(kernel, R, r, N=(10 ** 6, 10 ** 6)):
    cfg = box_cfg(n_sd=2, kernel=kernel, dV=1e3, dt=1.0, seed=0)
    s = make_state(list(N), np.array([R * R, r * r]))
    return coalesce(cfg, s, step=0).max_p


def long_cgs(R, r):
    """Long's (1974) efficiency as he states it, with the radii in cm:
    E = 4.5e4 R^2 (1 - 3e-4 / r); the oracle writes it in SI units."""
    Rc, rc = R * 100.0, r * 100.0
    return 4.5e4 * Rc * Rc * (1.0 - 3e-4 / rc)


@pytest.mark.parametrize("R,r,E", [(60e-6, 55e-6, 1.0),                                   # R >= 50 um
                                   (40e-6, 2e-6, 1e-3),                                    # floor
                                   (20e-6, 10e-6, long_cgs(20e-6, 10e-6)),                 # 0.126
                                   (45e-6, 40e-6, long_cgs(45e-6, 40e-6)),                 # 0.843
                                   (49.5e-6, 45e-6, 1.0)])                                 # formula > 1: cap
def test_efficiency_is_the_ratio_to_the_geometric_kernel(R, r, E):
    assert 0 < E <= 1
    assert max_p("long", R, r) == pytest.approx(E * max_p("geometric", R, r), rel=1e-13)


def test_large_drops_collide_as_in_the_geometric_kernel():
    rng = np.random.default_rng(4)
    n = 64
    N = rng.integers(1, 10 ** 6, size=n)
    rw2 = rng.uniform(55e-6, 400e-6, size=n) ** 2
    out = []
    for kernel in ("geometric", "long"):
        s = make_state(N, rw2)
        st = coalesce(box_cfg(n_sd=n, kernel=kernel, dV=1e2, dt=1.0, seed=4), s, step=2, sstp=10)
        out.append((s, st))
    (a, sa), (b, sb) = out
    assert sa.n_coll == sb.n_coll > 0 and sa.max_p == sb.max_p
    assert np.array_equal(a.N, b.N) and np.array_equal(a.rw2, b.rw2)
