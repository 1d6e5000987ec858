"""Pins of the oracle's multiple coalescence (the treatment of P_ij > 1 that
the paper plans in Sec. 5.1.4, from Shima et al. 2009, Sec. 4.1.4 there)
against results fixed by probability and arithmetic:

* unbiasedness beyond P = 1: the expected loss of droplets per substep is
  sum_{i<j} N_i N_j K_ij dt/dV for any P as long as floor(N_L/N_S) never
  caps the number of events, while the paper's one-event scheme falls
  short of it once P > 1;
* the event count takes only floor(P) and floor(P) + 1, the latter with
  frequency P - floor(P);
* exact integers N_L - gamma N_S, merged r^3 = r_S^3 + gamma r_L^3, the cap
  at floor(N_L/N_S) and the zero left by equal multiplicities;
* where every P <= 1 the result is the paper's scheme bit for bit.
"""
import itertools
import math

import numpy as np
import pytest

from oracle_helpers import box_cfg, coalesce, make_state


def _golovin_b_for(N, rw2, p_max, dV=1.0, dt=1.0):
    """Golovin constant that makes the largest scaled P of the cell p_max."""
    n = len(N)
    V = 4.0 / 3.0 * math.pi * np.asarray(rw2) ** 1.5
    scale = n * (n - 1) / (2 * (n // 2))
    Kmax = max(max(N[i], N[j]) * (V[i] + V[j]) for i, j in itertools.combinations(range(n), 2))
    return p_max / (Kmax * dt / dV * scale), V


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (5, 2), (6, 3)])
def test_expected_loss_unbiased_beyond_p_one(n, seed):
    rng = np.random.default_rng(seed)
    # multiplicities a factor of ~16 apart, so floor(N_L/N_S) >= 8 is above
    # every gamma that P <= 3.5 can draw and no event count is capped; the
    # larger multiplicities go with the smaller droplets
    N = 1000 * 16 ** np.arange(n) + rng.integers(0, 1000, size=n)
    rw2 = (30e-6 / 2.0 ** np.arange(n) * rng.uniform(0.8, 1.2, size=n)) ** 2
    b, V = _golovin_b_for(N, rw2, 3.5)
    cfg = box_cfg(n_sd=n, b=b, seed=seed)
    scale = n * (n - 1) / (2 * (n // 2))
    pairs = list(itertools.combinations(range(n), 2))
    # every pair is drawn with probability 1/scale and loses gamma N_S
    # droplets, E[gamma] = P; the one-event scheme has E[gamma] = min(P, 1)
    expected = sum(N[i] * N[j] * b * (V[i] + V[j]) for i, j in pairs)
    P = {(i, j): max(N[i], N[j]) * b * (V[i] + V[j]) * scale for i, j in pairs}
    expected_one = sum(min(P[(i, j)], 1.0) * min(N[i], N[j]) / scale for i, j in pairs)
    assert max(P.values()) > 1.0
    trials = 20000
    loss = {0: np.empty(trials), 1: np.empty(trials)}
    for multi in (0, 1):
        for step in range(trials):
            s = make_state(N, rw2)
            st = coalesce(cfg, s, step=step, multi=multi)
            loss[multi][step] = N.sum() - s.N.astype(np.int64).sum()
        assert st.max_p <= 3.5 * (1 + 1e-12)
    se = {m: loss[m].std(ddof=1) / math.sqrt(trials) for m in (0, 1)}
    # (a pair with P > 1 alone loses the same count every trial: se = 0)
    assert abs(loss[1].mean() - expected) <= 4.5 * se[1] + 1e-9 * expected
    assert abs(loss[0].mean() - expected_one) <= 4.5 * se[0] + 1e-9 * expected_one
    if n <= 3:  # here the two expectations are far apart: the pin is sharp
        assert expected - expected_one > 20 * max(se[0], se[1])


def test_event_count_is_floor_or_ceil_of_p():
    N = np.array([1000, 7])
    rw2 = np.array([4e-12, 9e-12])
    b, V = _golovin_b_for(N, rw2, 5.5)
    cfg = box_cfg(n_sd=2, b=b)
    trials = 4000
    gammas = np.empty(trials, np.int64)
    for step in range(trials):
        s = make_state(N, rw2, rd3=np.array([2e-24, 3e-24]), kappa=np.array([0.2, 1.2]))
        st = coalesce(cfg, s, step=step, multi=1)
        assert st.n_coll == 1 and st.n_pgt1 == 1
        NL = int(s.N[0])
        assert int(s.N[1]) == 7
        assert (1000 - NL) % 7 == 0
        g = (1000 - NL) // 7
        gammas[step] = g
        # the smaller-N super-droplet took g droplets of the larger one
        assert s.rw2[1] ** 1.5 == pytest.approx(9e-12 ** 1.5 + g * 4e-12 ** 1.5, rel=1e-14)
        assert s.rd3[1] == pytest.approx(3e-24 + g * 2e-24, rel=1e-15)
        assert s.kappa[1] == pytest.approx((1.2 * 3 + 0.2 * 2 * g) / (3 + 2 * g), rel=1e-14)
        # the larger keeps its radii; water is conserved
        assert s.rw2[0] == 4e-12 and s.rd3[0] == 2e-24
        m0 = (N * rw2 ** 1.5).sum()
        assert (s.N.astype(float) * s.rw2 ** 1.5).sum() == pytest.approx(m0, rel=1e-14)
    assert set(np.unique(gammas)) == {5, 6}
    # P - floor(P) = 0.5 up to rounding: binomial, 5 sigma
    assert abs((gammas == 6).mean() - 0.5) < 5 * math.sqrt(0.25 / trials)
    assert gammas.mean() == pytest.approx(5.5, abs=5 * math.sqrt(0.25 / trials))


def test_event_count_capped_by_multiplicity_ratio():
    rw2 = np.array([4e-12, 9e-12])
    b, _ = _golovin_b_for(np.array([10, 3]), rw2, 5.5)
    for step in range(50):
        s = make_state([10, 3], rw2)
        coalesce(box_cfg(n_sd=2, b=b), s, step=step, multi=1)
        assert list(s.N) == [1, 3]
        assert s.rw2[1] ** 1.5 == pytest.approx(9e-12 ** 1.5 + 3 * 4e-12 ** 1.5, rel=1e-14)


def test_equal_multiplicities_still_leave_a_zero():
    rw2 = np.array([1e-12, 4e-12])
    b, _ = _golovin_b_for(np.array([5, 5]), rw2, 2.7)
    for step in range(20):
        s = make_state([5, 5], rw2)
        coalesce(box_cfg(n_sd=2, b=b), s, step=step, multi=1)
        assert sorted(s.N.tolist()) == [0, 5]
        merged = int(np.nonzero(s.N)[0][0])
        assert s.rw2[merged] ** 1.5 == pytest.approx(1e-18 + 8e-18, rel=1e-14)


def test_reduces_to_one_event_scheme_when_p_at_most_one():
    rng = np.random.default_rng(5)
    n = 64
    N = rng.integers(1, 10 ** 6, size=n)
    rw2 = np.exp(rng.uniform(np.log(2e-6), np.log(60e-6), size=n)) ** 2
    rd3 = np.exp(rng.uniform(np.log(1e-8), np.log(1e-7), size=n)) ** 3
    kappa = rng.uniform(0.1, 1.2, size=n)
    b, _ = _golovin_b_for(N, rw2, 0.4, dt=0.1)  # dt'' = dt / 10 substeps; merges raise P
    cfg = box_cfg(n_sd=n, b=b, seed=5)
    out = []
    for multi in (0, 1):
        s = make_state(N, rw2, rd3=rd3, kappa=kappa)
        n_coll = 0
        for step in range(5):
            st = coalesce(cfg, s, step=step, sstp=10, multi=multi)
            assert st.max_p <= 1.0
            n_coll += st.n_coll
        assert n_coll > 20
        out.append(s)
    a, c = out
    assert np.array_equal(a.N, c.N)
    assert np.array_equal(a.rw2, c.rw2) and np.array_equal(a.rd3, c.rd3) and np.array_equal(a.kappa, c.kappa)


def test_invariants_many_multiple_events():
    rng = np.random.default_rng(9)
    n = 300
    N = rng.integers(1, 10 ** 9, size=n)
    rw2 = np.exp(rng.uniform(np.log(2e-6), np.log(300e-6), size=n)) ** 2
    rd3 = np.exp(rng.uniform(np.log(1e-8), np.log(1e-7), size=n)) ** 3
    cfg = box_cfg(n_sd=n, kernel="geometric", dV=1e-3, dt=5.0, seed=9)
    s = make_state(N, rw2, rd3=rd3, kappa=np.full(n, 0.61))
    m_w0 = (N * rw2 ** 1.5).sum()
    m_d0 = (N * rd3).sum()
    st = coalesce(cfg, s, step=1, sstp=10, multi=1)
    assert st.n_pgt1 > 20 and st.n_coll > 50
    Na = s.N.astype(np.int64)
    assert (Na >= 0).all() and Na.sum() < N.sum()
    assert (Na * s.rw2 ** 1.5).sum() == pytest.approx(m_w0, rel=1e-13)
    assert (Na * s.rd3).sum() == pytest.approx(m_d0, rel=1e-13)
    np.testing.assert_allclose(s.kappa, 0.61, rtol=1e-14)
