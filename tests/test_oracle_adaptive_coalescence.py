"""Pins of the oracle's adaptive coalescence substeps (the paper plans to
control the substep from P_ij, Sec. 5.1.4): per cell and step,
max(sstp_coal, ceil(P_bound)) substeps, at most coal_adapt, with P_bound an
upper bound of eq. P_ij over every pair the cell could form.

* the bound holds: with the chosen count, a brute-force pass over all
  n(n-1)/2 pairs finds no P_ij above 1;
* below the fixed count nothing changes (bit for bit), and the cap holds;
* on the Golovin box with 100 s steps the adaptive count recovers the
  analytic second moment, which one substep per step misses by far.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle_helpers import box_cfg, coalesce, make_state


def _max_pair_p(kernel, N, rw2, b, dV, dt, t=None):
    """Largest eq. P_ij over all pairs, from the kernel's definition."""
    n = len(N)
    r = np.sqrt(rw2)
    V = 4.0 / 3.0 * math.pi * r ** 3
    v = np.array([oracle.vterm(x, t) for x in rw2]) if kernel == "geometric" else None
    scale = n * (n - 1) / (2 * (n // 2))
    best = 0.0
    for i, j in itertools.combinations(range(n), 2):
        K = b * (V[i] + V[j]) if kernel == "golovin" else math.pi * (r[i] + r[j]) ** 2 * abs(v[i] - v[j])
        best = max(best, max(N[i], N[j]) * K * dt / dV * scale)
    return best


@pytest.mark.parametrize("kernel,n,seed", [("golovin", 2, 0), ("golovin", 7, 1), ("golovin", 40, 2),
                                           ("geometric", 3, 3), ("geometric", 16, 4), ("geometric", 64, 5)])
def test_substeps_bound_every_pair(kernel, n, seed):
    rng = np.random.default_rng(seed)
    N = rng.integers(1, 10 ** 9, size=n)
    rw2 = np.exp(rng.uniform(np.log(2e-6), np.log(500e-6), size=n)) ** 2
    t = oracle.thermo(np.float64(300.0), np.float64(0.01), np.float64(1.0))
    # size the problem so that the largest pair P at one substep is ~20
    dt, b, dV = 5.0, 1.0, 1.0
    p1 = _max_pair_p(kernel, N, rw2, b, dV, dt, t)
    if kernel == "golovin":
        b = 20.0 / p1
    else:
        dV = p1 / 20.0
    cfg = box_cfg(n_sd=n, kernel=kernel, b=b, dV=dV, dt=dt, seed=seed)
    s = make_state(N, rw2)
    st = _coalesce_adapt(cfg, s, sstp=1, cap=100000)
    sub = st.n_coal_substeps
    pmax = _max_pair_p(kernel, N, rw2, b, dV, dt, t)
    assert pmax > 1.0  # the fixed single substep would have P > 1
    assert sub >= 1 and pmax / sub <= 1.0
    # every substep paired all n super-droplets (no multiplicity reached 0)
    assert st.n_pairs == sub * (n // 2)


def _coalesce_adapt(cfg, state, sstp, cap, step=0, multi=0):
    import ctypes as C
    dom = oracle.make_domain(cfg)
    o = oracle.make_opts(dict(adve=0, sedi=0, cond=0, coal=1, sstp_coal=sstp, coal_multi=multi, coal_adapt=cap))
    f = lambda v: np.full(1, v, np.float64)
    st = oracle.Stats()
    sd = state.struct()
    oracle.lib().orc_coalesce(C.byref(dom), C.byref(o), C.byref(sd), oracle._dp(f(300.0)), oracle._dp(f(0.01)),
                              oracle._dp(f(1.0)), step, C.byref(st))
    return st


def test_no_change_below_the_fixed_count_and_cap():
    rng = np.random.default_rng(8)
    n = 64
    N = rng.integers(1, 10 ** 6, size=n)
    rw2 = np.exp(rng.uniform(np.log(2e-6), np.log(40e-6), size=n)) ** 2
    cfg = box_cfg(n_sd=n, kernel="golovin", b=1e-3, dV=1e6, dt=1.0, seed=8)
    a, c = make_state(N, rw2), make_state(N, rw2)
    sa = coalesce(cfg, a, step=2, sstp=10)
    sc = _coalesce_adapt(cfg, c, sstp=10, cap=1000, step=2)
    assert sc.n_coal_substeps == 10 and sa.n_coal_substeps == 10
    assert np.array_equal(a.N, c.N) and np.array_equal(a.rw2, c.rw2)
    # a bound far above the cap: the cap wins
    big = box_cfg(n_sd=n, kernel="golovin", b=1e15, dV=1e6, dt=1.0, seed=8)
    st = _coalesce_adapt(big, make_state(N, rw2), sstp=2, cap=37)
    assert st.n_coal_substeps == 37


B, N0, RBAR, DV = 1500.0, 2.0 ** 23, 30.531e-6, 1e6
VBAR = 4.0 / 3.0 * math.pi * RBAR ** 3


def _golovin_moments(dt, adapt, seeds=4, T=1800.0):
    m0, m2 = [], []
    for seed in range(seeds):
        w = workloads.golovin_box(seed=seed)
        cfg = dict(w.cfg, dt=dt)
        o = oracle.Oracle(cfg)
        o.init(w.th, w.rv, w.rhod)
        opts = dict(w.opts, coal_adapt=adapt)
        for _ in range(int(T / dt)):
            o.step_async(opts)
        N = o.state.N.astype(float)
        V = 4.0 / 3.0 * math.pi * o.state.rw2 ** 1.5
        m0.append(N.sum() / DV)
        m2.append((N * V * V).sum() / DV)
    return np.mean(m0), np.mean(m2), o.stats.n_coal_substeps


def test_golovin_long_steps_adaptive_recovers_second_moment():
    """Golovin (1963): M0 = n0 exp(-b n0 Vbar t), M2 = 2 n0 Vbar^2 exp(2 b n0 Vbar t)."""
    T = 1800.0
    m0a = N0 * math.exp(-B * N0 * VBAR * T)
    m2a = 2.0 * N0 * VBAR ** 2 * math.exp(2.0 * B * N0 * VBAR * T)
    m0, m2, sub = _golovin_moments(100.0, 1000)
    assert sub > 18 * 5  # the adaptive count went well above one substep per step
    assert m0 == pytest.approx(m0a, rel=0.04)
    assert m2 == pytest.approx(m2a, rel=0.3)
    _, m2_fixed, sub_fixed = _golovin_moments(100.0, 0)
    assert sub_fixed == 18
    assert m2_fixed < 0.4 * m2a
