"""The CUDA library's condensation solvers compiled for the CPU (the
kernels' own source, tests/hostcheck) against the oracle's bisection of the
paper's implicit growth equation (Sec. 5.1.3, eq. rw2_implicit), solve by
solve, along oracle trajectories of the 2D case (eddy transport of theta
and r_v, sedimentation and coalescence between the steps) and of columns of
the 3D updraft.

On the CPU both sides take exp, pow and log from the same math library, so
these tests isolate the solver's logic: its FP32 sign decisions under error
bounds, the Newton/secant polish, the replay that keeps the bisection's
root.  The GPU tests compare the device's own fast solve with its bisection
over whole domains.
"""
import numpy as np
import pytest

import oracle
import workloads

hostcheck = pytest.importorskip("hostcheck")


def cells_of(w, s):
    i = np.clip(np.floor(s.x / w.cfg["dx"]).astype(np.int64), 0, w.cfg["nx"] - 1)
    k = np.clip(np.floor(s.z / w.cfg["dz"]).astype(np.int64), 0, w.cfg["nz"] - 1)
    return i * w.cfg["nz"] + k


def trajectory(nx=10, sd=32, steps=30, seed=3):
    """Yield (x0, rd3, kappa, cell, th, rv, rhod, dt') before every step of
    an oracle run of the 2D case (every super-droplet with N > 0)."""
    w = workloads.icmw_2d(nx=nx, sd_conc=sd, seed=seed)
    o = oracle.Oracle(w.cfg, omp=True)
    o.init(w.th, w.rv, w.rhod)
    th0, rv0 = w.th.mean(axis=0), w.rv.mean(axis=0)
    dtp = w.cfg["dt"] / w.opts["sstp_cond"]
    for _ in range(steps):
        o.euler_step(w.rhoCx, None, w.rhoCz, th0, rv0)
        s = o.state
        live = s.N > 0
        yield (s.rw2[live].copy(), s.rd3[live].copy(), s.kappa[live].copy(), cells_of(w, s)[live], o.th.copy(),
               o.rv.copy(), o.rhod, dtp)
        o.step_sync(w.opts)
        o.step_async(w.opts, w.rhoCx, None, w.rhoCz)


@pytest.fixture(scope="module")
def states():
    hostcheck.build()
    return list(trajectory())


@pytest.mark.parametrize("solver", [1, 3], ids=["fast", "certified"])
def test_fast_solve_is_the_bisection_within_1e12(states, solver):
    """Both forms of the fast solve: the fused kernel's, and the staged
    layout's, which also settles on a Newton step whose error bound (from
    the FP32 slope's error and curvature bounds) is below 2^-43 x."""
    n = worst = fallbacks = evals = certified = 0
    for args in states:
        ref = oracle.solve_batch(*args)
        got, c = hostcheck.solve(*args, solver=solver)
        rel = np.abs(got - ref) / ref
        assert (rel <= 1e-12).all(), f"{(rel > 1e-12).sum()} solves differ by more than 1e-12; worst {rel.max():.3e}"
        n += len(ref)
        worst = max(worst, rel.max())
        fallbacks += c["fallback"]
        evals += c["evals"]
        certified += c["certified"]
    print(f"{n} solves, worst relative difference {worst:.2e}, {fallbacks} exact fallbacks, "
          f"{evals / n:.3f} FP64 growth evaluations per solve, {certified} certified settles")
    assert n > 400_000
    assert evals / n < 2.5  # against about 50 for the bisection
    assert (certified > n // 100) == (solver == 3)


def test_staged_rounds_are_the_certified_solve(states):
    """The staged layout's per-record sequence (the start, then one round
    per FP64 evaluation, bracket ends that need the term-by-term residual
    deferred to a round of their own) gives the certified solve's result bit
    for bit: the deferral moves work between rounds, never its arithmetic."""
    n = 0
    for args in states[::3]:
        a, _ = hostcheck.solve(*args, solver=3)
        b, _ = hostcheck.solve(*args, solver=4)
        assert np.array_equal(a, b), f"{(a != b).sum()} of {a.size} differ"
        n += a.size
    assert n > 100_000


def trajectory_3d(steps=25, seed=0):
    """As trajectory(), along a run of 4 x 4 x 128 columns of the 3D updraft
    (the full height: haze below, activation near cloud base, cloud above)."""
    w = workloads.updraft_3d(nx=4, ny=4, nz=128, seed=seed)
    o = oracle.Oracle(w.cfg, omp=True)
    o.init(w.th, w.rv, w.rhod)
    dtp = w.cfg["dt"] / w.opts["sstp_cond"]
    c = w.cfg
    for _ in range(steps):
        o.euler_step(w.rhoCx, w.rhoCy, w.rhoCz)
        s = o.state
        live = s.N > 0
        i = np.clip(np.floor(s.x / c["dx"]).astype(np.int64), 0, c["nx"] - 1)
        j = np.clip(np.floor(s.y / c["dy"]).astype(np.int64), 0, c["ny"] - 1)
        k = np.clip(np.floor(s.z / c["dz"]).astype(np.int64), 0, c["nz"] - 1)
        cell = (i * c["ny"] + j) * c["nz"] + k
        yield (s.rw2[live].copy(), s.rd3[live].copy(), s.kappa[live].copy(), cell[live], o.th.copy(), o.rv.copy(),
               o.rhod, dtp)
        o.step_sync(w.opts)
        o.step_async(w.opts, w.rhoCx, w.rhoCy, w.rhoCz)


def test_certified_solve_along_a_3d_trajectory():
    """The staged layout's solve along the 3D updraft: every solve within
    1e-12 of the oracle's bisection, about 1.2 FP64 growth evaluations per
    solve, most settled by a certified Newton step; and the staged rounds
    give the same results bit for bit."""
    hostcheck.build()
    n = worst = evals = certified = 0
    cls = dict(polish=0, euler=0, tiny=0, exact=0, deferred_ends=0)
    for q, args in enumerate(trajectory_3d()):
        ref = oracle.solve_batch(*args)
        got, c = hostcheck.solve(*args, solver=3)
        rel = np.abs(got - ref) / ref
        assert (rel <= 1e-12).all(), f"{(rel > 1e-12).sum()} solves differ by more than 1e-12; worst {rel.max():.3e}"
        n += len(ref)
        worst = max(worst, rel.max())
        evals += c["evals"]
        certified += c["certified"]
        if q % 5 == 0:
            assert np.array_equal(got, hostcheck.solve(*args, solver=4)[0])
        for key, v in hostcheck.staged_stats(*args).items():
            cls[key] += v
    print(f"3D: {n} solves, worst relative difference {worst:.2e}, {evals / n:.3f} FP64 growth evaluations per "
          f"solve, {certified / n:.1%} certified settles")
    m = sum(cls[key] for key in ("polish", "euler", "tiny", "exact"))
    print("start classes:", {key: f"{v / m:.2%}" for key, v in cls.items()})
    assert n > 1_000_000
    assert evals / n < 1.5
    assert certified > n // 2
    assert cls["polish"] > 0.6 * m and 0.1 * m < cls["exact"] < 0.4 * m  # most solves start from the FP32 locate
    assert 0 < cls["deferred_ends"] < 0.02 * m  # the deferred bracket ends are rare


def test_host_bisection_is_the_oracle_bisection(states):
    """The library's bisection and the oracle's take the same halvings: equal
    to rounding of the growth rate's terms (the library's thermodynamics
    order some products differently)."""
    for args in states[::6]:
        ref = oracle.solve_batch(*args)
        got, _ = hostcheck.solve(*args, solver=0)
        np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_fp32_growth_error_bound_holds(states):
    """The FP32 growth rate's error bound covers its actual error against
    the FP64 growth rate at every super-droplet's r_w^2, and at points
    across each one's bracket [x0 - 2 dt' |g0|, x0 + 2 dt' |g0|], where the
    fast solve takes its FP32 sign decisions."""
    rng = np.random.default_rng(0)
    n = 0
    for x0, rd3, kappa, cell, th, rv, rhod, dtp in states[::3]:
        _, _, g0 = hostcheck.growth(x0, rd3, kappa, cell, th, rv, rhod)
        for frac in (0.0, -1.0, -0.5, 0.5, 1.0, None):
            u = rng.uniform(-1.0, 1.0, len(x0)) if frac is None else frac
            x = np.maximum(x0 + u * 2.0 * dtp * np.abs(g0), np.cbrt(rd3) ** 2 * (1 + 1e-6))
            g32, e32, g64 = hostcheck.growth(x, rd3, kappa, cell, th, rv, rhod)
            # the bound is taken on the FP32 value of x: compare with FP64 there
            _, _, g64f = hostcheck.growth(x.astype(np.float32).astype(np.float64), rd3, kappa, cell, th, rv, rhod)
            err = np.abs(g32.astype(np.float64) - g64f)
            assert (err <= e32).all(), f"{(err > e32).sum()} of {len(x)} above the bound"
            n += len(x)
    assert n > 1_000_000


def test_fp32_solve_of_the_mixed_mode_away_from_activation(states):
    """The mixed mode's FP32 solve, on the droplets it is given (all but
    those near Koehler activation in near-saturated air: r_w^2 < 9 r_c^2,
    r_c^2 = 3 kappa r_d^3 / A), stays within a few FP32 ulps of r_w^2 of the
    bisection's root for 99 % of solves (median about 1e-8)."""
    for x0, rd3, kappa, cell, th, rv, rhod, dtp in states[::5]:
        t = [oracle.thermo(a, b, c) for a, b, c in zip(th, rv, rhod)]
        A = np.array([q.A for q in t])[cell]
        sat = np.array([q.rho_v_eff >= 0.99 * q.rho_vs for q in t])[cell]
        away = ~(sat & (x0 < 9.0 * 3.0 * kappa * rd3 / A))
        args = (x0[away], rd3[away], kappa[away], cell[away], th, rv, rhod, dtp)
        ref = oracle.solve_batch(*args)
        got, _ = hostcheck.solve(*args, solver=2)
        rel = np.abs(got - ref) / ref
        assert np.median(rel) < 1e-7 and np.percentile(rel, 99) < 5e-6 and rel.max() < 1e-3
