"""Small helpers that drive single oracle routines on hand-made states."""
import ctypes as C

import numpy as np

import oracle


def box_cfg(n_sd=4, kernel="golovin", b=1.0, dV=1.0, dt=1.0, seed=0):
    side = dV ** (1.0 / 3.0)
    return dict(nx=0, ny=0, nz=0, dx=side, dy=side, dz=side, dt=dt, sd_conc=n_sd, kernel=kernel,
                golovin_b=b, init_dist="exponential", exp_mean_volume=1e-15, exp_n0=1.0,
                modes=[], seed=seed, physics=1)


def make_state(N, rw2, rd3=None, kappa=None, uid=None, x=None, y=None, z=None):
    n = len(N)
    s = oracle.State(n)
    s.N[:] = np.asarray(N, np.uint64)
    s.rw2[:] = rw2
    s.rd3[:] = 0.0 if rd3 is None else rd3
    s.kappa[:] = 0.0 if kappa is None else kappa
    s.uid[:] = np.arange(n, dtype=np.uint64) if uid is None else np.asarray(uid, np.uint64)
    for f, v in (("x", x), ("y", y), ("z", z)):
        getattr(s, f)[:] = 0.0 if v is None else v
    return s


def coalesce(cfg, state, step=0, sstp=1, th=300.0, rv=0.01, rhod=1.0, multi=0):
    """One orc_coalesce call on ``state`` (modified in place); returns stats.
    ``multi`` turns on multiple coalescence for P > 1."""
    dom = oracle.make_domain(cfg)
    o = oracle.make_opts(dict(adve=0, sedi=0, cond=0, coal=1, sstp_coal=sstp, coal_multi=multi))
    nc = int(oracle.lib().orc_n_cells(C.byref(dom)))
    f = lambda v: np.full(nc, v, np.float64)
    TH, RV, RD = f(th), f(rv), f(rhod)
    st = oracle.Stats()
    s = state.struct()
    oracle.lib().orc_coalesce(C.byref(dom), C.byref(o), C.byref(s), oracle._dp(TH), oracle._dp(RV),
                              oracle._dp(RD), step, C.byref(st))
    return st


def condense(cfg, state, th, rv, rhod, sstp=10, RH_max=44.0):
    """One orc_condense call; th and rv arrays are updated in place."""
    dom = oracle.make_domain(cfg)
    o = oracle.make_opts(dict(adve=0, sedi=0, cond=1, coal=0, sstp_cond=sstp, RH_max=RH_max))
    st = oracle.Stats()
    s = state.struct()
    oracle.lib().orc_condense(C.byref(dom), C.byref(o), C.byref(s), oracle._dp(th), oracle._dp(rv),
                              oracle._dp(rhod), C.byref(st))
    return st


def transport(cfg, state, th, rv, rhod, rhoCx=None, rhoCy=None, rhoCz=None, adve=1, sedi=1):
    dom = oracle.make_domain(cfg)
    o = oracle.make_opts(dict(adve=adve, sedi=sedi, cond=0, coal=0))
    st = oracle.Stats()
    s = state.struct()
    oracle.lib().orc_transport(C.byref(dom), C.byref(o), C.byref(s), oracle._dp(th), oracle._dp(rv),
                               oracle._dp(rhod), oracle._dp(rhoCx), oracle._dp(rhoCy), oracle._dp(rhoCz),
                               C.byref(st))
    return st


def recycle(state):
    st = oracle.Stats()
    s = state.struct()
    oracle.lib().orc_recycle(C.byref(s), C.byref(st))
    return st


def golovin_run(arg):
    """One seed of the Golovin box (Shima et al. 2009 set-up) in the oracle:
    (N, r_w^2) at each listed time.  arg = (seed, times, coal_multi); a
    top-level function so that a spawn-started process pool can run seeds
    side by side."""
    import workloads
    seed, times, multi = arg
    w = workloads.golovin_box(seed=seed)
    o = oracle.Oracle(w.cfg)
    o.init(w.th, w.rv, w.rhod)
    opts = dict(w.opts, coal_multi=multi)
    out = {}
    for t in range(1, max(times) + 1):
        o.step_async(opts)
        if t in times:
            out[t] = (o.state.N.astype(float).copy(), o.state.rw2.copy(), o.stats.n_pgt1)
    return out
