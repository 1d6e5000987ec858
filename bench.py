"""Benchmark of the super-droplet hot path (one full timestep = step_sync
with sstp_cond condensation substeps + step_async with recycling,
advection, sedimentation, regrouping and sstp_coal coalescence substeps).

Default workload: the large 3D kinematic domain, 128 x 128 x 128 cells of
20 m, 32 super-droplets per cell (67 108 864), bimodal ammonium-sulphate
aerosol, uniform updraft of 1 m/s with per-column perturbations, geometric
kernel, dt = 1 s, 10/10 substeps, FP64 state.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload updraft_3d|icmw_2d|golovin_box|ensemble|serve]

Prints one JSON line.  Metric: super-droplet-steps per second over all
ranks.  ``value`` is device time (CUDA events on the library's stream, L2
flushed between timed steps, inputs resident in HBM); ``e2e`` is the same
metric through the public API with host buffers (theta and r_v copied in and
out every step), wall clock.  Multi-GPU runs are independent replicas (one
domain per rank, weak scaling).

``--impl reference`` times the CPU oracle (serial and cell-parallel OpenMP
builds of the same source) on a bounded sample of the same workload, the way
the paper times its back-ends (Sec. 6): whole runs of a short and a long
step count, each the shortest of three, per step = (long - short) / (steps
between them).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "super-droplet-steps/s (coal+cond)"
UNIT = "SD-steps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 arithmetic of one SM per clock on this part: 1.25 TFLOP/s nominal at
# the 2070 MHz boost clock over 152 SMs is 2 DFMA (4 FP64 flops) per SM per
# clock; the bench also measures the throughput (sdm_probe_device) and takes
# that as the peak
FP64_FLOPS_PER_SM_CLK = 4.0
# Algorithmic FP64 work of the condensation solve per super-droplet and
# substep: about 4-6 evaluations of the growth rate of a safeguarded Newton
# solve at 60-100 flops each (an exponential and a few divisions included),
# 3-6 kflop per SD-step over 10 substeps; the midpoint, 450 flops per
# SD-substep, is the per-unit figure the roofline line uses
COND_ALGO_FLOPS_PER_SD_SUBSTEP = 450.0
# Algorithmic HBM bytes per SD-step of the coalescence + condensation step:
# condensation reads N, r_w^2, r_d^3, kappa and writes r_w^2 (40 B);
# coalescence reads those and the id and writes N, r_w^2, r_d^3, kappa
# (68 B); the regrouping reads the cell and moves the state (116 B in 2D,
# 132 B in 3D)
HBM_BYTES_PER_SD_STEP = {"icmw_2d": 40 + 68 + 116, "updraft_3d": 40 + 68 + 132, "golovin_box": 68 + 116}
# ncu on the condensation call: the FP64 flops it executes (2 DFMA + DADD +
# DMUL) per SD-substep, its DRAM bytes read + written per call per
# super-droplet and the share of its cycles the FP64 pipe is busy, with the
# capture they come from, by workload, precision and layout.  "fused": one
# k_condense launch; "staged": the chain of k_cs_* launches of one call (10
# substeps), whose solve records travel through HBM between the launches.
# Mixed precision too is bound by its FP64 part (the solves near
# activation): its FP32 work is about 1 % of the FP32 peak.
COND_FP64 = {
    ("icmw_2d", "fp64", "fused"): dict(kernel="k_condense", flops_per_sd_substep=649.85,
                                       dram_bytes_per_sd=11.835e6 / 360000, fp64_pipe_active=0.7175,
                                       capture="2D case, 360 000 SDs, one launch"),
    ("icmw_2d", "mixed", "fused"): dict(kernel="k_condense", flops_per_sd_substep=178.07,
                                        dram_bytes_per_sd=11.895e6 / 360000, fp64_pipe_active=0.5272,
                                        capture="2D case, 360 000 SDs, one launch"),
    ("updraft_3d", "fp64", "fused"): dict(kernel="k_condense", flops_per_sd_substep=667.07,
                                          dram_bytes_per_sd=331.62e6 / 8388608, fp64_pipe_active=0.7364,
                                          capture="3D updraft at 64^3 cells (8.4 M SDs), one launch; traffic "
                                                  "scaled by the SDs of a launch"),
    ("icmw_2d", "fp64", "staged"): dict(kernel="condensation chain (k_cs_*)", flops_per_sd_substep=312.37,
                                        dram_bytes_per_sd=5060.9, fp64_pipe_active=0.381,
                                        capture="2D case, 360 000 SDs, one call (81 launches)"),
    ("updraft_3d", "fp64", "staged"): dict(kernel="condensation chain (k_cs_*)", flops_per_sd_substep=301.30,
                                           dram_bytes_per_sd=6609.1, fp64_pipe_active=0.584,
                                           capture="3D updraft, 32x32x128 columns (4.2 M SDs), one call (81 "
                                                   "launches); traffic scaled by the SDs of a call"),
}
# the library's own choice of layout (cond_layout = auto): the staged chain
# for the FP64 fast solve from 2^17 super-droplets
STAGED_MIN_SD = 1 << 17


def cond_layout_of(args, n_sd: int) -> str:
    if args.precision != "fp64" or args.cond_layout == "fused":
        return "fused"
    return "staged" if args.cond_layout == "staged" or n_sd >= STAGED_MIN_SD else "fused"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="updraft_3d", choices=["icmw_2d", "updraft_3d", "golovin_box", "ensemble", "serve"])
    ap.add_argument("--members", type=int, default=256)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cells", type=int, default=128, help="updraft_3d: cells per dimension")
    ap.add_argument("--nz", type=int, default=None,
                    help="updraft_3d: levels, when they differ from --cells (a profile of fewer columns of the "
                         "full-height domain)")
    ap.add_argument("--probe-seconds", type=float, default=2.0,
                    help="length of the sustained FP64 throughput probe before the workload (shorter for profiling "
                         "runs, whose launch lists would otherwise hold its launches)")
    ap.add_argument("--cond-layout", default="auto", choices=["auto", "fused", "staged"],
                    help="condensation kernels: fused, staged, or chosen by domain size")
    ap.add_argument("--profile-one-step", action="store_true",
                    help="ensemble: bracket one graph-replayed step after the warm-up with cudaProfilerStart/Stop "
                         "(for an ncu kernel list taken with --profile-from-start off)")
    ap.add_argument("--serve-requests", type=int, default=500, help="serve: requests per window")
    ap.add_argument("--serve-scale", type=float, default=1.0 / 6.0,
                    help="serve: factor on the 300-1800 steps of a request")
    ap.add_argument("--serve-sample", type=int, default=24,
                    help="serve: requests solved alone to fit the sequential service time")
    ap.add_argument("--diag", action="store_true",
                    help="also run the diagnostics after every step (moments k = 0..3 and a 64-bin spectrum of "
                         "the wet radius), as an output step of a model would; off for the headline number")
    return ap.parse_args()


def make_workload(name: str, seed: int, cells: int = 128, cond_layout: str = "auto", nz: int | None = None):
    if name == "icmw_2d":
        w = workloads.icmw_2d(seed=seed)
    elif name == "updraft_3d":
        w = workloads.updraft_3d(nx=cells, ny=cells, nz=nz or cells, seed=seed)
    else:
        w = workloads.golovin_box(seed=seed)
    w.cfg["cond_layout"] = cond_layout
    return w


def workload_desc(w) -> dict:
    c = w.cfg
    d = dict(workload=f"{w.name}: {c['nx']}x{c['ny']}x{c['nz']} cells, {c['sd_conc']} SD/cell "
                      f"({w.n_sd} SDs), sstp_cond={w.opts['sstp_cond']}, sstp_coal={w.opts['sstp_coal']}, "
                      f"kernel={c['kernel']}, dt={c['dt']} s"
                      + (", theta and r_v transported by the eddy and relaxed (Eulerian stand-in)"
                         if w.name == "icmw_2d" else
                         ", theta and r_v transported by the updraft (Eulerian stand-in)" if w.name == "updraft_3d"
                         else ""),
             n_sd=w.n_sd, n_cells=w.n_cells, sd_per_cell=c["sd_conc"], processes="cond+adve+sedi+coal",
             l2="flushed (256 MiB write) before every timed step")
    return d


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm
def run_gpu(args, rank: int, world: int):
    import torch

    from paper_1310_1905_gb300 import sdm

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    w = make_workload(args.workload, seed=rank, cells=args.cells, cond_layout=args.cond_layout, nz=args.nz)
    opts = w.opts
    if args.workload == "golovin_box":
        opts = dict(w.opts)
    th = torch.tensor(w.th, dtype=torch.float64, device="cuda")
    rv = torch.tensor(w.rv, dtype=torch.float64, device="cuda")
    rhod = torch.tensor(w.rhod, dtype=torch.float64, device="cuda")
    Cs = [None if a is None else torch.tensor(a, dtype=torch.float64, device="cuda")
          for a in (w.rhoCx, w.rhoCy, w.rhoCz)]
    device = sdm.sdm_probe_device(args.probe_seconds)  # SM count and FP64 throughput, before the workload
    p = sdm.Particles(w.cfg, th, rv, rhod, *Cs, stream=stream.cuda_stream, precision=args.precision)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    edges = np.geomspace(1e-9, 1e-2, 65)
    spec = torch.empty((64, p.n_cells), dtype=torch.float64, device="cuda") if args.diag else None
    mom = torch.empty(p.n_cells, dtype=torch.float64, device="cuda") if args.diag else None
    # the kinematic framework's Eulerian component (the driver's part, the
    # paper's MPDATA) before every step, outside the timed step: theta and
    # r_v transported by the flow; in the 2D case also relaxed to their
    # initial level means (its set-up's forcing)
    euler = args.workload in ("icmw_2d", "updraft_3d")
    relax = args.workload == "icmw_2d"
    axes = tuple(range(np.ndim(w.th) - 1))
    th0, rv0 = (w.th.mean(axis=axes), w.rv.mean(axis=axes)) if relax else (None, None)

    def euler_step():
        if euler:
            p.euler_step(th, rv, Cs[0], Cs[1], Cs[2], th0, rv0)

    def step():
        if opts.get("cond", 1):
            p.step_sync(opts, th, rv)
        p.step_async(opts)
        p.wait()
        if args.diag:
            sdm.sdm_diag_rng(p.ctx, True, 0.0, 1.0)
            for k in range(4):
                sdm.sdm_diag_mom(p.ctx, k)
                sdm.sdm_outbuf(p.ctx, mom)
            sdm.sdm_diag_spectrum(p.ctx, True, edges, 3, spec)

    for _ in range(args.warmup):
        euler_step()
        step()
    torch.cuda.synchronize()
    dist_barrier(world)
    sdm.sdm_timing_enable(p.ctx, True)
    sdm.sdm_get_timing(p.ctx, reset=True)
    clocks = ClockSampler(dev)
    clocks.start()
    t_dev = 0.0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        euler_step()
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_dev = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    tim = sdm.sdm_get_timing(p.ctx, reset=True)
    sdm.sdm_timing_enable(p.ctx, False)
    t_max = dist_max(t_dev, world)
    stats = p.stats()
    res = dict(t_dev=t_max, timing=tim, clocks=clk, stats=stats, n_sd=p.n_sd, w=w, device=device)
    # ---- e2e through the public API with host buffers
    if not args.no_e2e:
        th_h, rv_h = w.th.copy(), w.rv.copy()
        rhod_h = w.rhod
        q = sdm.Particles(w.cfg, th_h, rv_h, rhod_h, w.rhoCx, w.rhoCy, w.rhoCz, precision=args.precision)
        th_pin = torch.from_numpy(th_h).pin_memory().numpy()
        rv_pin = torch.from_numpy(rv_h).pin_memory().numpy()

        def host_step():
            if opts.get("cond", 1):
                q.step_sync(opts, th_pin, rv_pin)
            q.step_async(opts)
            return q.wait()

        def host_euler():
            if euler:
                q.euler_step(th_pin, rv_pin, w.rhoCx, w.rhoCy, w.rhoCz, th0, rv0)

        for _ in range(args.warmup):
            host_euler()
            host_step()
        dist_barrier(world)
        t_e2e = 0.0
        for _ in range(args.steps):
            host_euler()  # the driver's part, outside the timed step like on the device
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            host_step()
            t_e2e += time.perf_counter() - t0
        res["t_e2e"] = dist_max(t_e2e, world)
        nbytes = w.th.size * 8
        res["h2d"] = (2 * nbytes) if opts.get("cond", 1) else 0
        res["d2h"] = (2 * nbytes if opts.get("cond", 1) else 0) + 96  # fields + the 96-byte stats record of the wait
        q.close()
    p.close()
    return res


def run_ensemble(args, rank: int, world: int) -> dict:
    """Batched ensemble (256 ragged 0D members, mixed precision by default):
    one graph-captured step for all members, against the same members
    stepped one after another as single-member solves."""
    import torch

    from paper_1310_1905_gb300.ensemble import Ensemble

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    members = workloads.ensemble_members(args.members, seed=rank)
    opts = dict(adve=0, sedi=0, cond=1, coal=1, RH_max=44.0, sstp_cond=10, sstp_coal=10)
    n_sd = sum(m["n_sd"] for m in members)
    prec = args.precision if args.precision != "fp64" else "mixed"
    ens = Ensemble(precision=prec, max_sd=n_sd + 1024, max_members=len(members))
    ids = [ens.add(m) for m in members]
    tile, thr, pth = ens.autotune(opts)
    ens.use_graph(True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    t = [0.0]

    def step(e, idmap):
        r = workloads.parcel_rhod(members, t[0] + 1.0)
        e.step(opts, rhod={idmap[k]: v for k, v in r.items() if k in idmap})
        e.wait()

    idmap = dict(enumerate(ids))
    for _ in range(args.warmup):
        step(ens, idmap)
        t[0] += 1.0
    torch.cuda.synchronize()
    if args.profile_one_step:
        torch.cuda.cudart().cudaProfilerStart()
        step(ens, idmap)
        t[0] += 1.0
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
    dist_barrier(world)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", 0)))
    clocks.start()
    t_tot = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(ens, idmap)
        t_tot += time.perf_counter() - t0
        t[0] += 1.0
    clk = clocks.stop()
    stats = ens.stats()
    ens.close()
    # sequential plain solves: every member its own one-member ensemble
    solo = []
    for k, m in enumerate(members):
        e = Ensemble(precision=prec, max_sd=m["n_sd"], max_members=1)
        solo.append((e, {k: e.add(m)}))
    seq_steps = max(1, min(3, args.steps))
    for e, im in solo:
        step(e, im)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(seq_steps):
        for e, im in solo:
            step(e, im)
    t_seq = time.perf_counter() - t0
    for e, _ in solo:
        e.close()
    return dict(t=dist_max(t_tot, world), n_sd=n_sd, steps=args.steps, clocks=clk, tile=(tile, thr, pth),
                seq_value=n_sd * seq_steps / t_seq, stats=stats, precision=prec, members=len(members))


def run_serve(args, rank: int) -> dict:
    """Served stream: Poisson arrivals of parcel/box requests, N_sd
    log-uniform in [1e3, 2e6], w in [0.1, 5] m/s, mixed precision, 500
    requests per window (--serve-requests), step counts 300-1800 scaled by
    --serve-scale (1/6 by default: 50-300 steps, so that a window takes a
    few minutes), served at the offered rate (200 req/s, above capacity)
    and at half the measured capacity.  Beside it, the same requests as
    sequential plain solves: a sample of them solved one by one, each alone
    on the GPU, gives the service time t = a steps + b n_sd steps, and a
    first-come-first-served single server on the same arrival times gives
    their latencies."""
    import torch

    from paper_1310_1905_gb300.ensemble import Ensemble
    from paper_1310_1905_gb300.serve import Server, poisson_requests

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.5)
    prec = args.precision if args.precision != "fp64" else "mixed"
    opts = dict(adve=0, sedi=0, cond=1, coal=1, RH_max=44.0, sstp_cond=10, sstp_coal=10)

    def rhod_fn(m, t):
        return float(workloads.hydrostatic_rhod(np.array([m["z0"] + m["w"] * t]), 289.0, 7.5e-3, 101500.0)[0])

    n_req = args.serve_requests
    lo, hi = max(1, round(300 * args.serve_scale)), max(1, round(1800 * args.serve_scale))
    members = workloads.ensemble_members(n_req, seed=100 + rank, n_min=1e3, n_max=2e6, parcel_fraction=0.8)
    out, arrivals = {}, {}
    cap = None
    for label, rate in (("offered_200_per_s", 200.0), ("half_capacity", None)):
        if rate is None:
            mean_work = np.mean([m["n_sd"] for m in members]) * 0.5 * (lo + hi)
            rate = 0.5 * cap / mean_work
        reqs = poisson_requests(members, rate, (lo, hi), seed=7, rhod_fn=rhod_fn)
        arrivals[label] = [(r.arrival, r.member["n_sd"], r.steps) for r in reqs]
        srv = Server(mem_budget_bytes=budget, precision=prec, opts=opts)
        st = srv.run(reqs)
        srv.close()
        st["rate_per_s"] = rate
        out[label] = st
        if cap is None:
            cap = st["sd_steps_per_s"]
    # sequential plain solves: service times of a sample, each request alone
    rng = np.random.default_rng(3)
    reqs = poisson_requests(members, 200.0, (lo, hi), seed=7, rhod_fn=rhod_fn)
    order = np.argsort([r.member["n_sd"] for r in reqs])
    sample = [reqs[int(i)] for i in order[np.linspace(0, len(order) - 1, args.serve_sample).astype(int)]]
    rows = []
    for k, r in enumerate([sample[0]] + sample):  # the first, untimed: module loading and graph capture
        e = Ensemble(precision=prec, max_sd=r.member["n_sd"], max_members=1)
        mid = e.add(r.member)
        e.use_graph(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(r.steps):
            e.step(opts, rhod={mid: r.rhod_of_t(k + 1.0)} if r.rhod_of_t else None)
            e.wait()
        if k > 0:
            rows.append((r.steps, r.member["n_sd"] * r.steps, time.perf_counter() - t0))
        e.close()
    # t = a steps + b SD-steps, least squares in relative error (rows / t)
    A = np.array([[s_, w_] for s_, w_, _ in rows], float)
    tt = np.array([t for *_, t in rows])
    coef, *_ = np.linalg.lstsq(A / tt[:, None], np.ones_like(tt), rcond=None)
    rel = np.abs(A @ coef - tt) / tt
    fit_err = dict(median=float(np.median(rel)), worst=float(rel.max()))
    seq = {}
    for label, arr in arrivals.items():
        t_free, lat, work = 0.0, [], 0.0
        for t_arr, n_sd, steps in arr:
            start = max(t_arr, t_free)
            t_free = start + coef[0] * steps + coef[1] * n_sd * steps
            lat.append(t_free - t_arr)
            work += n_sd * steps
        seq[label] = dict(p50_latency_s=float(np.percentile(lat, 50)), p99_latency_s=float(np.percentile(lat, 99)),
                          sd_steps_per_s=work / t_free)
    return dict(out=out, n_req=n_req, budget=budget, steps=(lo, hi), seq=seq, precision=prec,
                seq_model=dict(a_s_per_step=float(coef[0]), b_s_per_sd_step=float(coef[1]), samples=len(rows),
                               fit_rel_err=fit_err))


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(v, world):
    """The maximum of v over the ranks (the slowest rank's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(n_sd_per_rank: int, steps: int, world: int, t_max: float) -> float:
    """SD-steps/s of the whole job: every rank runs its own replica of the
    workload (seeded by its rank) for the same steps, and the job takes as
    long as its slowest rank."""
    return n_sd_per_rank * steps * world / t_max


# ---------------------------------------------------------------- oracle timing
def oracle_sample_workload(name: str, seed: int = 0, cells: int = 128):
    """A bounded sample of the workload for the CPU oracle: the 3D domain's
    full columns on a 2 x 2 horizontal patch (2 x 2 x 128 cells of 32 SDs;
    the flow has no horizontal component, so its columns are independent),
    4 of the 2D case's 75 columns, or the whole one-cell box."""
    if name == "updraft_3d":
        return workloads.updraft_3d(nx=2, ny=2, nz=cells, seed=seed)
    if name == "icmw_2d":
        return workloads.icmw_2d(nx=4, seed=seed)
    return workloads.golovin_box(seed=seed)


def oracle_timing(name: str, k_short: int, k_long: int, omp: bool, repeats: int = 3, cells: int = 128) -> dict:
    """The oracle as it stands, timed as the paper times its back-ends
    (Sec. 6): whole runs (initialisation + steps) of k_short and of k_long
    steps, each the shortest of ``repeats``, and per step
    (long - short) / (k_long - k_short), which cancels the initialisation.
    The Eulerian step of the kinematic driver runs between the steps, as on
    the GPU, and is left out of the run times."""
    import oracle
    w = oracle_sample_workload(name, cells=cells)
    threads = oracle.threads(0, omp=omp)
    relax = w.name == "icmw_2d"
    axes = tuple(range(np.ndim(w.th) - 1))
    th0, rv0 = (w.th.mean(axis=axes), w.rv.mean(axis=axes)) if relax else (None, None)

    def run(k):
        o = oracle.Oracle(w.cfg, omp=omp)
        t0 = time.perf_counter()
        o.init(w.th, w.rv, w.rhod)
        t = time.perf_counter() - t0
        for _ in range(k):
            if w.name != "golovin_box":
                o.euler_step(w.rhoCx, w.rhoCy, w.rhoCz, th0, rv0)
            t0 = time.perf_counter()
            if w.opts.get("cond", 1):
                o.step_sync(w.opts)
            o.step_async(w.opts, w.rhoCx, w.rhoCy, w.rhoCz)
            t += time.perf_counter() - t0
        return t

    t_short = min(run(k_short) for _ in range(repeats))
    t_long = min(run(k_long) for _ in range(repeats))
    per_step = max(t_long - t_short, 1e-9) / (k_long - k_short)
    return dict(value=w.n_sd / per_step, ms_per_step=per_step * 1e3, n_sd=w.n_sd, threads=threads,
                t_short=t_short, t_long=t_long, k_short=k_short, k_long=k_long, repeats=repeats,
                sample=f"{w.name}: {w.cfg['nx']}x{w.cfg['ny']}x{w.cfg['nz']} cells x {w.cfg['sd_conc']} SD "
                       f"({w.n_sd} SDs) of the same workload")


def host_cpu() -> dict:
    model = platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
    except Exception:
        pass
    return dict(nproc=os.cpu_count(), model=model, arch=platform.machine())


def cpu_baseline(name: str, k_short: int, k_long: int, cells: int = 128) -> dict:
    """Serial and cell-parallel oracle on the same sample; the OpenMP figure
    (all host cores) is the line's value, the serial one rides along."""
    par = oracle_timing(name, k_short, k_long, omp=True, cells=cells)
    ser = oracle_timing(name, k_short, k_long, omp=False, cells=cells)
    how = (f"shortest of {par['repeats']} whole runs of {k_short} and of {k_long} steps from initialisation, "
           f"per step = (long - short)/{k_long - k_short}")
    return dict(value=par["value"], unit=UNIT, cores=par["threads"], kind="oracle",
                sample=f"{par['sample']}; {how}; OpenMP cell-parallel build, {par['threads']} threads",
                ms_per_step=par["ms_per_step"], host=host_cpu(),
                serial=dict(value=ser["value"], unit=UNIT, cores=1, ms_per_step=ser["ms_per_step"],
                            sample=f"{ser['sample']}; {how}; serial build"))


def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")

    if args.impl == "reference":
        if rank == 0:
            name = args.workload if args.workload in ("updraft_3d", "icmw_2d", "golovin_box") else "updraft_3d"
            k_short = max(1, args.warmup)
            cb = cpu_baseline(name, k_short, k_short + max(1, args.steps), cells=args.cells)
            line = dict(impl="reference", metric=METRIC, value=cb["value"], unit=UNIT, n_gpus=args.gpus,
                        steps=args.steps, warmup=args.warmup, ms_per_step=cb["ms_per_step"], higher_is_better=True,
                        scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                        config=dict(workload=cb["sample"].split(";")[0], of=workload_desc(
                            make_workload(name, 0, args.cells))["workload"],
                            note="a bounded sample of the workload, normalised per SD-step (the cost is linear "
                                 "in the super-droplets, Sec. 6); ms_per_step is the sample's own"),
                        cpu_baseline=cb,
                        e2e=dict(value=cb["value"], unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    if args.workload == "serve":
        r = run_serve(args, rank)
        if rank == 0:
            sat = r["out"]["offered_200_per_s"]
            lo, hi = r["steps"]
            line = dict(metric=METRIC, value=sat["sd_steps_per_s"], unit=UNIT, n_gpus=world, steps=sat["steps"],
                        warmup=0, ms_per_step=sat["wall_s"] / max(1, sat["steps"]) * 1e3, higher_is_better=True,
                        scaling="weak", vs_baseline=None, dtype="f64/f32", data="synthetic",
                        config=dict(workload=f"served stream: {r['n_req']} Poisson requests per window, parcels "
                                             f"(80 %, w in [0.1, 5] m/s) and boxes, N_sd log-uniform in "
                                             f"[1e3, 2e6], {lo}-{hi} steps (300-1800 x {args.serve_scale:.4g}), "
                                             f"{r['precision']} precision, arena of {sat['arena_sd']} SDs "
                                             f"({sat['arena_bytes'] / 1e9:.1f} GB reserved, "
                                             f"{sat['bytes_per_sd']:.1f} B/SD)"),
                        latency={k: dict(p50_s=v["p50_latency_s"], p99_s=v["p99_latency_s"],
                                         rate_per_s=v["rate_per_s"], sd_steps_per_s=v["sd_steps_per_s"],
                                         mean_queue_wait_s=v["mean_queue_wait_s"], served=v["served"],
                                         peak_resident_sd=v["peak_resident_sd"], wall_s=v["wall_s"])
                                 for k, v in r["out"].items()},
                        sequential=dict(latency=r["seq"], model=r["seq_model"],
                                        how="each sampled request solved alone (one-member graph-replayed "
                                            "ensemble, its own steps), t = a steps + b SD-steps fitted, then a "
                                            "first-come-first-served single server on the same arrivals"),
                        timing="host wall clock over the whole window")
            print(json.dumps(line), flush=True)
        return
    if args.workload == "ensemble":
        r = run_ensemble(args, rank, world)
        if rank == 0:
            v = r["n_sd"] * r["steps"] * world / r["t"]
            line = dict(metric=METRIC, value=v, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                        ms_per_step=r["t"] / args.steps * 1e3, higher_is_better=True, scaling="weak",
                        vs_baseline=None, dtype="f64/f32" if r["precision"] == "mixed" else "f64",
                        data="synthetic",
                        config=dict(workload=f"ensemble: {r['members']} ragged 0D box/parcel members, N_sd "
                                             f"log-uniform in [1e3, 1e6] ({r['n_sd']} SDs), {r['precision']} "
                                             f"precision, graph-captured step, autotuned tile {r['tile']}",
                                    n_sd=r["n_sd"], l2="flushed before every timed step"),
                        clocks=r["clocks"], timing="host wall clock around step + wait (graph replay)",
                        sequential=dict(value=r["seq_value"], unit=UNIT,
                                        how="the same members, one single-member solve after another"),
                        speedup_vs_sequential=v / r["seq_value"])
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    res = run_gpu(args, rank, world)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    w = res["w"]
    total_sd_steps = res["n_sd"] * args.steps * world
    value = whole_job_value(res["n_sd"], args.steps, world, res["t_dev"])
    tim = res["timing"]
    pk = peaks()
    # dominant kernel: condensation, bound by FP64 arithmetic, one call of
    # it (one k_condense launch, or the staged chain of k_cs_* launches)
    # timed with CUDA events on the context's stream.  achieved = the
    # algorithmic FP64 flops of the solve per SD-substep x the SD-substeps
    # of one call / the call's time; peak = the FP64 FMA throughput
    # measured on this device (sustained: one call runs for most of a step)
    cond_ms = tim["cond_ms"] / max(1, tim["cond_launches"])
    clk = res["clocks"]
    dev = res["device"]
    sm_mhz = clk.get("sm_mhz") or pk.get("clocks_under_load", {}).get("sm_mhz_median") or 2070.0
    fp64_derived = FP64_FLOPS_PER_SM_CLK * dev["n_sm"] * sm_mhz * 1e6 / 1e12  # TFLOP/s at the sampled clock
    fp64_peak = dev["fp64_tflops_sustained"] or dev["fp64_tflops_burst"]
    units = res["n_sd"] * w.opts["sstp_cond"]
    hbm = pk.get("hbm_gbs", 6800.0)
    hbm_src = "of measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in pk else "of fallback 6800 GB/s"
    layout = cond_layout_of(args, res["n_sd"])
    if tim["cond_launches"] > 0:
        k = COND_FP64.get((args.workload, args.precision, layout))
        achieved = COND_ALGO_FLOPS_PER_SD_SUBSTEP * units / (cond_ms * 1e-3) / 1e12
        roof = dict(kernel=k["kernel"] if k else ("condensation chain (k_cs_*)" if layout == "staged"
                                                  else "k_condense"),
                    layout=layout, bound="alu", achieved=achieved, peak=fp64_peak, unit="TFLOP/s",
                    frac=achieved / fp64_peak, traffic=k["dram_bytes_per_sd"] * res["n_sd"] if k else None,
                    algorithmic_flops_per_sd_substep=COND_ALGO_FLOPS_PER_SD_SUBSTEP,
                    launch_ms=cond_ms, sd_substeps_per_launch=units,
                    peak_source="of measured: FP64 FMA chains on this device (sdm_probe_device), sustained "
                                f"{dev['fp64_tflops_sustained']:.3f}, burst {dev['fp64_tflops_burst']:.3f} TFLOP/s",
                    derived_peak=dict(value=fp64_derived, how=f"4 FP64 flop/SM/clk x {dev['n_sm']} SMs (device "
                                                              f"query) x {sm_mhz:.0f} MHz (sampled)"))
        if k:
            executed = k["flops_per_sd_substep"] * units / (cond_ms * 1e-3) / 1e12
            roof["executed"] = dict(flops_per_sd_substep=k["flops_per_sd_substep"], achieved=executed,
                                    frac=executed / fp64_peak, fp64_pipe_active=k["fp64_pipe_active"],
                                    counters=k["capture"])
    else:  # no condensation (the Golovin box): coalescence, 68 B per SD-step (read 36, write 32)
        coal_ms = tim["coal_ms"] / max(1, tim["coal_launches"])
        achieved = 68.0 * res["n_sd"] / (coal_ms * 1e-3) / 1e9
        roof = dict(kernel="k_coal", bound="hbm", achieved=achieved, peak=hbm, unit="GB/s", frac=achieved / hbm,
                    traffic=None, note="one cell of 8192 SDs: latency-bound, the state stays in L2",
                    peak_source=hbm_src)
    bps = HBM_BYTES_PER_SD_STEP.get(args.workload)
    hbm_cc = None
    if bps:
        gbs = bps * value / world / 1e9
        hbm_cc = dict(bytes_per_sd_step=bps, achieved=gbs, peak=hbm, unit="GB/s", frac=gbs / hbm,
                      peak_source=hbm_src,
                      what="algorithmic HBM bytes of the coal+cond step (condensation 40, coalescence 68, "
                           "regrouping) x SD-steps/s of one GPU")
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=res["t_dev"] / args.steps * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64" if args.precision == "fp64" else "f64/f32",
                data="synthetic", config=workload_desc(w), roofline=roof, hbm_coal_cond=hbm_cc, clocks=clk,
                device=dict(n_sm=dev["n_sm"], fp64_tflops_burst=dev["fp64_tflops_burst"],
                            fp64_tflops_sustained=dev["fp64_tflops_sustained"]),
                gpu_launches=int(tim["launches"]),
                phases_ms_per_step={k[:-3]: tim[k] / args.steps for k in tim
                                    if k.endswith("_ms") and k != "euler_ms"})
    if tim["euler_launches"]:
        line["driver"] = dict(euler_ms_per_step=tim["euler_ms"] / args.steps,
                              euler_launches=int(tim["euler_launches"]),
                              what="the kinematic framework's Eulerian component (donor-cell transport of theta "
                                   "and r_v; in 2D also the relaxation of the level means) before every step, "
                                   "outside the timed step and its launch count")
    if "t_e2e" in res:
        line["e2e"] = dict(value=total_sd_steps / res["t_e2e"], unit=UNIT, h2d_bytes_per_step=res["h2d"],
                           d2h_bytes_per_step=res["d2h"])
    if not args.no_cpu:
        try:
            line["cpu_baseline"] = cpu_baseline(args.workload, 1, 4, cells=args.cells)
        except Exception as e:  # the oracle is a baseline, never a fallback
            line["cpu_baseline"] = dict(value=None, unit=UNIT, cores=None, kind="oracle", sample=f"failed: {e}")
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
