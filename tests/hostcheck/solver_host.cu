// Host build of the CUDA library's condensation solvers (the kernels'
// own source, compiled for the CPU) for CPU tests of their logic: the
// fast solve's FP32 sign decisions, its polish and its replay against the
// bisection of the paper's procedure (Sec. 5.1.3, eq. rw2_implicit), solve
// by solve, along oracle trajectories.  Test infrastructure: nothing in the
// library loads it.
#include "../../paper_1310_1905_gb300/csrc/k_cond.cu"

using namespace sdm;

namespace {
Thermo cell_thermo(int64_t c, const double *th, const double *rv, const double *rhod, double RH_max) {
    return thermo_eval_f<true>(th[c], rv[c], rhod[c], RH_max, rhod_factor(rhod[c]));
}
}  // namespace

// solver: 0 the bisection (SDM_SOLVER_BISECT), 1 the fast solve
// (SDM_SOLVER_FAST), 2 the FP32 solve of the mixed mode, 3 the fast solve
// with certified Newton steps (the staged layout's), 4 the staged layout's
// sequence of rounds itself: its start (fs_start), then one cs_step per
// round as the eval kernels take them, with the rare bracket ends deferred
// to a round of their own.  counters: Euler steps, exact-bisection
// fallbacks, FP64 growth evaluations, certified settles.
extern "C" void hc_solve(int64_t n, const double *x0, const double *rd3, const double *kappa, const int64_t *cell,
                         const double *th, const double *rv, const double *rhod, double RH_max, double dtp,
                         int physics, int solver, double *x1, int64_t *counters) {
    SolveCounters cnt{0, 0, 0, 0};
    for (int64_t q = 0; q < n; ++q) {
        const Thermo t = cell_thermo(cell[q], th, rv, rhod, RH_max);
        const ThermoF tf = to_float(t);
        if (solver == 0) {
            int eu = 0;
            x1[q] = solve_rw2_bisect(x0[q], rd3[q], kappa[q], t, dtp, physics, &eu);
            cnt.euler += eu;
        } else if (solver == 1) {
            x1[q] = solve_rw2_fast<false>(x0[q], rd3[q], kappa[q], t, tf, dtp, physics, cnt);
        } else if (solver == 3) {
            x1[q] = solve_rw2_fast<true>(x0[q], rd3[q], kappa[q], t, tf, dtp, physics, cnt);
        } else if (solver == 4) {
            FastSolve S;
            S.x0 = x0[q];
            S.rd3 = rd3[q];
            S.kappa = kappa[q];
            int task = cs_task_of(fs_start<true>(S, tf, dtp, physics));
            bool done = false;
            for (int k = 0; k < kStagedRounds && !done; ++k) done = cs_step(task, S, t, tf, dtp, physics, cnt);
            x1[q] = done ? S.x1 : -1.0;
        } else {
            solve_rw2_f32(x0[q], rd3[q], kappa[q], tf, (float)dtp, physics, &x1[q], cnt);
        }
    }
    counters[0] = cnt.euler;
    counters[1] = cnt.fallback;
    counters[2] = cnt.evals;
    counters[3] = cnt.certified;
}

// The staged sequence's statistics: stats[0..3] the start classes
// (kStartPolish, kStartEuler, kStartTiny, kStartExact), stats[4] the
// records whose bracket end waited for a round of its own (kTaskG0End).
extern "C" void hc_staged_stats(int64_t n, const double *x0, const double *rd3, const double *kappa,
                                const int64_t *cell, const double *th, const double *rv, const double *rhod,
                                double RH_max, double dtp, int physics, int64_t *stats) {
    for (int k = 0; k < 5; ++k) stats[k] = 0;
    for (int64_t q = 0; q < n; ++q) {
        const Thermo t = cell_thermo(cell[q], th, rv, rhod, RH_max);
        const ThermoF tf = to_float(t);
        SolveCounters cnt{0, 0, 0, 0};
        FastSolve S;
        S.x0 = x0[q];
        S.rd3 = rd3[q];
        S.kappa = kappa[q];
        const int st = fs_start<true>(S, tf, dtp, physics);
        stats[st]++;
        int task = cs_task_of(st);
        bool done = false;
        for (int k = 0; k < kStagedRounds && !done; ++k) {
            const int before = task;
            done = cs_step(task, S, t, tf, dtp, physics, cnt);
            if (task == kTaskG0End && before != kTaskG0End) stats[4]++;
        }
    }
}

// The FP32 growth rate with its error bound, and the FP64 one, at x.
extern "C" void hc_growth(int64_t n, const double *x, const double *rd3, const double *kappa, const int64_t *cell,
                          const double *th, const double *rv, const double *rhod, double RH_max, int physics,
                          float *g32, float *err32, double *g64) {
    for (int64_t q = 0; q < n; ++q) {
        const Thermo t = cell_thermo(cell[q], th, rv, rhod, RH_max);
        const ThermoF tf = to_float(t);
        const GF f = growth_f3<kDgNone>((float)x[q], (float)rd3[q], (float)kappa[q], tf, physics);
        g32[q] = f.g;
        err32[q] = f.err;
        g64[q] = growth(x[q], rd3[q], kappa[q], t, physics);
    }
}
