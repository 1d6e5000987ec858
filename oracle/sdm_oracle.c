/*
 * CPU oracle for the per-timestep hot path of the particle-based (super-
 * droplet) scheme of Arabas et al., "libcloudph++ 0.2", Sec. 5.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, __graft_entry__.smoke()
 * and bench.py's cpu_baseline / reference legs may load this library.  It is a
 * plain, serial, double-precision restatement of the paper, written to be read
 * against it: no blocking, no fusion, no reordering beyond what the equations
 * state.  Compiled with -ffp-contract=off so that every product is rounded as
 * written.
 *
 * Readings of passages that the paper leaves silent, ambiguous or garbled are
 * marked "READING" below; the CUDA library follows the same readings.
 *
 * Functions whose exact formula the paper only cites (transition-regime
 * factors, ventilation, terminal velocity, viscosity) are pinned against
 * other published forms (Seinfeld & Pandis's Fuchs-Sutugin arrangement,
 * Pruppacher & Klett's ventilation coefficient, tabulated air viscosity)
 * and, for the fall speed, against Stokes' law and Gunn & Kinzer's
 * measurements within 12 %: see orc_growth() and orc_vterm().
 *
 * The same source, compiled with -fopenmp, is the oracle's cell-parallel
 * timing variant (the paper's OpenMP back-end, Sec. 6): the "omp" pragmas
 * below split the loops over grid cells (cells are independent within
 * condensation and coalescence) and over super-droplets (terminal velocity,
 * advection) between threads.  Each cell keeps its own counters, merged
 * after the cell, so both builds give the same results bit for bit; without
 * -fopenmp the pragmas are ignored.
 */
#include "sdm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

/* ---- physical constants --------------------------------------------------
 * Printed in the paper's list of symbols (Appendix B): rho_w, sigma_w, c_pd,
 * c_pv, c_l, l_v0.  READING for the rest (not printed): R_d, R_v, the triple
 * point T0 and p_vs(T0), gravity, p1000 (Appendix A gives 1000 hPa), the
 * reference diffusivities D0, K0, STP = 20 C and 1013.25 hPa (Sec. 2.2), and
 * the Khvorostyanov-Curry (2002) drag constants delta0, C0.                 */
static const double rho_w = 1000.0, sigma_w = 0.072;
static const double c_pd = 1005.0, c_pv = 1850.0, c_l = 4218.0, l_v0 = 2.5e6;
static const double R_d = 287.0, R_v = 461.5;
static const double T0 = 273.16, p_vs0 = 611.73, grav = 9.81, p1000 = 1.0e5;
static const double D0 = 2.26e-5, K0 = 2.4e-2;
static const double delta0 = 9.06, C0 = 0.292;

static double rho_stp(void) { return 101325.0 / (R_d * 293.15); }

/* (0,1) open-interval uniform from 64 random bits: 52 bits plus one half. */
double orc_u01(uint64_t v) { return ((double)(v >> 12) + 0.5) * 0x1p-52; }

/* Threads of the cell-parallel build (n > 0 sets them); 1 in the serial one. */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* add one cell's counters to the run's (one thread at a time) */
static void stats_merge(orc_stats *st, const orc_stats *c)
{
    if (!st) return;
#ifdef _OPENMP
#pragma omp critical(orc_stats_merge)
#endif
    {
        st->n_pairs += c->n_pairs; st->n_coll += c->n_coll; st->n_pgt1 += c->n_pgt1;
        st->n_recycled += c->n_recycled; st->n_euler += c->n_euler; st->n_bisect += c->n_bisect;
        if (c->max_p > st->max_p) st->max_p = c->max_p;
        st->rainfall += c->rainfall;
        st->n_coal_substeps += c->n_coal_substeps;
    }
}

static void draw(uint64_t seed, uint64_t uid, uint64_t substep, uint64_t step, uint64_t stream,
                 uint64_t out[4])
{
    const uint64_t ctr[4] = {uid, substep, step, stream};
    const uint64_t key[2] = {seed, 0};
    orc_philox4x64_10(ctr, key, out);
}

enum { STREAM_COAL = 1, STREAM_INIT = 3 };

/* ---- grid ---------------------------------------------------------------- */
static int64_t dimn(int n) { return n > 0 ? n : 1; }

int64_t orc_n_cells(const orc_domain *d) { return dimn(d->nx) * dimn(d->ny) * dimn(d->nz); }

static double cell_volume(const orc_domain *d) { return d->dx * d->dy * d->dz; }

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Cell i = floor(x / dx) in each present dimension (Sec. 5.1.2, eq. adv_w);
 * linear index row-major over (x, y, z), z fastest. */
int64_t orc_cell_of(const orc_domain *d, double x, double y, double z)
{
    int64_t i = d->nx > 0 ? clampi((int64_t)floor(x / d->dx), 0, d->nx - 1) : 0;
    int64_t j = d->ny > 0 ? clampi((int64_t)floor(y / d->dy), 0, d->ny - 1) : 0;
    int64_t k = d->nz > 0 ? clampi((int64_t)floor(z / d->dz), 0, d->nz - 1) : 0;
    return (i * dimn(d->ny) + j) * dimn(d->nz) + k;
}

/* ---- kappa groups: READING: one initial spectrum per distinct kappa ------
 * (Sec. 5.1.6: "externally mixed aerosol may be represented using multiple
 * spectra, each characterised by different kappa"), each sampled with
 * sd_conc super-droplets per cell.                                          */
static int group_kappas(const orc_domain *d, double *kap)
{
    if (d->init_dist == 1) { kap[0] = 0.0; return 1; }
    int g = 0;
    for (int m = 0; m < d->n_modes; ++m) {
        int seen = 0;
        for (int q = 0; q < g; ++q) if (kap[q] == d->modes[m].kappa) seen = 1;
        if (!seen) kap[g++] = d->modes[m].kappa;
    }
    return g;
}

int orc_n_groups(const orc_domain *d) { double k[ORC_MAX_MODES]; return group_kappas(d, k); }

/* ---- thermodynamics (Appendix A, Sec. 5.1.3) ----------------------------- */
void orc_thermo_eval(double th, double rv, double rhod, double RH_max, orc_thermo *t)
{
    t->th = th; t->rv = rv; t->rhod = rhod;
    /* T and p diagnosed from theta, r_v and rho_d (Appendix A) */
    t->T = pow(th * pow(rhod * R_d / p1000, R_d / c_pd), c_pd / (c_pd - R_d));
    t->p = rhod * (R_d + rv * R_v) * t->T;
    /* l_v(T) from the list of symbols */
    t->lv = l_v0 + (c_pv - c_l) * (t->T - T0);
    /* READING: p_vs from Clausius-Clapeyron integrated with the linear l_v(T) */
    double lnp = (l_v0 + (c_l - c_pv) * T0) / R_v * (1.0 / T0 - 1.0 / t->T)
               - (c_l - c_pv) / R_v * log(t->T / T0);
    t->rho_vs = p_vs0 * exp(lnp) / (R_v * t->T);
    t->rho_v = rv * rhod;
    /* RH limit for drop growth (opts_t::RH_max, Sec. 5.2.1) */
    t->rho_v_eff = fmin(t->rho_v, RH_max * t->rho_vs);
    /* d theta / d r_v = -theta l_v / (c_pd T)  (Sec. 3.1.2, Appendix A) */
    t->dth_drv = -th * t->lv / (c_pd * t->T);
    /* Kelvin-term parameter A = 2 sigma_w / (R_v T rho_w) (Appendix B) */
    t->A = 2.0 * sigma_w / (R_v * t->T * rho_w);
    /* heat-conduction part of 1/D_eff (Sec. 5.1.3, eq. maxmason) */
    t->Dterm = t->rho_vs * t->lv / t->T * (t->lv / (R_v * t->T) - 1.0);
    /* READING: moist-air density, Sutherland-type viscosity, kinetic mean
     * free paths lambda = 2 * diffusivity / mean molecular speed */
    t->rho_a = rhod * (1.0 + rv);
    t->mu = 1.72e-5 * (393.0 / (t->T + 120.0)) * pow(t->T / 273.0, 1.5);
    t->nu = t->mu / t->rho_a;
    t->lambda_D = 2.0 * D0 / sqrt(8.0 * R_v * t->T / PI);
    t->lambda_K = 2.0 * K0 / (t->rho_a * c_pd * sqrt(8.0 * R_d * t->T / PI));
    t->Sc = t->nu / D0;
    t->Pr = t->nu * t->rho_a * c_pd / K0;
    /* Best (Davies) number of a sphere of radius r is cX * r^3 */
    t->cX = 32.0 / 3.0 * (rho_w - t->rho_a) / t->rho_a * grav / (t->nu * t->nu);
}

/* READING of Khvorostyanov & Curry (2002) for a sphere: Reynolds number as a
 * function of the Best number X, Re = delta0^2/4 (sqrt(1 + c1 sqrt(X)) - 1)^2
 * with c1 = 4 / (delta0^2 sqrt(C0)); it tends to Stokes' Re = X/24 for small
 * X.  Pinned by that Stokes limit and by Gunn & Kinzer's (1949) measured
 * fall speeds within 12 % (the fit approximates such measurements). */
double orc_reynolds(double rw2, const orc_thermo *t)
{
    double r = sqrt(rw2);
    if (!(r > 0.0)) return 0.0;
    double X = t->cX * rw2 * r;
    double c1 = 4.0 / (delta0 * delta0 * sqrt(C0));
    double e = c1 * sqrt(X);
    double s = e / (sqrt(1.0 + e) + 1.0); /* sqrt(1 + e) - 1 without cancellation */
    return delta0 * delta0 / 4.0 * s * s;
}

/* terminal velocity v_t = Re nu / (2 r)  (Sec. 5.1.5) */
double orc_vterm(double rw2, const orc_thermo *t)
{
    double r = sqrt(rw2);
    if (!(r > 0.0)) return 0.0;
    return orc_reynolds(rw2, t) * t->nu / (2.0 * r);
}

/* Fuchs-Sutugin transition-regime factor with unit accommodation
 * (Sec. 5.1.3): beta = (1 + Kn) / (1 + (4/3 + 0.377) Kn + 4/3 Kn^2). */
static double fuchs_sutugin(double Kn)
{
    return (1.0 + Kn) / (1.0 + (4.0 / 3.0 + 0.377) * Kn + 4.0 / 3.0 * Kn * Kn);
}

/* dr_w^2/dt = 2 r_w dr_w/dt from the Maxwell-Mason eq. (maxmason):
 *   r dr/dt = D_eff / rho_w (rho_v - rho_o),
 *   1/D_eff = 1/D + 1/K rho_vs l_v / T (l_v / (R_v T) - 1),
 *   rho_o   = rho_vs a_w(r_w, r_d) exp(A / r_w)      (eq. rho_circ),
 *   a_w     = (r_w^3 - r_d^3) / (r_w^3 - r_d^3 (1 - kappa))  (Appendix B),
 *   D = D0 beta_M Sh/2, K = K0 beta_T Nu/2                (Sec. 5.1.3).
 * physics == 0 drops the corrections (beta = 1, Sh = Nu = 2).
 * READING: Sh = 1 + (1 + Re Sc)^(1/3) f(Re), Nu likewise with Pr, and
 * f = 1 for Re <= 1, Re^0.077 above (Clift et al. 1978).  Pinned by the
 * limits Kn -> 0 (beta -> 1) and Re -> 0 (Sh = Nu = 2), by Seinfeld &
 * Pandis's arrangement of beta (Kn 0.08-4) and by Pruppacher & Klett's
 * ventilation coefficient within 5 % (Re up to 170). */
double orc_growth(double x, double rd3, double kappa, const orc_thermo *t, int physics)
{
    double r = sqrt(x);
    double r3 = x * r;
    double aw = (r3 - rd3) / (r3 - rd3 * (1.0 - kappa));
    double rho_o = t->rho_vs * aw * exp(t->A / r);
    double D = D0, K = K0;
    if (physics) {
        double bM = fuchs_sutugin(t->lambda_D / r);
        double bT = fuchs_sutugin(t->lambda_K / r);
        double Re = orc_reynolds(x, t);
        double fRe = Re > 1.0 ? pow(Re, 0.077) : 1.0;
        double Sh = 1.0 + cbrt(1.0 + Re * t->Sc) * fRe;
        double Nu = 1.0 + cbrt(1.0 + Re * t->Pr) * fRe;
        D = D0 * bM * Sh / 2.0;
        K = K0 * bT * Nu / 2.0;
    }
    double Deff = 1.0 / (1.0 / D + t->Dterm / K);
    return 2.0 * Deff / rho_w * (t->rho_v_eff - rho_o);
}

static double rd2_of(double rd3) { double rd = cbrt(rd3); return rd * rd; }

/* Implicit-in-r_w^2 drop growth over one substep dt' (Sec. 5.1.3, eq.
 * rw2_implicit): find x with  x = x0 + dt' g(x).
 * READING: the bracket uses the substep dt' (the printed bracket omits it and
 * the printed equation says dt), a = max(r_d^2, x0 + min(2 dt' g(x0), 0)),
 * b = x0 + max(2 dt' g(x0), 0).  If f = x - x0 - dt' g(x) does not change
 * strict sign between a and b, return (a + b)/2 (the Euler step).  Otherwise
 * bisect, keeping the half whose ends differ in sign, until b - a <= 2^-52 b
 * or 200 halvings, and return the middle of the last interval. */
static double fres(double x, double x0, double rd3, double kappa, const orc_thermo *t,
                   double dtp, int physics)
{
    return x - x0 - dtp * orc_growth(x, rd3, kappa, t, physics);
}

double orc_solve_rw2(double x0, double rd3, double kappa, const orc_thermo *t, double dtp,
                     int physics, orc_stats *st)
{
    double g0 = orc_growth(x0, rd3, kappa, t, physics);
    double a = fmax(rd2_of(rd3), x0 + fmin(2.0 * dtp * g0, 0.0));
    double b = x0 + fmax(2.0 * dtp * g0, 0.0);
    double fa = fres(a, x0, rd3, kappa, t, dtp, physics);
    double fb = fres(b, x0, rd3, kappa, t, dtp, physics);
    if ((fa > 0.0) == (fb > 0.0)) {
        if (st) st->n_euler++;
        return 0.5 * (a + b);
    }
    double lo = a, hi = b;
    int plo = fa > 0.0;
    for (int it = 0; it < 200; ++it) {
        if (hi - lo <= 0x1p-52 * hi) break;
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (st) st->n_bisect++;
        int pm = fres(mid, x0, rd3, kappa, t, dtp, physics) > 0.0;
        if (pm == plo) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* One condensation substep's solves for listed super-droplets, each in its
 * cell's ambient state at (th, rv, rhod), with no feedback on the cell:
 * x1[q] = orc_solve_rw2(x0[q], ...).  A test driver for comparing solvers
 * solve by solve along an oracle trajectory. */
void orc_solve_batch(int64_t n, const double *x0, const double *rd3, const double *kappa,
                     const int64_t *cell, const double *th, const double *rv, const double *rhod,
                     double RH_max, double dtp, int physics, double *x1)
{
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
        orc_thermo t;
        int64_t c = cell[q];
        orc_thermo_eval(th[c], rv[c], rhod[c], RH_max, &t);
        x1[q] = orc_solve_rw2(x0[q], rd3[q], kappa[q], &t, dtp, physics, NULL);
    }
}

/* Wet radius in equilibrium with relative humidity RH: zero left-hand side of
 * eq. (maxmason), i.e. a_w exp(A/r) = RH (Sec. 5.1.6), found by bisection in
 * x = r^2 on [r_d^2, x_hi], where a_w(x_hi) = RH so that the Kelvin factor
 * makes the left side exceed RH there.  For RH < 1 the root is unique (the
 * stable, left branch of the Koehler curve). */
double orc_equilibrium_rw2(double rd3, double kappa, double RH, double T)
{
    double rd2 = rd2_of(rd3);
    if (!(kappa > 0.0) || !(RH > 0.0) || !(RH < 1.0) || !(rd3 > 0.0)) return rd2;
    double A = 2.0 * sigma_w / (R_v * T * rho_w);
    double rhi = cbrt(rd3 * (1.0 - RH * (1.0 - kappa)) / (1.0 - RH));
    double lo = rd2, hi = rhi * rhi;
    for (int it = 0; it < 200; ++it) {
        if (hi - lo <= 0x1p-52 * hi) break;
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        double r = sqrt(mid), r3 = mid * r;
        double S = (r3 - rd3) / (r3 - rd3 * (1.0 - kappa)) * exp(A / r);
        if (S > RH) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

/* ---- initialisation (Sec. 5.1.6) ------------------------------------------ */
/* dN/dln(r) at STP of one kappa group: sum of lognormal modes (eq. lognormal,
 * written per unit ln r). */
static double n_lnr(const orc_domain *d, double kap, double lnr)
{
    double s = 0.0;
    for (int m = 0; m < d->n_modes; ++m) {
        if (d->modes[m].kappa != kap) continue;
        double ls = log(d->modes[m].sigma);
        double q = (lnr - log(d->modes[m].rm)) / ls;
        s += d->modes[m].n_stp / (sqrt(2.0 * PI) * ls) * exp(-0.5 * q * q);
    }
    return s;
}

/* READING of "multiplicity >= 1 at the minimal and maximal radii": with
 * super-droplets uniform in ln r over [lo, hi], one stands for a slice
 * (hi - lo)/sd_conc of ln r, so its STP multiplicity is n(ln r) dlnr dV.
 * Starting from [1 nm, 10 um], the range is narrowed to the outermost radii
 * where that multiplicity is >= 1 (a 1000-point scan, then 100 bisections),
 * and the new width fed back; 8 such passes. */
int orc_rd_range(const orc_domain *d, int group, double *lnr_min, double *lnr_max)
{
    double kap[ORC_MAX_MODES];
    int G = group_kappas(d, kap);
    if (group < 0 || group >= G || d->sd_conc <= 0) return -1;
    const double L0 = log(1e-9), L1 = log(1e-5);
    const int NG = 1000;
    double dV = cell_volume(d);
    double lo = L0, hi = L1;
    for (int pass = 0; pass < 8; ++pass) {
        double dlnr = (hi - lo) / d->sd_conc;
        int jlo = -1, jhi = -1;
        for (int j = 0; j <= NG; ++j) {
            double l = L0 + (L1 - L0) * j / NG;
            if (n_lnr(d, kap[group], l) * dlnr * dV >= 1.0) { jlo = j; break; }
        }
        for (int j = NG; j >= 0; --j) {
            double l = L0 + (L1 - L0) * j / NG;
            if (n_lnr(d, kap[group], l) * dlnr * dV >= 1.0) { jhi = j; break; }
        }
        if (jlo < 0 || jhi < 0) return -2;
        double nlo = L0 + (L1 - L0) * jlo / NG, nhi = L0 + (L1 - L0) * jhi / NG;
        if (jlo > 0) { /* w(below) < 1 <= w(above) */
            double b0 = L0 + (L1 - L0) * (jlo - 1) / NG, b1 = nlo;
            for (int it = 0; it < 100; ++it) {
                double m = 0.5 * (b0 + b1);
                if (n_lnr(d, kap[group], m) * dlnr * dV >= 1.0) b1 = m; else b0 = m;
            }
            nlo = b1;
        }
        if (jhi < NG) { /* w(below) >= 1 > w(above) */
            double b0 = nhi, b1 = L0 + (L1 - L0) * (jhi + 1) / NG;
            for (int it = 0; it < 100; ++it) {
                double m = 0.5 * (b0 + b1);
                if (n_lnr(d, kap[group], m) * dlnr * dV >= 1.0) b0 = m; else b1 = m;
            }
            nhi = b0;
        }
        lo = nlo; hi = nhi;
    }
    *lnr_min = lo; *lnr_max = hi;
    return 0;
}

/* Initial super-droplets of the listed cells (Sec. 5.1.6).  READINGS: exactly
 * sd_conc super-droplets per cell per kappa group, each uniform within its
 * cell (a stratified form of the uniform initial positions); id
 * ((cell * G) + group) * sd_conc + k; random numbers from Philox with counter
 * (id, 0, 0, 3): words 0/1/2 give x/y/z, word 3 gives ln r_d (or the volume).
 * Multiplicity = max(1, floor(n(ln r) dlnr dV rho_d/rho_STP + 1/2)); wet
 * radius at Koehler equilibrium with the cell's RH, or RH = 0.95 where the
 * cell is supersaturated.  init_dist 1 is the box test: volumes exponential
 * with the given mean, dry mass zero, multiplicity n0 dV / sd_conc. */
int orc_init_cells(const orc_domain *d, const double *th, const double *rv, const double *rhod,
                   int64_t n_list, const int64_t *cells, orc_sds *out)
{
    return orc_init_cells_nreal(d, th, rv, rhod, n_list, cells, out, NULL);
}

/* The same, also returning (if nreal != NULL) each multiplicity before
 * rounding, so that tests can tell rounding-ambiguous values apart. */
int orc_init_cells_nreal(const orc_domain *d, const double *th, const double *rv,
                         const double *rhod, int64_t n_list, const int64_t *cells, orc_sds *out,
                         double *nreal)
{
    double kap[ORC_MAX_MODES], lmin[ORC_MAX_MODES], lmax[ORC_MAX_MODES];
    int G = group_kappas(d, kap);
    if (d->init_dist == 0)
        for (int g = 0; g < G; ++g)
            if (orc_rd_range(d, g, &lmin[g], &lmax[g]) != 0) return -1;
    double dV = cell_volume(d);
    int64_t NY = dimn(d->ny), NZ = dimn(d->nz);
    int64_t o = 0;
    for (int64_t q = 0; q < n_list; ++q) {
        int64_t c = cells[q];
        int64_t ci = c / (NY * NZ), cj = (c / NZ) % NY, ck = c % NZ;
        orc_thermo t;
        orc_thermo_eval(th[c], rv[c], rhod[c], 44.0, &t);
        double RH = t.rho_v / t.rho_vs;
        if (RH >= 1.0) RH = 0.95;
        for (int g = 0; g < G; ++g) {
            for (int k = 0; k < d->sd_conc; ++k, ++o) {
                uint64_t uid = ((uint64_t)c * G + g) * d->sd_conc + k;
                uint64_t w[4];
                draw(d->seed, uid, 0, 0, STREAM_INIT, w);
                out->uid[o] = uid;
                out->x[o] = d->nx > 0 ? ((double)ci + orc_u01(w[0])) * d->dx : 0.0;
                out->y[o] = d->ny > 0 ? ((double)cj + orc_u01(w[1])) * d->dy : 0.0;
                out->z[o] = d->nz > 0 ? ((double)ck + orc_u01(w[2])) * d->dz : 0.0;
                if (d->init_dist == 1) {
                    double V = -d->exp_mean_volume * log(orc_u01(w[3]));
                    double r = cbrt(3.0 * V / (4.0 * PI));
                    out->rw2[o] = r * r;
                    out->rd3[o] = 0.0;
                    out->kappa[o] = 0.0;
                    double v = d->exp_n0 * dV / d->sd_conc;
                    double n = floor(v + 0.5);
                    out->N[o] = n < 1.0 ? 1 : (uint64_t)n;
                    if (nreal) nreal[o] = v;
                } else {
                    double lnr = lmin[g] + orc_u01(w[3]) * (lmax[g] - lmin[g]);
                    double rd = exp(lnr);
                    double rd3 = rd * rd * rd;
                    double dlnr = (lmax[g] - lmin[g]) / d->sd_conc;
                    double v = n_lnr(d, kap[g], lnr) * dlnr * dV * rhod[c] / rho_stp();
                    double n = floor(v + 0.5);
                    out->N[o] = n < 1.0 ? 1 : (uint64_t)n;
                    if (nreal) nreal[o] = v;
                    out->rd3[o] = rd3;
                    out->kappa[o] = kap[g];
                    out->rw2[o] = orc_equilibrium_rw2(rd3, kap[g], RH, t.T);
                }
            }
        }
    }
    out->n = o;
    return 0;
}

/* ---- cell membership: per cell, super-droplet indices in id order -------- */
typedef struct { int64_t *start, *idx; } members;

static const uint64_t *g_uid_for_sort; /* qsort has no context argument in C99 */
static int cmp_idx_by_uid(const void *a, const void *b)
{
    uint64_t ua = g_uid_for_sort[*(const int64_t *)a], ub = g_uid_for_sort[*(const int64_t *)b];
    return ua < ub ? -1 : (ua > ub ? 1 : 0);
}

static members build_members(const orc_domain *d, const orc_sds *s)
{
    int64_t nc = orc_n_cells(d);
    members m;
    m.start = calloc((size_t)nc + 1, sizeof(int64_t));
    m.idx = malloc((size_t)(s->n > 0 ? s->n : 1) * sizeof(int64_t));
    int64_t *cell = malloc((size_t)(s->n > 0 ? s->n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < s->n; ++i) {
        cell[i] = orc_cell_of(d, s->x[i], s->y[i], s->z[i]);
        m.start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < nc; ++c) m.start[c + 1] += m.start[c];
    int64_t *fill = malloc((size_t)nc * sizeof(int64_t));
    memcpy(fill, m.start, (size_t)nc * sizeof(int64_t));
    for (int64_t i = 0; i < s->n; ++i) m.idx[fill[cell[i]]++] = i;
    g_uid_for_sort = s->uid;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < nc; ++c)
        qsort(m.idx + m.start[c], (size_t)(m.start[c + 1] - m.start[c]), sizeof(int64_t),
              cmp_idx_by_uid);
    free(fill);
    free(cell);
    return m;
}

static void free_members(members *m) { free(m->start); free(m->idx); }

/* ---- condensation: Sec. 5.1.3 ---------------------------------------------
 * sstp_cond substeps; in each, every super-droplet's r_w^2 is advanced with
 * the cell's theta and r_v held at the substep start, then the cell's r_v
 * and theta are updated with eq. (rhov_update):
 *   dr_v = -4 pi rho_w / (3 dV rho_d) sum N (r_w^3[new] - r_w^3[old]),
 *   dtheta = dr_v * dtheta/dr_v evaluated at the substep start.
 * READING: multiplicity-zero super-droplets (awaiting recycling) are skipped. */
void orc_condense(const orc_domain *d, const orc_opts *o, orc_sds *s, double *th, double *rv,
                  const double *rhod, orc_stats *st)
{
    members m = build_members(d, s);
    int64_t nc = orc_n_cells(d);
    double dV = cell_volume(d);
    double dtp = d->dt / o->sstp_cond;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < nc; ++c) {
        orc_stats cs;
        memset(&cs, 0, sizeof cs);
        for (int sub = 0; sub < o->sstp_cond; ++sub) {
            orc_thermo t;
            orc_thermo_eval(th[c], rv[c], rhod[c], o->RH_max, &t);
            double sum = 0.0;
            for (int64_t q = m.start[c]; q < m.start[c + 1]; ++q) {
                int64_t i = m.idx[q];
                if (s->N[i] == 0) continue;
                double x0 = s->rw2[i];
                double x1 = orc_solve_rw2(x0, s->rd3[i], s->kappa[i], &t, dtp, d->physics, &cs);
                s->rw2[i] = x1;
                sum += (double)s->N[i] * (x1 * sqrt(x1) - x0 * sqrt(x0));
            }
            double drv = -4.0 * PI * rho_w / (3.0 * dV * rhod[c]) * sum;
            rv[c] = t.rv + drv;
            th[c] = t.th + drv * t.dth_drv;
        }
        stats_merge(st, &cs);
    }
    free_members(&m);
}

/* ---- recycling of multiplicity-zero super-droplets (Sec. 5.1.4) ----------
 * READING: over the whole domain, the k-th zero-multiplicity super-droplet in
 * id order takes all attributes of the k-th donor in (multiplicity
 * descending, id ascending) order among donors with multiplicity >= 2; the
 * clone gets floor(N/2), the donor keeps the rest.  Zeros beyond the number
 * of such donors stay at zero. */
static const orc_sds *g_sds_for_sort;
static int cmp_donor(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    uint64_t Ni = g_sds_for_sort->N[i], Nj = g_sds_for_sort->N[j];
    if (Ni != Nj) return Ni > Nj ? -1 : 1;
    uint64_t ui = g_sds_for_sort->uid[i], uj = g_sds_for_sort->uid[j];
    return ui < uj ? -1 : (ui > uj ? 1 : 0);
}

void orc_recycle(orc_sds *s, orc_stats *st)
{
    int64_t nz = 0, nd = 0;
    for (int64_t i = 0; i < s->n; ++i) {
        if (s->N[i] == 0) nz++;
        else if (s->N[i] >= 2) nd++;
    }
    if (nz == 0 || nd == 0) return;
    int64_t *zi = malloc((size_t)nz * sizeof(int64_t)), *di = malloc((size_t)nd * sizeof(int64_t));
    int64_t a = 0, b = 0;
    for (int64_t i = 0; i < s->n; ++i) {
        if (s->N[i] == 0) zi[a++] = i;
        else if (s->N[i] >= 2) di[b++] = i;
    }
    g_uid_for_sort = s->uid;
    qsort(zi, (size_t)nz, sizeof(int64_t), cmp_idx_by_uid);
    g_sds_for_sort = s;
    qsort(di, (size_t)nd, sizeof(int64_t), cmp_donor);
    int64_t np = nz < nd ? nz : nd;
    for (int64_t q = 0; q < np; ++q) {
        int64_t z = zi[q], dn = di[q];
        s->rw2[z] = s->rw2[dn]; s->rd3[z] = s->rd3[dn]; s->kappa[z] = s->kappa[dn];
        s->x[z] = s->x[dn]; s->y[z] = s->y[dn]; s->z[z] = s->z[dn];
        s->N[z] = s->N[dn] / 2;
        s->N[dn] = s->N[dn] - s->N[z];
    }
    if (st) st->n_recycled += (uint64_t)np;
    free(zi);
    free(di);
}

/* ---- transport: Sec. 5.1.2 (advection) and 5.1.5 (sedimentation) -------- */

/* READING: the API passes rho_d * C on cell edges (Sec. 5.2.1); C on an edge
 * is that divided by the mean rho_d of the two cells sharing it (the single
 * adjacent cell on a non-periodic boundary). */
static double courant_x(const orc_domain *d, const double *rhod, const double *rhoC, int64_t ie,
                        int64_t j, int64_t k)
{
    int64_t NY = dimn(d->ny), NZ = dimn(d->nz);
    int64_t il = (ie - 1 + d->nx) % d->nx, ir = ie % d->nx;
    double re = 0.5 * (rhod[(il * NY + j) * NZ + k] + rhod[(ir * NY + j) * NZ + k]);
    return rhoC[(ie * NY + j) * NZ + k] / re;
}
static double courant_y(const orc_domain *d, const double *rhod, const double *rhoC, int64_t i,
                        int64_t je, int64_t k)
{
    int64_t NY = d->ny, NZ = dimn(d->nz);
    int64_t jl = (je - 1 + NY) % NY, jr = je % NY;
    double re = 0.5 * (rhod[(i * NY + jl) * NZ + k] + rhod[(i * NY + jr) * NZ + k]);
    return rhoC[(i * (NY + 1) + je) * NZ + k] / re;
}
static double courant_z(const orc_domain *d, const double *rhod, const double *rhoC, int64_t i,
                        int64_t j, int64_t ke)
{
    int64_t NY = dimn(d->ny), NZ = d->nz;
    int64_t kl = ke - 1 < 0 ? 0 : ke - 1, kr = ke > NZ - 1 ? NZ - 1 : ke;
    double re = 0.5 * (rhod[(i * NY + j) * NZ + kl] + rhod[(i * NY + j) * NZ + kr]);
    return rhoC[(i * NY + j) * (NZ + 1) + ke] / re;
}

/* Analytic solution of the backward-Euler step x' = x + dx C(x') with C
 * interpolated linearly between the edges of the cell holding x (eqs.
 * adv_implicit, adv_c, adv_w):
 *   x' = (x + dx (C_l - i dC)) / (1 - dC),  dC = C_r - C_l. */
static double advect_1d(double x, double h, int64_t i, double Cl, double Cr)
{
    double dC = Cr - Cl;
    return (x + h * (Cl - (double)i * dC)) / (1.0 - dC);
}

static double wrap(double x, double X)
{
    double w = fmod(x, X);
    if (w < 0.0) w += X;
    if (w >= X) w = 0.0;
    return w;
}

void orc_advect(const orc_domain *d, orc_sds *s, const double *rhod, const double *rhoCx,
                const double *rhoCy, const double *rhoCz)
{
    int64_t NY = dimn(d->ny), NZ = dimn(d->nz);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < s->n; ++q) {
        int64_t c = orc_cell_of(d, s->x[q], s->y[q], s->z[q]);
        int64_t i = c / (NY * NZ), j = (c / NZ) % NY, k = c % NZ;
        if (d->nx > 0 && rhoCx) {
            double xn = advect_1d(s->x[q], d->dx, i, courant_x(d, rhod, rhoCx, i, j, k),
                                  courant_x(d, rhod, rhoCx, i + 1, j, k));
            s->x[q] = wrap(xn, d->nx * d->dx);
        }
        if (d->ny > 0 && rhoCy) {
            double yn = advect_1d(s->y[q], d->dy, j, courant_y(d, rhod, rhoCy, i, j, k),
                                  courant_y(d, rhod, rhoCy, i, j + 1, k));
            s->y[q] = wrap(yn, d->ny * d->dy);
        }
        if (d->nz > 0 && rhoCz) {
            s->z[q] = advect_1d(s->z[q], d->dz, k, courant_z(d, rhod, rhoCz, i, j, k),
                                courant_z(d, rhod, rhoCz, i, j, k + 1));
        }
    }
}

/* Advection, then explicit-Euler sedimentation z -= v_t dt with v_t taken in
 * the cell the super-droplet occupied at the step start (Sec. 5.1.5).
 * Super-droplets that leave through the bottom or top get multiplicity zero;
 * READING: the liquid mass N (4/3) pi rho_w r_w^3 of bottom leavers is added
 * to the accumulated rainfall [kg]. */
void orc_transport(const orc_domain *d, const orc_opts *o, orc_sds *s, const double *th,
                   const double *rv, const double *rhod, const double *rhoCx,
                   const double *rhoCy, const double *rhoCz, orc_stats *st)
{
    double *vt = NULL;
    if (o->sedi && d->nz > 0) {
        vt = malloc((size_t)(s->n > 0 ? s->n : 1) * sizeof(double));
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < s->n; ++q) {
            int64_t c = orc_cell_of(d, s->x[q], s->y[q], s->z[q]);
            orc_thermo t;
            orc_thermo_eval(th[c], rv[c], rhod[c], 44.0, &t);
            vt[q] = orc_vterm(s->rw2[q], &t);
        }
    }
    if (o->adve) orc_advect(d, s, rhod, rhoCx, rhoCy, rhoCz);
    if (d->nz > 0) {
        double Z = d->nz * d->dz;
        for (int64_t q = 0; q < s->n; ++q) {
            if (vt) s->z[q] = s->z[q] - vt[q] * d->dt;
            if (s->z[q] < 0.0) {
                double r = sqrt(s->rw2[q]);
                if (st) st->rainfall += (double)s->N[q] * (4.0 / 3.0 * PI * rho_w * r * r * r);
                s->N[q] = 0;
                s->z[q] = 0.0;
            } else if (s->z[q] >= Z) {
                s->N[q] = 0;
                s->z[q] = Z;
            }
        }
    }
    free(vt);
}

/* ---- coalescence: Sec. 5.1.4 ----------------------------------------------- */
typedef struct { uint64_t key, uid, acc; int64_t i; } shuf;
static int cmp_shuf(const void *a, const void *b)
{
    const shuf *p = a, *q = b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->uid < q->uid ? -1 : (p->uid > q->uid ? 1 : 0);
}

/* collection kernel: geometric K = E pi (r_i + r_j)^2 |v_i - v_j| with E = 1,
 * or (box test) Golovin K = b (V_i + V_j) */
static double kernel_K(const orc_domain *d, const orc_thermo *t, double rw2a, double rw2b)
{
    if (d->kernel == 1) {
        double Va = 4.0 / 3.0 * PI * rw2a * sqrt(rw2a), Vb = 4.0 / 3.0 * PI * rw2b * sqrt(rw2b);
        return d->golovin_b * (Va + Vb);
    }
    double ra = sqrt(rw2a), rb = sqrt(rw2b);
    double dv = fabs(orc_vterm(rw2a, t) - orc_vterm(rw2b, t));
    double E = 1.0;
    if (d->kernel == 2) {
        /* hydrodynamic collection efficiency after Long (1974), a formula
         * standing in for the tabulated ones the paper cites (Sec. 5.1.4),
         * READING: R the larger, r the smaller radius; E = 1 for R >= 50 um,
         * else 4.5e4 R^2 (1 - 3e-4/r) with R, r in cm (4.5e8 R^2 (1 - 3e-6/r)
         * in m), floored at 1e-3 and capped at 1 */
        double R = ra > rb ? ra : rb, r = ra > rb ? rb : ra;
        if (R < 50e-6) {
            E = 4.5e8 * R * R * (1.0 - 3e-6 / r);
            if (E < 1e-3) E = 1e-3;
            if (E > 1.0) E = 1.0;
        }
    }
    return E * (PI * (ra + rb) * (ra + rb) * dv);
}

/* gamma collision events of all min(N_i, N_j) particles (Sec. 5.1.4; gamma
 * is 1 unless multiple coalescence is on).  READING of the garbled role
 * assignment: the super-droplet with the larger multiplicity L (the first
 * of the pair on a tie) keeps its radii and loses gamma times the other's
 * multiplicity; the other, S, keeps its multiplicity and takes the merged
 * radii: r_w^3 and r_d^3 of gamma L-droplets added to its own, kappa
 * averaged weighted by r_d^3. */
static void collide(orc_sds *s, int64_t a, int64_t b, uint64_t gamma)
{
    int64_t L = s->N[a] >= s->N[b] ? a : b;
    int64_t S = L == a ? b : a;
    s->N[L] -= gamma * s->N[S];
    double g = (double)gamma;
    double r3 = s->rw2[S] * sqrt(s->rw2[S]) + g * (s->rw2[L] * sqrt(s->rw2[L]));
    double r = cbrt(r3);
    s->rw2[S] = r * r;
    double dL = g * s->rd3[L];
    double m3 = s->rd3[S] + dL;
    if (m3 > 0.0) s->kappa[S] = (s->kappa[S] * s->rd3[S] + s->kappa[L] * dL) / m3;
    s->rd3[S] = m3;
}

/* Number of collision events of a pair with scaled probability P and
 * uniform number u.  The paper's scheme (Sec. 5.1.4): one event when u < P,
 * whatever P.  Multiple coalescence (Shima et al. 2009, Sec. 4.1.4 there),
 * which the paper plans for P > 1: gamma = floor(P), plus one when
 * u < P - floor(P), so that E[gamma] = P; at most floor(N_L/N_S) events can
 * take place. */
static uint64_t n_events(double P, double u, uint64_t NL, uint64_t NS, int multi)
{
    if (!multi) return u < P ? 1 : 0;
    if (!(P > 0.0)) return 0;
    uint64_t cap = NL / NS;
    double fl = floor(P);
    if (fl >= (double)cap) return cap;
    uint64_t g = (uint64_t)fl;
    if (u < P - fl) g++;
    return g < cap ? g : cap;
}

/* Adaptive coalescence substeps (the paper plans to control the substep
 * from P_ij, Sec. 5.1.4; READING): at the start of the step, per cell, an
 * upper bound of eq. P_ij over every pair the cell's n super-droplets with
 * N > 0 could form,
 *   P_bound = N_max K_bound dt / dV * n (n-1) / (2 floor(n/2)),
 * with K_bound = pi (2 r_max)^2 (v_max - v_min) for the geometric kernel
 * (no pair has larger radii or a larger speed difference) and
 * K_bound = b 2 V_max for Golovin's.  The cell takes
 * max(sstp_coal, ceil(P_bound)) substeps, at most coal_adapt, so that no
 * pair's P exceeds 1 at the first substep when the cap allows it. */
static int adaptive_substeps(const orc_domain *d, const orc_opts *o, const orc_thermo *t,
                             const orc_sds *s, const members *m, int64_t c, double dV)
{
    int64_t n = 0;
    uint64_t Nmax = 0;
    double rw2max = 0.0, vmax = 0.0, vmin = INFINITY;
    for (int64_t q = m->start[c]; q < m->start[c + 1]; ++q) {
        int64_t i = m->idx[q];
        if (s->N[i] == 0) continue;
        n++;
        if (s->N[i] > Nmax) Nmax = s->N[i];
        if (s->rw2[i] > rw2max) rw2max = s->rw2[i];
        if (d->kernel != 1) {
            double v = orc_vterm(s->rw2[i], t);
            if (v > vmax) vmax = v;
            if (v < vmin) vmin = v;
        }
    }
    if (n < 2) return o->sstp_coal;
    double rmax = sqrt(rw2max), K;
    if (d->kernel == 1) {
        K = d->golovin_b * (2.0 * (4.0 / 3.0 * PI * rw2max * rmax));
    } else {
        double two_r = 2.0 * rmax;
        K = PI * two_r * two_r * (vmax - vmin);
    }
    double scale = (double)n * (double)(n - 1) / (2.0 * (double)(n / 2));
    double Pb = (double)Nmax * K * d->dt / dV * scale;
    int sstp = o->sstp_coal;
    if (Pb > (double)sstp) sstp = Pb >= (double)o->coal_adapt ? o->coal_adapt : (int)ceil(Pb);
    return sstp < o->sstp_coal ? o->sstp_coal : sstp;
}

/* sstp_coal substeps per cell (or the adaptive count above).  In each: the
 * cell's n super-droplets with
 * non-zero multiplicity (READING: zero-multiplicity ones take no part) are
 * put in random order and paired (0,1), (2,3), ...; pair (i, j) collides
 * with probability (eq. P_ij)
 *   P = max(N_i, N_j) K(r_i, r_j) dt''/dV n (n-1) / (2 floor(n/2)),
 * i.e. when P exceeds a uniform number from (0,1).  P > 1 is counted but not
 * treated (no multiple coalescence, Sec. 5.1.4).
 * READING of the random draws: Philox with counter (id, substep, step, 1);
 * word 0 is the sort key (ties by id), word 1 of the pair's first member is
 * the uniform number. */
void orc_coalesce(const orc_domain *d, const orc_opts *o, orc_sds *s, const double *th,
                  const double *rv, const double *rhod, uint64_t step, orc_stats *st)
{
    members m = build_members(d, s);
    int64_t nc = orc_n_cells(d);
    double dV = cell_volume(d);
    shuf *all = malloc(sizeof(shuf) * (size_t)(s->n > 0 ? s->n : 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < nc; ++c) {
        shuf *buf = all + m.start[c];  /* room for the cell's members */
        orc_stats cs;
        memset(&cs, 0, sizeof cs);
        orc_stats *cst = st ? &cs : NULL;
        orc_thermo t;
        orc_thermo_eval(th[c], rv[c], rhod[c], 44.0, &t);
        int sstp = o->coal_adapt > 0 ? adaptive_substeps(d, o, &t, s, &m, c, dV) : o->sstp_coal;
        double dtpp = d->dt / sstp;
        if (cst) cst->n_coal_substeps += (uint64_t)sstp;
        for (int sub = 0; sub < sstp; ++sub) {
            int64_t n = 0;
            for (int64_t q = m.start[c]; q < m.start[c + 1]; ++q) {
                int64_t i = m.idx[q];
                if (s->N[i] == 0) continue;
                uint64_t w[4];
                draw(d->seed, s->uid[i], (uint64_t)sub, step, STREAM_COAL, w);
                buf[n].key = w[0]; buf[n].acc = w[1]; buf[n].uid = s->uid[i]; buf[n].i = i;
                n++;
            }
            if (n < 2) continue;
            qsort(buf, (size_t)n, sizeof(shuf), cmp_shuf);
            double scale = (double)n * (double)(n - 1) / (2.0 * (double)(n / 2));
            for (int64_t k = 0; k < n / 2; ++k) {
                int64_t a = buf[2 * k].i, b = buf[2 * k + 1].i;
                double K = kernel_K(d, &t, s->rw2[a], s->rw2[b]);
                uint64_t Nmax = s->N[a] > s->N[b] ? s->N[a] : s->N[b];
                uint64_t Nmin = s->N[a] > s->N[b] ? s->N[b] : s->N[a];
                double P = (double)Nmax * K * dtpp / dV * scale;
                if (cst) {
                    cst->n_pairs++;
                    if (P > 1.0) cst->n_pgt1++;
                    if (P > cst->max_p) cst->max_p = P;
                }
                uint64_t gamma = n_events(P, orc_u01(buf[2 * k].acc), Nmax, Nmin, o->coal_multi);
                if (gamma > 0) {
                    collide(s, a, b, gamma);
                    if (cst) cst->n_coll++;
                }
            }
        }
        stats_merge(st, &cs);
    }
    free(all);
    free_members(&m);
}

/* ---- time stepping (Sec. 5.2.1, Fig. uml_lgrngn) --------------------------- */
void orc_step_sync(const orc_domain *d, const orc_opts *o, orc_sds *s, double *th, double *rv,
                   const double *rhod, orc_stats *st)
{
    if (o->cond) orc_condense(d, o, s, th, rv, rhod, st);
}

void orc_step_async(const orc_domain *d, const orc_opts *o, orc_sds *s, const double *th,
                    const double *rv, const double *rhod, const double *rhoCx,
                    const double *rhoCy, const double *rhoCz, uint64_t step, orc_stats *st)
{
    orc_recycle(s, st);
    if (o->adve || o->sedi)
        orc_transport(d, o, s, th, rv, rhod, o->adve ? rhoCx : NULL, o->adve ? rhoCy : NULL,
                      o->adve ? rhoCz : NULL, st);
    if (o->coal) orc_coalesce(d, o, s, th, rv, rhod, step, st);
}

/* ---- parcel framework (Sec. 5.2.1: nx = ny = nz = 0, one cell) ------------
 * An adiabatic parcel (or a box, when rho_d never changes) advanced one
 * timestep.  READINGS:
 *  - the parcel keeps its dry-air mass m_d = rho_d dV: a new rho_d given for
 *    the step (step_sync's optional rho_d, "needs to be specified only if the
 *    Eulerian framework allows the density to vary in time") sets
 *    dV = m_d / rho_d before the step; a value equal to the current one
 *    changes nothing.  theta (the dry potential temperature) and r_v are
 *    carried over: T and p follow from them and the new rho_d (Appendix A);
 *  - the step begins with the recycling of zero-multiplicity super-droplets
 *    ("at the beginning of each timestep", Sec. 5.1.4), then condensation
 *    (step_sync), then coalescence; there is no transport.
 * The volume is kept as dx with dy = dz = 1, so that dx dy dz is m_d / rho_d
 * exactly. */
void orc_parcel_step(orc_domain *d, const orc_opts *o, orc_sds *s, double *th, double *rv, double *rhod,
                     double m_d, double rhod_new, uint64_t step, orc_stats *st)
{
    if (rhod_new > 0.0 && rhod_new != rhod[0]) {
        rhod[0] = rhod_new;
        d->dx = m_d / rhod_new;
        d->dy = 1.0;
        d->dz = 1.0;
    }
    orc_recycle(s, st);
    if (o->cond) orc_condense(d, o, s, th, rv, rhod, st);
    if (o->coal) orc_coalesce(d, o, s, th, rv, rhod, step, st);
}

/* ---- diagnostics (Sec. 5.2.1) ----------------------------------------------
 * M^k = (rho_d dV)^-1 sum over the cell's super-droplets with radius in
 * [r_min, r_max] of N r^k, for the wet (r_w) or dry (r_d) radius. */
void orc_moments(const orc_domain *d, const orc_sds *s, const double *rhod, int wet,
                 double r_min, double r_max, int k, double *out)
{
    int64_t nc = orc_n_cells(d);
    double dV = cell_volume(d);
    for (int64_t c = 0; c < nc; ++c) out[c] = 0.0;
    for (int64_t q = 0; q < s->n; ++q) {
        double r = wet ? sqrt(s->rw2[q]) : cbrt(s->rd3[q]);
        if (!(r >= r_min && r <= r_max)) continue;
        double p = 1.0;
        for (int e = 0; e < k; ++e) p *= r;
        out[orc_cell_of(d, s->x[q], s->y[q], s->z[q])] += (double)s->N[q] * p;
    }
    for (int64_t c = 0; c < nc; ++c) out[c] /= rhod[c] * dV;
}

/* Binned spectrum: the moment M^k of the diagnostics above for each of the
 * n_bins radius bins [edges[b], edges[b+1]) (READING: half-open, so that
 * every radius falls in at most one bin), out[b * n_cells + c]. */
void orc_spectrum(const orc_domain *d, const orc_sds *s, const double *rhod, int wet,
                  const double *edges, int n_bins, int k, double *out)
{
    int64_t nc = orc_n_cells(d);
    double dV = cell_volume(d);
    for (int64_t i = 0; i < nc * n_bins; ++i) out[i] = 0.0;
    for (int64_t q = 0; q < s->n; ++q) {
        double r = wet ? sqrt(s->rw2[q]) : cbrt(s->rd3[q]);
        int b = -1;
        for (int e = 0; e < n_bins; ++e)
            if (r >= edges[e] && r < edges[e + 1]) b = e;
        if (b < 0) continue;
        double p = 1.0;
        for (int e = 0; e < k; ++e) p *= r;
        out[b * nc + orc_cell_of(d, s->x[q], s->y[q], s->z[q])] += (double)s->N[q] * p;
    }
    for (int b = 0; b < n_bins; ++b)
        for (int64_t c = 0; c < nc; ++c) out[b * nc + c] /= rhod[c] * dV;
}

/* ---- Eulerian component of the kinematic framework (Sec. 2.1-2.2) ----------
 * The paper transports theta and r_v with MPDATA (libmpdata++), outside the
 * particle scheme.  READING: a first-order donor-cell (upwind) scheme stands
 * in for it, in flux form with the same rho_d C Courant fields the particles
 * use (edge arrays of the Arakawa-C grid):
 *   rho_d psi' = rho_d psi - sum over the cell's edges of the outward
 *                (rho_d C)_edge psi_up,
 * psi_up the value in the cell the flow comes from.  Periodic in x and y;
 * on a z boundary edge the value is the inside cell's (zero gradient).
 * rho_d is stationary (Sec. 2.1: the flow is divergence free in the rho_d
 * weighted sense), so psi' = (rho_d psi') / rho_d. */
static double up_flux(double C, double left, double right) { return C * (C >= 0.0 ? left : right); }

void orc_upwind(const orc_domain *d, double *psi, const double *rhod, const double *rhoCx,
                const double *rhoCy, const double *rhoCz)
{
    int64_t NX = dimn(d->nx), NY = dimn(d->ny), NZ = dimn(d->nz), nc = NX * NY * NZ;
    double *old = malloc(sizeof(double) * (size_t)nc);
    for (int64_t c = 0; c < nc; ++c) old[c] = psi[c];
    for (int64_t i = 0; i < NX; ++i)
        for (int64_t j = 0; j < NY; ++j)
            for (int64_t k = 0; k < NZ; ++k) {
                int64_t c = (i * NY + j) * NZ + k;
                double out = 0.0;  /* net outward flux of rho_d psi */
                if (d->nx > 0 && rhoCx) {
                    int64_t il = (i - 1 + NX) % NX, ir = (i + 1) % NX;
                    double Cl = rhoCx[(i * NY + j) * NZ + k], Cr = rhoCx[((i + 1) * NY + j) * NZ + k];
                    out += up_flux(Cr, old[c], old[(ir * NY + j) * NZ + k]);
                    out -= up_flux(Cl, old[(il * NY + j) * NZ + k], old[c]);
                }
                if (d->ny > 0 && rhoCy) {
                    int64_t jl = (j - 1 + NY) % NY, jr = (j + 1) % NY;
                    double Cl = rhoCy[(i * (NY + 1) + j) * NZ + k], Cr = rhoCy[(i * (NY + 1) + j + 1) * NZ + k];
                    out += up_flux(Cr, old[c], old[(i * NY + jr) * NZ + k]);
                    out -= up_flux(Cl, old[(i * NY + jl) * NZ + k], old[c]);
                }
                if (d->nz > 0 && rhoCz) {
                    double below = k > 0 ? old[c - 1] : old[c], above = k < NZ - 1 ? old[c + 1] : old[c];
                    double Cb = rhoCz[(i * NY + j) * (NZ + 1) + k], Ct = rhoCz[(i * NY + j) * (NZ + 1) + k + 1];
                    out += up_flux(Ct, old[c], above);
                    out -= up_flux(Cb, below, old[c]);
                }
                psi[c] = (rhod[c] * old[c] - out) / rhod[c];
            }
    free(old);
}

/* Relaxation of the horizontal means (Sec. 2.2): at every level the mean
 * <psi> over x (and y) moves toward the initial profile psi0 by
 *   dt (psi0 - <psi>) / tau,  tau = tau_rlx exp(z / z_rlx),
 * z at the level's cell centres, added to every cell of the level (explicit
 * Euler).  READING: the printed source term carries the opposite sign,
 * which would drive the mean away from the initial profile the text says it
 * is relaxed to. */
void orc_relax(const orc_domain *d, double *psi, const double *psi0, double tau_rlx, double z_rlx)
{
    int64_t NX = dimn(d->nx), NY = dimn(d->ny), NZ = dimn(d->nz);
    for (int64_t k = 0; k < NZ; ++k) {
        double sum = 0.0;
        for (int64_t i = 0; i < NX; ++i)
            for (int64_t j = 0; j < NY; ++j) sum += psi[(i * NY + j) * NZ + k];
        double mean = sum / (double)(NX * NY);
        double z = (k + 0.5) * d->dz;
        double tau = tau_rlx * exp(z / z_rlx);
        double inc = d->dt * (psi0[k] - mean) / tau;
        for (int64_t i = 0; i < NX; ++i)
            for (int64_t j = 0; j < NY; ++j) psi[(i * NY + j) * NZ + k] += inc;
    }
}

/* READING: super-droplet "concentration" is the count of super-droplets with
 * non-zero multiplicity in each cell. */
void orc_sd_conc(const orc_domain *d, const orc_sds *s, double *out)
{
    int64_t nc = orc_n_cells(d);
    for (int64_t c = 0; c < nc; ++c) out[c] = 0.0;
    for (int64_t q = 0; q < s->n; ++q)
        if (s->N[q] > 0) out[orc_cell_of(d, s->x[q], s->y[q], s->z[q])] += 1.0;
}
