/*
 * CPU oracle for the super-droplet (particle-based) warm-rain scheme of
 * Arabas, Jaruga, Pawlowska & Grabowski, "libcloudph++ 0.2", Sec. 5.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  This is a plain, serial,
 * double-precision restatement of the paper's equations used to check the
 * CUDA library.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load it.  It shares no code with the
 * CUDA library and includes none of its headers.
 *
 * Super-droplet storage: structure of arrays with an explicit 64-bit id per
 * super-droplet.  The oracle never relies on storage order: cell membership
 * comes from positions, and every order-dependent choice is made by id.
 */
#ifndef SDM_ORACLE_H
#define SDM_ORACLE_H
#include <stdint.h>

#define ORC_MAX_MODES 8

typedef struct {
    double rm;    /* lognormal mode radius [m]                       */
    double sigma; /* geometric standard deviation [1]                 */
    double n_stp; /* concentration at STP [m^-3]                       */
    double kappa; /* hygroscopicity [1]                                */
} orc_mode;

typedef struct {
    int nx, ny, nz;                /* cells per dimension; 0 = dimension absent */
    double dx, dy, dz, dt;         /* grid steps [m], timestep [s]             */
    int sd_conc;                   /* super-droplets per cell per kappa group  */
    int kernel;                    /* 0 geometric (E = 1), 1 Golovin, 2 Long    */
    double golovin_b;              /* Golovin constant [s^-1]                  */
    int init_dist;                 /* 0 lognormal dry modes, 1 exp. wet volume  */
    double exp_mean_volume;        /* mean droplet volume [m^3]  (init_dist 1) */
    double exp_n0;                 /* droplet concentration [m^-3] (init_dist 1) */
    int n_modes;
    orc_mode modes[ORC_MAX_MODES];
    uint64_t seed;
    int physics;                   /* 0 bare Maxwell-Mason, 1 with corrections */
} orc_domain;

typedef struct {
    int adve, sedi, cond, coal;
    double RH_max;
    int sstp_cond, sstp_coal;
    int coal_multi;                /* 1: multiple coalescence for P_ij > 1      */
    int coal_adapt;                /* > 0: adaptive coalescence substeps, at most this many */
} orc_opts;

typedef struct {
    uint64_t n_pairs, n_coll, n_pgt1, n_recycled, n_euler, n_bisect;
    double max_p;
    double rainfall;
    uint64_t n_coal_substeps;      /* cell-substeps of coalescence taken        */
} orc_stats;

typedef struct {
    int64_t n;
    uint64_t *uid, *N;
    double *rw2, *rd3, *kappa, *x, *y, *z;
} orc_sds;

/* per-cell thermodynamic state (Appendix A and Sec. 5.1.3) */
typedef struct {
    double th, rv, rhod;
    double T, p, lv, rho_v, rho_vs, rho_v_eff, dth_drv, A, Dterm;
    double rho_a, mu, nu, lambda_D, lambda_K, Sc, Pr, cX;
} orc_thermo;

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
double orc_u01(uint64_t v);
int orc_threads(int n);  /* threads of the -fopenmp build (n > 0 sets them); 1 otherwise */

int64_t orc_n_cells(const orc_domain *d);
int orc_n_groups(const orc_domain *d);
int64_t orc_cell_of(const orc_domain *d, double x, double y, double z);

void orc_thermo_eval(double th, double rv, double rhod, double RH_max, orc_thermo *t);
double orc_reynolds(double rw2, const orc_thermo *t);
double orc_vterm(double rw2, const orc_thermo *t);
double orc_growth(double x, double rd3, double kappa, const orc_thermo *t, int physics);
double orc_solve_rw2(double x0, double rd3, double kappa, const orc_thermo *t, double dtp,
                     int physics, orc_stats *st);
void orc_solve_batch(int64_t n, const double *x0, const double *rd3, const double *kappa,
                     const int64_t *cell, const double *th, const double *rv, const double *rhod,
                     double RH_max, double dtp, int physics, double *x1);
double orc_equilibrium_rw2(double rd3, double kappa, double RH, double T);

int orc_rd_range(const orc_domain *d, int group, double *lnr_min, double *lnr_max);
int orc_init_cells(const orc_domain *d, const double *th, const double *rv, const double *rhod,
                   int64_t n_list, const int64_t *cells, orc_sds *out);
int orc_init_cells_nreal(const orc_domain *d, const double *th, const double *rv,
                         const double *rhod, int64_t n_list, const int64_t *cells, orc_sds *out,
                         double *nreal);

void orc_condense(const orc_domain *d, const orc_opts *o, orc_sds *s, double *th, double *rv,
                  const double *rhod, orc_stats *st);
void orc_recycle(orc_sds *s, orc_stats *st);
void orc_advect(const orc_domain *d, orc_sds *s, const double *rhod, const double *rhoCx,
                const double *rhoCy, const double *rhoCz);
void orc_transport(const orc_domain *d, const orc_opts *o, orc_sds *s, const double *th,
                   const double *rv, const double *rhod, const double *rhoCx,
                   const double *rhoCy, const double *rhoCz, orc_stats *st);
void orc_coalesce(const orc_domain *d, const orc_opts *o, orc_sds *s, const double *th,
                  const double *rv, const double *rhod, uint64_t step, orc_stats *st);
void orc_step_sync(const orc_domain *d, const orc_opts *o, orc_sds *s, double *th, double *rv,
                   const double *rhod, orc_stats *st);
void orc_step_async(const orc_domain *d, const orc_opts *o, orc_sds *s, const double *th,
                    const double *rv, const double *rhod, const double *rhoCx,
                    const double *rhoCy, const double *rhoCz, uint64_t step, orc_stats *st);
void orc_parcel_step(orc_domain *d, const orc_opts *o, orc_sds *s, double *th, double *rv, double *rhod,
                     double m_d, double rhod_new, uint64_t step, orc_stats *st);
void orc_moments(const orc_domain *d, const orc_sds *s, const double *rhod, int wet,
                 double r_min, double r_max, int k, double *out);
void orc_sd_conc(const orc_domain *d, const orc_sds *s, double *out);
void orc_upwind(const orc_domain *d, double *psi, const double *rhod, const double *rhoCx,
                const double *rhoCy, const double *rhoCz);
void orc_relax(const orc_domain *d, double *psi, const double *psi0, double tau_rlx, double z_rlx);
void orc_spectrum(const orc_domain *d, const orc_sds *s, const double *rhod, int wet,
                  const double *edges, int n_bins, int k, double *out);

#endif
