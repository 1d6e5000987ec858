/*
 * sdm.h - C ABI of the GB300 (sm_103a) super-droplet microphysics library.
 *
 * The library advances the particle-based ("super-droplet") warm-rain scheme
 * of Arabas, Jaruga, Pawlowska & Grabowski, "libcloudph++ 0.2" (GMD 2015),
 * Sec. 5, on one GPU.  The calls restate the paper's particles_t interface
 * (Sec. 5.2.1, listings of opts_t, opts_init_t, arrinfo_t, particles_t and
 * factory()) as plain C: init, step_sync, step_async, diagnostics.
 *
 * Conventions for every entry point:
 *  - Every call returns an sdm_status; nothing is thrown across the ABI.
 *    On failure sdm_last_error(ctx) holds a one-line message (a context-less
 *    failure of sdm_init is reported by sdm_last_error(NULL)).
 *  - Eulerian fields are caller-owned float64 arrays described by sdm_arr
 *    (host or device memory).  Super-droplet state and the output buffer are
 *    library-owned device memory.
 *  - All GPU work of a context runs on the stream given to sdm_init, in
 *    issue order.  Calls on one context must not be made concurrently from
 *    several host threads.
 *  - There is no CPU fallback: without a usable CUDA device sdm_init fails
 *    with SDM_ECUDA.
 */
#ifndef SDM_H
#define SDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SDM_OK = 0,
    SDM_EINVAL = 1,   /* invalid argument (message says which)                  */
    SDM_ENOMEM = 2,   /* device or host allocation failed                       */
    SDM_ECUDA = 3,    /* a CUDA runtime call failed                             */
    SDM_ETIMEOUT = 4, /* sdm_wait deadline passed; the work is still in flight  */
    SDM_ENUMERIC = 5, /* a kernel flagged a non-finite value                    */
    SDM_ESTATE = 6,   /* call out of order (e.g. step_sync before sdm_wait)     */
    SDM_ENOTSUP = 7   /* valid but not supported by this build (message says)   */
} sdm_status;

typedef struct sdm_ctx sdm_ctx;

/* Description of a caller-owned n-dimensional float64 array, the paper's
 * arrinfo_t (Sec. 5.2.1): data_zero points at element (0,...,0); element
 * (i,j,k) is at data_zero + i*strides[0] + j*strides[1] + k*strides[2]
 * (strides in elements, one per present dimension, in (x, y, z) order).
 * data_zero == NULL means "argument absent" (arrinfo_t::is_null).
 * on_device: 0 = host memory, 1 = device memory of the context's GPU. */
typedef struct {
    double *data_zero;
    const int64_t *strides;
    int on_device;
} sdm_arr;

/* One lognormal mode of the initial dry spectrum (Sec. 2.2 eq. lognormal,
 * opts_init_t::dry_distros): mode radius [m], geometric standard deviation,
 * concentration at STP [m^-3], hygroscopicity kappa. */
typedef struct {
    double rm, sigma, n_stp, kappa;
} sdm_lognormal;

enum { SDM_KERNEL_GEOMETRIC = 0, SDM_KERNEL_GOLOVIN = 1, SDM_KERNEL_LONG = 2 };
enum { SDM_INIT_LOGNORMAL = 0, SDM_INIT_EXPONENTIAL = 1 };
enum { SDM_PRECISION_FP64 = 0, SDM_PRECISION_MIXED = 1 };
enum { SDM_BACKEND_SERIAL = 0, SDM_BACKEND_OPENMP = 1, SDM_BACKEND_CUDA = 2 };
enum { SDM_SOLVER_BISECT = 0, SDM_SOLVER_FAST = 1 };
enum { SDM_COND_AUTO = 0, SDM_COND_FUSED = 1, SDM_COND_STAGED = 2 };

/* Options fixed for the life of a simulation (opts_init_t, Sec. 5.2.1).
 * nx, ny, nz: cells per dimension, 0 = dimension absent (all 0: parcel/box,
 *   one cell); dx, dy, dz [m]; dt [s].
 * sd_conc: super-droplets per cell per distinct kappa at initialisation
 *   (sd_conc_mean); they are placed uniformly at random within each cell.
 * kernel: SDM_KERNEL_GEOMETRIC (the paper's kernel_t::geometric, E = 1),
 *   SDM_KERNEL_GOLOVIN (K = golovin_b (V_i + V_j), for the box test) or
 *   SDM_KERNEL_LONG (the geometric kernel times the Long 1974 efficiency:
 *   E = 1 for a larger radius R >= 50 um, else 4.5e8 R^2 (1 - 3e-6 / r) in
 *   SI units held within [1e-3, 1]; the paper tabulates its efficiencies,
 *   Sec. 5.1.4).  Any other value: SDM_EINVAL.
 * init_dist: SDM_INIT_LOGNORMAL uses modes[0..n_modes); SDM_INIT_EXPONENTIAL
 *   draws wet volumes from an exponential law of mean exp_mean_volume [m^3]
 *   with exp_n0 droplets per m^3 and no dry mass (box test).
 * seed: key of the counter-based random numbers (runs are reproducible).
 * physics: 0 bare Maxwell-Mason growth, 1 with the transition-regime and
 *   ventilation corrections of Sec. 5.1.3.
 * precision: SDM_PRECISION_FP64 or SDM_PRECISION_MIXED.
 * backend: must be SDM_BACKEND_CUDA (factory(), Sec. 5.2.1; the other
 *   back-ends return SDM_EINVAL).
 * cond_solver: SDM_SOLVER_BISECT runs the paper's bisection (Sec. 5.1.3) in
 *   FP64 throughout; SDM_SOLVER_FAST (the default in the bindings) takes the
 *   same bracket, the same midpoints and the same sign decisions, decided in
 *   FP32 where an error bound proves the sign, then finishes with a
 *   bracketed FP64 Newton/secant iteration to the same sign change.
 * cond_layout: how the fast FP64 condensation runs on the GPU:
 *   SDM_COND_FUSED, one kernel per step carrying every solve;
 *   SDM_COND_STAGED, per substep a chain of small kernels (FP32 starts,
 *   rounds of FP64 evaluations over compacted lists, the cell sums), whose
 *   solves also settle on Newton steps with a certified error below 2^-43
 *   of r_w^2 and take the ventilation factors in FP32 where that moves the
 *   result by less than 2^-45 (both layouts stay within 1e-12 of the
 *   bisection's root); SDM_COND_AUTO (0): staged from 2^17 super-droplets,
 *   else fused.  Other solvers and the mixed mode always run fused.
 * sd_reserve: extra super-droplet slots (N = 0) beyond the initial ones,
 *   kept free for arrivals from the neighbouring slabs of an x_open context
 *   (sdm_import): their ids carry the top bit (2^31), which marks a slot
 *   recycling leaves alone.  0 by default.
 * x_open: 0 (default): periodic in x.  1: the context is one slab of a
 *   domain decomposed in x (the paper has no counterpart; in its calling
 *   sequence, Sec. 5.2, decomposition is the solver's): super-droplets advected past x = 0 or
 *   x = nx dx keep their position, outside [0, nx dx), until
 *   sdm_export_leavers takes them out, and the Courant numbers of the two
 *   boundary edges divide by the rho_d of their one adjacent cell. */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, dt;
    int sd_conc;
    int kernel;
    double golovin_b;
    int init_dist;
    double exp_mean_volume, exp_n0;
    int n_modes;
    const sdm_lognormal *modes;
    uint64_t seed;
    int physics;
    int precision;
    int backend;
    int cond_solver;
    int x_open;
    int cond_layout;
    int64_t sd_reserve;
} sdm_opts_init;

/* Per-step options (opts_t, Sec. 5.2.1; defaults 1,1,1,1, 44, 10, 10, 0, 0):
 * process toggles, RH limit for drop growth, substep counts.
 * coal_multi = 0 is the paper's scheme: a pair with P_ij > 1 still has one
 * collision event (Sec. 5.1.4).  coal_multi = 1 turns on the multiple
 * coalescence that Sec. 5.1.4 plans (Shima et al. 2009, Sec. 4.1.4 there):
 * gamma = floor(P_ij) events, plus one when the pair's uniform number is
 * below P_ij - floor(P_ij), at most floor(N_L / N_S); the merged droplet
 * takes gamma droplets of the larger-multiplicity super-droplet.  Where
 * every P_ij <= 1 both give the same result bit for bit.
 * coal_adapt > 0 turns on adaptive coalescence substeps, the substep control
 * from P_ij that Sec. 5.1.4 also plans: per cell and step, from an upper
 * bound of P_ij over every pair the cell could form at the start of the step
 * (largest multiplicity, largest radius, terminal-velocity range),
 * max(sstp_coal, ceil(P_bound)) substeps, at most coal_adapt.  0 keeps
 * sstp_coal everywhere.  Single contexts only: sdm_ens_step returns
 * SDM_EINVAL for coal_adapt > 0 (its substeps are one captured graph). */
typedef struct {
    int adve, sedi, cond, coal;
    double RH_max;
    int sstp_cond, sstp_coal;
    int coal_multi;
    int coal_adapt;
} sdm_opts;

/* Counters accumulated since sdm_init (or the last sdm_stats_reset). */
typedef struct {
    uint64_t n_pairs;       /* candidate pairs examined                        */
    uint64_t n_coll;        /* collision events                                */
    uint64_t n_pgt1;        /* pairs with P_ij > 1 (no multiple coalescence)    */
    uint64_t n_recycled;    /* zero-multiplicity super-droplets re-populated   */
    uint64_t n_euler;       /* growth solves that took the Euler branch        */
    uint64_t n_fallback;    /* growth solves finished by full bisection        */
    uint64_t n_steps;       /* completed step_async calls                      */
    uint64_t n_zero;        /* multiplicity-zero super-droplets now            */
    double max_p;           /* largest P_ij seen                               */
    double rainfall;        /* liquid mass through the bottom [kg]              */
    uint64_t n_coal_substeps; /* cell-substeps of coalescence taken (cells x
                                 substeps summed over steps; single contexts,
                                 0 for ensembles)                              */
} sdm_stats;

/* Per-phase device time [ms] accumulated while timing is on; measured with
 * CUDA events on the context's stream around each group of launches.
 * cond_launches and coal_launches count the calls of the condensation and
 * coalescence phases (each a chain of one or more kernels: cond_ms /
 * cond_launches is one condensation call's time); launches counts the
 * particle scheme's kernels (steps and diagnostics); euler_ms and
 * euler_launches the Eulerian stand-in (sdm_euler_step), which is the
 * driver's part, apart. */
typedef struct {
    double cond_ms, recycle_ms, move_ms, sort_ms, coal_ms, diag_ms, copy_ms;
    uint64_t cond_launches, coal_launches, launches;
    double euler_ms;
    uint64_t euler_launches;
} sdm_timing;

/* ---- life cycle --------------------------------------------------------- */

/* factory() + particles_t::init (Sec. 5.2.1, 5.1.6): allocate the
 * super-droplets on the device and initialise them from the dry spectrum
 * (or the exponential box spectrum), at Koehler equilibrium with the cell
 * humidity (RH = 0.95 where supersaturated).
 * th, rv, rhod: theta [K], r_v [kg/kg], rho_d [kg/m^3] on cell centres,
 *   shape (nx, ny, nz) without absent dimensions (one value for a box).
 * rhoCx, rhoCy, rhoCz: rho_d times the Courant number on Arakawa-C edges,
 *   shapes (nx+1, ny, nz), (nx, ny+1, nz), (nx, ny, nz+1); absent (NULL
 *   data_zero) where the dimension is absent or the flow is zero.
 * stream: cudaStream_t to use (NULL: the library creates one).
 * out: receives the new context.  SDM_EINVAL on bad options, SDM_ENOMEM
 *   if the state does not fit, SDM_ECUDA without a usable GPU. */
sdm_status sdm_init(const sdm_opts_init *opts, sdm_arr th, sdm_arr rv, sdm_arr rhod,
                    sdm_arr rhoCx, sdm_arr rhoCy, sdm_arr rhoCz, void *stream, sdm_ctx **out);

/* Free all device memory of the context (waits for its stream first). */
sdm_status sdm_destroy(sdm_ctx *ctx);

/* Last error message of ctx (or of the last failed sdm_init for NULL). */
const char *sdm_last_error(const sdm_ctx *ctx);

/* ---- time stepping ------------------------------------------------------ */

/* particles_t::step_sync (Sec. 5.1.3, 5.2.1): condensation/evaporation in
 * sstp_cond substeps, each an implicit-in-r_w^2 growth solve per
 * super-droplet followed by the per-cell update of r_v and theta, eq.
 * (rhov_update).  th and rv are read and overwritten.  rhoCx/y/z, when
 * present, replace the flow used by the next step_async; rhod, when present,
 * replaces rho_d.  Host arrays are complete when the call returns; device
 * arrays are complete in stream order.  SDM_ESTATE if a step_async has not
 * been waited for. */
sdm_status sdm_step_sync(sdm_ctx *ctx, const sdm_opts *opts, sdm_arr th, sdm_arr rv,
                         sdm_arr rhoCx, sdm_arr rhoCy, sdm_arr rhoCz, sdm_arr rhod);

/* particles_t::step_async (Sec. 5.1.2, 5.1.4, 5.1.5): recycling of
 * zero-multiplicity super-droplets, advection, sedimentation, regrouping by
 * cell and sstp_coal substeps of Monte-Carlo coalescence.  Enqueues the work
 * and returns; sdm_wait completes it. */
sdm_status sdm_step_async(sdm_ctx *ctx, const sdm_opts *opts);

/* Wait at most timeout_s seconds (< 0: no limit) for the context's stream.
 * rainfall_out (nullable) receives the accumulated rainfall [kg] (the paper's
 * step_async return value).  SDM_ETIMEOUT leaves the work in flight.
 * SDM_ENOTSUP if a cell held more than 8192 super-droplets in a context whose
 * initial cells hold at most 8192 (such a context reserves no scratch for
 * larger cells; one initialised with larger cells reserves 48 bytes per
 * super-droplet and pairs any cell). */
sdm_status sdm_wait(sdm_ctx *ctx, double timeout_s, double *rainfall_out);

/* ---- the kinematic framework's Eulerian component (Sec. 2.1-2.2) --------
 * Not part of the particle scheme: the paper's driver transports theta and
 * r_v with MPDATA (libmpdata++).  This stand-in lets a driver of this
 * library run the ICMW set-up on the device:
 *   advect: one first-order donor-cell (upwind) step of theta and r_v in
 *     flux form with the same rho_d C Courant fields (Arakawa-C edge arrays,
 *     as for sdm_step_sync): rho_d psi' = rho_d psi - sum over the cell's
 *     edges of the outward (rho_d C)_edge psi_up, psi_up taken in the cell
 *     the flow comes from; periodic in x and y, a z boundary edge takes the
 *     inside cell's value; rho_d is stationary (Sec. 2.1);
 *   relax: then each level's horizontal mean moves toward the initial
 *     profile, psi += dt (psi0 - <psi>) / tau, tau = tau_rlx exp(z / z_rlx),
 *     z at the level's cell centres (Sec. 2.2: 300 s and 200 m).
 * th0, rv0: host arrays of nz values (nz = 1 without a z dimension). */
typedef struct {
    int advect, relax;
    double tau_rlx, z_rlx;
    const double *th0, *rv0;
} sdm_euler_opts;

/* One Eulerian step on the caller's theta and r_v (host or device arrays,
 * overwritten; complete on return for host arrays, ordered on the context's
 * stream for device ones).  SDM_ESTATE while step_async is in flight;
 * SDM_EINVAL for missing fields, or relaxation without profiles or with a
 * non-positive time or height scale.  Allocates two small device buffers on
 * its first call. */
sdm_status sdm_euler_step(sdm_ctx *ctx, const sdm_euler_opts *opts, sdm_arr th, sdm_arr rv, sdm_arr rhoCx,
                          sdm_arr rhoCy, sdm_arr rhoCz);

/* ---- diagnostics (Sec. 5.2.1, diag_* and outbuf) ------------------------ */

/* Select super-droplets with wet (wet=1) or dry (wet=0) radius in
 * [r_min, r_max] for the following sdm_diag_mom calls. */
sdm_status sdm_diag_rng(sdm_ctx *ctx, int wet, double r_min, double r_max);

/* k-th moment (0 <= k <= 8) per cell, M = (rho_d dV)^-1 sum N r^k over the
 * selected super-droplets, into the output buffer.  SDM_ESTATE before the
 * first sdm_diag_rng. */
sdm_status sdm_diag_mom(sdm_ctx *ctx, int k);

/* Number of super-droplets with non-zero multiplicity per cell, into the
 * output buffer. */
sdm_status sdm_diag_sd_conc(sdm_ctx *ctx);

/* The ambient state per cell that the condensation solve sees (Appendix A:
 * T and p diagnosed from theta, r_v and rho_d; Sec. 5.1.3: the saturation
 * vapour density), from the context's current theta, r_v and rho_d, into
 * the output buffer.  what: 0 = T [K], 1 = p [Pa], 2 = rho_vs [kg m^-3],
 * 3 = RH = rho_v / rho_vs (not capped by RH_max).  SDM_EINVAL for another
 * value. */
sdm_status sdm_diag_ambient(sdm_ctx *ctx, int what);

/* Copy the output buffer (n_cells float64, row-major (x, y, z)) to dst,
 * host (dst_on_device = 0, complete on return) or device memory. */
sdm_status sdm_outbuf(sdm_ctx *ctx, double *dst, int dst_on_device);

/* Binned spectrum: the moment of sdm_diag_mom (Sec. 5.2.1) for n_bins
 * radius bins in one pass,
 *   dst[b * n_cells + c] = (rho_d dV)^-1 sum N r^k
 * over the super-droplets of cell c whose wet (wet = 1) or dry (wet = 0)
 * radius lies in [edges[b], edges[b+1]) (half-open: a radius falls in at
 * most one bin).  edges: host array of n_bins + 1 strictly increasing radii
 * [m], edges[0] >= 0; 1 <= n_bins <= 256; 0 <= k <= 8 (SDM_EINVAL
 * otherwise).  dst:
 * n_bins * n_cells float64, bin-major, in host memory (dst_on_device = 0;
 * complete on return) or device memory (ordered on the context's stream).
 * Leaves the output buffer and the sdm_diag_rng selection untouched.  A
 * call with more bins than every earlier one allocates the context's
 * spectrum buffer (n_bins * n_cells float64), kept until sdm_destroy. */
sdm_status sdm_diag_spectrum(sdm_ctx *ctx, int wet, const double *edges, int n_bins, int k, double *dst,
                             int dst_on_device);

/* ---- state access (tests, checkpoint / resume) --------------------------- */

enum {
    SDM_ATTR_N = 0,     /* uint64 multiplicity               */
    SDM_ATTR_RW2 = 1,   /* float64 wet radius squared [m^2]  */
    SDM_ATTR_RD3 = 2,   /* float64 dry radius cubed [m^3]    */
    SDM_ATTR_KAPPA = 3, /* float64 hygroscopicity            */
    SDM_ATTR_X = 4,     /* float64 positions [m]             */
    SDM_ATTR_Y = 5,
    SDM_ATTR_Z = 6,
    SDM_ATTR_UID = 7    /* uint32 super-droplet id           */
};

/* Number of super-droplets and cells of the context. */
sdm_status sdm_sizes(const sdm_ctx *ctx, int64_t *n_sd, int64_t *n_cells);

/* Copy one attribute of all n_sd super-droplets (storage order, the same for
 * every attribute) to host memory dst (n elements, n == n_sd).  Completes
 * before returning. */
sdm_status sdm_get_attr(sdm_ctx *ctx, int attr, void *dst, int64_t n);

/* Overwrite one attribute from host memory (storage order as returned by
 * sdm_get_attr).  Positions changed this way regroup the super-droplets at
 * the next step, diagnostic or sdm_get_attr, not before: a checkpoint
 * (every attribute from sdm_get_attr, the step from sdm_get_step, theta and
 * r_v) restores into any context of the same set-up through sdm_set_attr
 * calls in any order and sdm_set_step, and the run then continues bit for
 * bit as if uninterrupted. */
sdm_status sdm_set_attr(sdm_ctx *ctx, int attr, const void *src, int64_t n);

/* Copy the library's current theta and r_v (n_cells each) to host memory. */
sdm_status sdm_get_fields(sdm_ctx *ctx, double *th, double *rv);

/* Step counter used in the random-number counters (completed step_async
 * calls); set it to resume a checkpointed run bit-identically. */
sdm_status sdm_get_step(const sdm_ctx *ctx, uint64_t *step);
sdm_status sdm_set_step(sdm_ctx *ctx, uint64_t step);

/* ---- decomposed domains: the exchange of super-droplets between slabs ----
 * The paper's library holds one domain and leaves decomposition to the
 * solver that calls it (Sec. 5.2, example calling sequence); these calls are
 * the device side of the exchange a
 * sharded driver needs (the paper has no counterpart).  With x_open set, a
 * timestep is: sdm_step_sync; sdm_step_transport (recycling, advection,
 * sedimentation); sdm_export_leavers, the exchange with the neighbouring
 * slabs (decomp.exchange in the Python package), sdm_import; then
 * sdm_step_coalesce (regrouping and coalescence) and sdm_wait.  Without
 * exports or imports sdm_step_transport + sdm_step_coalesce give the
 * results of sdm_step_async bit for bit. */

/* A block of super-droplets in flight between contexts: n entries per array.
 * y or z may be NULL when the context lacks that dimension.  on_device: 1 =
 * device memory of the context's GPU, 0 = host memory. */
typedef struct {
    uint64_t *N;
    uint32_t *uid;
    double *rw2, *rd3, *kappa, *x, *y, *z;
    int on_device;
} sdm_sd_block;

/* The first half of sdm_step_async: recycling of zero multiplicities,
 * advection and sedimentation with exits (Sec. 5.1.2, 5.1.4, 5.1.5),
 * enqueued on the context's stream.  SDM_ESTATE while an sdm_step_async or
 * sdm_step_coalesce is in flight or a transport is pending. */
sdm_status sdm_step_transport(sdm_ctx *ctx, const sdm_opts *opts);

/* The second half: regrouping by cell (from the positions, if super-droplets
 * were exported or imported in between) and sstp_coal coalescence substeps
 * (opts->coal), then the step counter advances; complete with sdm_wait.
 * SDM_ESTATE without a pending sdm_step_transport. */
sdm_status sdm_step_coalesce(sdm_ctx *ctx, const sdm_opts *opts);

/* Take out every super-droplet with N > 0 and x outside [0, nx dx) (only
 * an x_open context has such): their attributes go to dst, in storage
 * order, and their slots are left with N = 0 for sdm_import to fill; the
 * emptied slot's id gets the top bit (2^31), the mark of a slot
 * that recycling leaves to arrivals (the leaver keeps its id, which must
 * stay unique among live super-droplets).  cap: the block's room; *n_out:
 * how many were taken.  Completes
 * before returning.  SDM_ENOMEM (nothing taken, *n_out the number waiting)
 * if cap is too small, SDM_EINVAL if the context is not x_open. */
sdm_status sdm_export_leavers(sdm_ctx *ctx, sdm_sd_block dst, int64_t cap, int64_t *n_out);

/* Put n super-droplets (attributes as sdm_export_leavers writes them, x
 * already in this context's coordinates, [0, nx dx); ids below 2^31) into
 * slots with N = 0, the k-th into the k-th such slot in storage order.  Completes before
 * returning.  SDM_ENOMEM (nothing written) if fewer than n slots are free,
 * SDM_EINVAL for a position outside the domain. */
sdm_status sdm_import(sdm_ctx *ctx, sdm_sd_block src, int64_t n);

/* ---- regrouping of caller-held particles -------------------------------- */

/* Counting sort of particles by grid cell, the regrouping that the cell-wise
 * pairing (Sec. 5.1.4) and cell sums (Sec. 5.1.3, eq. rhov_update) rest on.
 * cell: n cell indices in [0, n_cells) (device memory, uint32).
 * perm: out, n particle indices grouped by cell (device); the order within
 *   a cell is unspecified.  offsets: out, n_cells + 1 entries (device):
 *   cell c holds perm[offsets[c] .. offsets[c+1]).
 * Work runs on stream (cudaStream_t, NULL = legacy default stream); scratch
 * is allocated and freed on that stream; the call completes before it
 * returns.  SDM_EINVAL if a cell index is out of range (nothing is written
 * for it) or an argument is invalid, SDM_ENOMEM if scratch is unavailable. */
sdm_status sdm_cell_sort(const uint32_t *cell, int64_t n, int32_t n_cells, uint32_t *perm,
                         uint32_t *offsets, void *stream);

/* The same sort for callers that cannot allocate device memory while they
 * run (inside a captured CUDA graph, in a stream-ordered region where a
 * cudaMalloc would synchronise, or under a memory pool fixed at start-up).
 * The paper has no counterpart: this is a systems variant of the call above.
 * It allocates nothing: its scratch is one fixed file-scope device array of
 * about 10 MB, reserved on every GPU that loads the library until the
 * process exits.  Limits: n <= 2097152 particles and n_cells <= 524288
 * cells per call, else SDM_EINVAL (message in sdm_last_error(NULL)).
 * A call outside stream capture resolves the array's device address on the
 * current device (a cudaDeviceReset may move it); a call inside a capture
 * uses the address the last uncaptured call on that device resolved, so make
 * the first call on a device, and the first after a cudaDeviceReset, before
 * any stream capture.  The work is only enqueued on stream: nothing is
 * synchronised.  All calls share the one array, so calls whose work overlaps
 * on the GPU (other streams, other host threads) race; order them on one
 * stream.  Cell indices out of range are skipped, not written: then
 * offsets[n_cells] < n. */
sdm_status sdm_cell_sort_noalloc(const uint32_t *cell, int64_t n, int32_t n_cells, uint32_t *perm,
                                 uint32_t *offsets, void *stream);

/* ---- device probe ------------------------------------------------------- */

/* What sdm_probe_device measures on the current device. */
typedef struct {
    int n_sm;                     /* multiprocessors (cudaDevAttrMultiProcessorCount)          */
    int blocks;                   /* blocks of the probe launch (n_sm x resident blocks per SM) */
    double fp64_tflops_burst;     /* FP64 FMA throughput, best of 5 launches of ~20 ms [TFLOP/s] */
    double fp64_tflops_sustained; /* the same over back-to-back launches for sustained_s       */
    double sustained_s;           /* length of the sustained measurement [s]                    */
} sdm_device_peaks;

/* Measures the FP64 arithmetic throughput of the current device with chains
 * of independent fused multiply-adds (2 flops each), on a stream of its own,
 * timed with CUDA events: the ceiling for the FP64-bound condensation solve
 * (Sec. 5.1.3).  The paper has no counterpart: a measurement utility.
 * sustain_s in [0, 60]: length of the back-to-back run (0 skips it).  It
 * allocates a few KB of device memory and frees it, and synchronises its own
 * stream.  SDM_EINVAL for bad arguments, SDM_ECUDA if a CUDA call fails
 * (message in sdm_last_error(NULL)). */
sdm_status sdm_probe_device(double sustain_s, sdm_device_peaks *out);

/* Counters (completes the stream first). */
sdm_status sdm_get_stats(sdm_ctx *ctx, sdm_stats *out);

/* Turn per-phase CUDA-event timing on (1) or off (0); read and reset it. */
sdm_status sdm_timing_enable(sdm_ctx *ctx, int on);
sdm_status sdm_get_timing(sdm_ctx *ctx, sdm_timing *out, int reset);

/* ---- batched ensembles of 0D members -------------------------------------
 * Many independent box or adiabatic-parcel simulations (the particles_t
 * parcel set-up, nx = ny = nz = 0, Sec. 5.2.1) advanced together by one set
 * of launches per step, capturable as one CUDA graph.  Each member draws its
 * random numbers from its own seed, ids and step count, so its result does
 * not depend on which other members share the batch.  Parcels conserve
 * their dry-air mass: a new rho_d changes their volume to m_d / rho_d. */
typedef struct sdm_ens sdm_ens;

/* One member.  n_sd super-droplets in one cell of volume dV [m^3] at theta,
 * r_v, rho_d; initial spectrum as in sdm_opts_init (1..4 lognormal modes
 * that share one kappa, or the exponential box spectrum); seed keys its
 * random numbers. */
typedef struct {
    int64_t n_sd;
    double dV;
    double th, rv, rhod;
    int init_dist;
    int n_modes;
    sdm_lognormal modes[4];
    double exp_mean_volume, exp_n0;
    uint64_t seed;
} sdm_member;

/* Options shared by the members (see sdm_opts_init) and the capacity of the
 * device arena: at most max_sd super-droplets and max_members members are
 * resident at a time; sdm_ens_create reserves the memory for them. */
typedef struct {
    double dt;
    int kernel;
    double golovin_b;
    int physics, precision, cond_solver;
    int64_t max_sd;
    int32_t max_members;
} sdm_ens_opts;

sdm_status sdm_ens_create(const sdm_ens_opts *opts, void *stream, sdm_ens **out);
sdm_status sdm_ens_destroy(sdm_ens *e);
/* The device memory the ensemble's arena reserved at creation (held until
 * sdm_ens_destroy), its capacity in super-droplets and in members: what a
 * server admits requests against.  A repacking after removals also takes,
 * for its duration, a few bytes per member more.  The paper has no
 * counterpart (serving). */
sdm_status sdm_ens_memory(const sdm_ens *e, size_t *device_bytes, int64_t *cap_sd, int32_t *cap_members);
const char *sdm_ens_last_error(const sdm_ens *e);

/* Admit a member (initialised on the device, Sec. 5.1.6); *id receives its
 * handle.  SDM_ENOMEM when the arena cannot hold it (nothing changes). */
sdm_status sdm_ens_add(sdm_ens *e, const sdm_member *m, int32_t *id);

/* Retire a member; its memory is reused from the next step on. */
sdm_status sdm_ens_remove(sdm_ens *e, int32_t id);

/* Ids of the resident members (up to cap) and their count, and the number
 * of resident super-droplets. */
sdm_status sdm_ens_members(const sdm_ens *e, int32_t *ids, int32_t cap, int32_t *n, int64_t *n_sd);

/* One full timestep of every resident member: recycling, sstp_cond
 * condensation substeps with the per-member vapour/theta feedback,
 * sstp_coal coalescence substeps (opts->adve and opts->sedi have no meaning
 * in 0D).  ids/rhod (n entries, host memory, nullable) give a new rho_d for
 * some members before the step (parcels).  Enqueues and returns. */
sdm_status sdm_ens_step(sdm_ens *e, const sdm_opts *opts, const int32_t *ids, const double *rhod,
                        int32_t n);

/* Wait at most timeout_s seconds (< 0: no limit) for the last step. */
sdm_status sdm_ens_wait(sdm_ens *e, double timeout_s);

/* Per-member moments (as sdm_diag_mom, per unit dry-air mass) into host
 * out[n] for the listed ids; completes before returning. */
sdm_status sdm_ens_moments(sdm_ens *e, int wet, double r_min, double r_max, int k, const int32_t *ids,
                           double *out, int32_t n);

/* Current theta and r_v of the listed members (host arrays). */
sdm_status sdm_ens_fields(sdm_ens *e, const int32_t *ids, double *th, double *rv, int32_t n);

/* One attribute (SDM_ATTR_N, _RW2, _RD3, _KAPPA, _UID) of one member's
 * super-droplets, in id order, into host dst (n = the member's n_sd). */
sdm_status sdm_ens_get_attr(sdm_ens *e, int32_t id, int attr, void *dst, int64_t n);

/* Replay steps from a captured CUDA graph (1) or launch them one by one
 * (0, the default).  The graph is re-captured when membership or options
 * change. */
sdm_status sdm_ens_use_graph(sdm_ens *e, int on);

/* Choose the launch shapes by timing candidates on the resident members
 * (their state and counters are restored afterwards): the condensation tile
 * size and block size (one substep's solves), then, if opts->coal, the
 * block size of the coalescence pair kernel (one substep's keys, sort and
 * pairs).  A captured step graph is dropped and re-captured at the next
 * step.  Outputs may be NULL.  The paper has no counterpart (batching). */
sdm_status sdm_ens_autotune(sdm_ens *e, const sdm_opts *opts, int *tile_out, int *threads_out,
                            int *pair_threads_out);

/* Counters accumulated over all members since creation. */
sdm_status sdm_ens_stats(sdm_ens *e, sdm_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* SDM_H */
