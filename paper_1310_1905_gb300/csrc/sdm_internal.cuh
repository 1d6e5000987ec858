// Internal declarations of the super-droplet library (sm_103a).
//
// Device physics restates the paper (Arabas et al., libcloudph++ 0.2):
// Sec. 5.1.3 (phase changes), 5.1.4 (coalescence), 5.1.5 (sedimentation),
// 5.1.6 (initialisation), Appendix A (T, p from theta, r_v, rho_d) and the
// list of symbols.  Where the paper is silent the library takes the same
// readings as its test oracle (listed in the project's design notes).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/sdm.h"

#define SDM_HD __host__ __device__ __forceinline__

namespace sdm {

// ---------------------------------------------------------------- constants
// list of symbols: rho_w, sigma_w, c_pd, c_pv, c_l, l_v0; the rest are the
// library's readings of values the paper does not print
namespace phys {
constexpr double pi = 3.14159265358979323846;
constexpr double rho_w = 1000.0, sigma_w = 0.072;
constexpr double c_pd = 1005.0, c_pv = 1850.0, c_l = 4218.0, l_v0 = 2.5e6;
constexpr double R_d = 287.0, R_v = 461.5;
constexpr double T0 = 273.16, p_vs0 = 611.73, grav = 9.81, p1000 = 1.0e5;
constexpr double D0 = 2.26e-5, K0 = 2.4e-2;
constexpr double delta0 = 9.06, C0 = 0.292;
constexpr double rho_stp = 101325.0 / (R_d * 293.15);
}  // namespace phys

constexpr int kMaxModes = 8;
constexpr int kBigCellCap = 8192;  // largest cell handled by the block path

// ---------------------------------------------------------------- RNG
// Philox4x64-10 (Salmon et al., SC'11): counter (id, substep, step, stream)
// under key (seed, 0); streams: 1 coalescence, 3 initialisation.
enum { kStreamCoal = 1, kStreamInit = 3 };

struct u64x4 {
    uint64_t v[4];
};

__device__ __forceinline__ u64x4 philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                            uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t h0 = __umul64hi(M0, c0), l0 = M0 * c0;
        const uint64_t h1 = __umul64hi(M1, c2), l1 = M1 * c2;
        const uint64_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
    }
    u64x4 o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}

// open-interval (0,1) uniform: 52 random bits plus one half, times 2^-52
SDM_HD double u01(uint64_t v) {
    return ((double)(v >> 12) + 0.5) * 0x1p-52;
}

// ---------------------------------------------------------------- thermo
struct Thermo {
    double th, rv, rhod;
    double T, lv, rho_v, rho_vs, rho_v_eff, dth_drv, A, Dterm;
    double rho_a, nu, lambda_D, lambda_K, Sc, Pr, cX;
};

// 1 / sqrt(x): the device's reciprocal square root (host builds, used by
// test harnesses, divide)
SDM_HD double rsqrt_hd(double x) {
#ifdef __CUDA_ARCH__
    return rsqrt(x);
#else
    return 1.0 / sqrt(x);
#endif
}

// (rho_d R_d / p1000)^(R_d / c_pd): the rho_d factor of T in Appendix A,
// constant over a step (rho_d changes only between steps)
SDM_HD double rhod_factor(double rhod) {
    using namespace phys;
    return pow(rhod * R_d / p1000, R_d / c_pd);
}

// Appendix A: T and p from theta, r_v, rho_d; Sec. 5.1.3 quantities.
// cond = true (the condensation kernels): T, rho_vs, A and dtheta/dr_v take
// exactly the operations below, since the growth rate's cancellation and the
// theta update depend on their last bits; the air's transport properties
// (mu, nu, lambda_D, lambda_K, Sc, Pr, c_X) and Dterm, which only scale
// D_eff, use reciprocals and x sqrt(x) for (T/273)^1.5 and so differ from
// the cond = false values (the coalescence ambient) by rounding.
template <bool cond = false>
SDM_HD Thermo thermo_eval_f(double th, double rv, double rhod, double RH_max, double rhod_f) {
    using namespace phys;
    Thermo t;
    t.th = th;
    t.rv = rv;
    t.rhod = rhod;
    t.T = pow(th * rhod_f, c_pd / (c_pd - R_d));
    t.lv = l_v0 + (c_pv - c_l) * (t.T - T0);
    const double rT = 1.0 / t.T;
    // Clausius-Clapeyron integrated with the linear l_v(T)
    const double lnp = (l_v0 + (c_l - c_pv) * T0) / R_v * (1.0 / T0 - rT) -
                       (c_l - c_pv) / R_v * log(t.T / T0);
    t.rho_vs = p_vs0 * exp(lnp) / (R_v * t.T);
    t.rho_v = rv * rhod;
    t.rho_v_eff = fmin(t.rho_v, RH_max * t.rho_vs);
    t.dth_drv = -th * t.lv / (c_pd * t.T);
    t.A = 2.0 * sigma_w / (R_v * t.T * rho_w);
    t.rho_a = rhod * (1.0 + rv);
    const double Tr = t.T / 273.0;
    if (cond) {
        t.Dterm = t.rho_vs * t.lv * rT * (t.lv * rT * (1.0 / R_v) - 1.0);
        const double mu = 1.72e-5 * (393.0 / (t.T + 120.0)) * (Tr * sqrt(Tr));
        const double ra = 1.0 / t.rho_a;
        t.nu = mu * ra;
        t.lambda_D = 2.0 * D0 * rsqrt_hd(8.0 / pi * R_v * t.T);
        t.lambda_K = 2.0 * K0 / c_pd * ra * rsqrt_hd(8.0 / pi * R_d * t.T);
        t.Sc = t.nu * (1.0 / D0);
        t.Pr = t.nu * t.rho_a * (c_pd / K0);
        const double rnu = 1.0 / t.nu;
        t.cX = 32.0 / 3.0 * grav * (rho_w - t.rho_a) * ra * (rnu * rnu);
    } else {
        t.Dterm = t.rho_vs * t.lv / t.T * (t.lv / (R_v * t.T) - 1.0);
        const double mu = 1.72e-5 * (393.0 / (t.T + 120.0)) * pow(Tr, 1.5);
        t.nu = mu / t.rho_a;
        t.lambda_D = 2.0 * D0 / sqrt(8.0 * R_v * t.T / pi);
        t.lambda_K = 2.0 * K0 / (t.rho_a * c_pd * sqrt(8.0 * R_d * t.T / pi));
        t.Sc = t.nu / D0;
        t.Pr = t.nu * t.rho_a * c_pd / K0;
        t.cX = 32.0 / 3.0 * (rho_w - t.rho_a) / t.rho_a * grav / (t.nu * t.nu);
    }
    return t;
}

SDM_HD Thermo thermo_eval(double th, double rv, double rhod, double RH_max) {
    return thermo_eval_f<false>(th, rv, rhod, RH_max, rhod_factor(rhod));
}

// Khvorostyanov & Curry (2002) sphere: Re(X), X = cX r^3 (Best number)
// Re from r_w^2 and r_w = sqrt(r_w^2) (callers that keep r pass it)
SDM_HD double reynolds_r(double rw2, double r, double cX) {
    using namespace phys;
    if (!(r > 0.0)) return 0.0;
    const double X = cX * rw2 * r;
    const double c1 = 4.0 / (delta0 * delta0 * sqrt(C0));
    const double e = c1 * sqrt(X);
    const double s = e / (sqrt(1.0 + e) + 1.0);
    return delta0 * delta0 / 4.0 * s * s;
}

SDM_HD double reynolds(double rw2, double cX) { return reynolds_r(rw2, sqrt(rw2), cX); }

// terminal velocity v_t = Re nu / (2 r)
SDM_HD double vterm_r(double rw2, double r, double nu, double cX) {
    if (!(r > 0.0)) return 0.0;
    return reynolds_r(rw2, r, cX) * nu / (2.0 * r);
}

SDM_HD double vterm(double rw2, double nu, double cX) { return vterm_r(rw2, sqrt(rw2), nu, cX); }

// the same terminal velocity in FP32 (mixed-precision mode)
SDM_HD float vterm_f(float rw2, float nu, float cX) {
    const float r = sqrtf(rw2);
    if (!(r > 0.0f)) return 0.0f;
    const float X = cX * rw2 * r;
    const float c1 = (float)(4.0 / (phys::delta0 * phys::delta0 * 0.54037024344425184));  // sqrt(C0)
    const float e = c1 * sqrtf(X);
    const float s = e / (sqrtf(1.0f + e) + 1.0f);
    const float Re = (float)(phys::delta0 * phys::delta0 / 4.0) * s * s;
    return Re * nu / (2.0f * r);
}

// Collection efficiency of the Long (1974) kernel (the paper's collision
// efficiencies come from tables, Sec. 5.1.4; this closed form stands in):
// with R the larger and r the smaller radius, E = 1 for R >= 50 um, else
// 4.5e8 R^2 (1 - 3e-6 / r) in SI units, held within [1e-3, 1].  Products
// and one quotient only, so no contraction changes its rounding.
SDM_HD double long_E(double ra, double rb) {
    const double R = ra > rb ? ra : rb, r = ra > rb ? rb : ra;
    if (R >= 50e-6) return 1.0;
    double E = 4.5e8 * R * R * (1.0 - 3e-6 / r);
    if (E < 1e-3) E = 1e-3;
    if (E > 1.0) E = 1.0;
    return E;
}

SDM_HD float long_Ef(float ra, float rb) {
    const float R = ra > rb ? ra : rb, r = ra > rb ? rb : ra;
    if (R >= 50e-6f) return 1.0f;
    float E = 4.5e8f * R * R * (1.0f - 3e-6f / r);
    return E < 1e-3f ? 1e-3f : (E > 1.0f ? 1.0f : E);
}

// 24 random bits plus one half, times 2^-24: open (0,1) in FP32
SDM_HD float u01f(uint64_t v) { return ((float)(uint32_t)(v >> 40) + 0.5f) * 5.9604645e-8f; }

// The upscaling factor of eq. P_ij, n (n-1) / (2 floor(n/2)), is n - 1 for
// even n and n for odd n.  Its FP64 evaluation from the formula is exact
// for n < 2^26 (exact product, exact integer quotient), so this integer
// form gives the same double while keeping the FP64 pipe free (on GB300 it
// runs at 1/64 of the FP32 rate).
SDM_HD double pair_scale(int64_t n) { return (double)((n & 1) ? n : n - 1); }

// Collision events of a pair with scaled probability P (eq. P_ij), uniform
// draw w and multiplicities NL >= NS > 0.  The paper's scheme (Sec. 5.1.4):
// one event when u < P.  Multiple coalescence (multi = 1; Shima et al.
// 2009): floor(P), plus one when u < P - floor(P) (exact in either
// precision for P >= 1), at most floor(NL / NS).  Below P = 1 both are the
// single test u < P, so the 64-bit division is only taken for P >= 1.  In
// mixed precision P holds an FP32 value and the test uses the 24-bit draw.
__device__ __forceinline__ unsigned long long n_events(double P, uint64_t w, unsigned long long NL,
                                                       unsigned long long NS, int multi, int mixed) {
    const bool hit = mixed ? u01f(w) < (float)P : u01(w) < P;
    if (!multi || !(P >= 1.0)) return hit ? 1ull : 0ull;
    const unsigned long long cap = NL / NS;
    const double fl = floor(P);
    if (fl >= (double)cap) return cap;
    unsigned long long g = (unsigned long long)fl;
    if (mixed ? u01f(w) < (float)P - (float)fl : u01(w) < P - fl) g++;
    return g < cap ? g : cap;
}

SDM_HD double fuchs_sutugin(double Kn) {
    return (1.0 + Kn) / (1.0 + (4.0 / 3.0 + 0.377) * Kn + 4.0 / 3.0 * Kn * Kn);
}

// dr_w^2/dt = 2 D_eff / rho_w (rho_v - rho_o), eq. (maxmason), (rho_circ)
SDM_HD double growth(double x, double rd3, double kappa, const Thermo &t,
                                         int physics) {
    using namespace phys;
    const double r = sqrt(x);
    const double r3 = x * r;
    const double aw = (r3 - rd3) / (r3 - rd3 * (1.0 - kappa));
    const double rho_o = t.rho_vs * aw * exp(t.A / r);
    double D = D0, K = K0;
    if (physics) {
        const double bM = fuchs_sutugin(t.lambda_D / r);
        const double bT = fuchs_sutugin(t.lambda_K / r);
        const double Re = reynolds(x, t.cX);
        const double fRe = Re > 1.0 ? pow(Re, 0.077) : 1.0;
        const double Sh = 1.0 + cbrt(1.0 + Re * t.Sc) * fRe;
        const double Nu = 1.0 + cbrt(1.0 + Re * t.Pr) * fRe;
        D = D0 * bM * Sh / 2.0;
        K = K0 * bT * Nu / 2.0;
    }
    const double Deff = 1.0 / (1.0 / D + t.Dterm / K);
    return 2.0 * Deff / rho_w * (t.rho_v_eff - rho_o);
}

SDM_HD double rd2_of(double rd3) {
    const double rd = cbrt(rd3);
    return rd * rd;
}

// ---------------------------------------------------------------- context
struct DevStats {
    unsigned long long n_pairs, n_coll, n_pgt1, n_recycled, n_euler, n_fallback, n_zero;
    unsigned long long max_p_bits;  // max of non-negative doubles via uint order
    double rainfall;
    unsigned int flags;  // kFlag* bits
    unsigned int n_big;  // cells routed to the block coalescence path
    unsigned int n_rc_zero, n_rc_donor;
    unsigned long long n_coal_substeps;  // cell-substeps of coalescence taken
};
enum : unsigned { kFlagNumeric = 1u, kFlagBigCell = 2u };
// The top bit of an id marks a free slot kept for arrivals from other slabs
// (sdm_export_leavers leaves it on the slot it empties; sd_reserve slots
// start with it): recycling leaves such slots alone, sdm_import overwrites
// the id.  Live super-droplets' ids stay below 2^31.
constexpr uint32_t kUidVacant = 0x80000000u;

struct Grid {
    int nx, ny, nz;     // 0 = absent
    int NX, NY, NZ;     // max(n, 1)
    double dx, dy, dz;  // cell sizes
    double dt, dV;
    int n_cells;
    int x_open;         // 1: a slab of a domain decomposed in x (no periodic wrap in x)
};

struct SdArrays {  // one buffer of the structure-of-arrays state
    unsigned long long *N;
    double *rw2, *rd3, *kappa, *x, *y, *z;
    uint32_t *uid;
};

struct PhaseTimer {
    cudaEvent_t a, b;
    int phase;
};

}  // namespace sdm

struct sdm_ctx {
    sdm_opts_init oi;
    std::vector<sdm_lognormal> modes;
    int G = 1;
    std::vector<double> gkappa, lnr_min, lnr_max;
    sdm::Grid grid;
    int64_t n_sd = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    sdm::SdArrays buf[2];
    int cur = 0;
    uint32_t *newcell = nullptr, *slot = nullptr, *perm = nullptr;
    uint32_t *count = nullptr, *offset = nullptr, *bigcells = nullptr;
    // coalescence scratch for cells above kBigCellCap (keys, pair words and
    // accept draws, 2 n_sd each, a cell at twice its offset): allocated where
    // the initial cells are that large
    unsigned long long *huge = nullptr;
    double *th = nullptr, *rv = nullptr, *rhod = nullptr, *amb = nullptr, *outbuf = nullptr;
    double *rhoC[3] = {nullptr, nullptr, nullptr};
    uint32_t *scan_tmp = nullptr;
    void *rc_tmp = nullptr;
    size_t rc_tmp_bytes = 0;
    void *rc_sel = nullptr;  // recycling's radix-select state and histogram (4 KB)
    sdm::DevStats *dstats = nullptr;
    sdm::DevStats *hstats = nullptr;  // pinned landing area of stats copies
    sdm::DevStats mirror{};           // last copy pulled from the device
    uint64_t host_recycled = 0;       // super-droplets re-populated so far
    cudaEvent_t done_event = nullptr; // end of the last step_async

    bool async_in_flight = false;
    bool layout_dirty = false;
    bool transported = false;   // sdm_step_transport done, sdm_step_coalesce pending
    uint32_t *xch_flag = nullptr, *xch_off = nullptr, *xch_tmp = nullptr;  // exchange scratch (n_sd + 1)
    bool rng_set = false;
    int diag_wet = 1;
    double diag_rmin = 0.0, diag_rmax = 0.0;
    double *spec_buf = nullptr, *spec_edges = nullptr;  // binned spectrum: n_bins x n_cells, n_bins + 1
    void *cs_rec[2] = {nullptr, nullptr};               // staged condensation: solve records, ping-pong
    void *cs_cell = nullptr;                            // and the per-cell ambient state
    double *cs_x1 = nullptr;                            // and each super-droplet's new r_w^2
    unsigned *cs_cnt = nullptr;                         // and the round counts
    uint32_t *cond_order = nullptr;                     // condensation: warps longest-first
    float *cond_cost = nullptr;                         // and their cost in the last launch
    int64_t cond_nw = 0;
    bool cond_order_on = true;
    double *euler_tmp = nullptr, *euler_prof = nullptr;  // Eulerian stand-in: old field, th0 and rv0 profiles
    double *cedge[3] = {nullptr, nullptr, nullptr};       // Courant numbers of the edges, per step
    int spec_cap = 0;                                   // bins spec_buf holds
    uint64_t step = 0;
    uint64_t known_zeros = 0;
    std::string err;

    bool timing = false;
    std::vector<sdm::PhaseTimer> timers;
    std::vector<cudaEvent_t> event_pool;
    sdm_timing tacc{};
};

namespace sdm {

// launch wrappers (each returns the first CUDA error of its launches)
cudaError_t launch_init(sdm_ctx *c);
// *launches: the kernels it enqueued
cudaError_t launch_condense(sdm_ctx *c, const sdm_opts &o, int *launches);
cudaError_t launch_ambient(sdm_ctx *c);
cudaError_t launch_move(sdm_ctx *c, const sdm_opts &o);
cudaError_t launch_regroup(sdm_ctx *c);  // scan + perm (after move)
cudaError_t launch_coalesce(sdm_ctx *c, const sdm_opts &o, bool coal);
cudaError_t launch_recycle_compact(sdm_ctx *c);
bool recycle_small(const sdm_ctx *c);
cudaError_t launch_recycle_small(sdm_ctx *c);
cudaError_t launch_recycle_apply(sdm_ctx *c, uint32_t nz, uint32_t nd);
cudaError_t launch_moments(sdm_ctx *c, int k);
cudaError_t launch_sd_conc(sdm_ctx *c);
cudaError_t launch_cond_ambient(sdm_ctx *c, int what);
cudaError_t launch_exchange_count(sdm_ctx *c, int leavers, uint32_t *total_host);
cudaError_t launch_export(sdm_ctx *c, const sdm_sd_block &dst);
cudaError_t launch_import(sdm_ctx *c, const sdm_sd_block &src, int64_t n);
cudaError_t launch_block_check(sdm_ctx *c, const sdm_sd_block &src, int64_t n, unsigned *bad_host);
constexpr int kMaxSpectrumBins = 256;
// records per tile of the ensemble's radix sort: the histogram table its
// callers allocate holds 256 counts per tile of this size
constexpr int kRsTileRecords = 2048;
cudaError_t launch_upwind(const double *old, double *out, const double *rhod, const double *Cx, const double *Cy,
                          const double *Cz, const Grid &g, cudaStream_t st);
cudaError_t launch_relax(double *psi, const double *psi0, const Grid &g, double tau_rlx, double z_rlx,
                         cudaStream_t st);
cudaError_t launch_spectrum(sdm_ctx *c, int wet, int n_bins, int k);
cudaError_t launch_field_gather(double *dst, const double *src, const int64_t *strides, int ndim,
                                const int *shape, cudaStream_t s);
cudaError_t launch_field_scatter(double *dst, const double *src, const int64_t *strides,
                                 int ndim, const int *shape, cudaStream_t s);

cudaError_t scan_counts(const uint32_t *count, uint32_t *offset, uint32_t *tmp, int n,
                        cudaStream_t st);

// ---- batched ensembles of 0D members (ens.cu)
struct MemberDev {
    uint32_t off, n;         // super-droplet range
    uint32_t tile0, ntiles;  // condensation tiles
    uint32_t zeros;          // multiplicities that reached zero, not yet recycled
    double dV, md;           // volume [m^3], dry-air mass [kg]
    double th, rv, rhod;
    double nu, cX;           // air viscosity and Best-number factor for v_t
    unsigned long long seed, step;
};

struct EnsCondParams {
    double dt;
    int sstp, physics, solver, mixed;
    double RH_max;
};

// the largest block k_ens_cond_tiles launches with for these parameters
int ens_cond_max_threads(const EnsCondParams &p);

// one substep of condensation for every tile (k_cond.cu)
cudaError_t launch_ens_cond_tiles(SdArrays s, const MemberDev *M, const uint32_t *tile_member,
                                  const uint32_t *tile_beg, const uint32_t *tile_end, double *tile_sum,
                                  int n_tiles, int threads, EnsCondParams p, DevStats *st,
                                  cudaStream_t stream);
cudaError_t cell_sort_with_scratch(const uint32_t *cell, int64_t n, uint32_t n_cells, uint32_t *perm,
                                   uint32_t *offsets, uint32_t *count, uint32_t *slot,
                                   uint32_t *scan_tmp, unsigned *bad, cudaStream_t st);

// sort of (key_hi, key_lo, payload) records ascending by (key_hi, key_lo)
struct SortRec {
    unsigned long long hi;
    uint32_t lo, val;
};
cudaError_t sort_records(SortRec *rec, uint32_t n, uint32_t n_pow2, cudaStream_t s);

// message returned by sdm_last_error(NULL) on this thread
void sdm_set_global_error(const std::string &msg);

// initial dry-radius range of one kappa group (host; shared by contexts and
// ensemble members): the outermost ln r where n(ln r) dlnr dV >= 1
bool rd_range_modes(const std::vector<sdm_lognormal> &modes, double kap, int64_t sd_conc, double dV,
                    double *lo_out, double *hi_out);

// A kernel's dynamic shared-memory limit, raised once per device (the
// attribute belongs to each device's copy of the function): done holds one
// bit per device id below 64; devices beyond set it on every call.
template <class F>
inline cudaError_t smem_attr_once(F *kern, int bytes, std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load() & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit);
    return e;
}

inline unsigned grid_for(int64_t n, int block) {
    return (unsigned)((n + block - 1) / block);
}

}  // namespace sdm
