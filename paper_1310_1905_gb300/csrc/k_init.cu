// Initialisation of the super-droplets (paper Sec. 5.1.6), one thread per
// super-droplet.  The state is created sorted by cell: id = ((cell * G) +
// kappa group) * sd_conc + k, so cell c owns ids [c G sd_conc, (c+1) G sd_conc).
#include "sdm_internal.cuh"

namespace sdm {

struct InitParams {
    Grid g;
    int sd_conc, G, init_dist, n_modes;
    uint64_t seed;
    double exp_mean_volume, exp_n0;
    double lrm[kMaxModes], lsig[kMaxModes], n_stp[kMaxModes], mkappa[kMaxModes];
    double gkappa[kMaxModes], lmin[kMaxModes], lmax[kMaxModes];
};

// dN/dln r at STP of one kappa group: sum of the lognormal modes
__device__ double n_lnr(const InitParams &p, double kap, double lnr) {
    double s = 0.0;
    for (int m = 0; m < p.n_modes; ++m) {
        if (p.mkappa[m] != kap) continue;
        const double ls = p.lsig[m];
        const double q = (lnr - p.lrm[m]) / ls;
        s = __dadd_rn(s, __dmul_rn(p.n_stp[m] / (sqrt(2.0 * phys::pi) * ls), exp(-0.5 * q * q)));
    }
    return s;
}

// equilibrium wet radius squared: a_w(r) exp(A/r) = RH by bisection on
// [r_d^2, x_hi] with a_w(x_hi) = RH (Sec. 5.1.6, zero growth in eq. maxmason)
__device__ double equilibrium_rw2(double rd3, double kappa, double RH, double T) {
    using namespace phys;
    const double rd2 = rd2_of(rd3);
    if (!(kappa > 0.0) || !(RH > 0.0) || !(RH < 1.0) || !(rd3 > 0.0)) return rd2;
    const double A = 2.0 * sigma_w / (R_v * T * rho_w);
    const double rhi = cbrt(rd3 * (1.0 - RH * (1.0 - kappa)) / (1.0 - RH));
    double lo = rd2, hi = rhi * rhi;
    for (int it = 0; it < 200; ++it) {
        if (hi - lo <= 0x1p-52 * hi) break;
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        const double r = sqrt(mid), r3 = mid * r;
        const double S = (r3 - rd3) / (r3 - rd3 * (1.0 - kappa)) * exp(A / r);
        if (S > RH) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

__global__ void k_init(SdArrays s, int64_t n, InitParams p, const double *th, const double *rv,
                       const double *rhod) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Grid &g = p.g;
    const uint64_t uid = (uint64_t)i;
    const int64_t per_cell = (int64_t)p.G * p.sd_conc;
    const int64_t c = i / per_cell;
    const int grp = (int)((i / p.sd_conc) % p.G);
    const int64_t ci = c / ((int64_t)g.NY * g.NZ), cj = (c / g.NZ) % g.NY, ck = c % g.NZ;
    const u64x4 w = philox4x64(uid, 0, 0, kStreamInit, p.seed, 0);
    s.uid[i] = (uint32_t)uid;
    if (g.nx > 0) s.x[i] = ((double)ci + u01(w.v[0])) * g.dx;
    if (g.ny > 0) s.y[i] = ((double)cj + u01(w.v[1])) * g.dy;
    if (g.nz > 0) s.z[i] = ((double)ck + u01(w.v[2])) * g.dz;
    if (p.init_dist == SDM_INIT_EXPONENTIAL) {
        const double V = -p.exp_mean_volume * log(u01(w.v[3]));
        const double r = cbrt(3.0 * V / (4.0 * phys::pi));
        s.rw2[i] = r * r;
        s.rd3[i] = 0.0;
        s.kappa[i] = 0.0;
        const double nn = floor(p.exp_n0 * g.dV / p.sd_conc + 0.5);
        s.N[i] = nn < 1.0 ? 1ull : (unsigned long long)nn;
        return;
    }
    const double lmin = p.lmin[grp], lmax = p.lmax[grp];
    // no fused multiply-add here: the lognormal's slope amplifies a one-ulp
    // change of ln r about a hundredfold in the multiplicity
    const double lnr = __dadd_rn(lmin, __dmul_rn(u01(w.v[3]), lmax - lmin));
    const double rd = exp(lnr);
    const double rd3 = rd * rd * rd;
    const double dlnr = (lmax - lmin) / p.sd_conc;
    const double nn = floor(n_lnr(p, p.gkappa[grp], lnr) * dlnr * g.dV * rhod[c] / phys::rho_stp + 0.5);
    s.N[i] = nn < 1.0 ? 1ull : (unsigned long long)nn;
    s.rd3[i] = rd3;
    s.kappa[i] = p.gkappa[grp];
    const Thermo t = thermo_eval(th[c], rv[c], rhod[c], 44.0);
    double RH = t.rho_v / t.rho_vs;
    if (RH >= 1.0) RH = 0.95;
    s.rw2[i] = equilibrium_rw2(rd3, p.gkappa[grp], RH, t.T);
}

__global__ void k_init_offsets(uint32_t *offset, int n_cells, uint32_t per_cell) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c <= n_cells) offset[c] = (uint32_t)c * per_cell;
}

// the reserved slots (sdm_opts_init::sd_reserve) after the initial ones:
// N = 0, no water, at the domain's origin, ids after the initial ones with
// the mark of a slot kept for arrivals
__global__ void k_init_reserve(SdArrays s, int64_t first, int64_t n, Grid g) {
    const int64_t q = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    s.N[q] = 0;
    s.rw2[q] = 0.0;
    s.rd3[q] = 0.0;
    s.kappa[q] = 0.0;
    if (g.nx > 0) s.x[q] = 0.0;
    if (g.ny > 0) s.y[q] = 0.0;
    if (g.nz > 0) s.z[q] = 0.0;
    s.uid[q] = (uint32_t)q | kUidVacant;
}

cudaError_t launch_init(sdm_ctx *c) {
    InitParams p{};
    p.g = c->grid;
    p.sd_conc = c->oi.sd_conc;
    p.G = c->G;
    p.init_dist = c->oi.init_dist;
    p.n_modes = (int)c->modes.size();
    p.seed = c->oi.seed;
    p.exp_mean_volume = c->oi.exp_mean_volume;
    p.exp_n0 = c->oi.exp_n0;
    for (int m = 0; m < p.n_modes; ++m) {
        p.lrm[m] = log(c->modes[m].rm);  // host logs, as in the oracle
        p.lsig[m] = log(c->modes[m].sigma);
        p.n_stp[m] = c->modes[m].n_stp;
        p.mkappa[m] = c->modes[m].kappa;
    }
    for (int g = 0; g < c->G; ++g) {
        p.gkappa[g] = c->gkappa[g];
        p.lmin[g] = c->lnr_min.empty() ? 0.0 : c->lnr_min[g];
        p.lmax[g] = c->lnr_max.empty() ? 0.0 : c->lnr_max[g];
    }
    const int B = 256;
    const int64_t n_init = c->n_sd - c->oi.sd_reserve;
    k_init<<<grid_for(n_init, B), B, 0, c->stream>>>(c->buf[c->cur], n_init, p, c->th, c->rv, c->rhod);
    if (c->oi.sd_reserve > 0)
        k_init_reserve<<<grid_for(c->oi.sd_reserve, B), B, 0, c->stream>>>(c->buf[c->cur], n_init, c->n_sd, c->grid);
    k_init_offsets<<<grid_for(c->grid.n_cells + 1, B), B, 0, c->stream>>>(
        c->offset, c->grid.n_cells, (uint32_t)(c->G * c->oi.sd_conc));
    return cudaGetLastError();
}

}  // namespace sdm
