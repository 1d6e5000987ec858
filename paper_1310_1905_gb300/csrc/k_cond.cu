// Condensation / evaporation (paper Sec. 5.1.3): one warp per grid cell,
// all sstp_cond substeps in one launch.  In each substep every lane advances
// its super-droplets' r_w^2 with the implicit growth equation (eq.
// rw2_implicit), the warp sums N (r_w^3[new] - r_w^3[old]) and every lane
// applies eq. (rhov_update) to its register copy of the cell's r_v, theta.
#include "sdm_internal.cuh"

namespace sdm {

__device__ __forceinline__ double fres(double x, double x0, double rd3, double kappa,
                                       const Thermo &t, double dtp, int physics) {
    return x - x0 - dtp * growth(x, rd3, kappa, t, physics);
}

// The paper's predictor-corrector: bracket [a, b] from the derivative at
// x0 with the factor 2, the Euler step (a+b)/2 when f does not change strict
// sign over it, bisection to b - a <= 2^-52 b otherwise.
__device__ double solve_rw2_bisect(double x0, double rd3, double kappa, const Thermo &t,
                                   double dtp, int physics, int *euler) {
    const double g0 = growth(x0, rd3, kappa, t, physics);
    const double a = fmax(rd2_of(rd3), x0 + fmin(2.0 * dtp * g0, 0.0));
    const double b = x0 + fmax(2.0 * dtp * g0, 0.0);
    const double fa = fres(a, x0, rd3, kappa, t, dtp, physics);
    const double fb = fres(b, x0, rd3, kappa, t, dtp, physics);
    if ((fa > 0.0) == (fb > 0.0)) {
        *euler = 1;
        return 0.5 * (a + b);
    }
    double lo = a, hi = b;
    const bool plo = fa > 0.0;
    for (int it = 0; it < 200; ++it) {
        if (hi - lo <= 0x1p-52 * hi) break;
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        const bool pm = fres(mid, x0, rd3, kappa, t, dtp, physics) > 0.0;
        if (pm == plo) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void k_condense(SdArrays s, const uint32_t *offset, double *th, double *rv,
                           const double *rhod, Grid g, int sstp, double RH_max, int physics,
                           DevStats *st) {
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= g.n_cells) return;
    const int c = warp;
    const uint32_t beg = offset[c], end = offset[c + 1];
    double thc = th[c], rvc = rv[c];
    const double rd = rhod[c];
    const double dtp = g.dt / sstp;
    int n_euler = 0;
    bool bad = false;
    for (int sub = 0; sub < sstp; ++sub) {
        const Thermo t = thermo_eval(thc, rvc, rd, RH_max);
        double sum = 0.0;
        for (uint32_t i = beg + lane; i < end; i += 32) {
            const unsigned long long N = s.N[i];
            if (N == 0) continue;
            const double x0 = s.rw2[i];
            int eu = 0;
            const double x1 = solve_rw2_bisect(x0, s.rd3[i], s.kappa[i], t, dtp, physics, &eu);
            n_euler += eu;
            bad |= !isfinite(x1);
            s.rw2[i] = x1;
            sum += (double)N * (x1 * sqrt(x1) - x0 * sqrt(x0));
        }
        sum = warp_sum(sum);
        const double drv = -4.0 * phys::pi * phys::rho_w / (3.0 * g.dV * rd) * sum;
        rvc = t.rv + drv;
        thc = t.th + drv * t.dth_drv;
    }
    bad |= !isfinite(rvc) || !isfinite(thc);
    unsigned ne = __reduce_add_sync(0xffffffffu, (unsigned)n_euler);
    const unsigned anybad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        th[c] = thc;
        rv[c] = rvc;
        if (ne) atomicAdd(&st->n_euler, (unsigned long long)ne);
        if (anybad) atomicOr(&st->flags, kFlagNumeric);
    }
}

cudaError_t launch_condense(sdm_ctx *c, const sdm_opts &o) {
    const int B = 128;
    const int64_t threads = (int64_t)c->grid.n_cells * 32;
    k_condense<<<grid_for(threads, B), B, 0, c->stream>>>(c->buf[c->cur], c->offset, c->th, c->rv,
                                                          c->rhod, c->grid, o.sstp_cond, o.RH_max,
                                                          c->oi.physics, c->dstats);
    return cudaGetLastError();
}

}  // namespace sdm
