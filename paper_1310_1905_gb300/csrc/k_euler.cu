// The kinematic framework's Eulerian component (Sec. 2.1-2.2), the part the
// paper leaves to its MPDATA solver: a first-order donor-cell (upwind) stand
// in for the transport of theta and r_v by the same rho_d C Courant fields
// the particles use, in flux form,
//   rho_d psi' = rho_d psi - sum over the cell's edges of the outward
//                (rho_d C)_edge psi_up,
// psi_up the value in the cell the flow comes from (periodic in x and y; on
// a z boundary edge the inside cell's value), psi' = (rho_d psi') / rho_d;
// and the relaxation of each level's horizontal mean toward the initial
// profile, dt (psi0 - <psi>) / tau, tau = tau_rlx exp(z / z_rlx).
#include "sdm_internal.cuh"

namespace sdm {

__device__ __forceinline__ double up_flux(double C, double left, double right) {
    return C * (C >= 0.0 ? left : right);
}

// one thread per cell, reading the old field and writing the new one
__global__ void k_upwind(const double *__restrict__ old, double *__restrict__ out, const double *__restrict__ rhod,
                         const double *Cx, const double *Cy, const double *Cz, Grid g) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.n_cells) return;
    const int i = c / (g.NY * g.NZ), j = (c / g.NZ) % g.NY, k = c % g.NZ;
    const double p = old[c];
    double o = 0.0;  // net outward flux of rho_d psi
    if (g.nx > 0 && Cx) {
        const int il = (i - 1 + g.NX) % g.NX, ir = (i + 1) % g.NX;
        const double Cl = Cx[((int64_t)i * g.NY + j) * g.NZ + k], Cr = Cx[((int64_t)(i + 1) * g.NY + j) * g.NZ + k];
        o += up_flux(Cr, p, old[((int64_t)ir * g.NY + j) * g.NZ + k]);
        o -= up_flux(Cl, old[((int64_t)il * g.NY + j) * g.NZ + k], p);
    }
    if (g.ny > 0 && Cy) {
        const int jl = (j - 1 + g.NY) % g.NY, jr = (j + 1) % g.NY;
        const double Cl = Cy[((int64_t)i * (g.NY + 1) + j) * g.NZ + k];
        const double Cr = Cy[((int64_t)i * (g.NY + 1) + j + 1) * g.NZ + k];
        o += up_flux(Cr, p, old[((int64_t)i * g.NY + jr) * g.NZ + k]);
        o -= up_flux(Cl, old[((int64_t)i * g.NY + jl) * g.NZ + k], p);
    }
    if (g.nz > 0 && Cz) {
        const double below = k > 0 ? old[c - 1] : p, above = k < g.NZ - 1 ? old[c + 1] : p;
        const double Cb = Cz[((int64_t)i * g.NY + j) * (g.NZ + 1) + k];
        const double Ct = Cz[((int64_t)i * g.NY + j) * (g.NZ + 1) + k + 1];
        o += up_flux(Ct, p, above);
        o -= up_flux(Cb, below, p);
    }
    out[c] = (rhod[c] * p - o) / rhod[c];
}

// one warp per level: the mean over the level's NX NY cells (lane-strided
// sums, then a butterfly: a fixed order), then the increment on every cell
__global__ void k_relax(double *psi, const double *psi0, Grid g, double tau_rlx, double z_rlx) {
    const int k = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= g.NZ) return;
    const int nh = g.NX * g.NY;
    double sum = 0.0;
    for (int h = lane; h < nh; h += 32) sum += psi[(int64_t)h * g.NZ + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const double mean = sum / (double)nh;
    const double tau = tau_rlx * exp((k + 0.5) * g.dz / z_rlx);
    const double inc = g.dt * (psi0[k] - mean) / tau;
    for (int h = lane; h < nh; h += 32) psi[(int64_t)h * g.NZ + k] += inc;
}

cudaError_t launch_upwind(const double *old, double *out, const double *rhod, const double *Cx, const double *Cy,
                          const double *Cz, const Grid &g, cudaStream_t st) {
    const int B = 256;
    k_upwind<<<grid_for(g.n_cells, B), B, 0, st>>>(old, out, rhod, Cx, Cy, Cz, g);
    return cudaGetLastError();
}

cudaError_t launch_relax(double *psi, const double *psi0, const Grid &g, double tau_rlx, double z_rlx,
                         cudaStream_t st) {
    const int B = 128;
    k_relax<<<grid_for((int64_t)g.NZ * 32, B), B, 0, st>>>(psi, psi0, g, tau_rlx, z_rlx);
    return cudaGetLastError();
}

}  // namespace sdm
