// Transport and regrouping: per-cell ambient for terminal velocities,
// per-super-droplet advection (Sec. 5.1.2, eqs. adv_implicit, adv_c, adv_w)
// and sedimentation (Sec. 5.1.5) with the new cell index and a counting-sort
// slot, then an exclusive scan of the cell counts and the permutation.
#include "sdm_internal.cuh"

namespace sdm {

__global__ void k_ambient(double *amb, const double *th, const double *rv, const double *rhod,
                          int n_cells) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const Thermo t = thermo_eval(th[c], rv[c], rhod[c], 44.0);
    amb[2 * c] = t.nu;
    amb[2 * c + 1] = t.cX;
}

cudaError_t launch_ambient(sdm_ctx *c) {
    const int B = 256;
    k_ambient<<<grid_for(c->grid.n_cells, B), B, 0, c->stream>>>(c->amb, c->th, c->rv, c->rhod,
                                                                 c->grid.n_cells);
    return cudaGetLastError();
}

__device__ __forceinline__ int64_t clampi(int64_t v, int64_t lo, int64_t hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

__device__ __forceinline__ int cell_of(const Grid &g, double x, double y, double z) {
    const int64_t i = g.nx > 0 ? clampi((int64_t)floor(x / g.dx), 0, g.nx - 1) : 0;
    const int64_t j = g.ny > 0 ? clampi((int64_t)floor(y / g.dy), 0, g.ny - 1) : 0;
    const int64_t k = g.nz > 0 ? clampi((int64_t)floor(z / g.dz), 0, g.nz - 1) : 0;
    return (int)((i * g.NY + j) * g.NZ + k);
}

// Courant number on an edge: rho_d C divided by the mean rho_d of the two
// cells sharing the edge (the adjacent cell on a closed boundary, and on the
// x boundaries of a slab)
__device__ __forceinline__ double courant_x(const Grid &g, const double *rhod, const double *C,
                                            int ie, int j, int k) {
    const int il = g.x_open ? (ie > 0 ? ie - 1 : 0) : (ie - 1 + g.nx) % g.nx;
    const int ir = g.x_open ? (ie < g.nx ? ie : g.nx - 1) : ie % g.nx;
    const double re = 0.5 * (rhod[((int64_t)il * g.NY + j) * g.NZ + k] +
                             rhod[((int64_t)ir * g.NY + j) * g.NZ + k]);
    return C[((int64_t)ie * g.NY + j) * g.NZ + k] / re;
}
__device__ __forceinline__ double courant_y(const Grid &g, const double *rhod, const double *C,
                                            int i, int je, int k) {
    const int jl = (je - 1 + g.ny) % g.ny, jr = je % g.ny;
    const double re = 0.5 * (rhod[((int64_t)i * g.NY + jl) * g.NZ + k] +
                             rhod[((int64_t)i * g.NY + jr) * g.NZ + k]);
    return C[((int64_t)i * (g.NY + 1) + je) * g.NZ + k] / re;
}
__device__ __forceinline__ double courant_z(const Grid &g, const double *rhod, const double *C,
                                            int i, int j, int ke) {
    const int kl = ke - 1 < 0 ? 0 : ke - 1, kr = ke > g.nz - 1 ? g.nz - 1 : ke;
    const double re = 0.5 * (rhod[((int64_t)i * g.NY + j) * g.NZ + kl] +
                             rhod[((int64_t)i * g.NY + j) * g.NZ + kr]);
    return C[((int64_t)i * g.NY + j) * (g.NZ + 1) + ke] / re;
}

// x' = (x + dx (C_l - i dC)) / (1 - dC): the analytic backward-Euler step
__device__ __forceinline__ double advect_1d(double x, double h, int i, double Cl, double Cr) {
    const double dC = Cr - Cl;
    return (x + h * (Cl - (double)i * dC)) / (1.0 - dC);
}

// periodic wrap into [0, X): w = fmod(x, X), plus X if negative, 0 if that
// rounds to X.  Within one period of the domain (every Courant number below
// 1) the same value comes from a comparison and at most one exact
// subtraction or one rounded addition: FP64 fmod is a loop of FP64 work.
__device__ __forceinline__ double wrap(double x, double X) {
    if (x >= 0.0 && x < X) return x;
    if (x > -X && x < 0.0) {  // fmod returns x itself
        const double w = x + X;
        return w >= X ? 0.0 : w;
    }
    if (x >= X && x < 2.0 * X) return x - X;  // exact: X <= x <= 2X
    double w = fmod(x, X);
    if (w < 0.0) w += X;
    if (w >= X) w = 0.0;
    return w;
}

// The Courant number of every edge, C = (rho_d C) / rho_d,edge (courant_x,
// _y, _z), once per step: the super-droplets of a cell share its edges, so
// k_move reads them instead of dividing per super-droplet.  The same
// operations on the same operands: the values are those courant_* give.
__global__ void k_courant(Grid g, const double *rhod, const double *Cx, const double *Cy, const double *Cz,
                          double *Ex, double *Ey, double *Ez) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (Cx) {
        const int64_t n = (int64_t)(g.nx + 1) * g.NY * g.NZ;
        if (t < n) {
            const int ie = (int)(t / ((int64_t)g.NY * g.NZ)), j = (int)((t / g.NZ) % g.NY), k = (int)(t % g.NZ);
            Ex[t] = courant_x(g, rhod, Cx, ie, j, k);
        }
    }
    if (Cy) {
        const int64_t n = (int64_t)g.NX * (g.ny + 1) * g.NZ;
        if (t < n) {
            const int i = (int)(t / ((int64_t)(g.ny + 1) * g.NZ)), je = (int)((t / g.NZ) % (g.ny + 1));
            const int k = (int)(t % g.NZ);
            Ey[t] = courant_y(g, rhod, Cy, i, je, k);
        }
    }
    if (Cz) {
        const int64_t n = (int64_t)g.NX * g.NY * (g.nz + 1);
        if (t < n) {
            const int i = (int)(t / ((int64_t)g.NY * (g.nz + 1))), j = (int)((t / (g.nz + 1)) % g.NY);
            const int ke = (int)(t % (g.nz + 1));
            Ez[t] = courant_z(g, rhod, Cz, i, j, ke);
        }
    }
}

struct MoveParams {
    Grid g;
    int adve, sedi, transport, mixed;
    const double *Cx, *Cy, *Cz;  // Courant numbers of the edges (k_courant)
};

__global__ void k_move(SdArrays s, int64_t n, MoveParams p, const double *rhod, const double *amb,
                       uint32_t *count, uint32_t *newcell, uint32_t *slot, DevStats *st) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rain = 0.0;
    if (q < n) {
        const Grid &g = p.g;
        double x = g.nx > 0 ? s.x[q] : 0.0, y = g.ny > 0 ? s.y[q] : 0.0, z = g.nz > 0 ? s.z[q] : 0.0;
        const int c = cell_of(g, x, y, z);
        const int i = c / (g.NY * g.NZ), j = (c / g.NZ) % g.NY, k = c % g.NZ;
        double vt = 0.0;
        const bool sedi = p.sedi && g.nz > 0;
        if (sedi)
            vt = p.mixed ? (double)vterm_f((float)s.rw2[q], (float)amb[2 * c], (float)amb[2 * c + 1])
                         : vterm(s.rw2[q], amb[2 * c], amb[2 * c + 1]);
        if (p.adve) {
            if (g.nx > 0 && p.Cx) {
                x = advect_1d(x, g.dx, i, p.Cx[((int64_t)i * g.NY + j) * g.NZ + k],
                              p.Cx[((int64_t)(i + 1) * g.NY + j) * g.NZ + k]);
                if (!g.x_open) x = wrap(x, g.nx * g.dx);  // a slab keeps its leavers outside for the export
            }
            if (g.ny > 0 && p.Cy)
                y = wrap(advect_1d(y, g.dy, j, p.Cy[((int64_t)i * (g.NY + 1) + j) * g.NZ + k],
                                   p.Cy[((int64_t)i * (g.NY + 1) + j + 1) * g.NZ + k]),
                         g.ny * g.dy);
            if (g.nz > 0 && p.Cz)
                z = advect_1d(z, g.dz, k, p.Cz[((int64_t)i * g.NY + j) * (g.NZ + 1) + k],
                              p.Cz[((int64_t)i * g.NY + j) * (g.NZ + 1) + k + 1]);
        }
        if (p.transport && g.nz > 0) {
            const double Z = g.nz * g.dz;
            if (sedi) z = z - vt * g.dt;
            if (z < 0.0) {
                const double r = sqrt(s.rw2[q]);
                rain = (double)s.N[q] * (4.0 / 3.0 * phys::pi * phys::rho_w * r * r * r);
                s.N[q] = 0;
                z = 0.0;
            } else if (z >= Z) {
                s.N[q] = 0;
                z = Z;
            }
        }
        if (g.nx > 0) s.x[q] = x;
        if (g.ny > 0) s.y[q] = y;
        if (g.nz > 0) s.z[q] = z;
        const int nc = cell_of(g, x, y, z);
        newcell[q] = (uint32_t)nc;
        // one cell: the slot is the storage index, so the counting sort keeps
        // the order (the coalescence gather then finds it in id order)
        const uint32_t sl = atomicAdd(count + nc, 1u);
        slot[q] = g.n_cells == 1 ? (uint32_t)q : sl;
    }
    // rainfall: warp-reduce, one atomic per warp that saw any
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rain += __shfl_xor_sync(0xffffffffu, rain, o);
    if ((threadIdx.x & 31) == 0 && rain != 0.0) atomicAdd(&st->rainfall, rain);
}

cudaError_t launch_move(sdm_ctx *c, const sdm_opts &o) {
    MoveParams p;
    p.g = c->grid;
    p.adve = o.adve;
    p.sedi = o.sedi;
    p.mixed = c->oi.precision == SDM_PRECISION_MIXED;
    p.transport = o.adve || o.sedi;
    p.Cx = p.Cy = p.Cz = nullptr;
    const int B = 256;
    cudaError_t e;
    if (o.adve && (c->rhoC[0] || c->rhoC[1] || c->rhoC[2])) {
        const Grid &g = c->grid;
        const int64_t ne[3] = {(int64_t)(g.nx + 1) * g.NY * g.NZ, (int64_t)g.NX * (g.ny + 1) * g.NZ,
                               (int64_t)g.NX * g.NY * (g.nz + 1)};
        int64_t nmax = 0;
        for (int d = 0; d < 3; ++d) {
            if (!c->rhoC[d]) continue;
            if (!c->cedge[d]) {
                e = cudaMalloc(&c->cedge[d], 8 * (size_t)ne[d]);
                if (e != cudaSuccess) return e;
            }
            nmax = ne[d] > nmax ? ne[d] : nmax;
        }
        k_courant<<<grid_for(nmax, B), B, 0, c->stream>>>(g, c->rhod, c->rhoC[0], c->rhoC[1], c->rhoC[2], c->cedge[0],
                                                          c->cedge[1], c->cedge[2]);
        p.Cx = c->rhoC[0] ? c->cedge[0] : nullptr;
        p.Cy = c->rhoC[1] ? c->cedge[1] : nullptr;
        p.Cz = c->rhoC[2] ? c->cedge[2] : nullptr;
    }
    e = cudaMemsetAsync(c->count, 0, sizeof(uint32_t) * (c->grid.n_cells + 1), c->stream);
    if (e != cudaSuccess) return e;
    k_move<<<grid_for(c->n_sd, B), B, 0, c->stream>>>(c->buf[c->cur], c->n_sd, p, c->rhod, c->amb,
                                                       c->count, c->newcell, c->slot, c->dstats);
    return cudaGetLastError();
}

// ---- exclusive scan of the cell counts (three passes, 1024 cells a block)
constexpr int kScanB = 1024;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_tot,
                                                         uint32_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t a = lane < nw ? warp_tot[lane] : 0u;
        uint32_t ai = a;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, ai, o);
            if (lane >= o) ai += t;
        }
        if (lane < nw) warp_tot[lane] = ai - a;
        if (lane == nw - 1) *total = ai;
    }
    __syncthreads();
    return incl - v + warp_tot[w];
}

__global__ void k_scan_local(const uint32_t *count, uint32_t *offset, uint32_t *bsum, int n) {
    __shared__ uint32_t wt[32];
    __shared__ uint32_t tot;
    const int i = blockIdx.x * kScanB + threadIdx.x;
    const uint32_t v = i < n ? count[i] : 0u;
    const uint32_t ex = block_exclusive_scan(v, wt, &tot);
    if (i < n) offset[i] = ex;
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_top(uint32_t *bsum, int nb, uint32_t *offset_end, int n) {
    __shared__ uint32_t wt[32];
    __shared__ uint32_t tot;
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += kScanB) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? bsum[i] : 0u;
        const uint32_t ex = block_exclusive_scan(v, wt, &tot);
        if (i < nb) bsum[i] = ex + carry;
        __syncthreads();
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) offset_end[n] = carry;
}

__global__ void k_scan_add(uint32_t *offset, const uint32_t *bsum, int n) {
    const int i = blockIdx.x * kScanB + threadIdx.x;
    if (i < n) offset[i] += bsum[blockIdx.x];
}

__global__ void k_perm(const uint32_t *newcell, const uint32_t *slot, const uint32_t *offset,
                       uint32_t *perm, int64_t n) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) perm[offset[newcell[q]] + slot[q]] = (uint32_t)q;
}

// exclusive scan of n counts into offset[0..n], offset[n] = total;
// tmp holds n/1024 + 2 words
cudaError_t scan_counts(const uint32_t *count, uint32_t *offset, uint32_t *tmp, int n,
                        cudaStream_t st) {
    const int nb = (n + kScanB - 1) / kScanB;
    k_scan_local<<<nb, kScanB, 0, st>>>(count, offset, tmp, n);
    k_scan_top<<<1, kScanB, 0, st>>>(tmp, nb, offset, n);
    k_scan_add<<<nb, kScanB, 0, st>>>(offset, tmp, n);
    return cudaGetLastError();
}

cudaError_t launch_regroup(sdm_ctx *c) {
    cudaError_t e = scan_counts(c->count, c->offset, c->scan_tmp, c->grid.n_cells, c->stream);
    if (e != cudaSuccess) return e;
    const int B = 256;
    k_perm<<<grid_for(c->n_sd, B), B, 0, c->stream>>>(c->newcell, c->slot, c->offset, c->perm,
                                                       c->n_sd);
    return cudaGetLastError();
}

}  // namespace sdm
