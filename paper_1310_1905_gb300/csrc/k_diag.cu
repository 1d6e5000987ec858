// Diagnostics (paper Sec. 5.2.1): per-cell moments of the wet or dry
// spectrum over a radius range, M^k = (rho_d dV)^-1 sum N r^k, the count
// of super-droplets with non-zero multiplicity, and the binned spectrum
// (that moment for many radius bins in one pass).
// Also the strided gather/scatter of caller-owned device fields (arrinfo_t).
#include "sdm_internal.cuh"

namespace sdm {

// Both moment kernels take 32 consecutive cells per block of 8 warps, 4
// cells per warp.  The super-droplets of a warp's 4 cells are one
// contiguous range of the cell-sorted state, which the warp streams in
// chunks of 32 (independent, coalesced loads); each lane knows the cell of
// its super-droplet from the 5 offsets.  Per-cell results gather in shared
// memory and leave the block as coalesced rows of 32 cells.  Every sum runs
// in a fixed order, so results do not depend on scheduling.
// On GB300 FP64 arithmetic runs at 1/64 of the FP32 rate, and these kernels
// are bound by it (the radius is an FP64 square or cube root), not by HBM:
// the sums are arranged to spend as few FP64 additions as possible.
constexpr int kDiagCells = 32, kDiagWarps = 8, kCellsPerWarp = kDiagCells / kDiagWarps;

__device__ __forceinline__ double diag_radius(const SdArrays &s, uint32_t i, int wet) {
    return wet ? sqrt(s.rw2[i]) : cbrt(s.rd3[i]);
}

__device__ __forceinline__ double pow_k(double r, int k) {
    double p = 1.0;
    for (int e = 0; e < k; ++e) p *= r;
    return p;
}

__global__ void __launch_bounds__(kDiagWarps * 32)
    k_moments(SdArrays s, const uint32_t *offset, const double *rhod, Grid g, int wet, double rmin, double rmax,
              int k, double *out) {
    __shared__ uint32_t s_off[kDiagCells + 1];
    __shared__ double s_res[kDiagCells];
    const int c0 = blockIdx.x * kDiagCells;
    const int nc = min(kDiagCells, g.n_cells - c0);
    if (threadIdx.x <= nc) s_off[threadIdx.x] = offset[c0 + threadIdx.x];
    __syncthreads();
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = wib * kCellsPerWarp;
    static_assert(kCellsPerWarp == 4, "the reduction below folds 4 cells");
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (j0 < nc) {
        const int jn = min(kCellsPerWarp, nc - j0);
        uint32_t o[kCellsPerWarp + 1];
#pragma unroll
        for (int j = 0; j <= kCellsPerWarp; ++j) o[j] = s_off[j0 + min(j, jn)];
        // a lane meets its cells in increasing order: one running sum, moved
        // into the cell's accumulator (selects, no arithmetic) when it changes
        double run = 0.0;
        int cj = 0;
        for (uint32_t i = o[0] + lane; i < o[kCellsPerWarp]; i += 32) {
            const int j = (i >= o[1]) + (i >= o[2]) + (i >= o[3]);
            if (j != cj) {
                a0 = cj == 0 ? run : a0;
                a1 = cj == 1 ? run : a1;
                a2 = cj == 2 ? run : a2;
                run = 0.0;
                cj = j;
            }
            const double r = diag_radius(s, i, wet);
            if (r >= rmin && r <= rmax) run += (double)s.N[i] * pow_k(r, k);
        }
        a0 = cj == 0 ? run : a0;
        a1 = cj == 1 ? run : a1;
        a2 = cj == 2 ? run : a2;
        a3 = cj == 3 ? run : a3;
    }
    // reduce-scatter over the lanes: across 16 each half keeps two cells,
    // across 8 one, then a butterfly (6 additions per lane, not 20)
    const bool hi16 = lane & 16, hi8 = lane & 8;
    double k0 = hi16 ? a2 : a0, k1 = hi16 ? a3 : a1;
    const double g0 = hi16 ? a0 : a2, g1 = hi16 ? a1 : a3;
    k0 += __shfl_xor_sync(0xffffffffu, g0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, g1, 16);
    double x = hi8 ? k1 : k0;
    x += __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
#pragma unroll
    for (int d = 4; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    if ((lane & 7) == 0) s_res[j0 + 2 * (int)hi16 + (int)hi8] = x;
    __syncthreads();
    if (threadIdx.x < nc) out[c0 + threadIdx.x] = s_res[threadIdx.x] / (rhod[c0 + threadIdx.x] * g.dV);
}

__global__ void k_sd_conc(SdArrays s, const uint32_t *offset, Grid g, double *out) {
    const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= g.n_cells) return;
    unsigned cnt = 0;
    for (uint32_t i = offset[c] + lane; i < offset[c + 1]; i += 32) cnt += s.N[i] > 0;
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) out[c] = (double)cnt;
}

// Binned spectrum: the moment of k_moments for every bin [e_b, e_b+1) at
// once, out[b * n_cells + c].  Per chunk of 32 super-droplets each lane
// finds its bin by binary search; the lanes that share a (cell, bin) key
// find each other (match_any) and the lowest of them adds the others'
// values in lane order, then adds the group's sum into the block's
// shared-memory table of 32 cells x n_bins (one FP64 addition per member,
// against five per distinct key for butterflies).
__global__ void __launch_bounds__(kDiagWarps * 32)
    k_spectrum(SdArrays s, const uint32_t *offset, const double *rhod, Grid g, const double *edges, int n_bins,
               int wet, int k, double *out) {
    extern __shared__ double s_dyn[];
    double *s_edges = s_dyn;                      // n_bins + 1
    double *s_acc = s_dyn + kMaxSpectrumBins + 1;  // kDiagCells rows of `stride`
    __shared__ uint32_t s_off[kDiagCells + 1];
    __shared__ double s_inv[kDiagCells];
    const int stride = n_bins | 1;                 // odd row stride: fewer bank conflicts on the way out
    const int c0 = blockIdx.x * kDiagCells;
    const int nc = min(kDiagCells, g.n_cells - c0);
    for (int i = threadIdx.x; i <= n_bins; i += blockDim.x) s_edges[i] = edges[i];
    for (int i = threadIdx.x; i < kDiagCells * stride; i += blockDim.x) s_acc[i] = 0.0;
    if (threadIdx.x <= nc) s_off[threadIdx.x] = offset[c0 + threadIdx.x];
    // one FP64 division per cell, not one per bin (a division is about a
    // dozen FP64 operations); the product with the reciprocal is within two
    // ulps of the quotient
    if (threadIdx.x < nc) s_inv[threadIdx.x] = 1.0 / (rhod[c0 + threadIdx.x] * g.dV);
    __syncthreads();
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = wib * kCellsPerWarp;
    if (j0 < nc) {
        const int jn = min(kCellsPerWarp, nc - j0);
        uint32_t o[kCellsPerWarp + 1];
#pragma unroll
        for (int j = 0; j <= kCellsPerWarp; ++j) o[j] = s_off[j0 + min(j, jn)];
        const double lo_edge = s_edges[0], hi_edge = s_edges[n_bins];
        for (uint32_t i0 = o[0]; i0 < o[kCellsPerWarp]; i0 += 32) {
            const uint32_t i = i0 + lane;
            int key = -1;
            double v = 0.0;
            if (i < o[kCellsPerWarp]) {
                const double r = diag_radius(s, i, wet);
                if (r >= lo_edge && r < hi_edge) {
                    // edges are >= 0 and so is r here (r >= edges[0]; -0.0
                    // made +0.0): their bit patterns order like their
                    // values, and the search compares integers, not FP64
                    const long long rb = __double_as_longlong(r + 0.0);
                    int lo = 0, hi = n_bins;  // s_edges[lo] <= r < s_edges[hi]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (__double_as_longlong(s_edges[mid]) <= rb) lo = mid;
                        else hi = mid;
                    }
                    int j = 0;
#pragma unroll
                    for (int q = 1; q < kCellsPerWarp; ++q) j += i >= o[q];
                    key = (j0 + j) * stride + lo;
                    v = (double)s.N[i] * pow_k(r, k);
                }
            }
            const unsigned grp = __match_any_sync(0xffffffffu, key);
            const bool lead = key >= 0 && (__ffs(grp) - 1) == lane;
            const int gmax = (int)__reduce_max_sync(0xffffffffu, key >= 0 ? (unsigned)__popc(grp) : 0u);
            unsigned rest = grp & (grp - 1);  // the group without its lowest lane
            double x = v;
            for (int it = 1; it < gmax; ++it) {
                const int src = lead && rest ? __ffs(rest) - 1 : lane;
                const double y = __shfl_sync(0xffffffffu, v, src);
                if (lead && rest) {
                    x += y;
                    rest &= rest - 1;
                }
            }
            if (lead) s_acc[key] += x;
        }
    }
    __syncthreads();
    // bin-major rows: 32 consecutive cells of one bin per warp store
    for (int t = threadIdx.x; t < n_bins * kDiagCells; t += blockDim.x) {
        const int b = t / kDiagCells, j = t % kDiagCells;
        if (j < nc) out[(int64_t)b * g.n_cells + c0 + j] = s_acc[j * stride + b] * s_inv[j];
    }
}

size_t spectrum_smem_bytes(int n_bins) {
    return sizeof(double) * ((size_t)kMaxSpectrumBins + 1 + (size_t)kDiagCells * (size_t)(n_bins | 1));
}

cudaError_t launch_spectrum(sdm_ctx *c, int wet, int n_bins, int k) {
    const size_t smem = spectrum_smem_bytes(n_bins);
    static std::atomic<unsigned long long> attr_done{0};
    const cudaError_t e = smem_attr_once(k_spectrum, (int)spectrum_smem_bytes(kMaxSpectrumBins), attr_done);
    if (e != cudaSuccess) return e;
    const int nb = (c->grid.n_cells + kDiagCells - 1) / kDiagCells;
    k_spectrum<<<nb, kDiagWarps * 32, smem, c->stream>>>(c->buf[c->cur], c->offset, c->rhod, c->grid, c->spec_edges,
                                                         n_bins, wet, k, c->spec_buf);
    return cudaGetLastError();
}

cudaError_t launch_moments(sdm_ctx *c, int k) {
    const int nb = (c->grid.n_cells + kDiagCells - 1) / kDiagCells;
    k_moments<<<nb, kDiagWarps * 32, 0, c->stream>>>(c->buf[c->cur], c->offset, c->rhod, c->grid, c->diag_wet,
                                                     c->diag_rmin, c->diag_rmax, k, c->outbuf);
    return cudaGetLastError();
}

cudaError_t launch_sd_conc(sdm_ctx *c) {
    const int B = 256;
    k_sd_conc<<<grid_for((int64_t)c->grid.n_cells * 32, B), B, 0, c->stream>>>(
        c->buf[c->cur], c->offset, c->grid, c->outbuf);
    return cudaGetLastError();
}

struct Shape3 {
    int n[3];
    int64_t s[3];
    int ndim;
};

__global__ void k_field_gather(double *dst, const double *src, Shape3 sh, int64_t total) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int64_t rem = t, off = 0;
    for (int d = sh.ndim - 1; d >= 0; --d) {
        const int64_t i = rem % sh.n[d];
        rem /= sh.n[d];
        off += i * sh.s[d];
    }
    dst[t] = src[off];
}

__global__ void k_field_scatter(double *dst, const double *src, Shape3 sh, int64_t total) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int64_t rem = t, off = 0;
    for (int d = sh.ndim - 1; d >= 0; --d) {
        const int64_t i = rem % sh.n[d];
        rem /= sh.n[d];
        off += i * sh.s[d];
    }
    dst[off] = src[t];
}

static Shape3 make_shape(const int64_t *strides, int ndim, const int *shape, int64_t *total) {
    Shape3 sh{};
    sh.ndim = ndim;
    *total = 1;
    for (int d = 0; d < ndim; ++d) {
        sh.n[d] = shape[d];
        sh.s[d] = strides[d];
        *total *= shape[d];
    }
    return sh;
}

cudaError_t launch_field_gather(double *dst, const double *src, const int64_t *strides, int ndim,
                                const int *shape, cudaStream_t st) {
    int64_t total;
    const Shape3 sh = make_shape(strides, ndim, shape, &total);
    const int B = 256;
    k_field_gather<<<grid_for(total, B), B, 0, st>>>(dst, src, sh, total);
    return cudaGetLastError();
}

cudaError_t launch_field_scatter(double *dst, const double *src, const int64_t *strides, int ndim,
                                 const int *shape, cudaStream_t st) {
    int64_t total;
    const Shape3 sh = make_shape(strides, ndim, shape, &total);
    const int B = 256;
    k_field_scatter<<<grid_for(total, B), B, 0, st>>>(dst, src, sh, total);
    return cudaGetLastError();
}

}  // namespace sdm
