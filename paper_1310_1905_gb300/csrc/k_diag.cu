// Diagnostics (paper Sec. 5.2.1): per-cell moments of the wet or dry
// spectrum over a radius range, M^k = (rho_d dV)^-1 sum N r^k, and the count
// of super-droplets with non-zero multiplicity; one warp per cell.  The
// binned spectrum computes that moment for many radius bins in one pass.
// Also the strided gather/scatter of caller-owned device fields (arrinfo_t).
#include "sdm_internal.cuh"

namespace sdm {

__global__ void k_moments(SdArrays s, const uint32_t *offset, const double *rhod, Grid g, int wet,
                          double rmin, double rmax, int k, double *out) {
    const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= g.n_cells) return;
    double sum = 0.0;
    for (uint32_t i = offset[c] + lane; i < offset[c + 1]; i += 32) {
        const double r = wet ? sqrt(s.rw2[i]) : cbrt(s.rd3[i]);
        if (!(r >= rmin && r <= rmax)) continue;
        double p = 1.0;
        for (int e = 0; e < k; ++e) p *= r;
        sum += (double)s.N[i] * p;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) out[c] = sum / (rhod[c] * g.dV);
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
// once, out[b * n_cells + c].  One warp per cell; the warp's bins sit in
// shared memory.  Each group of 32 super-droplets finds its bins by binary
// search, then every distinct bin of the group is summed by a butterfly
// over the lanes (the others add zero): the order of the additions is
// fixed, so the result does not depend on scheduling.
constexpr int kSpecWarps = 4;

__global__ void __launch_bounds__(kSpecWarps * 32)
    k_spectrum(SdArrays s, const uint32_t *offset, const double *rhod, Grid g, const double *edges, int n_bins,
               int wet, int k, double *out) {
    __shared__ double s_edges[kMaxSpectrumBins + 1];
    __shared__ double s_acc[kSpecWarps][kMaxSpectrumBins];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i <= n_bins; i += blockDim.x) s_edges[i] = edges[i];
    for (int i = lane; i < n_bins; i += 32) s_acc[wib][i] = 0.0;
    __syncthreads();
    const int c = blockIdx.x * kSpecWarps + wib;
    if (c >= g.n_cells) return;
    const double lo_edge = s_edges[0], hi_edge = s_edges[n_bins];
    const uint32_t end = offset[c + 1];
    for (uint32_t i0 = offset[c]; i0 < end; i0 += 32) {
        const uint32_t i = i0 + lane;
        int b = -1;
        double v = 0.0;
        if (i < end) {
            const double r = wet ? sqrt(s.rw2[i]) : cbrt(s.rd3[i]);
            if (r >= lo_edge && r < hi_edge) {
                int lo = 0, hi = n_bins;  // s_edges[lo] <= r < s_edges[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (s_edges[mid] <= r) lo = mid;
                    else hi = mid;
                }
                b = lo;
                double p = 1.0;
                for (int e = 0; e < k; ++e) p *= r;
                v = (double)s.N[i] * p;
            }
        }
        unsigned todo = __ballot_sync(0xffffffffu, b >= 0);
        while (todo) {
            const int bl = __shfl_sync(0xffffffffu, b, __ffs(todo) - 1);
            double x = b == bl ? v : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) s_acc[wib][bl] += x;
            todo &= ~__ballot_sync(0xffffffffu, b == bl);
        }
    }
    __syncwarp();
    const double den = rhod[c] * g.dV;
    for (int b = lane; b < n_bins; b += 32) out[(int64_t)b * g.n_cells + c] = s_acc[wib][b] / den;
}

cudaError_t launch_spectrum(sdm_ctx *c, int wet, int n_bins, int k) {
    const int nb = (c->grid.n_cells + kSpecWarps - 1) / kSpecWarps;
    k_spectrum<<<nb, kSpecWarps * 32, 0, c->stream>>>(c->buf[c->cur], c->offset, c->rhod, c->grid, c->spec_edges,
                                                      n_bins, wet, k, c->spec_buf);
    return cudaGetLastError();
}

cudaError_t launch_moments(sdm_ctx *c, int k) {
    const int B = 256;
    k_moments<<<grid_for((int64_t)c->grid.n_cells * 32, B), B, 0, c->stream>>>(
        c->buf[c->cur], c->offset, c->rhod, c->grid, c->diag_wet, c->diag_rmin, c->diag_rmax, k,
        c->outbuf);
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
