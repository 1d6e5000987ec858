// Diagnostics (paper Sec. 5.2.1): per-cell moments of the wet or dry
// spectrum over a radius range, M^k = (rho_d dV)^-1 sum N r^k, and the count
// of super-droplets with non-zero multiplicity; one warp per cell.
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
