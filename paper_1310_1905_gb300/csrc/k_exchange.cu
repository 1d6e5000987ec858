// The device side of the exchange of super-droplets between the slabs of a
// domain decomposed in x (the paper leaves decomposition to the solver that
// calls the library, Sec. 5.2): the leavers of a slab (N > 0, x outside
// [0, X)) are compacted, in storage order, into a block and their slots
// freed; arrivals take the free slots (N = 0), the k-th arrival the k-th
// free slot in storage order.  Both go through one flag pass and the
// library's exclusive scan, so the order is deterministic.
#include "sdm_internal.cuh"

namespace sdm {

__global__ void k_xch_flag(SdArrays s, int64_t n, Grid g, int leavers, uint32_t *flag) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const unsigned long long N = s.N[q];
    bool f;
    if (leavers) {
        const double x = s.x[q], X = g.nx * g.dx;
        f = N > 0 && !(x >= 0.0 && x < X);
    } else {
        f = N == 0;
    }
    flag[q] = f ? 1u : 0u;
}

__global__ void k_xch_export(SdArrays s, int64_t n, Grid g, const uint32_t *flag, const uint32_t *off,
                             sdm_sd_block b) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n || !flag[q]) return;
    const uint32_t k = off[q];
    b.N[k] = s.N[q];
    b.uid[k] = s.uid[q];
    b.rw2[k] = s.rw2[q];
    b.rd3[k] = s.rd3[q];
    b.kappa[k] = s.kappa[q];
    b.x[k] = s.x[q];
    if (g.ny > 0 && b.y) b.y[k] = s.y[q];
    if (g.nz > 0 && b.z) b.z[k] = s.z[q];
    s.N[q] = 0;
    s.uid[q] |= kUidVacant;  // its id lives on with the leaver: the slot waits for an arrival
}

__global__ void k_xch_import(SdArrays s, int64_t n, Grid g, const uint32_t *flag, const uint32_t *off,
                             sdm_sd_block b, int64_t m) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n || !flag[q]) return;
    const uint32_t k = off[q];
    if ((int64_t)k >= m) return;
    s.N[q] = b.N[k];
    s.uid[q] = b.uid[k];
    s.rw2[q] = b.rw2[k];
    s.rd3[q] = b.rd3[k];
    s.kappa[q] = b.kappa[k];
    s.x[q] = b.x[k];
    if (g.ny > 0) s.y[q] = b.y[k];
    if (g.nz > 0) s.z[q] = b.z[k];
}

// positions outside the domain, N = 0 or a marked id in an arriving block
__global__ void k_xch_check(sdm_sd_block b, int64_t m, Grid g, unsigned *bad) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    bool ok = b.N[k] > 0 && !(b.uid[k] & kUidVacant) && b.x[k] >= 0.0 && b.x[k] < g.nx * g.dx;
    if (g.ny > 0) ok = ok && b.y[k] >= 0.0 && b.y[k] < g.ny * g.dy;
    if (g.nz > 0) ok = ok && b.z[k] >= 0.0 && b.z[k] < g.nz * g.dz;
    if (!ok) atomicOr(bad, 1u);
}

static cudaError_t ensure_scratch(sdm_ctx *c) {
    cudaError_t e = cudaSuccess;
    if (!c->xch_flag) e = cudaMalloc(&c->xch_flag, 4 * ((size_t)c->n_sd + 1));
    if (e == cudaSuccess && !c->xch_off) e = cudaMalloc(&c->xch_off, 4 * ((size_t)c->n_sd + 1));
    if (e == cudaSuccess && !c->xch_tmp) e = cudaMalloc(&c->xch_tmp, 4 * ((size_t)c->n_sd / 1024 + 4));
    return e;
}

// flag the leavers (leavers = 1) or the free slots (0) and scan the flags;
// the total comes back to the host (the call synchronises the stream)
cudaError_t launch_exchange_count(sdm_ctx *c, int leavers, uint32_t *total_host) {
    cudaError_t e = ensure_scratch(c);
    if (e != cudaSuccess) return e;
    const int B = 256;
    k_xch_flag<<<grid_for(c->n_sd, B), B, 0, c->stream>>>(c->buf[c->cur], c->n_sd, c->grid, leavers, c->xch_flag);
    e = scan_counts(c->xch_flag, c->xch_off, c->xch_tmp, (int)c->n_sd, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(total_host, c->xch_off + c->n_sd, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e;
}

cudaError_t launch_export(sdm_ctx *c, const sdm_sd_block &dst) {
    const int B = 256;
    k_xch_export<<<grid_for(c->n_sd, B), B, 0, c->stream>>>(c->buf[c->cur], c->n_sd, c->grid, c->xch_flag,
                                                            c->xch_off, dst);
    return cudaGetLastError();
}

cudaError_t launch_import(sdm_ctx *c, const sdm_sd_block &src, int64_t n) {
    const int B = 256;
    k_xch_import<<<grid_for(c->n_sd, B), B, 0, c->stream>>>(c->buf[c->cur], c->n_sd, c->grid, c->xch_flag,
                                                            c->xch_off, src, n);
    return cudaGetLastError();
}

cudaError_t launch_block_check(sdm_ctx *c, const sdm_sd_block &src, int64_t n, unsigned *bad_host) {
    cudaError_t e = ensure_scratch(c);
    if (e != cudaSuccess) return e;
    unsigned *bad = c->xch_tmp;  // one word of the scan scratch, not in use here
    e = cudaMemsetAsync(bad, 0, 4, c->stream);
    const int B = 256;
    if (e == cudaSuccess && n > 0) k_xch_check<<<grid_for(n, B), B, 0, c->stream>>>(src, n, c->grid, bad);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(bad_host, bad, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e;
}

}  // namespace sdm
