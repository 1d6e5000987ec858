// Standalone counting sort of particles by grid cell (the regrouping step
// that makes the cell-wise pairing of Sec. 5.1.4 and the cell sums of
// Sec. 5.1.3 possible): histogram with per-cell atomics that also hand out
// a slot, exclusive scan of the counts, scatter of particle indices.
#include "sdm_internal.cuh"

namespace sdm {

__global__ void k_count_slots(const uint32_t *cell, int64_t n, uint32_t n_cells, uint32_t *count,
                              uint32_t *slot, unsigned *bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c = cell[i];
    if (c >= n_cells) {  // reported, never written out of bounds
        atomicOr(bad, 1u);
        slot[i] = 0xffffffffu;
        return;
    }
    slot[i] = atomicAdd(count + c, 1u);
}

__global__ void k_scatter_perm(const uint32_t *cell, const uint32_t *slot, const uint32_t *offset,
                               int64_t n, uint32_t n_cells, uint32_t *perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c = cell[i];
    if (c >= n_cells) return;
    perm[offset[c] + slot[i]] = (uint32_t)i;
}

cudaError_t cell_sort_with_scratch(const uint32_t *cell, int64_t n, uint32_t n_cells, uint32_t *perm,
                                   uint32_t *offsets, uint32_t *count, uint32_t *slot,
                                   uint32_t *scan_tmp, unsigned *bad, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint32_t) * ((size_t)n_cells + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const int B = 256;
    if (n > 0) k_count_slots<<<grid_for(n, B), B, 0, st>>>(cell, n, n_cells, count, slot, bad);
    e = scan_counts(count, offsets, scan_tmp, (int)n_cells, st);
    if (e != cudaSuccess) return e;
    if (n > 0) k_scatter_perm<<<grid_for(n, B), B, 0, st>>>(cell, slot, offsets, n, n_cells, perm);
    return cudaGetLastError();
}

}  // namespace sdm

using namespace sdm;

extern "C" sdm_status sdm_cell_sort(const uint32_t *cell, int64_t n, int32_t n_cells, uint32_t *perm,
                                    uint32_t *offsets, void *stream) {
    if (n < 0 || n_cells < 1 || (n > 0 && (!cell || !perm)) || !offsets) return SDM_EINVAL;
    if (n >= (int64_t)0xffffffffLL) return SDM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nb = (size_t)n_cells / 1024 + 2;
    const size_t bytes = sizeof(uint32_t) * ((size_t)n_cells + 1 + (size_t)n + nb) + 256;
    void *scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return SDM_ENOMEM;
    }
    uint32_t *count = (uint32_t *)scratch;
    uint32_t *slot = count + n_cells + 1;
    uint32_t *tmp = slot + n;
    unsigned *bad = (unsigned *)(tmp + nb);
    cudaError_t e = cell_sort_with_scratch(cell, n, (uint32_t)n_cells, perm, offsets, count, slot, tmp,
                                           bad, st);
    unsigned hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return SDM_ECUDA;
    return hbad ? SDM_EINVAL : SDM_OK;
}
