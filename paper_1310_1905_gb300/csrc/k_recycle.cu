// Recycling of zero-multiplicity super-droplets (paper Sec. 5.1.4): the
// k-th zero in id order takes every attribute of the k-th donor in
// (multiplicity descending, id ascending) order among donors with N >= 2;
// the clone gets floor(N/2), the donor keeps the rest.
//
// Only run when the previous step left zeros (the host knows the count from
// sdm_wait).  Zeros and donors are compacted, then both lists are sorted.
#include "sdm_internal.cuh"

namespace sdm {

__global__ void k_rc_compact(SdArrays s, int64_t n, SortRec *zrec, SortRec *drec, DevStats *st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long N = s.N[i];
    if (N == 0) {
        const unsigned q = atomicAdd(&st->n_rc_zero, 1u);
        zrec[q] = SortRec{(unsigned long long)s.uid[i], 0u, (uint32_t)i};
    } else if (N >= 2) {
        const unsigned q = atomicAdd(&st->n_rc_donor, 1u);
        drec[q] = SortRec{~N, s.uid[i], (uint32_t)i};  // ascending ~N = descending N
    }
}

__global__ void k_rc_apply(SdArrays s, const SortRec *zrec, const SortRec *drec, uint32_t np) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    const uint32_t z = zrec[q].val, d = drec[q].val;
    s.rw2[z] = s.rw2[d];
    s.rd3[z] = s.rd3[d];
    s.kappa[z] = s.kappa[d];
    if (s.x) s.x[z] = s.x[d];
    if (s.y) s.y[z] = s.y[d];
    if (s.z) s.z[z] = s.z[d];
    const unsigned long long Nd = s.N[d];
    s.N[z] = Nd / 2;
    s.N[d] = Nd - Nd / 2;
}

cudaError_t launch_recycle_compact(sdm_ctx *c) {
    cudaError_t e = cudaMemsetAsync(&c->dstats->n_rc_zero, 0, 2 * sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return e;
    SortRec *zrec = (SortRec *)c->rc_tmp;
    SortRec *drec = zrec + (c->rc_tmp_bytes / sizeof(SortRec)) / 2;
    const int B = 256;
    k_rc_compact<<<grid_for(c->n_sd, B), B, 0, c->stream>>>(c->buf[c->cur], c->n_sd, zrec, drec,
                                                            c->dstats);
    return cudaGetLastError();
}

static uint32_t pow2_at_least(uint32_t n) {
    uint32_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

cudaError_t launch_recycle_apply(sdm_ctx *c, uint32_t nz, uint32_t nd) {
    SortRec *zrec = (SortRec *)c->rc_tmp;
    SortRec *drec = zrec + (c->rc_tmp_bytes / sizeof(SortRec)) / 2;
    cudaError_t e = sort_records(zrec, nz, pow2_at_least(nz), c->stream);
    if (e == cudaSuccess) e = sort_records(drec, nd, pow2_at_least(nd), c->stream);
    if (e != cudaSuccess) return e;
    const uint32_t np = nz < nd ? nz : nd;
    const int B = 256;
    k_rc_apply<<<grid_for(np, B), B, 0, c->stream>>>(c->buf[c->cur], zrec, drec, np);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    c->host_recycled += np;
    c->tacc.launches += 1 + (nz > 1 ? 2 : 0) + (nd > 1 ? 2 : 0);  // apply, fills and sorts
    return cudaSuccess;
}

// ---- bitonic sort of SortRec records by (hi, lo), padded to a power of two
__device__ __forceinline__ bool srec_gt(const SortRec &a, const SortRec &b) {
    return a.hi > b.hi || (a.hi == b.hi && (a.lo > b.lo || (a.lo == b.lo && a.val > b.val)));
}

__global__ void k_fill_max(SortRec *r, uint32_t from, uint32_t to) {
    const uint32_t i = from + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < to) r[i] = SortRec{~0ull, ~0u, ~0u};
}

constexpr int kSmemSort = 8192;  // records sorted in one block (128 KB)

__global__ void __launch_bounds__(1024) k_sort_smem(SortRec *r, uint32_t npow2) {
    extern __shared__ SortRec s[];
    for (uint32_t i = threadIdx.x; i < npow2; i += blockDim.x) s[i] = r[i];
    __syncthreads();
    for (uint32_t k = 2; k <= npow2; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < npow2; i += blockDim.x) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const SortRec a = s[i], b = s[ixj];
                    if (srec_gt(a, b) == up) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t i = threadIdx.x; i < npow2; i += blockDim.x) r[i] = s[i];
}

__global__ void k_sort_step(SortRec *r, uint32_t npow2, uint32_t k, uint32_t j) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npow2) return;
    const uint32_t ixj = i ^ j;
    if (ixj > i) {
        const bool up = (i & k) == 0;
        const SortRec a = r[i], b = r[ixj];
        if (srec_gt(a, b) == up) {
            r[i] = b;
            r[ixj] = a;
        }
    }
}

cudaError_t sort_records(SortRec *rec, uint32_t n, uint32_t npow2, cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    const int B = 256;
    if (npow2 > n) k_fill_max<<<grid_for(npow2 - n, B), B, 0, st>>>(rec, n, npow2);
    if (npow2 <= (uint32_t)kSmemSort) {
        static bool attr_set = false;
        const int bytes = (int)(sizeof(SortRec) * kSmemSort);
        if (!attr_set) {
            const cudaError_t e =
                cudaFuncSetAttribute(k_sort_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess) return e;
            attr_set = true;
        }
        k_sort_smem<<<1, 1024, sizeof(SortRec) * npow2, st>>>(rec, npow2);
        return cudaGetLastError();
    }
    for (uint32_t k = 2; k <= npow2; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1)
            k_sort_step<<<grid_for(npow2, B), B, 0, st>>>(rec, npow2, k, j);
    return cudaGetLastError();
}

}  // namespace sdm
