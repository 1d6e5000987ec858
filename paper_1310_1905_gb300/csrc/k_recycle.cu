// Recycling of zero-multiplicity super-droplets (paper Sec. 5.1.4): the
// k-th zero in id order takes every attribute of the k-th donor in
// (multiplicity descending, id ascending) order among donors with N >= 2;
// the clone gets floor(N/2), the donor keeps the rest.
//
// Only run when the previous step left zeros (the host knows the count from
// sdm_wait).  The nz zeros are compacted and sorted by id.  Of the donors
// only the first nz in that order are needed: a radix select on N (eight
// 8-bit digits, from the top) and then on the id among ties at the
// threshold finds them without sorting every super-droplet, and only those
// nz are compacted and sorted.
#include "sdm_internal.cuh"

namespace sdm {

constexpr int kSmemSort = 8192;  // records sorted in one block (128 KB)

// zeros compacted; donors (N >= 2) counted
__global__ void k_rc_compact(SdArrays s, int64_t n, SortRec *zrec, DevStats *st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool donor = false;
    if (i < n) {
        const unsigned long long N = s.N[i];
        if (N == 0 && !(s.uid[i] & kUidVacant)) {  // a slot kept for arrivals is no zero to fill
            const unsigned q = atomicAdd(&st->n_rc_zero, 1u);
            zrec[q] = SortRec{(unsigned long long)s.uid[i], 0u, (uint32_t)i};
        }
        donor = N >= 2;
    }
    const unsigned nd = __popc(__ballot_sync(0xffffffffu, donor));
    if ((threadIdx.x & 31) == 0 && nd) atomicAdd(&st->n_rc_donor, nd);
}

// Radix select of the first k donors in (N descending, id ascending) order.
struct RcSelect {
    unsigned long long prefix, mask;  // the N digits fixed so far
    unsigned k;                       // donors still to take at the current prefix
    unsigned uprefix, umask;          // the id digits fixed so far (ties at N = prefix)
};

// digit histogram of the donors that match the fixed digits: of N (by_id =
// 0) or, among N = prefix, of the id (by_id = 1)
__global__ void k_rc_hist(SdArrays s, int64_t n, const RcSelect *sel, int shift, int by_id, unsigned *hist) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const RcSelect S = *sel;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long N = s.N[i];
        if (N < 2) continue;
        if (!by_id) {
            if ((N & S.mask) == S.prefix) atomicAdd(&h[(unsigned)(N >> shift) & 255u], 1u);
        } else if (N == S.prefix) {
            const unsigned u = s.uid[i];
            if ((u & S.umask) == S.uprefix) atomicAdd(&h[(u >> shift) & 255u], 1u);
        }
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// fix the next digit: N from the largest bin down, ids from the smallest up
__global__ void k_rc_pick(RcSelect *sel, unsigned *hist, int shift, int by_id) {
    if (threadIdx.x != 0) return;
    RcSelect S = *sel;
    unsigned acc = 0;
    for (int j = 0; j < 256; ++j) {
        const int b = by_id ? j : 255 - j;
        const unsigned c = hist[b];
        if (acc + c >= S.k) {
            S.k -= acc;
            if (!by_id) {
                S.prefix |= (unsigned long long)b << shift;
                S.mask |= 255ull << shift;
            } else {
                S.uprefix |= (unsigned)b << shift;
                S.umask |= 255u << shift;
            }
            break;
        }
        acc += c;
    }
    *sel = S;
    for (int b = 0; b < 256; ++b) hist[b] = 0;
}

// the selected donors: N > T, or N = T with id <= U (take_all: every N >= 2)
__global__ void k_rc_donors(SdArrays s, int64_t n, const RcSelect *sel, int take_all, SortRec *drec,
                            DevStats *st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long N = s.N[i];
    if (N < 2) return;
    bool take = take_all;
    if (!take) {
        const RcSelect S = *sel;
        take = N > S.prefix || (N == S.prefix && s.uid[i] <= S.uprefix);
    }
    if (take) {
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

// records ordered by (hi, lo), ties by val
__device__ __forceinline__ bool srec_gt(const SortRec &a, const SortRec &b) {
    return a.hi > b.hi || (a.hi == b.hi && (a.lo > b.lo || (a.lo == b.lo && a.val > b.val)));
}

// The whole recycling in one block where the state has at most kSmemSort
// super-droplets, with no count travelling to the host.  The zeros are
// compacted (key: the id).  Of the donors only the first np = min(zeros,
// donors) in (N descending, id ascending) order are needed: a radix select
// over the key (~N, id), eight 8-bit digits of ~N from the top and then
// four of the id, finds the np-th smallest key T, and the donors with keys
// up to T are appended (key: ~N, which for any multiplicity below 2^63 lies
// above every id).  One bitonic sort of the zeros and those donors puts the
// zeros first, by id, then the donors in order; the k-th zero takes the
// k-th donor.
__global__ void __launch_bounds__(1024) k_rc_small(SdArrays s, int n, DevStats *st) {
    extern __shared__ SortRec r[];
    __shared__ unsigned s_m, s_nz, s_nd, s_k, hist[256];
    __shared__ unsigned long long s_phi, s_mhi;  // fixed digits of ~N and their mask
    __shared__ unsigned s_plo, s_mlo;            // fixed digits of the id and their mask
    if (threadIdx.x == 0) {
        s_m = s_nz = s_nd = 0;
        s_phi = s_mhi = 0ull;
        s_plo = s_mlo = 0u;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long N = s.N[i];
        if (N == 0 && !(s.uid[i] & kUidVacant)) {
            r[atomicAdd(&s_m, 1u)] = SortRec{(unsigned long long)s.uid[i], 0u, (uint32_t)i};
            atomicAdd(&s_nz, 1u);
        } else if (N >= 2) {
            atomicAdd(&s_nd, 1u);
        }
    }
    __syncthreads();
    const unsigned nz = s_nz, nd = s_nd, np = nz < nd ? nz : nd;
    if (np == 0) return;
    const bool take_all = nd <= nz;
    if (!take_all) {
        if (threadIdx.x == 0) s_k = np;  // the rank (from 1) still to find under the fixed digits
        for (int pass = 0; pass < 12; ++pass) {
            const bool on_id = pass >= 8;
            const int shift = on_id ? 24 - 8 * (pass - 8) : 56 - 8 * pass;
            if (threadIdx.x < 256) hist[threadIdx.x] = 0;
            __syncthreads();
            const unsigned long long phi = s_phi, mhi = s_mhi;
            const unsigned plo = s_plo, mlo = s_mlo;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const unsigned long long N = s.N[i];
                if (N < 2) continue;
                const unsigned long long hi = ~N;
                const unsigned lo = s.uid[i];
                if ((hi & mhi) != phi || (lo & mlo) != plo) continue;
                const unsigned d = on_id ? (lo >> shift) & 0xffu : (unsigned)((hi >> shift) & 0xffu);
                atomicAdd(&hist[d], 1u);
            }
            __syncthreads();
            if (threadIdx.x < 32) {  // the bin holding rank k, from the smallest digit up
                const int lane = threadIdx.x;
                unsigned v[8], tot = 0;
                for (int j = 0; j < 8; ++j) tot += (v[j] = hist[lane * 8 + j]);
                unsigned incl = tot;
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                const unsigned k = s_k;
                unsigned before = incl - tot;
                const bool mine = before < k && k <= incl;
                if (mine) {
                    int j = 0;
                    while (before + v[j] < k) before += v[j++];
                    const unsigned d = (unsigned)(lane * 8 + j);
                    s_k = k - before;
                    if (on_id) {
                        s_plo |= d << shift;
                        s_mlo |= 0xffu << shift;
                    } else {
                        s_phi |= (unsigned long long)d << shift;
                        s_mhi |= 0xffull << shift;
                    }
                }
            }
            __syncthreads();
        }
    }
    // the selected donors after the zeros: every donor, or those with keys up to T
    const unsigned long long thi = s_phi;
    const unsigned tlo = s_plo;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long N = s.N[i];
        if (N < 2) continue;
        const unsigned long long hi = ~N;
        const unsigned lo = s.uid[i];
        if (take_all || hi < thi || (hi == thi && lo <= tlo))
            r[atomicAdd(&s_m, 1u)] = SortRec{hi, lo, (uint32_t)i};
    }
    __syncthreads();
    const unsigned m = s_m;
    const unsigned npa = m - nz < np ? m - nz : np;  // = np (keys are unique); never read past the donors
    unsigned np2 = 1;
    while (np2 < m) np2 <<= 1;
    for (unsigned i = m + threadIdx.x; i < np2; i += blockDim.x) r[i] = SortRec{~0ull, ~0u, ~0u};
    __syncthreads();
    for (unsigned k = 2; k <= np2; k <<= 1) {
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            for (unsigned i = threadIdx.x; i < np2; i += blockDim.x) {
                const unsigned ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const SortRec a = r[i], b = r[ixj];
                    if (srec_gt(a, b) == up) {
                        r[i] = b;
                        r[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (unsigned q = threadIdx.x; q < npa; q += blockDim.x) {
        const uint32_t z = r[q].val, d = r[nz + q].val;
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
    if (threadIdx.x == 0) atomicAdd(&st->n_recycled, (unsigned long long)npa);
}

bool recycle_small(const sdm_ctx *c) { return c->n_sd <= kSmemSort; }

cudaError_t launch_recycle_small(sdm_ctx *c) {
    static std::atomic<unsigned long long> attr_done{0};
    const int bytes = (int)(sizeof(SortRec) * kSmemSort);
    cudaError_t e = smem_attr_once(k_rc_small, bytes, attr_done);
    if (e != cudaSuccess) return e;
    k_rc_small<<<1, 1024, bytes, c->stream>>>(c->buf[c->cur], (int)c->n_sd, c->dstats);
    return cudaGetLastError();
}

cudaError_t launch_recycle_compact(sdm_ctx *c) {
    cudaError_t e = cudaMemsetAsync(&c->dstats->n_rc_zero, 0, 2 * sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return e;
    SortRec *zrec = (SortRec *)c->rc_tmp;
    const int B = 256;
    k_rc_compact<<<grid_for(c->n_sd, B), B, 0, c->stream>>>(c->buf[c->cur], c->n_sd, zrec, c->dstats);
    return cudaGetLastError();
}

static uint32_t pow2_at_least(uint32_t n) {
    uint32_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

// nz zeros and nd donors counted by launch_recycle_compact
cudaError_t launch_recycle_apply(sdm_ctx *c, uint32_t nz, uint32_t nd) {
    SortRec *zrec = (SortRec *)c->rc_tmp;
    SortRec *drec = zrec + (c->rc_tmp_bytes / sizeof(SortRec)) / 2;
    RcSelect *sel = (RcSelect *)(c->rc_sel);
    unsigned *hist = (unsigned *)(sel + 1);
    const uint32_t np = nz < nd ? nz : nd;
    const int B = 256;
    // every donor is taken, or they all fit one block's shared-memory sort:
    // sort them all and use the first np
    const int take_all = nd <= nz || nd <= (uint32_t)kSmemSort;
    const uint32_t ns = take_all ? nd : np;  // donor records compacted and sorted
    const int hist_blocks = 4 * 152;
    int launches = 0;
    if (!take_all) {
        RcSelect init{0ull, 0ull, np, 0u, 0u};
        cudaError_t e = cudaMemcpyAsync(sel, &init, sizeof(init), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned), c->stream);
        if (e != cudaSuccess) return e;
        for (int by_id = 0; by_id < 2; ++by_id) {
            for (int shift = by_id ? 24 : 56; shift >= 0; shift -= 8) {
                k_rc_hist<<<hist_blocks, 256, 0, c->stream>>>(c->buf[c->cur], c->n_sd, sel, shift, by_id, hist);
                k_rc_pick<<<1, 32, 0, c->stream>>>(sel, hist, shift, by_id);
                launches += 2;
            }
        }
    }
    cudaError_t e = cudaMemsetAsync(&c->dstats->n_rc_donor, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return e;
    k_rc_donors<<<grid_for(c->n_sd, B), B, 0, c->stream>>>(c->buf[c->cur], c->n_sd, sel, take_all, drec, c->dstats);
    e = sort_records(zrec, nz, pow2_at_least(nz), c->stream);
    if (e == cudaSuccess) e = sort_records(drec, ns, pow2_at_least(ns), c->stream);
    if (e != cudaSuccess) return e;
    k_rc_apply<<<grid_for(np, B), B, 0, c->stream>>>(c->buf[c->cur], zrec, drec, np);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    c->host_recycled += np;
    c->tacc.launches += launches + 2 + (nz > 1 ? 2 : 0) + (ns > 1 ? 2 : 0);  // select, donors, apply, sorts
    return cudaSuccess;
}

// ---- bitonic sort of SortRec records by (hi, lo), padded to a power of two

__global__ void k_fill_max(SortRec *r, uint32_t from, uint32_t to) {
    const uint32_t i = from + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < to) r[i] = SortRec{~0ull, ~0u, ~0u};
}

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
        static std::atomic<unsigned long long> attr_done{0};
        const cudaError_t e = smem_attr_once(k_sort_smem, (int)(sizeof(SortRec) * kSmemSort), attr_done);
        if (e != cudaSuccess) return e;
        k_sort_smem<<<1, 1024, sizeof(SortRec) * npow2, st>>>(rec, npow2);
        return cudaGetLastError();
    }
    for (uint32_t k = 2; k <= npow2; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1)
            k_sort_step<<<grid_for(npow2, B), B, 0, st>>>(rec, npow2, k, j);
    return cudaGetLastError();
}

}  // namespace sdm
