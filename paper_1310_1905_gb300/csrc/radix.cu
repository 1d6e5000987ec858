// Stable LSD radix sort of (key, value) records with 8-bit digits, used to
// put every member of a batched ensemble into the random order that its
// pairing needs (Sec. 5.1.4): the key words are sorted digit by digit from
// the least significant, then the member index, so that the final order is
// (member, key, original position) - the order of the oracle's
// (key, id) sort inside each member, since members store ids ascending.
//
// One pass: per-tile digit histograms (256 bins), an exclusive scan of the
// digit-major histogram table, then a stable scatter in which every tile
// ranks its elements by digit in their original order.
#include <utility>

#include "sdm_internal.cuh"

namespace sdm {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;                       // items per thread
constexpr int kRsTile = kRsThreads * kRsItems;     // 4096 records per tile
constexpr int kRsWarps = kRsThreads / 32;

template <class K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift) {
    return (uint32_t)(k >> shift) & 0xffu;
}

template <class K>
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const K *key, int64_t n, int shift, uint32_t *hist,
                                                        int n_tiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int i = 0; i < kRsItems; ++i) {
        const int64_t q = base + (int64_t)i * kRsThreads + threadIdx.x;
        if (q < n) atomicAdd(&h[digit_of(key[q], shift)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];  // digit-major
}

// K: the type of the word being sorted on; P: a passenger word moved along
template <class K, class P>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const K *key_in, const uint32_t *val_in,
                                                           const P *aux_in, K *key_out,
                                                           uint32_t *val_out, P *aux_out,
                                                           int64_t n, int shift, const uint32_t *offs,
                                                           int n_tiles) {
    __shared__ uint32_t base_d[256];      // running position of each digit
    __shared__ uint32_t wcnt[kRsWarps][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    base_d[threadIdx.x] = offs[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
    const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
    for (int i = 0; i < kRsItems; ++i) {
        for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
        __syncthreads();
        const int64_t q = tile0 + (int64_t)i * kRsThreads + threadIdx.x;
        const bool ok = q < n;
        K k = 0;
        uint32_t dg = 0xffffffffu;
        if (ok) {
            k = key_in[q];
            dg = digit_of(k, shift);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const unsigned lower = peers & ((1u << lane) - 1u);
        if (ok && lower == 0) wcnt[w][dg] = __popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t pos = base_d[dg] + __popc(lower);
            for (int v = 0; v < w; ++v) pos += wcnt[v][dg];
            key_out[pos] = k;
            val_out[pos] = val_in[q];
            if (aux_in) aux_out[pos] = aux_in[q];
        }
        __syncthreads();
        // advance the running bases by this round's counts
        uint32_t add = 0;
        for (int v = 0; v < kRsWarps; ++v) add += wcnt[v][threadIdx.x];
        base_d[threadIdx.x] += add;
        __syncthreads();
    }
}

// Sort n records by (aux, key) where aux < 2^(8*aux_bytes) and only the
// low key_bytes bytes of key are significant.  Buffers a (input, output)
// and b (scratch) each hold n keys, values and aux words; hist holds
// 256 * tiles + tiles/1024 + 2 words of scan space.
template <class K>
cudaError_t radix_sort_pairs(K *key_a, uint32_t *val_a, uint32_t *aux_a, K *key_b, uint32_t *val_b,
                             uint32_t *aux_b, int64_t n, int key_bytes, int aux_bytes, uint32_t *hist,
                             uint32_t *scan_tmp, cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    const int tiles = (int)((n + kRsTile - 1) / kRsTile);
    K *ka = key_a, *kb = key_b;
    uint32_t *va = val_a, *vb = val_b, *xa = aux_a, *xb = aux_b;
    int passes = 0;
    for (int byte = 0; byte < key_bytes + aux_bytes; ++byte) {
        const bool on_aux = byte >= key_bytes;
        const int shift = 8 * (on_aux ? byte - key_bytes : byte);
        if (!on_aux) {
            k_rs_hist<K><<<tiles, kRsThreads, 0, st>>>(ka, n, shift, hist, tiles);
            cudaError_t e = scan_counts(hist, hist, scan_tmp, 256 * tiles, st);
            if (e != cudaSuccess) return e;
            k_rs_scatter<K, uint32_t><<<tiles, kRsThreads, 0, st>>>(ka, va, xa, kb, vb, xb, n, shift, hist, tiles);
        } else {
            // sort by aux: aux acts as the key, the key rides along
            k_rs_hist<uint32_t><<<tiles, kRsThreads, 0, st>>>(xa, n, shift, hist, tiles);
            cudaError_t e = scan_counts(hist, hist, scan_tmp, 256 * tiles, st);
            if (e != cudaSuccess) return e;
            k_rs_scatter<uint32_t, K><<<tiles, kRsThreads, 0, st>>>(xa, va, ka, xb, vb, kb, n, shift, hist, tiles);
        }
        std::swap(ka, kb);
        std::swap(va, vb);
        std::swap(xa, xb);
        ++passes;
    }
    if (passes & 1) {  // result must end in the a buffers
        cudaMemcpyAsync(key_a, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(val_a, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(aux_a, xa, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
    }
    return cudaGetLastError();
}

}  // namespace sdm

namespace sdm {
template cudaError_t radix_sort_pairs<unsigned long long>(unsigned long long *, uint32_t *, uint32_t *,
                                                          unsigned long long *, uint32_t *, uint32_t *,
                                                          int64_t, int, int, uint32_t *, uint32_t *,
                                                          cudaStream_t);
template cudaError_t radix_sort_pairs<uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *, uint32_t *,
                                                uint32_t *, int64_t, int, int, uint32_t *, uint32_t *,
                                                cudaStream_t);
}  // namespace sdm
