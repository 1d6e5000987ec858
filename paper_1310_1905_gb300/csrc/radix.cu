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
// one thread per digit bin in the histogram and in the scatter's per-digit
// bookkeeping, and whole items per thread in a tile
static_assert(kRsThreads == 256, "the kernels index the 256 digit bins by thread");
static_assert(kRsTileRecords % kRsThreads == 0, "a tile is a whole number of items per thread");
constexpr int kRsItems = kRsTileRecords / kRsThreads;  // items per thread
constexpr int kRsTile = kRsTileRecords;                // records per tile
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

// The stable scatter of one pass (K: the word sorted on; P: a passenger
// word moved along), with the tile staged in shared memory: every tile
// ranks its records by digit in their original order (warp match_any), puts
// them there in digit order, and then every digit's run leaves as
// consecutive writes (a direct scatter writes each record to its own bin,
// about one 32-byte transaction per record).  offs is the
// exclusive scan of the digit-major tile histogram, so a tile's count of
// digit d is the step to the next entry.
template <class K, class P>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter_staged(const K *key_in, const uint32_t *val_in,
                                                                  const P *aux_in, K *key_out,
                                                                  uint32_t *val_out, P *aux_out, int64_t n,
                                                                  int shift, const uint32_t *offs,
                                                                  int n_tiles) {
    extern __shared__ __align__(16) unsigned char sm[];
    K *skey = reinterpret_cast<K *>(sm);
    uint32_t *sval = reinterpret_cast<uint32_t *>(skey + kRsTile);
    P *saux = reinterpret_cast<P *>(sval + kRsTile);
    __shared__ uint32_t start[256], gbase[256], run[256];
    __shared__ uint32_t wcnt[kRsWarps][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, d0 = threadIdx.x;
    const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
    const int cnt_tile = n - tile0 < kRsTile ? (int)(n - tile0) : kRsTile;
    {
        const int64_t idx = (int64_t)d0 * n_tiles + blockIdx.x;
        const uint32_t o = offs[idx];
        const uint32_t next = idx + 1 < (int64_t)256 * n_tiles ? offs[idx + 1] : (uint32_t)n;
        gbase[d0] = o;
        start[d0] = next - o;  // the tile's count of this digit, scanned below
        run[d0] = 0;
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the 256 counts by one warp
        uint32_t v[8], tot = 0;
        for (int j = 0; j < 8; ++j) {
            v[j] = start[lane * 8 + j];
            tot += v[j];
        }
        uint32_t incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        uint32_t acc = incl - tot;
        for (int j = 0; j < 8; ++j) {
            start[lane * 8 + j] = acc;
            acc += v[j];
        }
    }
    __syncthreads();
    for (int i = 0; i < kRsItems; ++i) {
        for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
        __syncthreads();
        const int j = i * kRsThreads + threadIdx.x;
        const bool ok = j < cnt_tile;
        K k = 0;
        uint32_t dg = 0xffffffffu;
        if (ok) {
            k = key_in[tile0 + j];
            dg = digit_of(k, shift);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const unsigned lower = peers & ((1u << lane) - 1u);
        if (ok && lower == 0) wcnt[w][dg] = __popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t pos = start[dg] + run[dg] + __popc(lower);
            for (int v = 0; v < w; ++v) pos += wcnt[v][dg];
            skey[pos] = k;
            sval[pos] = val_in[tile0 + j];
            if (aux_in) saux[pos] = aux_in[tile0 + j];
        }
        __syncthreads();
        uint32_t add = 0;
        for (int v = 0; v < kRsWarps; ++v) add += wcnt[v][threadIdx.x];
        run[threadIdx.x] += add;
        __syncthreads();
    }
    for (int j = threadIdx.x; j < cnt_tile; j += kRsThreads) {
        const K k = skey[j];
        const uint32_t d = digit_of(k, shift);
        const uint32_t pos = gbase[d] + (uint32_t)j - start[d];
        key_out[pos] = k;
        val_out[pos] = sval[j];
        if (aux_in) aux_out[pos] = saux[j];
    }
}

template <class K, class P>
static size_t staged_smem() {
    return (size_t)kRsTile * (sizeof(K) + sizeof(uint32_t) + sizeof(P));
}

template <class K, class P>
static cudaError_t staged_attr() {
    static std::atomic<unsigned long long> done{0};
    return smem_attr_once(k_rs_scatter_staged<K, P>, (int)staged_smem<K, P>(), done);
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
            e = staged_attr<K, uint32_t>();
            if (e != cudaSuccess) return e;
            k_rs_scatter_staged<K, uint32_t><<<tiles, kRsThreads, staged_smem<K, uint32_t>(), st>>>(
                ka, va, xa, kb, vb, xb, n, shift, hist, tiles);
        } else {
            // sort by aux: aux acts as the key, the key rides along
            k_rs_hist<uint32_t><<<tiles, kRsThreads, 0, st>>>(xa, n, shift, hist, tiles);
            cudaError_t e = scan_counts(hist, hist, scan_tmp, 256 * tiles, st);
            if (e != cudaSuccess) return e;
            e = staged_attr<uint32_t, K>();
            if (e != cudaSuccess) return e;
            k_rs_scatter_staged<uint32_t, K><<<tiles, kRsThreads, staged_smem<uint32_t, K>(), st>>>(
                xa, va, ka, xb, vb, kb, n, shift, hist, tiles);
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
