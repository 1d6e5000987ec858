// Allocation-free variant of the cell sort, for callers that cannot
// allocate device memory while they run: code inside a captured CUDA graph
// or a stream-ordered region where a cudaMalloc would synchronise or be
// refused, and hosts whose memory pools are fixed at start-up.  Its scratch
// is a file-scope device array, reserved on every GPU that loads the library
// until the process exits.
#include <mutex>

#include "sdm_internal.cuh"

namespace sdm {

constexpr int64_t kStaticSortMaxN = int64_t(1) << 21;      // particles per call
constexpr int32_t kStaticSortMaxCells = int32_t(1) << 19;  // cells per call
constexpr size_t kStaticSortWords =
    (size_t)kStaticSortMaxCells + 1 + (size_t)kStaticSortMaxN + (size_t)kStaticSortMaxCells / 1024 + 2 + 64;

// counts | slots | scan partials | flag  (about 10 MB)
static __device__ __align__(256) uint32_t g_sort_scratch[kStaticSortWords];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
uint32_t *g_scratch_addr[kMaxDevices] = {};

// Host code cannot use g_sort_scratch's name as a device address; resolve
// it on the current device.  Outside stream capture every call resolves it
// afresh (a cudaDeviceReset reloads the module, and the array may then sit
// elsewhere); inside a capture the address cached by the last such call on
// this device is used, so the first call on a device must come before any
// capture.
cudaError_t scratch_for_current_device(cudaStream_t st, uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = (uint32_t *)p;
    }
    if (!g_scratch_addr[dev]) return cudaErrorStreamCaptureUnsupported;
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}
}  // namespace

}  // namespace sdm

using namespace sdm;

extern "C" sdm_status sdm_cell_sort_noalloc(const uint32_t *cell, int64_t n, int32_t n_cells,
                                            uint32_t *perm, uint32_t *offsets, void *stream) {
    if (n < 0 || n_cells < 1 || (n > 0 && (!cell || !perm)) || !offsets) {
        sdm_set_global_error("sdm_cell_sort_noalloc: invalid argument");
        return SDM_EINVAL;
    }
    if (n > kStaticSortMaxN || n_cells > kStaticSortMaxCells) {
        sdm_set_global_error("sdm_cell_sort_noalloc: at most 2097152 particles and 524288 cells per call");
        return SDM_EINVAL;
    }
    uint32_t *scratch = nullptr;
    if (scratch_for_current_device((cudaStream_t)stream, &scratch) != cudaSuccess) {
        cudaGetLastError();
        sdm_set_global_error("sdm_cell_sort_noalloc: device scratch is not reachable");
        return SDM_ECUDA;
    }
    uint32_t *count = scratch;
    uint32_t *slot = count + n_cells + 1;
    uint32_t *tmp = slot + n;
    unsigned *flag = (unsigned *)(tmp + (size_t)n_cells / 1024 + 2);
    // the counts are cleared on the stream inside the call (they keep the
    // previous call's values otherwise)
    const cudaError_t e = cell_sort_with_scratch(cell, n, (uint32_t)n_cells, perm, offsets, count, slot,
                                                 tmp, flag, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        sdm_set_global_error(std::string("sdm_cell_sort_noalloc: ") + cudaGetErrorString(e));
        return SDM_ECUDA;
    }
    return SDM_OK;
}
