// Device probe: the multiprocessor count and the FP64 arithmetic throughput
// the current GPU sustains, measured with a chain of independent fused
// multiply-adds.  The condensation solve (Sec. 5.1.3) is bound by FP64
// arithmetic on this part, and this figure is the peak its roofline is
// taken against.  Not a step of the method: a measurement utility.
#include <cmath>

#include "sdm_internal.cuh"

namespace sdm {

constexpr int kProbeChains = 8;      // independent accumulators per thread
constexpr int kProbeThreads = 256;
constexpr int kProbeIters = 4096;    // 2 * kProbeChains flops each

__global__ void __launch_bounds__(kProbeThreads) k_probe_dfma(double m, double c, double *sink) {
    double a[kProbeChains];
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) a[j] = fma(a[j], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) s += a[j];
    // never true for the arguments used; keeps the chains alive
    if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace sdm

using namespace sdm;

extern "C" sdm_status sdm_probe_device(double sustain_s, sdm_device_peaks *out) {
    if (!out || !(sustain_s >= 0.0) || sustain_s > 60.0) {
        sdm_set_global_error("sdm_probe_device: out must be non-NULL and 0 <= sustain_s <= 60");
        return SDM_EINVAL;
    }
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_dfma, kProbeThreads, 0);
    cudaStream_t st = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    double *sink = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int blocks = n_sm * (per_sm > 0 ? per_sm : 1);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(double) * (size_t)blocks);
    const double flops = 2.0 * kProbeChains * (double)kProbeIters * kProbeThreads * (double)blocks;
    double best_ms = 1e30, sus_ms = 0.0;
    int sus_launches = 0;
    auto launch = [&]() { k_probe_dfma<<<blocks, kProbeThreads, 0, st>>>(0.99999999, 1e-8, sink); };
    if (e == cudaSuccess) {
        launch();  // warm-up
        e = cudaStreamSynchronize(st);
    }
    for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
        cudaEventRecord(t0, st);
        launch();
        cudaEventRecord(t1, st);
        e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && ms > 0.0f && ms < best_ms) best_ms = ms;
    }
    if (e == cudaSuccess && sustain_s > 0.0) {
        sus_launches = (int)std::ceil(sustain_s * 1e3 / best_ms);
        if (sus_launches < 1) sus_launches = 1;
        cudaEventRecord(t0, st);
        for (int k = 0; k < sus_launches; ++k) launch();
        cudaEventRecord(t1, st);
        e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        sus_ms = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (sink) cudaFree(sink);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sdm_set_global_error(std::string("sdm_probe_device: ") + cudaGetErrorString(e));
        return SDM_ECUDA;
    }
    out->n_sm = n_sm;
    out->blocks = blocks;
    out->fp64_tflops_burst = flops / (best_ms * 1e-3) / 1e12;
    out->fp64_tflops_sustained = sus_launches > 0 ? flops * sus_launches / (sus_ms * 1e-3) / 1e12 : 0.0;
    out->sustained_s = sus_ms * 1e-3;
    return SDM_OK;
}
