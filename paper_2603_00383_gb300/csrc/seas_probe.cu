// Device probe for roofline reporting: the FP64 fused multiply-add rate of the GPU, measured with a kernel of
// independent FMA chains (no memory traffic).  Not part of the method; it supplies the denominator of the FP64
// path's roofline, which no copy or GEMM benchmark gives.
#include "seas.h"
#include "seas_internal.h"

#include <cstdio>
#include <string>

namespace seas {
namespace {

constexpr int kProbeChains = 8;      // independent FMA chains per thread (enough to cover the pipe latency)

__global__ void __launch_bounds__(kThreads) k_fp64_fma_probe(double *sink, int iters, double a, double b) {
    double x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += x[k];
    if (s == -1.0) sink[blockIdx.x] = s;       // never true (x stays near 1): keeps the chains live
}

}  // namespace
}  // namespace seas

using namespace seas;

extern "C" seas_status seas_measure_fp64_peak(int device, double *fma_per_second) {
    if (!fma_per_second) return SEAS_EINVAL;
    *fma_per_second = 0.0;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return device < 0 || (count > 0 && device >= count) ? SEAS_EINVAL : SEAS_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SEAS_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return SEAS_ECUDA;
    const int grid = sms * 8, iters = 8192;
    double *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    seas_status status = SEAS_ECUDA;
    double best_ms = 0.0;
    if (cudaMalloc(&sink, sizeof(double) * grid) != cudaSuccess) goto done;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) goto done;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    for (int rep = 0; rep < 4; ++rep) {        // the first launch warms the clocks up and is not counted
        cudaEventRecord(e0, st);
        k_fp64_fma_probe<<<grid, kThreads, 0, st>>>(sink, iters, 0.9999999, 1e-7);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) goto done;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) goto done;
        if (rep > 0 && (best_ms == 0.0 || ms < best_ms)) best_ms = ms;
    }
    if (cudaGetLastError() != cudaSuccess || best_ms <= 0.0) goto done;
    *fma_per_second = (double)grid * kThreads * kProbeChains * (double)iters / (best_ms * 1e-3);
    status = SEAS_OK;
done:
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    return status;
}
