// peak.cu -- mppi_fp32_fma_probe(): the FP32 FMA rate of this GPU, measured.
//
// The rollout kernels are bound by the FP32 pipe, so their roofline needs the
// pipe's attainable rate.  This probe runs independent FMA chains on every
// SM (scalar fmaf, or the paired f32x2 form the quadrotor kernel also uses)
// long enough to settle the clock, and times them with CUDA events.  Each
// thread carries 8 independent chains, which hides the FMA latency with a
// few warps per SM sub-partition.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "mppi_internal.h"

namespace mppi {
namespace {

constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 512;

__device__ float g_probe_sink[1];

// a <- a * b + c per chain; b < 1 keeps the values bounded.  The sink write
// keeps the compiler from removing the loop (the condition is never true for
// these inputs, but it cannot know that).
__global__ void __launch_bounds__(kProbeThreads) fma_probe_scalar(int iters, float b, float c) {
    float a[kProbeChains];
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) a[j] = threadIdx.x * 1e-3f + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) s += a[j];
    if (s == -1.2345e30f) g_probe_sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) fma_probe_pair(int iters, float b, float c) {
    unsigned long long a[kProbeChains];
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) a[j] = pack2(threadIdx.x * 1e-3f + j, j + 0.5f);
    const unsigned long long B = pack2(b, b), C = pack2(c, c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) a[j] = fma2(a[j], B, C);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) {
        float x, y;
        unpack2(a[j], x, y);
        s += x + y;
    }
    if (s == -1.2345e30f) g_probe_sink[0] = s;
}

}  // namespace
}  // namespace mppi

extern "C" mppi_status mppi_fp32_fma_probe(int pair, int iters, float *ms_out,
                                           double *flops_out) {
    using namespace mppi;
    if (!ms_out || !flops_out || iters < 1 || iters > (1 << 24) || (pair != 0 && pair != 1))
        return MPPI_ERR_INVALID_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *fn = pair ? reinterpret_cast<const void *>(fma_probe_pair)
                          : reinterpret_cast<const void *>(fma_probe_scalar);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kProbeThreads, 0);
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return MPPI_ERR_CUDA;
    }
    const float b = 0.999f, c = 1e-3f;
    // one launch to warm up, then the timed one (on the legacy stream,
    // synchronously: this is a measurement, not part of a step)
    if (pair)
        fma_probe_pair<<<blocks, kProbeThreads>>>(iters / 8 + 1, b, c);
    else
        fma_probe_scalar<<<blocks, kProbeThreads>>>(iters / 8 + 1, b, c);
    cudaEventRecord(e0);
    if (pair)
        fma_probe_pair<<<blocks, kProbeThreads>>>(iters, b, c);
    else
        fma_probe_scalar<<<blocks, kProbeThreads>>>(iters, b, c);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    *ms_out = ms;
    *flops_out = 2.0 * (pair ? 2.0 : 1.0) * kProbeChains * static_cast<double>(iters) *
                 static_cast<double>(blocks) * kProbeThreads;
    return MPPI_OK;
}
