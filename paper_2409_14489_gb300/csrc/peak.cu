// peak.cu -- measured FP32 fused multiply-add rate of the current device (the denominator of
// the chain kernel's ALU roofline).  A measurement utility, not part of the paper's method.
//
// Every thread runs kChains independent FFMA dependency chains for kIters iterations; the grid
// holds 2048 threads per SM (4 CTAs of 512), so each SM sub-partition always has independent
// FFMAs to issue and the launch time is the FMA pipe's time.  The rate is the best of several
// launches timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include "../../include/cbessfm.h"
#include "internal.h"

namespace cbessfm {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 8192;
constexpr int kThreads = 512;
constexpr int kCtasPerSm = 4;

// written only if the sum comes out as a value it cannot take, so the chains are not removed
__device__ float g_peak_sink;

__global__ void __launch_bounds__(kThreads) fp32_peak_kernel(float m, float c) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (float)threadIdx.x * 1e-3f + (float)i;
#pragma unroll 4
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == -1.2345e-30f) g_peak_sink = s;
}

}  // namespace
}  // namespace cbessfm

using namespace cbessfm;

extern "C" cbessfm_status cbessfm_measure_fp32_peak(int repeats, double* flops, int* sm_count,
                                                   cbessfm_stream stream) {
    clear_error();
    if (!flops || !sm_count || repeats < 1 || repeats > 1000)
        return fail(CBESSFM_ERR_INVALID_ARG, "measure_fp32_peak: NULL output or repeats not in 1..1000");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const dim3 grid(sms * kCtasPerSm);
    float best_ms = 0.f;
    // one untimed launch first (clocks ramp, instruction cache)
    if (e == cudaSuccess) {
        fp32_peak_kernel<<<grid, kThreads, 0, st>>>(0.999f, 1e-3f);
        e = cudaGetLastError();
    }
    for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, st);
        if (e != cudaSuccess) break;
        fp32_peak_kernel<<<grid, kThreads, 0, st>>>(0.999f, 1e-3f);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "measure_fp32_peak");
    const double lane_fmas = (double)grid.x * kThreads * (double)kIters * kChains;
    *flops = 2.0 * lane_fmas / (best_ms * 1e-3);
    *sm_count = sms;
    return CBESSFM_OK;
}
