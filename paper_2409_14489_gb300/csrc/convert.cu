// convert.cu -- widening of 16-bit sample storage to complex64 and narrowing back, for the forms
// whose inner fields are complex64 (the streamed form's passes, the checkpointed forward): the
// first pass reads the widened copy, the last pass's complex64 result is narrowed into the
// caller's 16-bit output.  Rounding to 16 bits is round-to-nearest, as in the chain kernel's own
// 16-bit store.  HBM-bound copies: 8 bytes in and 16 bytes out per sample, or the reverse.
#include "fwd_kernel.cuh"
#include "internal.h"
#include "storage_convert.h"

namespace cbessfm {
namespace {

template <int ST>
__global__ void widen_kernel(const uint2* __restrict__ in, float4* __restrict__ out, long long n) {
    using S = Storage<ST>;
    using Pol = typename S::Pol;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const uint2 v = __ldg(in + k);
        const float2 x = S::to_f32(*reinterpret_cast<const Pol*>(&v.x));
        const float2 y = S::to_f32(*reinterpret_cast<const Pol*>(&v.y));
        out[k] = make_float4(x.x, x.y, y.x, y.y);
    }
}

template <int ST>
__global__ void narrow_kernel(const float4* __restrict__ in, uint2* __restrict__ out, long long n) {
    using S = Storage<ST>;
    using Pol = typename S::Pol;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const float4 v = __ldg(in + k);
        const Pol x = S::from_f32(make_float2(v.x, v.y));
        const Pol y = S::from_f32(make_float2(v.z, v.w));
        uint2 w;
        w.x = *reinterpret_cast<const unsigned int*>(&x);
        w.y = *reinterpret_cast<const unsigned int*>(&y);
        out[k] = w;
    }
}

unsigned grid_for(long long n) {
    const long long g = (n + 255) / 256;
    return (unsigned)(g < 65536 ? (g > 0 ? g : 1) : 65536);
}

}  // namespace

cudaError_t launch_widen(int storage, const void* in, float4* out, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const uint2* src = static_cast<const uint2*>(in);
    if (storage == CBESSFM_F16x4)
        widen_kernel<1><<<grid_for(n), 256, 0, st>>>(src, out, n);
    else if (storage == CBESSFM_BF16x4)
        widen_kernel<2><<<grid_for(n), 256, 0, st>>>(src, out, n);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_narrow(int storage, const float4* in, void* out, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    uint2* dst = static_cast<uint2*>(out);
    if (storage == CBESSFM_F16x4)
        narrow_kernel<1><<<grid_for(n), 256, 0, st>>>(in, dst, n);
    else if (storage == CBESSFM_BF16x4)
        narrow_kernel<2><<<grid_for(n), 256, 0, st>>>(in, dst, n);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace cbessfm
