// storage_convert.h -- complex64 paths of 16-bit plans: the forward launch with complex64 fields
// whatever the plan's storage (fwd.cu; the plan prepares those kernels at creation) and the
// widening / narrowing copies between 16-bit storage and complex64 float4 samples (convert.cu).
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace cbessfm {

cudaError_t launch_forward_c64(const PlanImpl& p, const ChainArgs& a, cudaStream_t stream);
// storage: CBESSFM_F16x4 or CBESSFM_BF16x4; n samples of 8 bytes <-> n float4
cudaError_t launch_widen(int storage, const void* in, float4* out, long long n, cudaStream_t st);
cudaError_t launch_narrow(int storage, const float4* in, void* out, long long n, cudaStream_t st);

}  // namespace cbessfm
