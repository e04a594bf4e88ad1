// fwd_launch.h -- per-(N', storage) launch entry points of the forward chain kernel.
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace cbessfm {

template <int NP, int ST>
cudaError_t fwd_launch(const ChainArgs& a, int threads, cudaStream_t stream);
template <int NP, int ST>
cudaError_t fwd_prepare(int smem_bytes);
template <int NP, int ST>
cudaError_t fwd_persistent_launch(const ChainArgs* jobs, const int2* items, int n_items,
                                  unsigned int* counter, int n_sb, int G, int region_bytes,
                                  int tbl_bytes, int per_pol, int threads, int grid,
                                  cudaStream_t stream);
template <int NP, int ST>
cudaError_t fwd_persistent_occupancy(int threads, int smem_bytes, int* ctas_per_sm);

#define CBESSFM_FWD_EXTERN(NP)                                                            \
    extern template cudaError_t fwd_launch<NP, 0>(const ChainArgs&, int, cudaStream_t);   \
    extern template cudaError_t fwd_launch<NP, 1>(const ChainArgs&, int, cudaStream_t);   \
    extern template cudaError_t fwd_launch<NP, 2>(const ChainArgs&, int, cudaStream_t);   \
    extern template cudaError_t fwd_prepare<NP, 0>(int);                                  \
    extern template cudaError_t fwd_prepare<NP, 1>(int);                                  \
    extern template cudaError_t fwd_prepare<NP, 2>(int);                                  \
    extern template cudaError_t fwd_persistent_launch<NP, 0>(const ChainArgs*, const int2*, int, \
        unsigned int*, int, int, int, int, int, int, int, cudaStream_t);                            \
    extern template cudaError_t fwd_persistent_launch<NP, 1>(const ChainArgs*, const int2*, int, \
        unsigned int*, int, int, int, int, int, int, int, cudaStream_t);                            \
    extern template cudaError_t fwd_persistent_launch<NP, 2>(const ChainArgs*, const int2*, int, \
        unsigned int*, int, int, int, int, int, int, int, cudaStream_t);                            \
    extern template cudaError_t fwd_persistent_occupancy<NP, 0>(int, int, int*);          \
    extern template cudaError_t fwd_persistent_occupancy<NP, 1>(int, int, int*);          \
    extern template cudaError_t fwd_persistent_occupancy<NP, 2>(int, int, int*);
CBESSFM_FWD_EXTERN(16)
CBESSFM_FWD_EXTERN(32)
CBESSFM_FWD_EXTERN(64)
CBESSFM_FWD_EXTERN(128)
CBESSFM_FWD_EXTERN(256)
CBESSFM_FWD_EXTERN(512)
CBESSFM_FWD_EXTERN(1024)
CBESSFM_FWD_EXTERN(2048)
#undef CBESSFM_FWD_EXTERN

}  // namespace cbessfm
