// fwd_inst_256_512.cu -- explicit instantiations of the forward chain kernel for N' in {256, 512}.
#include "fwd_kernel.cuh"

namespace cbessfm {

#define CBESSFM_FWD_INST(NP)                                                            \
    template cudaError_t fwd_launch<NP, 0>(const ChainArgs&, int, cudaStream_t);        \
    template cudaError_t fwd_launch<NP, 1>(const ChainArgs&, int, cudaStream_t);        \
    template cudaError_t fwd_launch<NP, 2>(const ChainArgs&, int, cudaStream_t);        \
    template cudaError_t fwd_prepare<NP, 0>(int);                                       \
    template cudaError_t fwd_prepare<NP, 1>(int);                                       \
    template cudaError_t fwd_prepare<NP, 2>(int);                                       \
    template cudaError_t fwd_persistent_launch<NP, 0>(const ChainArgs*, const int2*, int,  \
        unsigned int*, int, int, int, int, int, int, int, cudaStream_t);                          \
    template cudaError_t fwd_persistent_launch<NP, 1>(const ChainArgs*, const int2*, int,  \
        unsigned int*, int, int, int, int, int, int, int, cudaStream_t);                          \
    template cudaError_t fwd_persistent_launch<NP, 2>(const ChainArgs*, const int2*, int,  \
        unsigned int*, int, int, int, int, int, int, int, cudaStream_t);                          \
    template cudaError_t fwd_persistent_occupancy<NP, 0>(int, int, int*);               \
    template cudaError_t fwd_persistent_occupancy<NP, 1>(int, int, int*);               \
    template cudaError_t fwd_persistent_occupancy<NP, 2>(int, int, int*);
CBESSFM_FWD_INST(256)
CBESSFM_FWD_INST(512)
#undef CBESSFM_FWD_INST

}  // namespace cbessfm
