// adj_taps.cu -- launches of the Manakov adjoint without the ratio gradient (taps and input
// only), a translation unit of its own so it compiles beside adj.cu.
#include "adj_kernel.cuh"

namespace cbessfm {
namespace {

template <int NP>
cudaError_t launch_np(const ChainArgs& a, int threads, cudaStream_t st) {
    const long long total = (long long)a.batch * a.n_blocks;
    const long long grid = (total + a.G - 1) / a.G;
    if (grid <= 0) return cudaSuccess;
    // the G block regions + staged twiddles
    const size_t smem = (size_t)a.G * a.region_bytes + chain_tw_bytes(fft_tw_size(NP));
    cudaError_t e = cudaFuncSetAttribute(cbessfm_adj_kernel<NP, false, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cbessfm_adj_kernel<NP, false, false><<<(unsigned)grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adj_taps(int np, const ChainArgs& a, int threads, cudaStream_t st) {
    switch (np) {
        case 16: return launch_np<16>(a, threads, st);
        case 32: return launch_np<32>(a, threads, st);
        case 64: return launch_np<64>(a, threads, st);
        case 128: return launch_np<128>(a, threads, st);
        case 256: return launch_np<256>(a, threads, st);
        case 512: return launch_np<512>(a, threads, st);
        case 1024: return launch_np<1024>(a, threads, st);
        case 2048: return launch_np<2048>(a, threads, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cbessfm
