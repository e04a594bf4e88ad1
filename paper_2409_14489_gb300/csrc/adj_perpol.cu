// adj_perpol.cu -- launches of the per-polarization NLPR's checkpointed forward and adjoint
// (Eqs. (NLPR_polx/poly)); a translation unit of its own so it compiles beside adj.cu.
#include "adj_kernel.cuh"

namespace cbessfm {
namespace {

template <int NP>
cudaError_t launch_np(bool adjoint, const ChainArgs& a, int threads, cudaStream_t st) {
    const long long total = (long long)a.batch * a.n_blocks;
    const long long grid = (total + a.G - 1) / a.G;
    if (grid <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.G * a.region_bytes;
    if (adjoint) {
        const size_t smem_a = smem + chain_tw_bytes(fft_tw_size(NP));   // + staged twiddles
        cudaError_t e = cudaFuncSetAttribute(cbessfm_adj_kernel<NP, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a);
        if (e != cudaSuccess) return e;
        cbessfm_adj_kernel<NP, true><<<(unsigned)grid, threads, smem_a, st>>>(a);
    } else {
        const size_t smem_f = smem + a.tbl_bytes;        // + the chain's per-CTA tables
        cudaError_t e = cudaFuncSetAttribute(cbessfm_fwd_ckpt_kernel<NP, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f);
        if (e != cudaSuccess) return e;
        cbessfm_fwd_ckpt_kernel<NP, true><<<(unsigned)grid, threads, smem_f, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adj_per_pol(int np, bool adjoint, const ChainArgs& a, int threads,
                               cudaStream_t st) {
    switch (np) {
        case 16: return launch_np<16>(adjoint, a, threads, st);
        case 32: return launch_np<32>(adjoint, a, threads, st);
        case 64: return launch_np<64>(adjoint, a, threads, st);
        case 128: return launch_np<128>(adjoint, a, threads, st);
        case 256: return launch_np<256>(adjoint, a, threads, st);
        case 512: return launch_np<512>(adjoint, a, threads, st);
        case 1024: return launch_np<1024>(adjoint, a, threads, st);
        case 2048: return launch_np<2048>(adjoint, a, threads, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cbessfm
