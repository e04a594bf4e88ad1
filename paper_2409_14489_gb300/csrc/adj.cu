// adj.cu -- reverse-mode gradient (adjoint) of the CB-ESSFM chain (differentiation form): the
// C-ABI entry points, the workspace layout, the launches and the FP64 reductions.  The adjoint
// kernel itself is in adj_kernel.cuh (Manakov form launched here, per-polarization form from
// adj_perpol.cu).
//
// The paper trains its taps offline with finite-difference gradients (Sec. III-B) and names
// automatic differentiation as the way to per-step taps; this file is the hand-written adjoint
// of the forward chain kernel.  Gradient convention: G_z = dL/dRe(z) + j dL/dIm(z), so a
// complex-linear map y = A x back-propagates as G_x = A^H G_y.
//
// cbessfm_backpropagate_checkpointed runs the forward chain and keeps, per OLS block, the
// spectrum after the first GVD, each step's time samples before its rotation, and the spectrum
// after the last GVD.  cbessfm_grad then walks each block backwards, one CTA slot per block:
//
//   G_X = DEMUX(DFT_N(G_out on the kept samples))                 (adjoint of MUX + IDFT)
//   for s = N_st-1 .. 0:
//     G_W = conj(T_s) G_X ; G_v = IDFT_unnorm(G_W)                (adjoint of T_s DFT)
//     recompute u_s (checkpoint), P = |x|^2 + |y|^2, theta, psi = exp(j theta) - 1
//     G_theta_i[k] = -Im(sum_pol conj(G_v) v),  v = u (1 + psi)
//     dL/dw[s][i][l][m] = sum_k G_theta_i[k] P_l[k - m]          (per-block partial)
//     G_P_l[n] = sum_i sum_m w[s][i][l][m] G_theta_i[n + m]       (FIR with transposed taps)
//     G_X = NP G_W + DFT_unnorm(conj(psi) G_v + 2 G_P u)          (= DFT_unnorm(G_u))
//     the step's term of dL/drho from D_Z = DFT(psi u) and that last DFT (see the kernel)
//   G_in = IDFT_unnorm_N(MUX(conj(T_first) G_X))                  (adjoint of T_first DEMUX DFT)
//
// Per-block partial tap gradients (FP32) are summed over blocks in FP64 by a second kernel; the
// splitting-ratio terms are summed per thread in FP32 and over threads and blocks in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "block_count.h"
#include "adj_kernel.cuh"
#include "internal.h"
#include "trace.h"
#include "storage_convert.h"

namespace cbessfm {

// FP64 sum of the per-block partial gradients: out[k] = sum_b part[b][k].  A CTA takes 32
// consecutive coefficients (coalesced rows) and 8 interleaved slices of the blocks; the 8 slice
// sums of a coefficient are then added in a fixed order, so the result does not depend on
// scheduling.  (One thread per coefficient over all blocks left most SMs idle: 0.12 ms on c4.)
constexpr int kRedK = 32, kRedB = 8;
__global__ void __launch_bounds__(kRedK * kRedB)
    reduce_blocks_kernel(const float* __restrict__ part, long long n_blocks, int stride,
                         int n_coeffs, double* __restrict__ out_coeffs,
                         double* __restrict__ out_ratio) {
    __shared__ double s_sum[kRedB][kRedK + 1];
    const int kx = threadIdx.x % kRedK, by = threadIdx.x / kRedK;
    const int k = blockIdx.x * kRedK + kx;
    double acc = 0.0;
    if (k < n_coeffs) {
        for (long long b = by; b < n_blocks; b += kRedB) acc += (double)part[b * stride + k];
    } else if (k == n_coeffs) {
        // the ratio partial of each block is stored as a double in two float slots
        for (long long b = by; b < n_blocks; b += kRedB)
            acc += *reinterpret_cast<const double*>(part + b * stride + k);
    }
    s_sum[by][kx] = acc;
    __syncthreads();
    if (by == 0 && k <= n_coeffs) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kRedB; ++q) t += s_sum[q][kx];
        if (k < n_coeffs) {
            out_coeffs[k] = t;
        } else if (out_ratio != nullptr) {
            *out_ratio = t;
        }
    }
}

// Per-block tap-gradient sums carry padded tap positions; gather the real ones.
__global__ void unpad_kernel(const double* __restrict__ padded, int rows, int ntaps_pad, int ntaps,
                             double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rows * ntaps) return;
    const int r = k / ntaps, m = k - r * ntaps;
    out[k] = padded[(size_t)r * ntaps_pad + m];
}

// taps_t[s][l][i][q] = taps[s][i][l][ntaps - 1 - q] (zero beyond ntaps)
__global__ void transpose_taps_kernel(const float* __restrict__ taps, float* __restrict__ taps_t,
                                      int n_st, int n_sb, int ntaps, int ntaps_pad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = n_st * n_sb * n_sb * ntaps_pad;
    if (k >= total) return;
    const int q = k % ntaps_pad;
    const int rest = k / ntaps_pad;
    const int i = rest % n_sb;
    const int l = (rest / n_sb) % n_sb;
    const int s = rest / (n_sb * n_sb);
    taps_t[k] = q < ntaps ? taps[((size_t)(s * n_sb + i) * n_sb + l) * ntaps_pad + (ntaps - 1 - q)]
                          : 0.f;
}

cudaError_t launch_transpose_taps(const PlanImpl& p, cudaStream_t st) {
    const int total = p.n_st * p.n_sb * p.n_sb * p.ntaps_pad;
    if (total == 0) return cudaSuccess;
    transpose_taps_kernel<<<(total + 255) / 256, 256, 0, st>>>(p.d_taps, p.d_taps_t, p.n_st, p.n_sb,
                                                               p.ntaps, p.ntaps_pad);
    return cudaGetLastError();
}

namespace {

template <int NP, bool ADJ>
cudaError_t launch_np_adj(const ChainArgs& a, int threads, cudaStream_t st) {
    const long long total = (long long)a.batch * a.n_blocks;
    const long long grid = (total + a.G - 1) / a.G;
    if (grid <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.G * a.region_bytes;
    if (a.per_pol) return launch_adj_per_pol(NP, ADJ, a, threads, st);   // adj_perpol.cu
    if (ADJ && a.want_ratio == 0) return launch_adj_taps(NP, a, threads, st);   // adj_taps.cu
    if constexpr (ADJ) {
        const size_t smem_a = smem + chain_tw_bytes(fft_tw_size(NP));   // + staged twiddles
        cudaError_t e = cudaFuncSetAttribute(cbessfm_adj_kernel<NP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a);
        if (e != cudaSuccess) return e;
        cbessfm_adj_kernel<NP><<<(unsigned)grid, threads, smem_a, st>>>(a);
    } else {
        const size_t smem_f = smem + a.tbl_bytes;        // + the chain's per-CTA tables
        cudaError_t e = cudaFuncSetAttribute(cbessfm_fwd_ckpt_kernel<NP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f);
        if (e != cudaSuccess) return e;
        cbessfm_fwd_ckpt_kernel<NP><<<(unsigned)grid, threads, smem_f, st>>>(a);
    }
    return cudaGetLastError();
}

template <bool ADJ>
cudaError_t dispatch(int np, const ChainArgs& a, int threads, cudaStream_t st) {
    switch (np) {
        case 16: return launch_np_adj<16, ADJ>(a, threads, st);
        case 32: return launch_np_adj<32, ADJ>(a, threads, st);
        case 64: return launch_np_adj<64, ADJ>(a, threads, st);
        case 128: return launch_np_adj<128, ADJ>(a, threads, st);
        case 256: return launch_np_adj<256, ADJ>(a, threads, st);
        case 512: return launch_np_adj<512, ADJ>(a, threads, st);
        case 1024: return launch_np_adj<1024, ADJ>(a, threads, st);
        case 2048: return launch_np_adj<2048, ADJ>(a, threads, st);
        default: return cudaErrorInvalidValue;
    }
}

int round_up_i(long long v, int m) { return (int)((v + m - 1) / m * m); }

// Shared-memory region of one block for the adjoint: exchange, intensity, (cos, sin), G_theta
// (swizzled with halo, and plain), G_P rows and the accumulators.
// The per-polarization form adds, from the next 128-byte boundary, the Px - Py rows and the
// D = G_tx - G_ty rows (swizzled, with halo) and the G_Dp rows.
int adj_region_bytes(const PlanImpl& p) {
    const int NP = p.n_fft, nsb = p.n_sb;
    long long bytes = round_up_i(16LL * xpad_len(p.N), 128) + 4LL * nsb * p.pstride +
                      8LL * nsb * xpad_len(NP) + 4LL * nsb * p.pstride + 8LL * nsb * NP +
                      4LL * (nsb * nsb * p.ntaps_pad + 4);
    if (p.per_pol) bytes = round_up_i(bytes, 128) + 8LL * nsb * p.pstride + 4LL * nsb * NP;
    return round_up_i(bytes, 128);
}

// Workspace: checkpoints | adjoint scratch (two fields per block) | per-block partial
// gradients | FP64 sums | for 16-bit plans, complex64 copies of the forward's input and output.
struct Layout {
    size_t ckpt_bytes, stash_bytes, part_bytes, padded_bytes, conv_bytes, total;
    long long n_blk;
    int part_stride;
};

// callers first refuse calls of more than 2^31 - 1 blocks (too_many_blocks), which bounds every
// size below
Layout layout(const PlanImpl& p, long long n_samples, int batch) {
    Layout l{};
    const long long nb = blocks_for(n_samples, p.V);
    l.n_blk = nb * batch;
    l.ckpt_bytes = (size_t)l.n_blk * (size_t)(p.n_st + 2) * 16 * p.N;
    l.stash_bytes = p.n_st > 0 ? (size_t)l.n_blk * 2 * 16 * p.N : 0;
    l.part_stride = p.n_st * p.n_sb * p.n_sb * p.ntaps_pad + 4;
    l.part_bytes = (size_t)l.n_blk * l.part_stride * sizeof(float);
    l.padded_bytes = ((size_t)l.part_stride * sizeof(double) + 255) / 256 * 256;
    l.ckpt_bytes = (l.ckpt_bytes + 255) / 256 * 256;
    l.stash_bytes = (l.stash_bytes + 255) / 256 * 256;
    l.part_bytes = (l.part_bytes + 255) / 256 * 256;
    l.conv_bytes = p.storage != CBESSFM_C64
                       ? 2 * (((size_t)n_samples * batch * 16 + 255) / 256 * 256) : 0;
    l.total = l.ckpt_bytes + l.stash_bytes + l.part_bytes + l.padded_bytes + l.conv_bytes;
    return l;
}

cbessfm_status check_common(const cbessfm_plan* plan, int64_t n_samples, int batch,
                            const void* workspace, size_t ws_bytes, const PlanImpl** pp) {
    const PlanImpl* p = plan_impl(plan);
    if (p == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "plan is NULL");
    if (n_samples < 1 || batch < 1) return fail(CBESSFM_ERR_INVALID_ARG, "n_samples and batch must be >= 1");
    if (too_many_blocks(blocks_for(n_samples, p->V), batch))
        return fail(CBESSFM_ERR_UNSUPPORTED, "too many blocks");
    if (workspace == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) & 255u)
        return fail(CBESSFM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    const Layout l = layout(*p, n_samples, batch);
    if (ws_bytes < l.total)
        return fail(CBESSFM_ERR_INVALID_ARG, "workspace of %zu bytes is smaller than %zu", ws_bytes, l.total);
    if (adj_region_bytes(*p) + chain_tw_bytes(fft_tw_size(p->n_fft)) > kMaxDynSmem)
        return fail(CBESSFM_ERR_UNSUPPORTED, "the adjoint of a %d-sample block%s does not fit shared memory",
                    p->N, p->per_pol ? " with the per-polarization NLPR" : "");
    *pp = p;
    return CBESSFM_OK;
}

}  // namespace
}  // namespace cbessfm

using namespace cbessfm;

extern "C" {

cbessfm_status cbessfm_grad_workspace_size(const cbessfm_plan* plan, int64_t n_samples, int batch,
                                           size_t* bytes) {
    clear_error();
    const PlanImpl* p = plan_impl(plan);
    if (p == nullptr || bytes == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "plan/bytes is NULL");
    if (n_samples < 1 || batch < 1) return fail(CBESSFM_ERR_INVALID_ARG, "n_samples and batch must be >= 1");
    if (too_many_blocks(blocks_for(n_samples, p->V), batch))
        return fail(CBESSFM_ERR_UNSUPPORTED, "too many blocks");
    *bytes = layout(*p, n_samples, batch).total;
    return CBESSFM_OK;
}

cbessfm_status cbessfm_backpropagate_checkpointed(const cbessfm_plan* plan, const void* in, void* out,
                                                  int64_t n_samples, int batch, void* workspace,
                                                  size_t ws_bytes, cbessfm_stream stream) {
    TraceRange trace_range("cbessfm:backpropagate_checkpointed");
    clear_error();
    const PlanImpl* p = nullptr;
    cbessfm_status st = check_common(plan, n_samples, batch, workspace, ws_bytes, &p);
    if (st != CBESSFM_OK) return st;
    if (in == nullptr || out == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "in/out is NULL");
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u)
        return fail(CBESSFM_ERR_INVALID_ARG, "in/out must be 16-byte aligned");
    const bool wide = p->storage != CBESSFM_C64;  // 16-bit fields around the complex64 chain
    const unsigned long long bytes = (unsigned long long)n_samples * batch * (wide ? 8ull : 16ull);
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(in), o0 = reinterpret_cast<uintptr_t>(out);
    if (i0 < o0 + bytes && o0 < i0 + bytes) return fail(CBESSFM_ERR_ALIAS, "out overlaps in");
    const uintptr_t w0 = reinterpret_cast<uintptr_t>(workspace), w1 = w0 + ws_bytes;
    if ((i0 < w1 && w0 < i0 + bytes) || (o0 < w1 && w0 < o0 + bytes))
        return fail(CBESSFM_ERR_ALIAS, "workspace overlaps in or out");
    const cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const Layout l = layout(*p, n_samples, batch);
    unsigned char* conv = static_cast<unsigned char*>(workspace) + l.total - l.conv_bytes;
    float4* const in64 = reinterpret_cast<float4*>(conv);
    float4* const out64 = reinterpret_cast<float4*>(conv + l.conv_bytes / 2);
    const long long n_all = (long long)n_samples * batch;
    if (wide) {
        const cudaError_t e = launch_widen(p->storage, in, in64, n_all, cs);
        if (e != cudaSuccess) return cuda_fail(e, "checkpointed forward input widening");
    }
    ChainArgs a = make_chain_args(*p);
    a.in = wide ? static_cast<const void*>(in64) : in;
    a.out = wide ? static_cast<void*>(out64) : out;
    a.L = n_samples;
    a.batch = batch;
    a.n_blocks = (int)blocks_for(n_samples, p->V);
    a.ckpt = static_cast<float2*>(workspace);
    cudaError_t e = dispatch<false>(p->n_fft, a, p->threads, cs);
    if (e != cudaSuccess) return cuda_fail(e, "checkpointed forward launch");
    if (wide) {
        e = launch_narrow(p->storage, out64, out, n_all, cs);
        if (e != cudaSuccess) return cuda_fail(e, "checkpointed forward output narrowing");
    }
    return CBESSFM_OK;
}

cbessfm_status cbessfm_grad(const cbessfm_plan* plan, const void* grad_out, double* grad_coeffs,
                            double* grad_ratio, void* grad_in, void* workspace, size_t ws_bytes,
                            int64_t n_samples, int batch, cbessfm_stream stream) {
    TraceRange trace_range("cbessfm:grad");
    clear_error();
    const PlanImpl* p = nullptr;
    cbessfm_status st = check_common(plan, n_samples, batch, workspace, ws_bytes, &p);
    if (st != CBESSFM_OK) return st;
    if (grad_out == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "grad_out is NULL");
    if ((reinterpret_cast<uintptr_t>(grad_out) | reinterpret_cast<uintptr_t>(grad_in)) & 15u)
        return fail(CBESSFM_ERR_INVALID_ARG, "grad_out/grad_in must be 16-byte aligned");
    if (p->n_st > 0 && grad_coeffs == nullptr)
        return fail(CBESSFM_ERR_INVALID_ARG, "grad_coeffs is NULL");
    const cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const Layout l = layout(*p, n_samples, batch);
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    ChainArgs a = make_chain_args(*p);
    classic_tables(*p, a);                  // the adjoint runs the fft_slots plan
    a.L = n_samples;
    a.batch = batch;
    a.n_blocks = (int)blocks_for(n_samples, p->V);
    a.ckpt = reinterpret_cast<float2*>(ws);
    a.stash = reinterpret_cast<float2*>(ws + l.ckpt_bytes);
    a.gpart = reinterpret_cast<float*>(ws + l.ckpt_bytes + l.stash_bytes);
    a.gout = static_cast<const float2*>(grad_out);
    a.gin = static_cast<float2*>(grad_in);
    a.want_ratio = grad_ratio != nullptr ? 1 : 0;
    a.taps_t = p->d_taps_t;
    // the adjoint's own region and CTA shape
    a.region_bytes = adj_region_bytes(*p);
    a.nlpr_off = round_up_i(16LL * xpad_len(p->N), 128);
    const int tpf = p->n_fft / fft_slots(p->n_fft);
    const int tb = 2 * p->n_sb * tpf;
    a.G = choose_blocks_per_cta(tb, a.region_bytes, tpf, p->n_sb,
                                chain_tw_bytes(fft_tw_size(p->n_fft)));
    if (a.G < 1) return fail(CBESSFM_ERR_UNSUPPORTED, "no CTA shape for the adjoint");
    {
        const double rn = p->link.sample_rate / p->N;
        a.kd0 = (float)(2.0 * 9.86960440108935861883 * p->link.beta2 * p->step_length * rn * rn);
    }
    cudaError_t e = cudaSuccess;
    if (grad_in != nullptr)
        e = cudaMemsetAsync(grad_in, 0, (size_t)n_samples * batch * 16, cs);
    if (e == cudaSuccess) e = dispatch<true>(p->n_fft, a, a.G * tb, cs);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
    const int n_coeffs = p->n_st * p->n_sb * p->n_sb * p->ntaps_pad;
    double* padded = reinterpret_cast<double*>(ws + l.ckpt_bytes + l.stash_bytes + l.part_bytes);
    // padded[0 .. n_coeffs) = tap sums, padded[n_coeffs] = ratio sum
    reduce_blocks_kernel<<<(n_coeffs + 1 + kRedK - 1) / kRedK, kRedK * kRedB, 0, cs>>>(
        a.gpart, l.n_blk, l.part_stride, n_coeffs, padded, padded + n_coeffs);
    e = cudaGetLastError();
    if (e == cudaSuccess && grad_ratio != nullptr)
        e = cudaMemcpyAsync(grad_ratio, padded + n_coeffs, sizeof(double), cudaMemcpyDeviceToDevice, cs);
    const int rows = p->n_st * p->n_sb * p->n_sb;
    if (e == cudaSuccess && rows > 0) {
        unpad_kernel<<<(rows * p->ntaps + 255) / 256, 256, 0, cs>>>(padded, rows, p->ntaps_pad,
                                                                  p->ntaps, grad_coeffs);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(e, "gradient reduction");
    return CBESSFM_OK;
}

}  // extern "C"
