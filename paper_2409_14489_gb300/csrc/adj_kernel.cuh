// adj_kernel.cuh -- the adjoint kernel of the CB-ESSFM chain (differentiation form), shared by
// adj.cu (Manakov NLPR) and adj_perpol.cu (per-polarization NLPR) so the two forms compile in
// parallel.
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
#pragma once
#include <cuda_runtime.h>

#include "fwd_kernel.cuh"
#include "internal.h"

namespace cbessfm {

// The forward kernel's windowed FIR (fir8) with the 9-to-12-tap fast path.
// skip_l >= 0 leaves out row skip_l (the coupling-only sums of the per-polarization form).
template <int E>
__device__ __forceinline__ void fir8_acc(const ChainArgs& a, const float4* __restrict__ wbase,
                                         const float* __restrict__ rows0, int k0, float (&acc)[8],
                                         int skip_l = -1) {
    if (a.nchunks == 3) {
        fir8<E, 3>(a, wbase, rows0, a.pstride, k0, acc, skip_l);
    } else {
        fir8<E, 0>(a, wbase, rows0, a.pstride, k0, acc, skip_l);
    }
}

// Start moving `bytes` of global memory (16-byte aligned, a multiple of 16 bytes) into L2
// without waiting for them (a bulk prefetch; no completion to track).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// write value v of row sample n (and its circular halo copies) into swizzled row `row`
template <int NP, int E>
__device__ __forceinline__ void row_store(float* row, int mb, int n, int H, float v) {
    row[pswz<E>(mb + n)] = v;
    if (n < H) row[pswz<E>(mb + n + NP)] = v;
    if (n >= NP - H) row[pswz<E>(mb + n - NP)] = v;
}

// PERPOL: the adjoint of the per-polarization NLPR of Eqs. (NLPR_polx/poly).  The forward
// applies theta^x = theta + delta and theta^y = theta - delta, with theta the Manakov phase of
// the intensities P = Px + Py and delta = (1/3) sum_{l != i} w_il (Px_l - Py_l).  With S = G_tx
// + G_ty and D = G_tx - G_ty (the phase gradients of the two polarizations):
//   G_P_l = sum_i corr(w_il, S_i),  G_Dp_l = (1/3) sum_{i != l} corr(w_il, D_i),
//   G_Px = G_P + G_Dp,  G_Py = G_P - G_Dp,
//   dL/dw_il[m] = sum_k S_i[k] P_l[k - m] + [i != l] (1/3) sum_k D_i[k] (Px_l - Py_l)[k - m].
// The phase row then holds (theta^x, theta^y) per sample, and each polarization thread forms
// its own exp(j theta^p) - 1.
// RHO = false compiles the form without the ratio gradient (the taps-only launch of the Manakov
// form, adj_taps.cu), which also asks L2 for each step's checkpoint a step ahead.  RHO = true
// keeps the ratio work under the run-time flag a.want_ratio.
template <int NP, bool PERPOL = false, bool RHO = true>
__global__ void __launch_bounds__(640, 1) cbessfm_adj_kernel(const ChainArgs a) {
    constexpr int E = fft_slots(NP);
    constexpr int TPF = NP / E;
    constexpr int XL = 2 * xpad_len(NP);
    constexpr int CSL = NP + NP / 16;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ float2 s_rot[kRotTable];
    const ThreadPos tp = thread_pos<NP>(a.n_sb);
    for (int k = tp.tid; k < kRotTable; k += blockDim.x) s_rot[k] = __ldg(a.rot_tbl + k);
    // FFT twiddles staged after the G block regions
    float2* const s_tw = reinterpret_cast<float2*>(smem + (size_t)a.G * a.region_bytes);
    for (int k = tp.tid; k < fft_tw_size(NP); k += blockDim.x) s_tw[k] = __ldg(a.fft_tw + k);
    const int TB = tp.TB, g = tp.g, rem = tp.rem, p = tp.p, gi = tp.gi, j = tp.j;
    const int N = a.N, n_sb = a.n_sb;

    // ---- shared-memory layout of this block's region ----------------------------------------
    unsigned char* region = smem + (size_t)g * a.region_bytes;
    float2* e = reinterpret_cast<float2*>(region) + gi * XL + p;          // exchange [0, 17 N)
    float* prow0 = reinterpret_cast<float*>(region + a.nlpr_off);         // intensity rows
    float2* csbase = reinterpret_cast<float2*>(prow0 + n_sb * a.pstride); // (cos, sin) rows
    float* trow0 = reinterpret_cast<float*>(csbase + n_sb * CSL);         // G_theta rows
    float* gprow0 = trow0 + n_sb * a.pstride;                              // G_P rows [l][n]
    float* gtplain = gprow0 + n_sb * NP;                                   // G_theta rows [i][n]
    float* accw = gtplain + n_sb * NP;                                     // tap-gradient sums
    const int n_acc = n_sb * n_sb * a.ntaps_pad;
    double* acc_rho = reinterpret_cast<double*>(accw + n_acc);          // 16-byte aligned slot
    // per-polarization rows, from the next 128-byte boundary: Px - Py (swizzled, halo), D =
    // G_tx - G_ty (swizzled, halo) and G_Dp [l][n]
    float* const dprow0 = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(accw + n_acc + 4) + 127) & ~static_cast<uintptr_t>(127));
    float* const dtrow0 = dprow0 + n_sb * a.pstride;
    float* const gdprow0 = dtrow0 + n_sb * a.pstride;
    const int mb = a.H + a.p_off;

    const long long total = (long long)a.batch * a.n_blocks;
    const long long item = (long long)blockIdx.x * a.G + g;
    const bool real = item < total;
    const int seq = real ? (int)(item / a.n_blocks) : 0;
    const int blk = real ? (int)(item % a.n_blocks) : 0;
    const long long gblk = real ? item : 0;
    const GroupBar<NP, E> bar{1 + g * n_sb + gi};
    const float2* ck = a.ckpt + (size_t)gblk * (size_t)(a.n_st + 2) * 2 * N + (size_t)gi * NP * 2 + p;
    // taps-only form: one thread per block asks L2 for a step's checkpoint of time samples
    // (field c, 16 N bytes) a step ahead, so that the step's first read of it does not wait on
    // HBM (c4: 1.541 -> 1.503 ms; in the ratio form the same code slowed the launch)
    const float2* const ck_block = a.ckpt + (size_t)gblk * (size_t)(a.n_st + 2) * 2 * N;
    auto prefetch_ckpt = [&](int c) {
        if constexpr (!RHO) {
            if (real && rem == 0) prefetch_l2(ck_block + (size_t)c * 2 * N, 16u * (uint32_t)N);
        }
    };
    if (a.n_st > 0) prefetch_ckpt(a.n_st);                // the last step's, used first
    auto load_ckpt = [&](int c, float2 (&v)[E]) {
        const float2* src = ck + (size_t)c * 2 * N;
#pragma unroll
        for (int t = 0; t < E; ++t) v[t] = src[2 * (j + TPF * t)];
    };
    for (int k = rem; k < n_acc + 4; k += TB) accw[k] = 0.f;

    // ---- 1. stage dL/d(out) of the kept samples (zero elsewhere), DFT_N + DEMUX ----------
    float2* stage = reinterpret_cast<float2*>(region);                    // [N] (x, y) pairs
    const int lo = a.n_ov / 2;
    const long long base = (long long)blk * a.V - lo;
    for (int n = rem; n < 2 * N; n += TB) {
        const int smp = n >> 1;
        const long long gidx = base + smp;
        const bool keep = real && smp >= lo && smp < lo + a.V && gidx < a.L;
        stage[n] = keep ? a.gout[2 * ((long long)seq * a.L + gidx) + (n & 1)] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 x[E];
#pragma unroll
    for (int t = 0; t < E; ++t) x[t] = stage[2 * (n_sb * (j + TPF * t) + gi) + p];
    __syncthreads();
    fft_regs<NP, E, false, true>(x, j, e, s_tw, bar);
    bar();
#pragma unroll
    for (int t = 0; t < E; ++t) e[2 * xpad(j + TPF * t)] = x[t];
    __syncthreads();
    const int ci = -N / 2 + gi * NP + NP / 2;
    {
        // DEMUX as in the forward chain: W_N^(K r) = W_N^(K_0 r) times the slot factor of (r, t)
        const float2* eb = reinterpret_cast<const float2*>(region) + p;
        const float2* td = a.mix_td;
        int K0 = ci + j;
        K0 += (K0 < 0) ? N : 0;
#pragma unroll
        for (int t = 0; t < E; ++t) x[t] = make_float2(0.f, 0.f);
        for (int r = 0; r < n_sb; ++r) {
            const float2* er = eb + r * XL;
            const float2 w0 = __ldg(a.mix_tw + (size_t)r * N + K0);
#pragma unroll
            for (int t = 0; t < E; ++t) {
                const int kap = j + TPF * t;
                int K = ci + (kap < NP / 2 ? kap : kap - NP);
                K += (K < 0) ? N : 0;
                const float2 w = c_mul(w0, __ldg(td + r * E + t));
                x[t] = c_add(x[t], c_mul(er[2 * xpad(K & (NP - 1))], w));
            }
        }
    }
    __syncthreads();
    // x now holds G for the spectrum after the last GVD.
    // kdisp of slot t: 2 pi^2 beta2 L_step (R/N)^2 (2 c_i k' + k'^2), k' the centred lowpass bin
    // (the table value of the plan, with the integer part exact in FP32)
    auto kappa = [&](int t) {
        const int kap = j + TPF * t;
        const int kp = kap < NP / 2 ? kap : kap - NP;
        const int cc = -a.N / 2 + gi * NP + NP / 2;
        return a.kd0 * (float)(2 * cc * kp + kp * kp);
    };
    // Splitting-ratio gradient.  With Q(Z) = sum_bins kdisp Im(conj(G_Z) Z), the ratio enters
    // the first and the last GVD only, so dL/drho = Q(Z_0) - Q(Z_N) (Z_s: spectrum entering step
    // s, Z_N the final one).  Q is unchanged by a GVD, so the difference telescopes into one
    // term per step: Q(Z_s) - Q(W_s), W_s the spectrum leaving the rotation.  With
    // psi = exp(j theta) - 1, D_Z = DFT(psi u) and D_G = DFT(conj(psi) G_v + 2 G_P u),
    //   Q(Z_s) - Q(W_s) = sum kdisp Im(conj(D_G) Z_s - conj(G_W) D_Z),
    // where D_Z and D_G come from their own small sources.  On long links the two end terms
    // are thousands of times the result, and their FP32 rounding would dominate it.  Z_s is
    // rebuilt backwards, Z_s = NP conj(h_s) Z_(s+1) - D_Z / NP (|h_s| = 1/NP), from the final
    // spectrum, and the adjoint's own G for Z_s becomes NP G_W + D_G.  kdisp omits the
    // subband-centre part (an exact invariant), which also keeps the two terms of a step from
    // cancelling when theta is large.  Each thread sums its 16 bins of a term in FP32 (those
    // rounding errors are independent across threads and steps) and adds the partial to an
    // FP64 total once per term; GB300's FP64 rate makes per-bin FP64 arithmetic costly.
    double rho_part = 0.0;
    const float NPf = (float)NP;
    const float inv_NP = 1.0f / NPf;
    float2* const sg = a.stash + (size_t)gblk * 4 * N + (size_t)gi * NP * 2 + p;   // G_W
    float2* const sz = sg + 2 * N;                                               // Z_s

    // ---- 2. steps, last to first ----------------------------------------------------------
    float2* cs_mine = csbase + gi * CSL;                                    // psi rows
    // exp(j theta) - 1 of slot t for this thread's polarization: the row holds it (Manakov), or
    // (theta^x, theta^y) from which each polarization thread forms its own (per-polarization)
    auto psi_at = [&](int t) -> float2 {
        const float2 r = cs_mine[cpad(j + TPF * t)];
        if constexpr (PERPOL) {
            return rotation_psi(p ? r.y : r.x, s_rot);
        } else {
            return r;
        }
    };
    const int k0 = E * j + (E / 2) * p;                                    // FIR outputs k0 ..
#pragma unroll 1
    for (int s = a.n_st - 1; s >= 0; --s) {
        const float2* h = a.gvd + (size_t)((s < a.n_st - 1 ? 1 : 2) * n_sb + gi) * NP;
        // G_W = conj(h) G_(Z_(s+1)), kept in the block's scratch when dL/drho is wanted
        const bool rho = RHO && a.want_ratio != 0;
#pragma unroll
        for (int t = 0; t < E; ++t) {
            x[t] = c_mulc(x[t], __ldg(h + j + TPF * t));
            if (real && rho) sg[2 * (j + TPF * t)] = x[t];
        }
        if (s > 0) prefetch_ckpt(s);                       // the next step's (c = 1 + (s - 1))
        {
            float2 u[E];
            load_ckpt(1 + s, u);
            // while the FIR runs, this thread's slots of the exchange array keep what the
            // transform after it needs: the step's time samples (the source of D_Z) on the ratio
            // path, G_W otherwise (the ratio path has G_W in its scratch field).  The array is
            // idle until that transform, and no other thread still reads these slots: the last
            // pass of every transform loads exactly the thread's own slot elements, and before
            // the first step only barrier-separated DEMUX reads touched the array.
#pragma unroll
            for (int t = 0; t < E; ++t) e[2 * xpad(j + TPF * t)] = rho ? u[t] : x[t];
            float* prow = prow0 + gi * a.pstride;
            // both lanes of an x/y pair hold every slot's intensity after the shuffle: lane p
            // stores the slots t with t % 2 == p (no branch on the polarization)
#pragma unroll
            for (int t2 = 0; t2 < E; t2 += 2) {
                const float own0 = fmaf(u[t2].x, u[t2].x, u[t2].y * u[t2].y);
                const float own1 = fmaf(u[t2 + 1].x, u[t2 + 1].x, u[t2 + 1].y * u[t2 + 1].y);
                const float oth0 = __shfl_xor_sync(0xffffffffu, own0, 1);
                const float oth1 = __shfl_xor_sync(0xffffffffu, own1, 1);
                row_store<NP, E>(prow, mb, j + TPF * (t2 + p), a.H, p ? own1 + oth1 : own0 + oth0);
                if constexpr (PERPOL)                         // |x|^2 - |y|^2 of the same slot
                    row_store<NP, E>(dprow0 + gi * a.pstride, mb, j + TPF * (t2 + p), a.H,
                                     p ? oth1 - own1 : own0 - oth0);
            }
        }
        __syncthreads();
        {
            const float4* wb = reinterpret_cast<const float4*>(
                a.taps + (size_t)(s * n_sb + gi) * n_sb * a.ntaps_pad);
#pragma unroll
            for (int h8 = 0; h8 < E / 16; ++h8) {
                float acc[8];
                fir8_acc<E>(a, wb, prow0, k0 + 8 * h8, acc);
                float2* dst = cs_mine + cpad(k0 + 8 * h8);
                if constexpr (PERPOL) {
                    // delta = (1/3) sum_{l != i} w_il (Px_l - Py_l); the row keeps theta +- delta
                    float dl[8];
                    fir8_acc<E>(a, wb, dprow0, k0 + 8 * h8, dl, gi);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float d = dl[q] * (1.0f / 3.0f);
                        dst[q] = make_float2(acc[q] + d, acc[q] - d);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) dst[q] = rotation_psi(acc[q], s_rot);
                }
            }
        }
        __syncthreads();
        // Two inverse transforms share one call site: D_Z = conj(IDFT(conj(psi u))), then G_v.
        // Between them: Z_s = NP conj(h) Z_(s+1) - D_Z / NP, the G_W part of the ratio term, and
        // G_W back into x as the second transform's input.
        {
            const float2* z1 = s == a.n_st - 1 ? ck + (size_t)(a.n_st + 1) * 2 * N : sz;
            if (!rho) {
#pragma unroll
                for (int t = 0; t < E; ++t) x[t] = e[2 * xpad(j + TPF * t)];      // G_W
            }
#pragma unroll 1
            for (int ph = rho ? 0 : 1; ph < 2; ++ph) {
                if (ph == 0) {
#pragma unroll
                    for (int t = 0; t < E; ++t)                                    // u from e
                        x[t] = c_conj(c_mul(psi_at(t), e[2 * xpad(j + TPF * t)]));
                }
                fft_regs<NP, E, true, true>(x, j, e, s_tw, bar);
                if (ph == 0) {
                    float rs = 0.f;
#pragma unroll
                    for (int t0 = 0; t0 < E; t0 += 4) {
                        // four slots' scratch and table loads issued together before their
                        // stores (the pass is bound by L2 round trips: 0.46 ms of c4's 2.31)
                        float2 zv[4], hw[4], gv[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int o = 2 * (j + TPF * (t0 + q));
                            zv[q] = z1[o];
                            hw[q] = __ldg(h + j + TPF * (t0 + q));
                            gv[q] = sg[o];
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int t = t0 + q;
                            const int o = 2 * (j + TPF * t);
                            const float2 dz = c_conj(x[t]);
                            const float2 zs = c_sub(c_scale(c_mulc(zv[q], hw[q]), NPf), c_scale(dz, inv_NP));
                            if (real) sz[o] = zs;
                            rs = fmaf(-kappa(t), gv[q].x * dz.y - gv[q].y * dz.x, rs);
                            x[t] = gv[q];
                        }
                    }
                    rho_part += (double)rs;
                }
            }
        }
        {
            // G_theta and the first part of D_G's source, conj(psi) G_v
            float2 u[E];
            load_ckpt(1 + s, u);
            float* trow = trow0 + gi * a.pstride;
#pragma unroll
            for (int t = 0; t < E; ++t) {
                const float2 ps = psi_at(t);
                const float2 v = c_mul(u[t], make_float2(1.0f + ps.x, ps.y));
                const float own = -(x[t].x * v.y - x[t].y * v.x);          // -Im(conj(G_v) v)
                const float oth = __shfl_xor_sync(0xffffffffu, own, 1);
                const float gt = own + oth;                                 // S (Manakov: G_theta)
                // both lanes hold the sum: lane p stores the odd or even slots (no branch on p)
                if ((t & 1) == p) {
                    const int n = j + TPF * t;
                    row_store<NP, E>(trow, mb, n, a.H, gt);
                    gtplain[gi * NP + n] = gt;
                    if constexpr (PERPOL)                                   // D = G_tx - G_ty
                        row_store<NP, E>(dtrow0 + gi * a.pstride, mb, n, a.H, p ? oth - own : own - oth);
                }
                // conj(psi) G_v (the ratio path adds G_v back in the spectral domain as NP G_W)
                x[t] = rho ? c_mulc(x[t], ps) : c_mulc(x[t], make_float2(1.0f + ps.x, ps.y));
            }
        }
        __syncthreads();
        // x (conj(psi) G_v) waits in this thread's own slots of the exchange array, idle until the
        // step's last transform, so the correlation below has the registers to itself
#pragma unroll
        for (int t = 0; t < E; ++t) e[2 * xpad(j + TPF * t)] = x[t];
        {
            // dL/dw[s][i][l][m] = sum_k G_theta_i[k] P_l[k - m].  Each (i, l) pair is handled by
            // 16 consecutive lanes; lane `sub` takes the KW-sample chunks k0 = 16 KW r + KW sub
            // (its float4 loads are 16 bytes apart across lanes: no bank conflicts), loads one
            // intensity window for all 12 taps of the 9-to-12-tap case (KW + 12 - 1 samples), and
            // accumulates the 12 tap sums in registers; a 16-lane shuffle reduction then gives
            // each pair's sums to one lane, which stores them.  Other tap counts use the generic
            // loop below.
            const int nseg = NP / 16;
            const int n_pairs = n_sb * n_sb;
            // (the per-polarization form takes the generic loop, which also sums its D term)
            const int lanes = (!PERPOL && TB % 16 == 0 && a.nchunks == 3 && NP >= 64) ? TB : 0;
            for (int base_t = 0; lanes > 0 && base_t < n_pairs * 16; base_t += lanes) {
                const int t16 = base_t + rem;
                const bool act = t16 < n_pairs * 16;
                const int pair = act ? t16 >> 4 : 0, sub = t16 & 15;
                const int i = pair / n_sb, l = pair - i * n_sb;
                const float* gtr = gtplain + i * NP;
                const float* pr = prow0 + l * a.pstride;
                float acc[12];
#pragma unroll
                for (int m = 0; m < 12; ++m) acc[m] = 0.f;
                if (act) {
                    constexpr int KW = NP >= 128 ? 8 : 4;           // samples per lane and pass
#pragma unroll 2
                    for (int it = 0; it < NP / (16 * KW); ++it) {
                        const int k0 = KW * sub + 16 * KW * it;
                        float g[KW];
#pragma unroll
                        for (int c4 = 0; c4 < KW / 4; ++c4) {
                            const float4 g4 = *reinterpret_cast<const float4*>(gtr + k0 + 4 * c4);
                            g[4 * c4] = g4.x; g[4 * c4 + 1] = g4.y; g[4 * c4 + 2] = g4.z;
                            g[4 * c4 + 3] = g4.w;
                        }
                        // P_l[k0 + q - m], m = -nc + mi (mi in [0, 12)): window start
                        // k0 + nc - 11, aligned because (H + p_off + nc + 1) % 4 == 0
                        const int ws = mb + k0 + a.nc - 11;
                        float win[KW + 12];
#pragma unroll
                        for (int e4 = 0; e4 < KW / 4 + 3; ++e4) {
                            const float4 v = *reinterpret_cast<const float4*>(pr + pswz<E>(ws + 4 * e4));
                            win[4 * e4] = v.x; win[4 * e4 + 1] = v.y; win[4 * e4 + 2] = v.z;
                            win[4 * e4 + 3] = v.w;
                        }
#pragma unroll
                        for (int mi = 0; mi < 12; ++mi)
#pragma unroll
                            for (int q = 0; q < KW; ++q) acc[mi] = fmaf(g[q], win[q - mi + 11], acc[mi]);
                    }
                }
#pragma unroll
                for (int mi = 0; mi < 12; ++mi) {
#pragma unroll
                    for (int o = 8; o > 0; o >>= 1) acc[mi] += __shfl_xor_sync(0xffffffffu, acc[mi], o);
                }
                if (act && sub == 0) {
                    float* dst = accw + (i * n_sb + l) * a.ntaps_pad;
#pragma unroll
                    for (int mi = 0; mi < 12; ++mi) dst[mi] = acc[mi];
                }
            }
            if (lanes == 0) {
                // blocks narrower than 16 lanes (small N'): one atomic per segment and tap chunk.
                // corr(tr, pr, scale) adds scale sum_k tr_i[k] pr_l[k - m] for the 16 samples of
                // one segment and one four-tap chunk.
                auto corr = [&](const float* tr, const float* pr, int ks, int c, float scale,
                                float* acc) {
                    const int m = mb + ks + a.nc - 4 * c - 3;
                    float win[20];
#pragma unroll
                    for (int e4 = 0; e4 < 5; ++e4) {
                        const float4 v = *reinterpret_cast<const float4*>(pr + pswz<E>(m + 4 * e4));
                        win[4 * e4] = v.x; win[4 * e4 + 1] = v.y; win[4 * e4 + 2] = v.z;
                        win[4 * e4 + 3] = v.w;
                    }
                    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float gq = tr[pswz<E>(mb + ks + q)];
                        s0 = fmaf(gq, win[q + 3], s0);
                        s1 = fmaf(gq, win[q + 2], s1);
                        s2 = fmaf(gq, win[q + 1], s2);
                        s3 = fmaf(gq, win[q], s3);
                    }
                    atomicAdd(acc, scale * s0);
                    atomicAdd(acc + 1, scale * s1);
                    atomicAdd(acc + 2, scale * s2);
                    atomicAdd(acc + 3, scale * s3);
                };
                for (int w = rem; w < n_pairs * nseg; w += TB) {
                    const int pair = w / nseg, seg = w - pair * nseg;
                    const int i = pair / n_sb, l = pair - i * n_sb;
                    const int ks = 16 * seg;
                    for (int c = 0; c < a.nchunks; ++c) {
                        float* acc = accw + (i * n_sb + l) * a.ntaps_pad + 4 * c;
                        corr(trow0 + i * a.pstride, prow0 + l * a.pstride, ks, c, 1.0f, acc);
                        if constexpr (PERPOL) {
                            if (i != l)            // (1/3) sum_k D_i[k] (Px_l - Py_l)[k - m]
                                corr(dtrow0 + i * a.pstride, dprow0 + l * a.pstride, ks, c,
                                     1.0f / 3.0f, acc);
                        }
                    }
                }
            }
            // G_P_l[n] = sum_i sum_m' wt[s][l][i][m'] G_theta_i[n - m'] (transposed taps)
            const float4* wb = reinterpret_cast<const float4*>(
                a.taps_t + (size_t)(s * n_sb + gi) * n_sb * a.ntaps_pad);
#pragma unroll
            for (int h8 = 0; h8 < E / 16; ++h8) {
                float acc[8];
                fir8_acc<E>(a, wb, trow0, k0 + 8 * h8, acc);
                float4* dst = reinterpret_cast<float4*>(gprow0 + gi * NP + k0 + 8 * h8);
                dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
                dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
                if constexpr (PERPOL) {
                    // G_Dp_l[n] = (1/3) sum_{i != l} sum_m w_il[m] D_i[n + m]
                    fir8_acc<E>(a, wb, dtrow0, k0 + 8 * h8, acc, gi);
                    float4* dd = reinterpret_cast<float4*>(gdprow0 + gi * NP + k0 + 8 * h8);
                    const float third = 1.0f / 3.0f;
                    dd[0] = make_float4(third * acc[0], third * acc[1], third * acc[2], third * acc[3]);
                    dd[1] = make_float4(third * acc[4], third * acc[5], third * acc[6], third * acc[7]);
                }
            }
        }
        __syncthreads();
        {
            // publish and clear this step's tap-gradient sums
            if (real) {
                float* gp = a.gpart + (size_t)gblk * ((size_t)a.n_st * n_acc + 4) + (size_t)s * n_acc;
                for (int k = rem; k < n_acc; k += TB) gp[k] = accw[k];
            }
            float2 u[E];
            load_ckpt(1 + s, u);
            const float* gpr = gprow0 + gi * NP;
#pragma unroll
            for (int t = 0; t < E; ++t) {
                float gp2 = 2.f * gpr[j + TPF * t];
                if constexpr (PERPOL) {                       // G_Px = G_P + G_Dp, G_Py = G_P - G_Dp
                    const float gd = 2.f * gdprow0[gi * NP + j + TPF * t];
                    gp2 = p ? gp2 - gd : gp2 + gd;
                }
                const float2 xv = e[2 * xpad(j + TPF * t)];               // parked above
                x[t] = make_float2(fmaf(gp2, u[t].x, xv.x), fmaf(gp2, u[t].y, xv.y));
            }
        }
        __syncthreads();
        for (int k = rem; k < n_acc; k += TB) accw[k] = 0.f;
        // D_G = DFT(conj(psi) G_v + 2 G_P u); G for Z_s = NP G_W + D_G; the D_G part of the ratio
        fft_regs<NP, E, false, true>(x, j, e, s_tw, bar);
        if (rho) {
            float rs = 0.f;
#pragma unroll
            for (int t = 0; t < E; ++t) {
                const int o = 2 * (j + TPF * t);
                const float2 zs = sz[o];
                rs = fmaf(kappa(t), x[t].x * zs.y - x[t].y * zs.x, rs);
                const float2 gw = sg[o];
                x[t] = make_float2(fmaf(NPf, gw.x, x[t].x), fmaf(NPf, gw.y, x[t].y));
            }
            rho_part += (double)rs;
        }
    }

    // ---- 3. first GVD, adjoint of entry (MUX + IDFT_N), scatter to G_in ---------------------
    // the block's ratio sum: FP64 atomics on one shared word contend (a compare-and-swap per
    // update), so when every warp lies within one block the warp first sums its lanes
    if (TB % 32 == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rho_part += __shfl_xor_sync(0xffffffffu, rho_part, o);
        if ((tp.tid & 31) == 0) atomicAdd(acc_rho, rho_part);
    } else {
        atomicAdd(acc_rho, rho_part);             // warps may span several small blocks
    }
    {
        const float2* h = a.gvd + (size_t)gi * NP;
#pragma unroll
        for (int t = 0; t < E; ++t) x[t] = c_mulc(x[t], __ldg(h + j + TPF * t));
    }
    __syncthreads();
    if (real && rem == 0) {
        float* gp = a.gpart + (size_t)gblk * ((size_t)a.n_st * n_acc + 4) + (size_t)a.n_st * n_acc;
        *reinterpret_cast<double*>(gp) = *acc_rho;                       // 16-byte aligned
    }
    if (a.gin == nullptr) return;                                         // uniform
    {
        float2* ex = reinterpret_cast<float2*>(region) + p;
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const int kap = j + TPF * t;
            int K = ci + (kap < NP / 2 ? kap : kap - NP);
            if (K < 0) K += N;
            ex[2 * xpad(K)] = x[t];
        }
        __syncthreads();
        // MUX as in the forward chain: W_N^(K gi) = W_N^((j + NP q) gi) W_N^((N'/E) t gi)
        const float2* wr = a.mix_tw + (size_t)gi * N;
        const float2* tm = a.mix_tm + gi * E;
#pragma unroll
        for (int t = 0; t < E; ++t) x[t] = make_float2(0.f, 0.f);
        for (int q = 0; q < n_sb; ++q) {
            const float2 w0 = __ldg(wr + j + NP * q);
#pragma unroll
            for (int t = 0; t < E; ++t) {
                const int K = j + TPF * t + NP * q;
                const float2 w = c_mul(w0, __ldg(tm + t));
                x[t] = c_add(x[t], c_mulc(ex[2 * xpad(K)], w));
            }
        }
    }
    __syncthreads();
    fft_regs<NP, E, true, true>(x, j, e, s_tw, bar);
    if (real) {
        long long pos = base % a.L;
        if (pos < 0) pos += a.L;
        float* gin = reinterpret_cast<float*>(a.gin) + 4 * (long long)seq * a.L + 2 * p;
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const int n = n_sb * (j + TPF * t) + gi;
            long long q = pos + n;
            q -= (q / a.L) * a.L;
            atomicAdd(gin + 4 * q, x[t].x);
            atomicAdd(gin + 4 * q + 1, x[t].y);
        }
    }
}

// Launch of the per-polarization form (adj_perpol.cu): the checkpointed forward (adjoint =
// false) or the adjoint kernel over the blocks of `a`, with the region sizes set in `a`.
cudaError_t launch_adj_per_pol(int np, bool adjoint, const ChainArgs& a, int threads,
                               cudaStream_t st);
// Launch of the Manakov adjoint without the ratio gradient (adj_taps.cu).
cudaError_t launch_adj_taps(int np, const ChainArgs& a, int threads, cudaStream_t st);

}  // namespace cbessfm
