// fwd.cu -- fused CB-ESSFM forward chain kernel (sm_103a).
//
// One CTA processes G overlap-and-save blocks (Sec. III-A, Fig. 2); each block is handled by
// n_sb groups of NP/16 threads.  Per block:
//   1. bulk-copy (TMA) the N = n_sb * NP input samples into shared memory (two or more copies
//      when the block wraps around the periodic sequence);
//   2. full-band DFT of size N per polarization as n_sb polyphase DFTs of size NP (group r
//      transforms x[n_sb n' + r]) followed by the twiddled n_sb-point combination
//      X[K] = sum_r W_N^(K r) Y_r[K mod NP], evaluated directly at the bins of each subband
//      (this is the DEMUX of Fig. 3: group i ends up holding the N' bins of subband i);
//   3. first GVD, then N_st times {inverse DFT of size NP, intensity of both polarizations,
//      MIMO FIR of Eq. (NLPR-multiband-2pol), rotation exp(+j theta), DFT of size NP, GVD};
//   4. MUX (the inverse combination) and inverse polyphase DFTs, then a direct store of the
//      V valid samples as float4.
// All scale factors (1/N at entry, 1/NP per step) are folded into the GVD tables, which the
// plan builds in FP64 with the phase reduced modulo 2 pi.
#include "device_common.cuh"
#include "internal.h"

namespace cbessfm {

constexpr int kMaxG = 16;
// exp(j theta) by table look-up (the paper computes the exponential with a LUT): theta =
// 2 pi k / 256 + d with |d| <= pi / 256; the table entry is built in FP64 by the plan and the
// residual rotation is 1 - d^2/2 + j d (1 - d^2/6), whose truncation error (< 1e-9) is far below
// float rounding.  d comes from a two-constant Cody-Waite reduction: the step 2 pi / 256 =
// kRotStepHi + kRotStepLo with kRotStepHi exact in 8 bits, so k * kRotStepHi is exact for
// |k| < 2^16 (|theta| < 1600 rad).
constexpr int kRotTable = 256;
constexpr float kRotInvStep = 40.7436654315252059568f;     // 256 / (2 pi)
constexpr float kRotStepHi = 0.0245361328125f;              // 201 / 8192
constexpr float kRotStepLo = 7.5597936702587190e-6f;        // 2 pi / 256 - 201 / 8192

__device__ __forceinline__ float2 rotation_factor(float th, const float2* __restrict__ tbl) {
    const float kf = rintf(th * kRotInvStep);
    float d = fmaf(-kf, kRotStepHi, th);
    d = fmaf(-kf, kRotStepLo, d);
    const float2 t = tbl[(int)kf & (kRotTable - 1)];
    const float d2 = d * d;
    return c_mul(t, make_float2(fmaf(-0.5f, d2, 1.0f), d * fmaf(-0.16666666666666667f, d2, 1.0f)));
}
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz: never reached by a live copy

// Barrier over the 2 NP/16 threads (both polarizations) of one FFT group.  Groups of a warp or
// less share their warp with other groups running the same code, so a warp barrier suffices.
template <int NP>
struct GroupBar {
    int id;
    __device__ __forceinline__ void operator()() const {
        if constexpr (2 * (NP / 16) > 32) {
            named_bar(id, 2 * (NP / 16));
        } else {
            __syncwarp();
        }
    }
};

// Intensity rows are XOR-swizzled in 16-byte granules: float m of a row lives at
// m ^ (((m >> 5) & 1) << 2).  The FIR's lanes read float4 windows 32 bytes apart; the swizzle
// puts the two 32-float halves of every 8-lane group on complementary banks.
__device__ __forceinline__ int pswz(int m) { return m ^ (((m >> 5) & 1) << 2); }
// (cos, sin) rows carry one spare float2 per 16 so the 8-sample runs of adjacent lanes do not
// collide on a bank.
__device__ __forceinline__ int cpad(int k) { return k + (k >> 4); }

// Rotation factors for the 8 samples k = k0 .. k0 + 7 of subband i, step s:
// theta_i[k] = sum_l sum_m w[s][i][l][m + nc] P_l[k - m]; stores (cos theta, sin theta).
// P rows carry a circular halo of H samples on each side, so no index wraps here; each chunk of
// four taps reads a 12-sample window with aligned 16-byte loads.
__device__ __forceinline__ void nlpr_rotation8(const ChainArgs& a, const float* __restrict__ prow0,
                                               float2* __restrict__ cs_row,
                                               const float2* __restrict__ rot_tbl, int s, int i,
                                               int k0) {
    const float4* wbase = reinterpret_cast<const float4*>(
        a.taps + (size_t)(s * a.n_sb + i) * a.n_sb * a.ntaps_pad);
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.f;
    const int m0 = a.H + a.p_off + k0 + a.nc - 3;      // row index of the first window sample
    for (int l = 0; l < a.n_sb; ++l) {
        const float* pl = prow0 + l * a.pstride;
        const float4* wrow = wbase + l * a.nchunks;
        for (int c = 0; c < a.nchunks; ++c) {
            const float4 w4 = __ldg(wrow + c);
            const int m = m0 - 4 * c;
            float win[12];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const float4 v = *reinterpret_cast<const float4*>(pl + pswz(m + 4 * e));
                win[4 * e] = v.x; win[4 * e + 1] = v.y; win[4 * e + 2] = v.z; win[4 * e + 3] = v.w;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float t = acc[q];
                t = fmaf(w4.x, win[q + 3], t);   // m = -nc + 4c
                t = fmaf(w4.y, win[q + 2], t);   // m = -nc + 4c + 1
                t = fmaf(w4.z, win[q + 1], t);
                t = fmaf(w4.w, win[q], t);
                acc[q] = t;
            }
        }
    }
    float2* dst = cs_row + cpad(k0);                   // k0 % 16 in {0, 8}: no carry below
#pragma unroll
    for (int q = 0; q < 8; ++q) dst[q] = rotation_factor(acc[q], rot_tbl);
}

// Thread layout of one OLS block (TB = 2 n_sb NP/16 threads): rem = 2 jj + p with p the
// polarization (x/y partners are adjacent lanes) and jj = gi * NP/16 + j.
template <int NP>
__global__ void __launch_bounds__(640, 1) cbessfm_fwd_kernel(const ChainArgs a) {
    constexpr int TPF = NP / 16;
    constexpr int XL = 2 * xpad_len(NP);               // float2 per group exchange array
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[kMaxG];
    __shared__ float2 s_rot[kRotTable];

    const int tid = threadIdx.x;
    for (int k = tid; k < kRotTable; k += blockDim.x) s_rot[k] = __ldg(a.rot_tbl + k);
    const int TB = 2 * a.n_sb * TPF;
    const int g = tid / TB;
    const int rem = tid - g * TB;
    const int p = rem & 1;
    const int jj = rem >> 1;
    const int gi = jj / TPF;           // subband (steps) or polyphase component (entry/exit)
    const int j = jj - gi * TPF;
    unsigned char* region = smem + (size_t)g * a.region_bytes;
    float2* e = reinterpret_cast<float2*>(region) + gi * XL + p;

    const long long total = (long long)a.batch * a.n_blocks;
    const long long item = (long long)blockIdx.x * a.G + g;
    const bool real = item < total;
    const int seq = real ? (int)(item / a.n_blocks) : 0;
    const int blk = real ? (int)(item % a.n_blocks) : 0;
    const GroupBar<NP> bar{1 + g * a.n_sb + gi};

    // ---------------- 1. stage the block (bulk copies, circular wrap) ----------------------
    float2* stage = reinterpret_cast<float2*>(region);          // [N] samples as (x, y) pairs
    if (tid < a.G) mbar_init(&bars[tid], 1);
    mbar_fence_init();
    __syncthreads();
    if (real && rem == 0) {
        mbar_arrive_expect_tx(&bars[g], (uint32_t)a.N * 16u);
        long long pos = ((long long)blk * a.V - a.n_ov / 2) % a.L;
        if (pos < 0) pos += a.L;
        const float4* src = reinterpret_cast<const float4*>(a.in) + (long long)seq * a.L;
        float4* dst4 = reinterpret_cast<float4*>(region);
        int dst = 0;
        while (dst < a.N) {
            const int len = (int)min((long long)(a.N - dst), a.L - pos);
            bulk_copy_g2s(dst4 + dst, src + pos, (uint32_t)len * 16u, &bars[g]);
            dst += len;
            pos = 0;
        }
    }
    bool ok = true;
    if (real) {
        ok = mbar_wait_bounded(&bars[g], 0, kWaitCycles);
    } else {
        for (int n = rem; n < 2 * a.N; n += TB) stage[n] = make_float2(0.f, 0.f);
    }
    if (__syncthreads_or(!ok)) {
        if (!ok) atomicOr(a.status, kStatusTimeout);
        if (real) mbar_wait_bounded(&bars[g], 0, kWaitCycles);   // let in-flight copies land
        return;
    }

    float2 x[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) x[t] = stage[2 * (a.n_sb * (j + TPF * t) + gi) + p];
    __syncthreads();

    // ---------------- 2. full-band DFT + DEMUX -------------------------------------------
    fft_regs<NP, false>(x, j, e, a.fft_tw, bar);                  // Y_r, r = gi
    bar();
#pragma unroll
    for (int t = 0; t < 16; ++t) e[2 * xpad(j + TPF * t)] = x[t];
    __syncthreads();
    const int N = a.N;
    const int ci = -N / 2 + gi * NP + NP / 2;                      // centre bin of subband gi
    {
        // X_i[kap] = sum_r W_N^(K r) Y_r[K mod NP], K = (c_i + k') mod N; loop r outermost so that
        // only the 16 accumulators stay live.
        const float2* eb = reinterpret_cast<const float2*>(region) + p;
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = make_float2(0.f, 0.f);
        for (int r = 0; r < a.n_sb; ++r) {
            const float2* er = eb + r * XL;
            const float2* wr = a.mix_tw + (size_t)r * N;
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int kap = j + TPF * t;
                int K = ci + (kap < NP / 2 ? kap : kap - NP);
                K += (K < 0) ? N : 0;
                x[t] = c_add(x[t], c_mul(er[2 * xpad(K & (NP - 1))], __ldg(wr + K)));
            }
        }
    }
    __syncthreads();

    // ---------------- 3. GVD / NLPR steps --------------------------------------------------
    {
        const float2* h = a.gvd + (size_t)gi * NP;                  // first GVD (x 1/N)
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = c_mul(x[t], __ldg(h + j + TPF * t));
    }
    // intensity rows and (cos, sin) rows: after the exchange arrays when they fit (a.sep), else
    // aliased onto them (then two more block-wide barriers per step guard the reuse)
    float* prow0 = reinterpret_cast<float*>(region + a.nlpr_off);
    float2* csbase = reinterpret_cast<float2*>(prow0 + a.n_sb * a.pstride);
    const float2* cs_mine = csbase + gi * (NP + NP / 16);
    const int cs_base = (NP >= 256) ? cpad(j) : 0;
#pragma unroll 1
    for (int s = 0; s < a.n_st; ++s) {
        fft_regs<NP, true>(x, j, e, a.fft_tw, bar);               // subband time samples
        if (!a.sep) __syncthreads();
        {
            float* prow = prow0 + gi * a.pstride;
            const int mb = a.H + a.p_off;
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                float pw = fmaf(x[t].x, x[t].x, x[t].y * x[t].y);
                pw += __shfl_xor_sync(0xffffffffu, pw, 1);          // |x|^2 + |y|^2
                if (p == 0) {
                    const int n = j + TPF * t;
                    prow[pswz(mb + n)] = pw;
                    // circular halo: H <= NP (ntaps <= NP/2), so one copy per side suffices
                    if (n < a.H) prow[pswz(mb + n + NP)] = pw;
                    if (n >= NP - a.H) prow[pswz(mb + n - NP)] = pw;
                }
            }
        }
        __syncthreads();
        nlpr_rotation8(a, prow0, csbase + gi * (NP + NP / 16), s_rot, s, gi, 16 * j + 8 * p);
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const float2 rot = (NP >= 256) ? cs_mine[cs_base + (TPF + TPF / 16) * t]
                                           : cs_mine[cpad(j + TPF * t)];
            x[t] = c_mul(x[t], rot);
        }
        if (!a.sep) __syncthreads();
        fft_regs<NP, false>(x, j, e, a.fft_tw, bar);              // back to subband bins
        const float2* h = a.gvd + (size_t)((s < a.n_st - 1 ? 1 : 2) * a.n_sb + gi) * NP;
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = c_mul(x[t], __ldg(h + j + TPF * t));
    }

    // ---------------- 4. MUX + inverse full-band DFT + store --------------------------------
    __syncthreads();
    {
        float2* ex = reinterpret_cast<float2*>(region) + p;        // [2 xpad(K) + p]
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int kap = j + TPF * t;
            int K = ci + (kap < NP / 2 ? kap : kap - NP);
            if (K < 0) K += N;
            ex[2 * xpad(K)] = x[t];
        }
        __syncthreads();
        // Z_r[kap] = sum_q conj(W_N^(K r)) Xi[K], K = kap + NP q (q outermost, as above)
        const float2* wr = a.mix_tw + (size_t)gi * N;
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = make_float2(0.f, 0.f);
        for (int q = 0; q < a.n_sb; ++q) {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int K = j + TPF * t + NP * q;
                x[t] = c_add(x[t], c_mulc(ex[2 * xpad(K)], __ldg(wr + K)));
            }
        }
    }
    __syncthreads();
    fft_regs<NP, true>(x, j, e, a.fft_tw, bar);                   // x[n_sb n' + r], r = gi
    if (real) {
        float2* dst = reinterpret_cast<float2*>(a.out) + 2 * (long long)seq * a.L + p;
        const int lo = a.n_ov / 2;
        const long long base = (long long)blk * a.V - lo;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int n = a.n_sb * (j + TPF * t) + gi;
            if (n >= lo && n < lo + a.V) {
                const long long gidx = base + n;
                if (gidx < a.L) dst[2 * gidx] = x[t];
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// FP64 table builder: GVD factors of the three step kinds for every subband bin
// ------------------------------------------------------------------------------------------
__global__ void build_gvd_kernel(float2* __restrict__ gvd, float* __restrict__ kdisp, int n_sb,
                                 int np, double beta2, double rate, double dz0, double dz1,
                                 double dz2, double scale0, double scale12, double step_len) {
    const int per = n_sb * np;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 3 * per) return;
    const int tbl = idx / per;
    const int r = idx - tbl * per;
    const int i = r / np;
    const int kap = r - i * np;
    const long long N = (long long)n_sb * np;
    const long long b = -N / 2 + (long long)i * np + np / 2 + (kap < np / 2 ? kap : kap - np);
    const double f = (double)b * rate / (double)N;
    const double dz = tbl == 0 ? dz0 : (tbl == 1 ? dz1 : dz2);
    // phase / (2 pi) = pi beta2 dz f^2, reduced to [0, 1) turns before the sine and cosine
    const double turns = 3.14159265358979323846 * beta2 * dz * f * f;
    const double frac = turns - floor(turns);
    double sn, cs;
    sincospi(2.0 * frac, &sn, &cs);
    const double sc = tbl == 0 ? scale0 : scale12;
    gvd[idx] = make_float2((float)(cs * sc), (float)(sn * sc));
    if (tbl == 0 && kdisp != nullptr)
        kdisp[r] = (float)(2.0 * 9.86960440108935861883 * beta2 * step_len * f * f);
}

cudaError_t launch_build_gvd(const PlanImpl& p, cudaStream_t stream) {
    const int np = p.n_fft;
    const double Ls = p.step_length;
    double dz0, dz1, dz2;
    if (p.n_st == 0) {
        dz0 = p.link.span_length * p.link.n_spans;
        dz1 = dz2 = 0.0;
    } else {
        dz0 = (1.0 - p.ratio) * Ls;
        dz1 = Ls;
        dz2 = p.ratio * Ls;
    }
    const int total = 3 * p.n_sb * np;
    build_gvd_kernel<<<(total + 255) / 256, 256, 0, stream>>>(
        p.d_gvd, p.d_kdisp, p.n_sb, np, p.link.beta2, p.link.sample_rate, dz0, dz1, dz2,
        1.0 / (double)p.N, 1.0 / (double)np, Ls);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
template <int NP>
static cudaError_t launch_np(const PlanImpl& p, const ChainArgs& a, cudaStream_t stream) {
    const long long total = (long long)a.batch * a.n_blocks;
    const long long grid = (total + a.G - 1) / a.G;
    if (grid <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.G * a.region_bytes;
    cbessfm_fwd_kernel<NP><<<(unsigned)grid, p.threads, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int NP>
static cudaError_t prepare_np(int smem_bytes) {
    return cudaFuncSetAttribute(cbessfm_fwd_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_bytes);
}

cudaError_t prepare_forward(int np, int smem_bytes) {
    switch (np) {
        case 16: return prepare_np<16>(smem_bytes);
        case 32: return prepare_np<32>(smem_bytes);
        case 64: return prepare_np<64>(smem_bytes);
        case 128: return prepare_np<128>(smem_bytes);
        case 256: return prepare_np<256>(smem_bytes);
        case 512: return prepare_np<512>(smem_bytes);
        case 1024: return prepare_np<1024>(smem_bytes);
        case 2048: return prepare_np<2048>(smem_bytes);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_forward(const PlanImpl& p, const ChainArgs& a, cudaStream_t stream) {
    switch (p.n_fft) {
        case 16: return launch_np<16>(p, a, stream);
        case 32: return launch_np<32>(p, a, stream);
        case 64: return launch_np<64>(p, a, stream);
        case 128: return launch_np<128>(p, a, stream);
        case 256: return launch_np<256>(p, a, stream);
        case 512: return launch_np<512>(p, a, stream);
        case 1024: return launch_np<1024>(p, a, stream);
        case 2048: return launch_np<2048>(p, a, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cbessfm
