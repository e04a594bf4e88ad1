// fwd_kernel.cuh -- fused CB-ESSFM forward chain kernel (sm_103a), templated on N' and storage.
//
// One CTA processes G overlap-and-save blocks (Sec. III-A, Fig. 2); each block is handled by
// n_sb groups of 2 NP/E threads (one polarization per thread, E = 16 register slots, 32 for
// N' = 2048).  Per block:
//   1. bulk-copy (TMA) the N = n_sb * NP input samples into shared memory (two or more copies
//      when the block wraps around the periodic sequence; 8-byte samples whose segments are
//      not 16-byte aligned are loaded by the threads instead);
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
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "device_common.cuh"
#include "internal.h"

namespace cbessfm {

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
// exp(j theta) - 1 from the same reduction, without cancellation for small theta:
// t (1 + r1) - 1 = t r1 + (t - 1) with r1 = -d^2/2 + j d (1 - d^2/6) the residual minus one.
__device__ __forceinline__ float2 rotation_psi(float th, const float2* __restrict__ tbl) {
    const float kf = rintf(th * kRotInvStep);
    float d = fmaf(-kf, kRotStepHi, th);
    d = fmaf(-kf, kRotStepLo, d);
    const float2 t = tbl[(int)kf & (kRotTable - 1)];
    const float d2 = d * d;
    const float2 tr = c_mul(t, make_float2(-0.5f * d2, d * fmaf(-0.16666666666666667f, d2, 1.0f)));
    return make_float2(tr.x + (t.x - 1.0f), tr.y + t.y);
}

// Barrier over the 2 NP/E threads (both polarizations) of one FFT group.  Groups of a warp or
// less share their warp with other groups running the same code, so a warp barrier suffices.
template <int NP, int E>
struct GroupBar {
    int id;
    __device__ __forceinline__ void operator()() const {
        if constexpr (2 * (NP / E) > 32) {
            named_bar(id, 2 * (NP / E));
        } else {
            __syncwarp();
        }
    }
};

// Sample storage in HBM (cbessfm_storage): 0 = complex64 (float4 per 4D sample), 1 = four fp16,
// 2 = four bf16.  Arithmetic is FP32 in every case; one polarization of a sample is addressed as
// element 2 n + p of a two-component array.
template <int ST>
struct Storage;
template <>
struct Storage<0> {
    using Pol = float2;
    static constexpr int kSampleBytes = 16;
    __device__ static float2 to_f32(float2 v) { return v; }
    __device__ static float2 from_f32(float2 v) { return v; }
};
template <>
struct Storage<1> {
    using Pol = __half2;
    static constexpr int kSampleBytes = 8;
    __device__ static float2 to_f32(__half2 v) { return __half22float2(v); }
    __device__ static __half2 from_f32(float2 v) { return __float22half2_rn(v); }
};
template <>
struct Storage<2> {
    using Pol = __nv_bfloat162;
    static constexpr int kSampleBytes = 8;
    __device__ static float2 to_f32(__nv_bfloat162 v) { return __bfloat1622float2(v); }
    __device__ static __nv_bfloat162 from_f32(float2 v) { return __float22bfloat162_rn(v); }
};

// Intensity rows are XOR-swizzled in 16-byte granules: float m of a row lives at
// m ^ (((m >> 5) & MASK) << 2).  The FIR's lanes read float4 windows E/2 floats apart (32 bytes
// for E = 16, 64 bytes for E = 32); the swizzle spreads every 8-lane group over all banks.
template <int E>
__device__ __forceinline__ int pswz(int m) {
    constexpr int MASK = E == 16 ? 1 : 3;
    return m ^ (((m >> 5) & MASK) << 2);
}
// (cos, sin) rows carry one spare float2 per 16 (per 32 in the packed layout) so the 8-sample
// runs of adjacent lanes do not collide on a bank.
__device__ __forceinline__ int cpad(int k) { return k + (k >> 4); }

// Rotation factors for the 8 samples k = k0 .. k0 + 7 of subband i, step s:
// theta_i[k] = sum_l sum_m w[s][i][l][m + nc] P_l[k - m]; stores (cos theta, sin theta).
// P rows carry a circular halo of H samples on each side, so no index wraps here; each chunk of
// four taps reads a 12-sample window with aligned 16-byte loads.
// Windowed FIR of 8 outputs k0 .. k0 + 7 for one output row: acc[q] = sum over rows l and taps
// of w[l][m] row_l[k0 + q - m] (rows swizzled, with circular halo).  NCH > 0 fixes the number
// of four-tap chunks at compile time: one window of 8 + 4 NCH samples per row then serves all
// chunks.  NCH = 0 handles any chunk count with one 12-sample window per chunk.
// WS: the taps `wbase` are in shared memory (plain loads) instead of global memory.
// PAD1: the last 4-tap chunk holds one zero pad tap (ntaps = 4 NCH - 1, e.g. 11): its
// multiply-adds are skipped (adding 0 * P leaves the sum unchanged bit for bit).
// `rs`: floats from one row to the next.
template <int E, int NCH, bool WS = false, bool PAD1 = false>
__device__ __forceinline__ void fir8(const ChainArgs& a, const float4* __restrict__ wbase,
                                     const float* __restrict__ rows0, int rs, int k0,
                                     float (&acc)[8], int skip_l = -1) {
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.f;
    const int m0 = a.H + a.p_off + k0 + a.nc - 3;      // row index of chunk 0's window
    for (int l = 0; l < a.n_sb; ++l) {
        if (l == skip_l) continue;                     // uniform across the subband group
        const float* pl = rows0 + l * rs;
        if constexpr (NCH > 0) {
            // Chunk c reads the 11 window samples from 16-byte granule NCH - 1 - c on, so the
            // chunks run with a sliding window of three granules: granules NCH + 1, NCH and
            // NCH - 1 for chunk 0, then one more granule (lower) per chunk.  Only 12 window
            // samples and one chunk's taps are live next to the accumulators.
            const float4* wrow = wbase + l * NCH;
            const int m_lo = m0 - 4 * (NCH - 1);
            auto granule = [&](int e) {
                return *reinterpret_cast<const float4*>(pl + pswz<E>(m_lo + 4 * e));
            };
            float4 g0 = granule(NCH - 1), g1 = granule(NCH), g2 = granule(NCH + 1);
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                if (c > 0) {                               // slide down by one granule
                    g2 = g1;
                    g1 = g0;
                    g0 = granule(NCH - 1 - c);
                }
                const float4 w4 = WS ? wrow[c] : __ldg(wrow + c);
                const float win[12] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y,
                                       g1.z, g1.w, g2.x, g2.y, g2.z, g2.w};
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float t = acc[q];
                    t = fmaf(w4.x, win[q + 3], t);   // m = -nc + 4c
                    t = fmaf(w4.y, win[q + 2], t);   // m = -nc + 4c + 1
                    t = fmaf(w4.z, win[q + 1], t);
                    if (!(PAD1 && c == NCH - 1)) t = fmaf(w4.w, win[q], t);
                    acc[q] = t;
                }
            }
        } else {
            const float4* wrow = wbase + l * a.nchunks;
            for (int c = 0; c < a.nchunks; ++c) {
                const float4 w4 = __ldg(wrow + c);
                const int m = m0 - 4 * c;
                float win[12];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const float4 v = *reinterpret_cast<const float4*>(pl + pswz<E>(m + 4 * e));
                    win[4 * e] = v.x; win[4 * e + 1] = v.y; win[4 * e + 2] = v.z; win[4 * e + 3] = v.w;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float t = acc[q];
                    t = fmaf(w4.x, win[q + 3], t);
                    t = fmaf(w4.y, win[q + 2], t);
                    t = fmaf(w4.z, win[q + 1], t);
                    t = fmaf(w4.w, win[q], t);
                    acc[q] = t;
                }
            }
        }
    }
}

// Rotation factors for the 8 samples k = k0 .. k0 + 7 of subband i, step s:
// theta_i[k] = sum_l sum_m w[s][i][l][m + nc] P_l[k - m]; stores (cos theta, sin theta).
// `s_taps` is the step's tap buffer in shared memory when a.taps_smem is set.
template <int E>
__device__ __forceinline__ void fir8_any(const ChainArgs& a, const float* __restrict__ rows0,
                                         int rs, const float4* __restrict__ s_taps, int s, int i,
                                         int k0, float (&acc)[8], int skip_l) {
    if (a.taps_smem) {
        if (a.ntaps_pad == 2 * a.nc + 2)                                     // 11 taps
            fir8<E, 3, true, true>(a, s_taps + i * a.n_sb * 3, rows0, rs, k0, acc, skip_l);
        else                                                                 // 9, 10, 12 taps
            fir8<E, 3, true>(a, s_taps + i * a.n_sb * 3, rows0, rs, k0, acc, skip_l);
    } else {
        const float4* wbase = reinterpret_cast<const float4*>(
            a.taps + (size_t)(s * a.n_sb + i) * a.n_sb * a.ntaps_pad);
        if (a.nchunks == 3) {
            fir8<E, 3>(a, wbase, rows0, rs, k0, acc, skip_l);
        } else {
            fir8<E, 0>(a, wbase, rows0, rs, k0, acc, skip_l);
        }
    }
}

// Manakov form: the rotation factors of 8 samples.  Per-polarization form (PERPOL): the
// two angles theta^x = theta + delta and theta^y = theta - delta, where theta is the Manakov
// phase and delta = (1/3) sum_{l != i} w_il (Px_l - Py_l) (the D rows follow the P rows): with
// w_il = (3/2) c_il, Eqs. (NLPR_polx/poly) weigh XPM by (2 Px + Py) / 1.5 and (Px + 2 Py) / 1.5.
// CSH: the (cos, sin) row has one spare float2 per 2^CSH.
template <int E, bool PERPOL, int CSH = 4>
__device__ __forceinline__ void nlpr_rotation8(const ChainArgs& a, const float* __restrict__ prow0,
                                               int rs, float2* __restrict__ cs_row,
                                               const float2* __restrict__ rot_tbl,
                                               const float4* __restrict__ s_taps, int s, int i,
                                               int k0) {
    float acc[8];
    fir8_any<E>(a, prow0, rs, s_taps, s, i, k0, acc, -1);
    float2* dst = cs_row + k0 + (k0 >> CSH);           // k0 % 8 = 0: no carry below
    if constexpr (PERPOL) {
        float dl[8];
        fir8_any<E>(a, prow0 + a.n_sb * a.pstride, rs, s_taps, s, i, k0, dl, i);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float d = dl[q] * (1.0f / 3.0f);
            dst[q] = make_float2(acc[q] + d, acc[q] - d);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = rotation_factor(acc[q], rot_tbl);
    }
}

// x[t] *= h(b_t) for the E slots of thread j of subband group gi, with h read from a half
// table by |b| (`hh` = one kind of ArgsChain::gvd_half).  Slot t holds lowpass bin
// kap = j + (NP/E) t, centred bin b = ci + kap (kap < NP/2) or ci + kap - NP.  A subband lies
// wholly on one side of bin 0 except the centre one (ci = 0, odd subband counts), so each half
// of the slots reads one contiguous run, ascending or descending, at immediate offsets.
template <int NP, int E>
__device__ __forceinline__ void gvd_apply(float2 (&x)[E], const float2* __restrict__ hh, int j,
                                          int ci) {
    constexpr int TPF = NP / E;
    if (ci > 0) {
        const float2* p0 = hh + (ci + j);
        const float2* p1 = hh + (ci + j - NP);
#pragma unroll
        for (int t = 0; t < E; ++t) x[t] = c_mul(x[t], __ldg((t < E / 2 ? p0 : p1) + TPF * t));
    } else if (ci < 0) {
        const float2* p0 = hh + (-ci - j);
        const float2* p1 = hh + (-ci - j + NP);
#pragma unroll
        for (int t = 0; t < E; ++t) x[t] = c_mul(x[t], __ldg((t < E / 2 ? p0 : p1) - TPF * t));
    } else {
        const float2* p0 = hh + j;
        const float2* p1 = hh + (NP - j);
#pragma unroll
        for (int t = 0; t < E; ++t)
            x[t] = c_mul(x[t], __ldg(t < E / 2 ? p0 + TPF * t : p1 - TPF * t));
    }
}

// Position of a thread in its CTA: block g of the CTA, polarization p, FFT group gi (subband in
// the steps, polyphase component at entry/exit) and index j within the group.
struct ThreadPos {
    int tid, TB, g, rem, p, gi, j;
};

template <int NP, int E = fft_slots(NP)>
__device__ __forceinline__ ThreadPos thread_pos(int n_sb) {
    constexpr int TPF = NP / E;
    ThreadPos t;
    t.tid = threadIdx.x;
    t.TB = 2 * n_sb * TPF;
    t.g = t.tid / t.TB;
    t.rem = t.tid - t.g * t.TB;
    t.p = t.rem & 1;
    const int jj = t.rem >> 1;
    t.gi = jj / TPF;
    t.j = jj - t.gi * TPF;
    return t;
}

// The whole CB-ESSFM chain on one overlap-and-save block (block `blk` of sequence `seq` of the
// job described by `a`), run by the 2 n_sb NP/E threads of CTA slot tp.g.  All threads of the
// CTA call it together (it contains block-wide barriers); `real` = false runs a zero block and
// stores nothing.  `bar_g` is the slot's mbarrier, used with phase `parity`.  Returns false if a
// bounded wait for the staging copy gave up (the caller must then stop).
//
// E = chain_slots(NP, PERPOL) register slots per thread.  With the two-pass plan (N' = 1024, 32
// slots) the block uses the packed layout (kLayoutPacked): one exchange array per subband
// group, which between the inverse FFT's loads and the forward FFT's stores of a step also
// holds the group's intensity row and then its (cos, sin) row.  That keeps a 5-subband block
// under half of an SM's shared memory, so two CTAs share an SM and fill each other's barrier
// phases.
template <int NP, int ST, bool CKPT = false, bool PERPOL = false>
__device__ __forceinline__ bool chain_block(const ChainArgs& a, unsigned char* smem,
                                            int region_bytes, uint64_t* bar_g, uint32_t parity,
                                            const float2* __restrict__ s_rot,
                                            const float2* __restrict__ s_tw,
                                            float4* __restrict__ s_taps, const ThreadPos& tp,
                                            bool real, int seq, int blk) {
    using S = Storage<ST>;
    using Pol = typename S::Pol;
    constexpr int E = chain_slots(NP, PERPOL);         // register slots per thread
    constexpr bool PACKED = chain_packed(NP, PERPOL);  // two-pass FFT, packed layout
    constexpr int SH = fft_xsh(NP, E);                 // exchange padding: one per 2^SH
    constexpr int TPF = NP / E;                        // threads per (subband, polarization)
    constexpr int XL = 2 * xpad_len_s(NP, SH);         // float2 per group exchange array
    // (cos, sin) rows: one spare per 16, so the FIR lanes' stores (16 samples apart, x and y
    // lanes 16 apart in the packed layout) and the slot reads are both conflict-free
    constexpr int CSH = 4;
    constexpr int CSL = NP + (NP >> CSH);              // float2 per (cos, sin) row
    // DEMUX/MUX twiddles: 16 slots, one table value per polyphase row times a per-slot factor;
    // 32 slots of N' = 1024, one table value per thread and per-slot factors, the rows by powers
    // (see below); N' = 2048 reads every twiddle from the table (its 64 threads per group leave
    // no registers for the products: the powers took c5 from 1.651 to 1.689 ms)
    constexpr bool kFactor = E == 16;
    constexpr bool kPowers = E == 32 && NP == 1024;
    // 32-slot plans of N' = 1024 have at most 5 subbands (2 x 5 x 32 threads fill the CTA)
    constexpr int kMaxBands32 = 5;
    const int TB = tp.TB, g = tp.g, rem = tp.rem, p = tp.p, gi = tp.gi, j = tp.j;
    unsigned char* region = smem + (size_t)g * region_bytes;
    // packed layout: the group arrays lie region_bytes / n_sb apart (at least XL float2; more when
    // long filters need longer intensity rows than XL leaves room for)
    const int XLg = PACKED ? region_bytes / (8 * a.n_sb) : XL;
    float2* const grpA = reinterpret_cast<float2*>(region) + gi * XLg;  // this group's array A
    float2* e = grpA + p;
    const GroupBar<NP, E> bar{1 + g * a.n_sb + gi};
    // Ping-pong layout: a second exchange array B.  Three-pass FFTs exchange through A then B;
    // two-pass FFTs use A for the inverse and B for the forward transform of a step.  The
    // (cos, sin) rows then live in the array the inverse FFT read last, which stays idle until
    // the forward FFT's second exchange (or the next step's inverse FFT).
    constexpr int NPASS = fft_npasses(NP, E);
    const bool pp = !PACKED && a.layout == kLayoutPingPong;
    float2* const grpB = pp ? reinterpret_cast<float2*>(region + a.exb_off) + gi * XL : grpA;
    float2* const eB = grpB + p;
    float2* const inv1 = e;
    float2* const inv2 = NPASS > 2 ? eB : e;
    float2* const fwd1 = (NPASS > 2 || !pp) ? e : eB;
    float2* const fwd2 = eB;
    // Checkpoints for the adjoint (CKPT): per block, n_st + 2 fields of N complex pairs in the
    // slot order [c][gi][idx][p]: c = 0 the spectrum after the first GVD, c = 1 + s the time
    // samples of step s before its rotation, c = n_st + 1 the spectrum after the last GVD.
    float2* ck = nullptr;
    if constexpr (CKPT) {
        ck = a.ckpt + (size_t)((long long)seq * a.n_blocks + blk) * (size_t)(a.n_st + 2) * 2 * a.N +
             (size_t)gi * NP * 2 + p;
    }
    auto save_ckpt = [&](int c, const float2 (&v)[E]) {
        if constexpr (CKPT) {
            if (real) {
                float2* d = ck + (size_t)c * 2 * a.N;
#pragma unroll
                for (int t = 0; t < E; ++t) d[2 * (j + TPF * t)] = v[t];
            }
        }
    };

    // ---------------- 1. stage the block (circular wrap) ------------------------------------
    // complex64: bulk copies (TMA) completing on an mbarrier, one per contiguous segment.
    // 8-byte samples: coalesced 8-byte loads by the block's threads (a bulk copy needs 16-byte
    // aligned starts and lengths, which arbitrary block offsets do not give).
    const Pol* stage = reinterpret_cast<const Pol*>(region);    // [N] samples as (x, y) pairs
    const long long start = ((long long)blk * a.V - a.n_ov / 2) % a.L;
    const long long pos0 = start < 0 ? start + a.L : start;
    if constexpr (ST == 0) {
        if (rem == 0) {
            if (real) {
                // earlier generic-proxy accesses to this region come before the async copy
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar_g, (uint32_t)a.N * 16u);
                long long pos = pos0;
                const float4* src = reinterpret_cast<const float4*>(a.in) + (long long)seq * a.L;
                float4* dst4 = reinterpret_cast<float4*>(region);
                int dst = 0;
                while (dst < a.N) {
                    const int len = (int)min((long long)(a.N - dst), a.L - pos);
                    bulk_copy_g2s(dst4 + dst, src + pos, (uint32_t)len * 16u, bar_g);
                    dst += len;
                    pos = 0;
                }
            } else {
                mbar_arrive(bar_g);                    // complete the phase without a copy
            }
        }
        bool ok = true;
        if (real) {
            ok = mbar_wait_bounded(bar_g, parity, a.wait_cycles);
        } else {
            float4* z = reinterpret_cast<float4*>(region);
            for (int n = rem; n < a.N; n += TB) z[n] = make_float4(0.f, 0.f, 0.f, 0.f);
            ok = mbar_wait_bounded(bar_g, parity, a.wait_cycles);
        }
        if (__syncthreads_or(!ok)) {
            if (!ok) atomicOr(a.status, kStatusTimeout);
            // let in-flight copies land before the shared memory is given up (the default
            // bound: a live copy always completes long before it)
            mbar_wait_bounded(bar_g, parity, kWaitCycles);
            return false;
        }
    } else {
        // 8-byte samples: bulk copies when every segment starts and ends on a 16-byte boundary
        // (even L and an even start), coalesced 8-byte loads otherwise.  Either way the slot's
        // mbarrier completes one phase, so the persistent kernels' phase parity stays in step.
        const bool bulk = real && ((a.L | pos0) & 1) == 0;
        const uint2* src = reinterpret_cast<const uint2*>(a.in) + (long long)seq * a.L;
        uint2* st8 = reinterpret_cast<uint2*>(region);
        if (rem == 0) {
            if (bulk) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar_g, (uint32_t)a.N * 8u);
                long long pos = pos0;
                int dst = 0;
                while (dst < a.N) {
                    const int len = (int)min((long long)(a.N - dst), a.L - pos);
                    bulk_copy_g2s(st8 + dst, src + pos, (uint32_t)len * 8u, bar_g);
                    dst += len;
                    pos = 0;
                }
            } else {
                mbar_arrive(bar_g);
            }
        }
        if (!bulk) {
            for (int n = rem; n < a.N; n += TB) {
                long long q = pos0 + n;
                q -= (q / a.L) * a.L;
                st8[n] = real ? __ldg(src + q) : make_uint2(0u, 0u);
            }
        }
        const bool ok = mbar_wait_bounded(bar_g, parity, a.wait_cycles);
        if (__syncthreads_or(!ok)) {
            if (!ok) atomicOr(a.status, kStatusTimeout);
            mbar_wait_bounded(bar_g, parity, kWaitCycles);
            return false;
        }
    }

    float2 x[E];
#pragma unroll
    for (int t = 0; t < E; ++t) x[t] = S::to_f32(stage[2 * (a.n_sb * (j + TPF * t) + gi) + p]);
    __syncthreads();

    // ---------------- 2. full-band DFT + DEMUX -------------------------------------------
    fft_regs<NP, E, false, true>(x, j, e, s_tw, bar);              // Y_r, r = gi
    bar();
#pragma unroll
    for (int t = 0; t < E; ++t) e[2 * xpad_s<SH>(j + TPF * t)] = x[t];
    __syncthreads();
    const int N = a.N;
    const int ci = -N / 2 + gi * NP + NP / 2;                      // centre bin of subband gi
    {
        // X_i[kap] = sum_r W_N^(K r) Y_r[K mod NP], K = (c_i + k') mod N; loop r outermost so that
        // only the E accumulators stay live.  With K_0 = c_i + j (slot 0), K = K_0 + (N'/E) t, less
        // N' for t >= E/2, so W_N^(K r) = W_N^(K_0 r) times a factor of (r, t) only: one table
        // load per r and thread, the factors from a small table read alike by the whole warp.
        const float2* eb = reinterpret_cast<const float2*>(region) + p;
        const float2* td = a.mix_td;                                    // [n_sb][E]
        int K0 = ci + j;
        K0 += (K0 < 0) ? N : 0;
        if constexpr (!kPowers) {
#pragma unroll
            for (int t = 0; t < E; ++t) x[t] = make_float2(0.f, 0.f);
            for (int r = 0; r < a.n_sb; ++r) {
                const float2* er = eb + r * XLg;
                const float2 w0 = __ldg(a.mix_tw + (size_t)r * N + K0);    // W_N^(K_0 r)
#pragma unroll
                for (int t = 0; t < E; ++t) {
                    const int kap = j + TPF * t;
                    int K = ci + (kap < NP / 2 ? kap : kap - NP);
                    K += (K < 0) ? N : 0;
                    const float2 w = kFactor ? c_mul(w0, __ldg(td + r * E + t))
                                             : __ldg(a.mix_tw + (size_t)r * N + K);
                    x[t] = c_add(x[t], c_mul(er[2 * xpad_s<SH>(K & (NP - 1))], w));
                }
            }
        } else {
            // N' = 1024: slot t outermost, so only the finished slots' sums stay live, and
            // W_N^(K r) as the powers of W_N^K = W_N^(K_0) times slot t's row-1 factor: one
            // table gather per thread instead of one per (r, t) (at most 4 products deep)
            const float2 wk0 =
                a.n_sb > 1 ? __ldg(a.mix_tw + (size_t)N + K0) : make_float2(1.f, 0.f);
#pragma unroll
            for (int t = 0; t < E; ++t) {
                const int kap = j + TPF * t;
                int K = ci + (kap < NP / 2 ? kap : kap - NP);
                K += (K < 0) ? N : 0;
                const int kk = 2 * xpad_s<SH>(K & (NP - 1));
                float2 acc = eb[kk];                                         // r = 0
                if (a.n_sb > 1) {
                    const float2 w1 = c_mul(wk0, __ldg(td + E + t));         // W_N^K
                    float2 w = w1;
#pragma unroll
                    for (int r = 1; r < kMaxBands32; ++r) {
                        if (r < a.n_sb) {
                            acc = c_add(acc, c_mul(eb[r * XLg + kk], w));
                            if (r + 1 < a.n_sb) w = c_mul(w, w1);
                        }
                    }
                }
                x[t] = acc;
            }
        }
    }
    __syncthreads();

    // ---------------- 3. GVD / NLPR steps --------------------------------------------------
    const int half_len = a.N / 2 + 1;
    gvd_apply<NP, E>(x, a.gvd_first, j, ci);                       // first GVD (x 1/N)
    save_ckpt(0, x);
    // intensity rows and (cos, sin) rows: see the kLayout* constants.  Packed layout: the row of
    // subband l at the start of exchange array l (rows 2 XLg floats apart), the group's (cos, sin)
    // row right after its own intensity row.
    const bool alias = !PACKED && a.layout == kLayoutAlias;
    float* const prowA = PACKED ? reinterpret_cast<float*>(region)
                                : reinterpret_cast<float*>(region + a.nlpr_off);
    const int rs = PACKED ? 2 * XLg : a.pstride;                   // floats between rows
    float2* const cs_row =
        PACKED ? reinterpret_cast<float2*>(reinterpret_cast<float*>(grpA) + a.pstride)
        : pp   ? (NPASS > 2 ? grpB : grpA)
               : reinterpret_cast<float2*>(prowA + (PERPOL ? 2 : 1) * a.n_sb * a.pstride) + gi * CSL;
    const bool group_cs_bar = pp && a.pbuf_bytes > 0;
    const int cs_base = (TPF >= (1 << CSH)) ? j + (j >> CSH) : 0;
    // packed layout: parked slots after the group's (cos, sin) row, [kParkSlots][2 TPF] float2
    float2* const park = reinterpret_cast<float2*>(reinterpret_cast<float*>(grpA) + a.pstride) +
                         CSL + (2 * j + p);
    const int n4 = a.n_sb * a.n_sb * 3;               // float4 per step's taps (12 per row)
#pragma unroll 1
    for (int s = 0; s < a.n_st; ++s) {
        // stage this step's taps (asynchronous copies, completed before the intensity barrier);
        // buffer s & 1 was last read in step s - 2, before step s - 1's intensity barrier
        float4* const taps_buf = s_taps + (s & 1) * n4;
        if (a.taps_smem) {
            const float4* src = reinterpret_cast<const float4*>(a.taps) + (size_t)s * n4;
            for (int k = threadIdx.x; k < n4; k += blockDim.x) cp_async16(taps_buf + k, src + k);
            cp_async_commit();
        }
        // subband time samples; the packed layout's single array needs the barrier before the
        // first store (the previous forward FFT's loads)
        fft_regs<NP, E, true, true>(x, j, inv1, inv2, s_tw, bar, PACKED || !pp);
        save_ckpt(1 + s, x);
        if (alias) __syncthreads();
        if constexpr (PACKED) bar();      // the group's loads are done before its row is written
        float* const prow0 =
            group_cs_bar ? reinterpret_cast<float*>(region + a.nlpr_off + (s & 1) * a.pbuf_bytes)
                         : prowA;
        {
            float* prow = prow0 + gi * rs;
            const int mb = a.H + a.p_off;
            // With E = 16 the swizzle period is 64 floats: for NP/E a multiple of 64 every slot's
            // row index is base + (NP/E) t with one XOR constant, so the stores use immediate
            // offsets.  With E = 32 and NP/E = 32 the XOR term of slot t depends on t mod 4 only
            // (see below).  Either way the halo (H <= NP/E) can only meet slots 0 and E - 1.
            constexpr bool kFlat16 = (E == 16) && (TPF % 64 == 0);
            constexpr bool kFlat32 = (E == 32) && (TPF == 32) && !PERPOL;
            const bool flat = (kFlat16 || kFlat32) && a.H <= TPF;
            const int dstride = PERPOL ? a.n_sb * a.pstride : 0;     // D rows follow P rows
            // After the shuffle both lanes of an x/y pair hold |x|^2 + |y|^2 of every slot, so
            // lane p stores the slots t with t % 2 == p: one store instruction per two slots and
            // no branch on the polarization inside the unrolled loop.  The storing lane's D value
            // (|x|^2 - |y|^2, per-polarization form) takes its sign from p.
            auto slot_pair = [&](int t2, float& pw, float& dv) {   // values of slot t2 + p
                const float own0 = fmaf(x[t2].x, x[t2].x, x[t2].y * x[t2].y);
                const float own1 = fmaf(x[t2 + 1].x, x[t2 + 1].x, x[t2 + 1].y * x[t2 + 1].y);
                const float oth0 = __shfl_xor_sync(0xffffffffu, own0, 1);
                const float oth1 = __shfl_xor_sync(0xffffffffu, own1, 1);
                pw = p == 0 ? own0 + oth0 : oth1 + own1;
                dv = p == 0 ? own0 - oth0 : oth1 - own1;
            };
            auto halo = [&](int t2, float pw, float dv) {
                // the halo can only meet slot 0 (lane 0 at t2 = 0) and slot E - 1 (lane 1)
                if (t2 == 0 && p == 0 && j < a.H) {
                    prow[pswz<E>(mb + j + NP)] = pw;
                    if constexpr (PERPOL) prow[pswz<E>(mb + j + NP) + dstride] = dv;
                }
                if (t2 == E - 2 && p == 1 && j + TPF * (E - 1) >= NP - a.H) {
                    prow[pswz<E>(mb + j + TPF * (E - 1) - NP)] = pw;
                    if constexpr (PERPOL) prow[pswz<E>(mb + j + TPF * (E - 1) - NP) + dstride] = dv;
                }
            };
            if (kFlat16 && flat) {
                float* const pbase = prow + pswz<E>(mb + j) + TPF * p;
#pragma unroll
                for (int t2 = 0; t2 < E; t2 += 2) {
                    float pw, dv;
                    slot_pair(t2, pw, dv);
                    pbase[TPF * t2] = pw;
                    if constexpr (PERPOL) pbase[TPF * t2 + dstride] = dv;
                    halo(t2, pw, dv);
                }
            } else if (kFlat32 && flat) {
                // pswz<32>(m), m = u + 32 t with u = mb + j: m >> 5 = (u >> 5) + t, and the XOR
                // term (((u >> 5) + t) & 3) << 2 touches bits 2 and 3 only, so pswz(m) =
                // (u ^ X(t mod 4)) + 32 t.  Lane p stores t = p mod 2, i.e. t mod 4 in {p, p + 2}:
                // two bases per lane (32 p folded in), immediate offsets 32 t2.
                const int u = mb + j;
                float* const pb0 = prow + (u ^ ((((u >> 5) + p) & 3) << 2)) + 32 * p;
                float* const pb2 = prow + (u ^ ((((u >> 5) + p + 2) & 3) << 2)) + 32 * p;
#pragma unroll
                for (int t2 = 0; t2 < E; t2 += 2) {
                    float pw, dv;
                    slot_pair(t2, pw, dv);
                    ((t2 & 2) ? pb2 : pb0)[32 * t2] = pw;
                    halo(t2, pw, dv);
                }
            } else {
#pragma unroll
                for (int t = 0; t < E; ++t) {
                    const float own = fmaf(x[t].x, x[t].x, x[t].y * x[t].y);
                    const float oth = __shfl_xor_sync(0xffffffffu, own, 1);
                    if (p == 0) {
                        const int n = j + TPF * t;
                        const float pw = own + oth;                  // |x|^2 + |y|^2
                        prow[pswz<E>(mb + n)] = pw;
                        // circular halo: H <= NP (ntaps <= NP/2), so one copy per side suffices
                        if (n < a.H) prow[pswz<E>(mb + n + NP)] = pw;
                        if (n >= NP - a.H) prow[pswz<E>(mb + n - NP)] = pw;
                        if constexpr (PERPOL) {
                            const float dv = own - oth;              // |x|^2 - |y|^2
                            prow[pswz<E>(mb + n) + dstride] = dv;
                            if (n < a.H) prow[pswz<E>(mb + n + NP) + dstride] = dv;
                            if (n >= NP - a.H) prow[pswz<E>(mb + n - NP) + dstride] = dv;
                        }
                    }
                }
            }
        }
        if constexpr (PACKED) {
#pragma unroll
            for (int u = 0; u < kParkSlots; ++u) park[u * 2 * TPF] = x[E - kParkSlots + u];
        }
        if (a.taps_smem) cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int h8 = 0; h8 < E / 16; ++h8)
            nlpr_rotation8<E, PERPOL, CSH>(a, prow0, rs, cs_row, s_rot, taps_buf, s, gi,
                                           E * j + (E / 2) * p + 8 * h8);
        // (cos, sin) of subband gi are written and read by group gi only.  With two intensity
        // buffers nothing else is shared before the next step's intensity barrier: a group that
        // runs ahead writes the other buffer.  The packed layout needs the block barrier: every
        // group reads every intensity row, and the next exchange overwrites them.
        if (group_cs_bar) {
            bar();
        } else {
            __syncthreads();
        }
        if constexpr (PACKED) {
#pragma unroll
            for (int u = 0; u < kParkSlots; ++u) x[E - kParkSlots + u] = park[u * 2 * TPF];
        }
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const float2 r = (TPF >= (1 << CSH)) ? cs_row[cs_base + (TPF + (TPF >> CSH)) * t]
                                                 : cs_row[cpad(j + TPF * t)];
            // per-polarization form: r holds the two angles
            float2 rot = r;
            if constexpr (PERPOL) rot = rotation_factor(p == 0 ? r.x : r.y, s_rot);
            x[t] = c_mul(x[t], rot);
        }
        if (alias) __syncthreads();
        if constexpr (PACKED) bar();      // the group's (cos, sin) reads come before its stores
        fft_regs<NP, E, false, true>(x, j, fwd1, fwd2, s_tw, bar, !PACKED && !pp);
        gvd_apply<NP, E>(x, s < a.n_st - 1 ? a.gvd_half + half_len : a.gvd_last, j, ci);
    }

    if (a.n_st > 0) save_ckpt(a.n_st + 1, x);

    // ---------------- 4. MUX + inverse full-band DFT + store --------------------------------
    __syncthreads();
    {
        float2* ex = reinterpret_cast<float2*>(region) + p;        // [2 xpad(K) + p]
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const int kap = j + TPF * t;
            int K = ci + (kap < NP / 2 ? kap : kap - NP);
            if (K < 0) K += N;
            ex[2 * xpad_s<SH>(K)] = x[t];
        }
        __syncthreads();
        // Z_r[kap] = sum_q conj(W_N^(K r)) Xi[K], K = kap + NP q (q outermost, as above), with
        // W_N^(K r) = W_N^((j + NP q) r) W_N^((N'/E) t r): one table load per q and thread
        const float2* wr = a.mix_tw + (size_t)gi * N;
        const float2* tm = a.mix_tm + gi * E;                      // [n_sb][E], row gi
        if constexpr (!kPowers) {
#pragma unroll
            for (int t = 0; t < E; ++t) x[t] = make_float2(0.f, 0.f);
            for (int q = 0; q < a.n_sb; ++q) {
                const float2 w0 = __ldg(wr + j + NP * q);
#pragma unroll
                for (int t = 0; t < E; ++t) {
                    const int K = j + TPF * t + NP * q;
                    const float2 w = kFactor ? c_mul(w0, __ldg(tm + t)) : __ldg(wr + K);
                    x[t] = c_add(x[t], c_mulc(ex[2 * xpad_s<SH>(K)], w));
                }
            }
        } else {
            // N' = 1024, as in the DEMUX: W_N^(K gi) = W_N^((j + (N'/E) t) gi) W_N^(N' q gi), the
            // first factor from one gather and slot t's factor, the second as powers of
            // W_N^(N' gi)
            const float2 a0 = __ldg(wr + j);                                  // W_N^(j gi)
            const float2 b1 = a.n_sb > 1 ? __ldg(wr + NP) : make_float2(1.f, 0.f);
#pragma unroll
            for (int t = 0; t < E; ++t) {
                const int K0t = j + TPF * t;
                float2 w = c_mul(a0, __ldg(tm + t));                         // q = 0
                float2 acc = c_mulc(ex[2 * xpad_s<SH>(K0t)], w);
#pragma unroll
                for (int q = 1; q < kMaxBands32; ++q) {
                    if (q < a.n_sb) {
                        w = c_mul(w, b1);
                        acc = c_add(acc, c_mulc(ex[2 * xpad_s<SH>(K0t + NP * q)], w));
                    }
                }
                x[t] = acc;
            }
        }
    }
    __syncthreads();
    fft_regs<NP, E, true, true>(x, j, e, s_tw, bar);               // x[n_sb n' + r], r = gi
    if constexpr (PACKED) {
        // Through shared memory in sample order, then coalesced stores: consecutive threads write
        // consecutive samples (16 bytes each in complex64, 8 bytes in 16-bit storage).
        __syncthreads();                                           // every exchange load is done
        Pol* st = reinterpret_cast<Pol*>(region);
#pragma unroll
        for (int t = 0; t < E; ++t) st[2 * (a.n_sb * (j + TPF * t) + gi) + p] = S::from_f32(x[t]);
        __syncthreads();
        if (real) {
            using Smp = typename std::conditional<ST == 0, float4, uint2>::type;
            const long long base = (long long)blk * a.V;           // first kept sample
            const int nv = (int)min((long long)a.V, a.L - base);
            const Smp* src = reinterpret_cast<const Smp*>(region) + a.n_ov / 2;
            Smp* dst = reinterpret_cast<Smp*>(a.out) + (long long)seq * a.L + base;
            for (int n = rem; n < nv; n += TB) dst[n] = src[n];
        }
    } else if (real) {
        Pol* dst = reinterpret_cast<Pol*>(a.out) + 2 * (long long)seq * a.L + p;
        const int lo = a.n_ov / 2;
        const long long base = (long long)blk * a.V - lo;
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const int n = a.n_sb * (j + TPF * t) + gi;
            if (n >= lo && n < lo + a.V) {
                const long long gidx = base + n;
                if (gidx < a.L) dst[2 * gidx] = S::from_f32(x[t]);
            }
        }
    }
    return true;
}

// One launch over `a.batch` sequences of one plan: CTA b runs blocks b G .. b G + G - 1 of the
// flattened (sequence, block) list.
template <int NP, int ST, bool PERPOL = false>
__global__ void __launch_bounds__(chain_max_threads(NP, PERPOL), chain_min_ctas(NP, PERPOL))
    cbessfm_fwd_kernel(const ChainArgs a) {
    constexpr int E = chain_slots(NP, PERPOL);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[kMaxG];
    __shared__ float2 s_rot[kRotTable];
    const ThreadPos tp = thread_pos<NP, E>(a.n_sb);
    float2* const s_tw = reinterpret_cast<float2*>(smem + (size_t)a.G * a.region_bytes);
    float4* const s_taps = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(s_tw) +
                                                     chain_tw_bytes(fft_tw_size(NP, E)));
    for (int k = tp.tid; k < kRotTable; k += blockDim.x) s_rot[k] = __ldg(a.rot_tbl + k);
    for (int k = tp.tid; k < fft_tw_size(NP, E); k += blockDim.x) s_tw[k] = __ldg(a.fft_tw + k);
    if (tp.tid < a.G) mbar_init(&bars[tp.tid], 1);
    mbar_fence_init();
    __syncthreads();
    const long long total = (long long)a.batch * a.n_blocks;
    const long long item = (long long)(a.cta0 * a.G + blockIdx.x * a.G + tp.g);  // < 2^31
    const bool real = item < total;
    const int seq = real ? (int)(item / a.n_blocks) : 0;
    const int blk = real ? (int)(item % a.n_blocks) : 0;
    chain_block<NP, ST, false, PERPOL>(a, smem, a.region_bytes, &bars[tp.g], 0u, s_rot, s_tw,
                                       s_taps, tp, real, seq, blk);
}

// Forward launch that also writes the adjoint's checkpoints (complex64 storage), for the
// Manakov or the per-polarization NLPR.
template <int NP, bool PERPOL = false>
__global__ void __launch_bounds__(chain_max_threads(NP, PERPOL), chain_min_ctas(NP, PERPOL))
    cbessfm_fwd_ckpt_kernel(const ChainArgs a) {
    constexpr int E = chain_slots(NP, PERPOL);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[kMaxG];
    __shared__ float2 s_rot[kRotTable];
    const ThreadPos tp = thread_pos<NP, E>(a.n_sb);
    float2* const s_tw = reinterpret_cast<float2*>(smem + (size_t)a.G * a.region_bytes);
    float4* const s_taps = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(s_tw) +
                                                     chain_tw_bytes(fft_tw_size(NP, E)));
    for (int k = tp.tid; k < kRotTable; k += blockDim.x) s_rot[k] = __ldg(a.rot_tbl + k);
    for (int k = tp.tid; k < fft_tw_size(NP, E); k += blockDim.x) s_tw[k] = __ldg(a.fft_tw + k);
    if (tp.tid < a.G) mbar_init(&bars[tp.tid], 1);
    mbar_fence_init();
    __syncthreads();
    const long long total = (long long)a.batch * a.n_blocks;
    const long long item = (long long)blockIdx.x * a.G + tp.g;
    const bool real = item < total;
    const int seq = real ? (int)(item / a.n_blocks) : 0;
    const int blk = real ? (int)(item % a.n_blocks) : 0;
    chain_block<NP, 0, true, PERPOL>(a, smem, a.region_bytes, &bars[tp.g], 0u, s_rot, s_tw,
                                     s_taps, tp, real, seq, blk);
}

// Persistent form for a batch of jobs that share N', the subband count and the storage type:
// CTAs claim work items (job, first block) from `counter` in the order of `items` (sorted by
// decreasing cost on the host) until the list is exhausted.  Each item runs G consecutive blocks
// of one job; per-job parameters come from `jobs`.
template <int NP, int ST, bool PERPOL = false>
__global__ void __launch_bounds__(chain_max_threads(NP, PERPOL), chain_min_ctas(NP, PERPOL))
    cbessfm_fwd_persistent_kernel(const ChainArgs* __restrict__ jobs,
                                  const int2* __restrict__ items, int n_items,
                                  unsigned int* __restrict__ counter, int n_sb, int G,
                                  int region_bytes) {
    constexpr int E = chain_slots(NP, PERPOL);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[kMaxG];
    __shared__ float2 s_rot[kRotTable];
    __shared__ ChainArgs s_job;
    __shared__ int s_item;
    const ThreadPos tp = thread_pos<NP, E>(n_sb);
    float2* const s_tw = reinterpret_cast<float2*>(smem + (size_t)G * region_bytes);
    float4* const s_taps = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(s_tw) +
                                                     chain_tw_bytes(fft_tw_size(NP, E)));
    {   // every job of the launch has this N' and form, so any job's twiddle table will do
        const float2* tw = jobs[items[0].x].fft_tw;
        for (int k = tp.tid; k < fft_tw_size(NP, E); k += blockDim.x) s_tw[k] = __ldg(tw + k);
    }
    if (tp.tid < G) mbar_init(&bars[tp.tid], 1);
    mbar_fence_init();
    int rot_of = -1;                               // job whose rotation table is in s_rot
    for (uint32_t it = 0;; ++it) {
        if (tp.tid == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;
        const int2 w = items[item];
        for (int k = tp.tid; k < (int)(sizeof(ChainArgs) / sizeof(int)); k += blockDim.x)
            reinterpret_cast<int*>(&s_job)[k] = reinterpret_cast<const int*>(jobs + w.x)[k];
        __syncthreads();
        if (rot_of != w.x) {                           // uniform across the CTA
            for (int k = tp.tid; k < kRotTable; k += blockDim.x) s_rot[k] = __ldg(s_job.rot_tbl + k);
            rot_of = w.x;
            __syncthreads();
        }
        const int blk = w.y + tp.g;
        const bool real = blk < s_job.n_blocks;
        if (!chain_block<NP, ST, false, PERPOL>(s_job, smem, region_bytes, &bars[tp.g], it & 1u,
                                                s_rot, s_tw, s_taps, tp, real, 0,
                                                real ? blk : 0))
            return;
        __syncthreads();                               // s_item / s_job reuse
    }
}

// Launch helpers, instantiated per (NP, storage) in the fwd_inst_*.cu translation units.
template <int NP, int ST>
cudaError_t fwd_launch(const ChainArgs& a, int threads, cudaStream_t stream) {
    const long long total = (long long)a.batch * a.n_blocks;
    const long long ctas = (total + a.G - 1) / a.G;
    long long grid = ctas - a.cta0;
    if (a.n_ctas > 0 && a.n_ctas < grid) grid = a.n_ctas;
    if (grid <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.G * a.region_bytes + a.tbl_bytes;
    if constexpr (ST == 0) {
        if (a.per_pol) {
            cbessfm_fwd_kernel<NP, 0, true><<<(unsigned)grid, threads, smem, stream>>>(a);
            return cudaGetLastError();
        }
    }
    cbessfm_fwd_kernel<NP, ST><<<(unsigned)grid, threads, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int NP, int ST>
cudaError_t fwd_prepare(int smem_bytes) {
    cudaError_t e = cudaFuncSetAttribute(cbessfm_fwd_kernel<NP, ST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    // the packed layout runs two CTAs per SM: ask for the whole shared-memory carve-out
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cbessfm_fwd_kernel<NP, ST>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(cbessfm_fwd_persistent_kernel<NP, ST>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cbessfm_fwd_persistent_kernel<NP, ST>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if constexpr (ST == 0) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(cbessfm_fwd_kernel<NP, 0, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(cbessfm_fwd_persistent_kernel<NP, 0, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    }
    return e;
}

template <int NP, int ST>
cudaError_t fwd_persistent_launch(const ChainArgs* jobs, const int2* items, int n_items,
                                  unsigned int* counter, int n_sb, int G, int region_bytes,
                                  int tbl_bytes, int per_pol, int threads, int grid,
                                  cudaStream_t stream) {
    if (n_items <= 0 || grid <= 0) return cudaSuccess;
    const size_t smem = (size_t)G * region_bytes + tbl_bytes;
    if constexpr (ST == 0) {
        if (per_pol) {
            cbessfm_fwd_persistent_kernel<NP, 0, true><<<grid, threads, smem, stream>>>(
                jobs, items, n_items, counter, n_sb, G, region_bytes);
            return cudaGetLastError();
        }
    }
    cbessfm_fwd_persistent_kernel<NP, ST><<<grid, threads, smem, stream>>>(
        jobs, items, n_items, counter, n_sb, G, region_bytes);
    return cudaGetLastError();
}

template <int NP, int ST>
cudaError_t fwd_persistent_occupancy(int threads, int smem_bytes, int* ctas_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        ctas_per_sm, cbessfm_fwd_persistent_kernel<NP, ST>, threads, smem_bytes);
}

}  // namespace cbessfm
