// device_common.cuh -- device building blocks of the CB-ESSFM kernels (sm_103a).
//
//  * complex float2 arithmetic,
//  * radix-2/4/8/16/32 DFT butterflies on register slots,
//  * a Stockham FFT of size NP (16..2048) executed by NP/E threads that each own E (16 or 32)
//    register slots of one polarization, exchanging through padded shared memory between passes
//    (the x and y threads of the same slots sit in adjacent lanes and share the exchange array),
//  * mbarrier + bulk-copy (TMA) helpers with bounded waits.
//
// Slot convention (shared by the forward and adjoint kernels): thread j of an FFT group holds,
// in slot t (0..E-1), element j + (NP/E) * t of the sequence, both on the time side and on the
// frequency side.  The Stockham passes are arranged (radix 16 first and last) so that the first
// pass reads exactly these elements and the last pass produces exactly these elements; the
// pointwise steps (dispersion, rotation) therefore run on registers with no reordering.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cbessfm {

// ------------------------------------------------------------------------------------------
// complex helpers
// ------------------------------------------------------------------------------------------
// Complex sums as packed two-lane FP32 adds (sm_100 and later): one instruction for both
// components, each rounded as a scalar add.
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) {
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
// multiplication by the twiddle w of a forward (INV = false) or inverse (conj(w)) transform
template <bool INV>
__device__ __forceinline__ float2 c_tw(float2 a, float2 w) { return INV ? c_mulc(a, w) : c_mul(a, w); }
// multiplication by -i (forward) or +i (inverse): the quarter-turn twiddle
template <bool INV>
__device__ __forceinline__ float2 c_quarter(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

constexpr float kSqrtHalf = 0.70710678118654752440f;
// (cos, sin) pairs of the DFT kernels are rounded to keep |w| = 1 as closely as float spacing
// allows (not each to its nearest float): every step of the chain applies the same constants, so
// a norm error adds up coherently over the steps, while their phase errors largely cancel
// between the forward and inverse transforms.  cos(pi/8) is one float step above its nearest
// float, sin(pi/8) two below.
constexpr float kCos8 = 0x1.d906bep-1f;    // cos(pi/8) ~ 0.923879564
constexpr float kSin8 = 0x1.87de26p-2f;    // sin(pi/8) ~ 0.382683367

// a * exp(-+ j 2 pi m / 16) for the constant exponents a radix-16 butterfly needs
template <int M, bool INV>
__device__ __forceinline__ float2 tw16(float2 a) {
    constexpr int m = M & 15;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (m == 4) {
        return c_quarter<INV>(a);
    } else if constexpr (m == 8) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (m == 2) {               // (1 -+ j) / sqrt2
        return INV ? make_float2((a.x - a.y) * kSqrtHalf, (a.x + a.y) * kSqrtHalf)
                   : make_float2((a.x + a.y) * kSqrtHalf, (a.y - a.x) * kSqrtHalf);
    } else if constexpr (m == 6) {               // (-1 -+ j) / sqrt2
        return INV ? make_float2(-(a.x + a.y) * kSqrtHalf, (a.x - a.y) * kSqrtHalf)
                   : make_float2((a.y - a.x) * kSqrtHalf, -(a.x + a.y) * kSqrtHalf);
    } else {
        // general exponent: cos/sin of 2 pi m / 16 from the two octant constants
        constexpr float cs[16] = {1.f, kCos8, kSqrtHalf, kSin8, 0.f, -kSin8, -kSqrtHalf, -kCos8,
                                  -1.f, -kCos8, -kSqrtHalf, -kSin8, 0.f, kSin8, kSqrtHalf, kCos8};
        constexpr float sn[16] = {0.f, kSin8, kSqrtHalf, kCos8, 1.f, kCos8, kSqrtHalf, kSin8,
                                  0.f, -kSin8, -kSqrtHalf, -kCos8, -1.f, -kCos8, -kSqrtHalf, -kSin8};
        return c_tw<INV>(a, make_float2(cs[m], -sn[m]));
    }
}

// ------------------------------------------------------------------------------------------
// small DFTs (natural order in, natural order out)
// ------------------------------------------------------------------------------------------
template <bool INV>
__device__ __forceinline__ void dft2(float2& a0, float2& a1) {
    const float2 t = a0;
    a0 = c_add(t, a1);
    a1 = c_sub(t, a1);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    const float2 s02 = c_add(a0, a2), d02 = c_sub(a0, a2);
    const float2 s13 = c_add(a1, a3), d13 = c_sub(a1, a3);
    a0 = c_add(s02, s13);
    a2 = c_sub(s02, s13);
    // d02 +- q(d13) with q = -i (forward) or +i (inverse), by components: the swapped pair
    // q(d13) never has to be formed
    if constexpr (INV) {
        a1 = make_float2(d02.x - d13.y, d02.y + d13.x);
        a3 = make_float2(d02.x + d13.y, d02.y - d13.x);
    } else {
        a1 = make_float2(d02.x + d13.y, d02.y - d13.x);
        a3 = make_float2(d02.x - d13.y, d02.y + d13.x);
    }
}

template <bool INV>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
    dft4<INV>(v[0], v[2], v[4], v[6]);           // even samples -> E_k at v[0], v[2], v[4], v[6]
    dft4<INV>(v[1], v[3], v[5], v[7]);           // odd samples  -> O_k at v[1], v[3], v[5], v[7]
    const float2 o1 = tw16<2, INV>(v[3]), o2 = tw16<4, INV>(v[5]), o3 = tw16<6, INV>(v[7]);
    float2 x[8];
    x[0] = c_add(v[0], v[1]); x[4] = c_sub(v[0], v[1]);
    x[1] = c_add(v[2], o1);   x[5] = c_sub(v[2], o1);
    x[2] = c_add(v[4], o2);   x[6] = c_sub(v[4], o2);
    x[3] = c_add(v[6], o3);   x[7] = c_sub(v[6], o3);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = x[k];
}

// 16-point DFT as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
    dft4<INV>(v[0], v[4], v[8], v[12]);
    dft4<INV>(v[1], v[5], v[9], v[13]);
    dft4<INV>(v[2], v[6], v[10], v[14]);
    dft4<INV>(v[3], v[7], v[11], v[15]);
    // v[n2 + 4 k1] *= W16^(n2 k1)
    v[5] = tw16<1, INV>(v[5]);  v[9] = tw16<2, INV>(v[9]);   v[13] = tw16<3, INV>(v[13]);
    v[6] = tw16<2, INV>(v[6]);  v[10] = tw16<4, INV>(v[10]); v[14] = tw16<6, INV>(v[14]);
    v[7] = tw16<3, INV>(v[7]);  v[11] = tw16<6, INV>(v[11]); v[15] = tw16<9, INV>(v[15]);
    dft4<INV>(v[0], v[1], v[2], v[3]);
    dft4<INV>(v[4], v[5], v[6], v[7]);
    dft4<INV>(v[8], v[9], v[10], v[11]);
    dft4<INV>(v[12], v[13], v[14], v[15]);
    // X[k1 + 4 k2] sits at v[4 k1 + k2]: transpose the 4 x 4 index
    float2 x[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = x[k];
}

// a * exp(-+ j 2 pi m / 32): even exponents are those of the 16-point twiddle; odd ones take
// cos and sin of (2 m' + 1) pi / 16 from two pairs of constants
// norm-preserving pairs as kCos8 / kSin8: sin(pi/16) three float steps above its nearest float
constexpr float kCos16 = 0x1.f6297cp-1f;   // cos(pi/16) ~ 0.980785251
constexpr float kSin16 = 0x1.8f8b90p-3f;   // sin(pi/16) ~ 0.195090413
constexpr float kCos316 = 0x1.a9b662p-1f;  // cos(3 pi/16) ~ 0.831469595
constexpr float kSin316 = 0x1.1c73b4p-1f;  // sin(3 pi/16) ~ 0.555570245
template <int M, bool INV>
__device__ __forceinline__ float2 tw32(float2 a) {
    constexpr int m = M & 31;
    if constexpr ((m & 1) == 0) {
        return tw16<m / 2, INV>(a);
    } else {
        // cos and sin of 2 pi m / 32 for odd m
        constexpr float cs[16] = {kCos16, kCos316, kSin316, kSin16, -kSin16, -kSin316, -kCos316,
                                  -kCos16, -kCos16, -kCos316, -kSin316, -kSin16, kSin16, kSin316,
                                  kCos316, kCos16};
        constexpr float sn[16] = {kSin16, kSin316, kCos316, kCos16, kCos16, kCos316, kSin316,
                                  kSin16, -kSin16, -kSin316, -kCos316, -kCos16, -kCos16, -kCos316,
                                  -kSin316, -kSin16};
        return c_tw<INV>(a, make_float2(cs[m / 2], -sn[m / 2]));
    }
}

// 32-point DFT by decimation in time: the 16-point DFTs E and O of the even and odd samples,
// then X[k] = E[k] + W32^k O[k] and X[k + 16] = E[k] - W32^k O[k].
template <bool INV>
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
    float2 ev[16], od[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        ev[k] = v[2 * k];
        od[k] = v[2 * k + 1];
    }
    dft16<INV>(ev);
    dft16<INV>(od);
    float2 o[16];
    o[0] = od[0];           o[1] = tw32<1, INV>(od[1]);   o[2] = tw32<2, INV>(od[2]);
    o[3] = tw32<3, INV>(od[3]);   o[4] = tw32<4, INV>(od[4]);   o[5] = tw32<5, INV>(od[5]);
    o[6] = tw32<6, INV>(od[6]);   o[7] = tw32<7, INV>(od[7]);   o[8] = tw32<8, INV>(od[8]);
    o[9] = tw32<9, INV>(od[9]);   o[10] = tw32<10, INV>(od[10]); o[11] = tw32<11, INV>(od[11]);
    o[12] = tw32<12, INV>(od[12]); o[13] = tw32<13, INV>(od[13]); o[14] = tw32<14, INV>(od[14]);
    o[15] = tw32<15, INV>(od[15]);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        v[k] = c_add(ev[k], o[k]);
        v[k + 16] = c_sub(ev[k], o[k]);
    }
}

// radix-R DFT on slots s, s + S, ..., s + (R-1) S of an E-slot array (R * S == E)
template <int R, int S, bool INV, int E>
__device__ __forceinline__ void dft_slots(float2 (&a)[E], const int s) {
    if constexpr (R == 32) {
        static_assert(S == 1 && E == 32, "a radix-32 pass uses all 32 slots of a thread");
        dft32<INV>(a);
    } else if constexpr (R == 16) {
        if constexpr (S == 1) {
            dft16<INV>(a);
        } else {
            float2 v[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = a[s + r * S];
            dft16<INV>(v);
#pragma unroll
            for (int r = 0; r < 16; ++r) a[s + r * S] = v[r];
        }
    } else if constexpr (R == 8) {
        float2 v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = a[s + r * S];
        dft8<INV>(v);
#pragma unroll
        for (int r = 0; r < 8; ++r) a[s + r * S] = v[r];
    } else if constexpr (R == 4) {
        dft4<INV>(a[s], a[s + S], a[s + 2 * S], a[s + 3 * S]);
    } else if constexpr (R == 2) {
        dft2<INV>(a[s], a[s + S]);
    }
}

// ------------------------------------------------------------------------------------------
// FFT pass plans, keyed by the transform size NP and the register slots per thread E
// ------------------------------------------------------------------------------------------
// Three-stage plan (any E): 16 | NP/16 (NP <= 256) or 16 | NP/256 | 16 (NP <= 4096): two
// exchanges for NP > 256.  Two-pass plan (E = 32, NP = 1024): 32 | 32, one exchange, each pass
// a 32-point DFT on the thread's 32 slots.
__host__ __device__ constexpr bool fft_two32(int np, int e) { return e == 32 && np == 1024; }
__host__ __device__ constexpr int fft_npasses(int np, int e) {
    return fft_two32(np, e) ? 2 : (np <= 16 ? 1 : (np <= 256 ? 2 : 3));
}
__host__ __device__ constexpr int fft_radix(int np, int e, int p) {
    return fft_two32(np, e) ? 32
                            : (p == 0 ? 16 : (np <= 256 ? np / 16 : (p == 1 ? np / 256 : 16)));
}
__host__ __device__ constexpr int fft_ns(int np, int e, int p) {
    int ns = 1;
    for (int q = 0; q < p; ++q) ns *= fft_radix(np, e, q);
    return ns;
}
// twiddle table of pass p >= 1: [(r - 1) * Ns + a] = W_{Ns R}^(a r), r in [1, R), a in [0, Ns)
__host__ __device__ constexpr int fft_tw_offset(int np, int e, int p) {
    int o = 0;
    for (int q = 1; q < p; ++q) o += (fft_radix(np, e, q) - 1) * fft_ns(np, e, q);
    return o;
}
__host__ __device__ constexpr int fft_tw_size(int np, int e) {
    return fft_tw_offset(np, e, fft_npasses(np, e));
}
// Exchange-array padding: one spare complex per 2^sh.  The three-stage plan's strided pass
// writes are conflict-free with one per 16, the two-pass plan's (lanes 32 elements apart) with
// one per 32.
__host__ __device__ constexpr int fft_xsh(int np, int e) { return fft_two32(np, e) ? 5 : 4; }

// Slots per thread of the adjoint and of the per-polarization forward chain: 32 for 2048 points
// (so 5 subbands x 2 polarizations fit in 640 threads), 16 otherwise.
__host__ __device__ constexpr int fft_slots(int np) { return np >= 2048 ? 32 : 16; }
// Slots per thread of the Manakov forward chain: 32 for 1024 points as well (the two-pass plan,
// 320 threads for 5 subbands, two CTAs per SM), otherwise as fft_slots.
__host__ __device__ constexpr int fwd_slots(int np) { return np >= 1024 ? 32 : 16; }

// The forward chain kernels: register slots per thread of the Manakov (per_pol = false) or
// per-polarization form, whether the block uses the packed layout of the two-pass plan, and the
// launch shape the kernels are compiled for (threads per CTA at most, CTAs per SM at least).
__host__ __device__ constexpr int chain_slots(int np, bool per_pol) {
    return per_pol ? fft_slots(np) : fwd_slots(np);
}
__host__ __device__ constexpr bool chain_packed(int np, bool per_pol) {
    return fft_two32(np, chain_slots(np, per_pol));
}
__host__ __device__ constexpr int chain_max_threads(int np, bool per_pol) {
    return chain_packed(np, per_pol) ? 320 : 640;
}
__host__ __device__ constexpr int chain_min_ctas(int np, bool per_pol) {
    return chain_packed(np, per_pol) ? 2 : 1;
}

// the plans of fft_slots(np)
__host__ __device__ constexpr int fft_npasses(int np) { return fft_npasses(np, fft_slots(np)); }
__host__ __device__ constexpr int fft_radix(int np, int p) { return fft_radix(np, fft_slots(np), p); }
__host__ __device__ constexpr int fft_ns(int np, int p) { return fft_ns(np, fft_slots(np), p); }
__host__ __device__ constexpr int fft_tw_offset(int np, int p) {
    return fft_tw_offset(np, fft_slots(np), p);
}
__host__ __device__ constexpr int fft_tw_size(int np) { return fft_tw_size(np, fft_slots(np)); }

// padded shared-memory index: one spare complex per 16 keeps strided pass writes conflict-free
__device__ __forceinline__ int xpad(int n) { return n + (n >> 4); }
__host__ __device__ constexpr int xpad_len(int n) { return n + (n >> 4); }
// the same with one spare complex per 2^SH
template <int SH>
__device__ __forceinline__ int xpad_s(int n) { return n + (n >> SH); }
__host__ __device__ constexpr int xpad_len_s(int n, int sh) { return n + (n >> sh); }

// Butterflies of pass P: thread j handles butterflies b = j + (NP/E) s, s in [0, E/R); element r
// of butterfly s lives in slot s + r (E/R).  The first pass therefore reads, and the last pass
// writes, exactly the elements j + (NP/E) t of the slot convention.
// TWS: the twiddle table `tw` is in shared memory (plain loads) instead of global memory.
template <int NP, int E, int P, bool INV, bool TWS = false>
__device__ __forceinline__ void fft_pass(float2 (&x)[E], const int j,
                                         const float2* __restrict__ tw) {
    constexpr int R = fft_radix(NP, E, P), NS = fft_ns(NP, E, P), S = E / R;
    constexpr int TW = fft_tw_offset(NP, E, P);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if constexpr (P > 0) {
            const int a = (j + (NP / E) * s) & (NS - 1);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2* w = tw + TW + (r - 1) * NS + a;
                float2 wv;
                if constexpr (TWS) {
                    // volatile: keeps each load at its use (plain loads of the table let the
                    // compiler keep twiddles live across passes, at the cost of spills)
                    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                                 : "=f"(wv.x), "=f"(wv.y)
                                 : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(w))));
                } else {
                    wv = __ldg(w);
                }
                x[s + r * S] = c_tw<INV>(x[s + r * S], wv);
            }
        }
        dft_slots<R, S, INV, E>(x, s);
    }
}

// Exchange arrays interleave the two polarizations: element n of polarization p is at
// e[2 xpad(n) + p], so the x/y partner threads (adjacent lanes) touch adjacent words; xpad has
// one spare complex per 2^SH (SH = fft_xsh).  When NP/E >= 2^SH every element index of a pass
// is f(j) + c with c a compile-time constant and f(j) or c a multiple of 2^SH, so
// xpad(f(j) + c) = xpad(f(j)) + c + c/2^SH and each access is one base register plus an
// immediate offset.
template <int NP, int E, int P>
__device__ __forceinline__ void fft_store(float2* e, const float2 (&x)[E], const int j) {
    constexpr int R = fft_radix(NP, E, P), NS = fft_ns(NP, E, P), S = E / R;
    constexpr int SH = fft_xsh(NP, E);
    if constexpr (NP / E >= (1 << SH)) {
        // b = j + (NP/E) s;  n = (b / NS) NS R + (b mod NS) + q NS
        const int f = (j / NS) * NS * R + (j & (NS - 1));
        float2* eb = e + 2 * xpad_s<SH>(f);
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int c = ((NP / E) * s / NS) * NS * R + q * NS;
                eb[2 * (c + (c >> SH))] = x[s + q * S];
            }
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int b = j + (NP / E) * s;
            const int base = (b / NS) * NS * R + (b & (NS - 1));
#pragma unroll
            for (int q = 0; q < R; ++q) e[2 * xpad_s<SH>(base + q * NS)] = x[s + q * S];
        }
    }
}

template <int NP, int E, int P>
__device__ __forceinline__ void fft_load(const float2* e, float2 (&x)[E], const int j) {
    constexpr int R = fft_radix(NP, E, P), S = E / R;
    constexpr int SH = fft_xsh(NP, E);
    if constexpr (NP / E >= (1 << SH)) {
        const float2* eb = e + 2 * xpad_s<SH>(j);
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int c = (NP / E) * s + r * (NP / R);               // multiple of 2^SH
                x[s + r * S] = eb[2 * (c + (c >> SH))];
            }
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int b = j + (NP / E) * s;
#pragma unroll
            for (int r = 0; r < R; ++r) x[s + r * S] = e[2 * xpad_s<SH>(b + r * (NP / R))];
        }
    }
}

// Unnormalized DFT of size NP of one polarization held by the NP/E threads of one group.
// INV = false: X[k] = sum_n x[n] exp(-j 2 pi k n / NP);  INV = true: exp(+j ...).
// `bar` synchronizes the group (both polarizations); `e1` and `e2` are this thread's polarization
// views (base + p) of the group's interleaved exchange arrays for the first and the second
// exchange.  `war` adds the barrier before each store that protects the previous loads of the
// same array; a caller may drop it when every earlier load of that array is already ordered
// before the store by another barrier (ping-pong arrays, see the forward chain).
template <int NP, int E, bool INV, bool TWS = false, class Bar>
__device__ __forceinline__ void fft_regs(float2 (&x)[E], const int j, float2* e1, float2* e2,
                                         const float2* __restrict__ tw, Bar bar, bool war) {
    constexpr int NPASS = fft_npasses(NP, E);
    fft_pass<NP, E, 0, INV, TWS>(x, j, tw);
    if constexpr (NPASS > 1) {
        if (war) bar();
        fft_store<NP, E, 0>(e1, x, j);
        bar();
        fft_load<NP, E, 1>(e1, x, j);
        fft_pass<NP, E, 1, INV, TWS>(x, j, tw);
    }
    if constexpr (NPASS > 2) {
        if (war) bar();
        fft_store<NP, E, 1>(e2, x, j);
        bar();
        fft_load<NP, E, 2>(e2, x, j);
        fft_pass<NP, E, 2, INV, TWS>(x, j, tw);
    }
}
// The same transform through one exchange array with every barrier.
template <int NP, int E, bool INV, bool TWS = false, class Bar>
__device__ __forceinline__ void fft_regs(float2 (&x)[E], const int j, float2* e,
                                         const float2* __restrict__ tw, Bar bar) {
    fft_regs<NP, E, INV, TWS>(x, j, e, e, tw, bar, true);
}

// ------------------------------------------------------------------------------------------
// mbarrier + bulk copy (TMA, non-tensor form) with bounded waits
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for phase `parity` of `bar`, giving up after roughly `max_cycles` SM cycles.  A limit of
// 0 or less is a single non-blocking test (try_wait itself may suspend the thread for a while).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long max_cycles) {
    if (max_cycles <= 0) return mbar_test_wait(bar, parity);
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > max_cycles) return false;
    }
    return true;
}
// global -> shared bulk copy completing on `bar` (addresses 16-byte aligned, bytes % 16 == 0)
__device__ __forceinline__ void bulk_copy_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// order earlier generic-proxy shared-memory accesses before later async-proxy (TMA) ones
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16-byte asynchronous global -> shared copy (completed by cp_async_wait_all in this thread)
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src_gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)),
                 "l"(src_gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// named barrier over `count` threads (a multiple of 32)
__device__ __forceinline__ void named_bar(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// device status bits
constexpr unsigned int kStatusTimeout = 1u;

}  // namespace cbessfm
