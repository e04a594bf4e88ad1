// api.cu -- C-ABI entry points: plan construction (FP64 tables), validation, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "device_common.cuh"
#include "abi_guard.h"
#include "block_count.h"
#include "internal.h"
#include "trace.h"
#include "storage_convert.h"


namespace cbessfm {
namespace {

thread_local char g_last_error[512];   // fixed size: reporting an error never allocates

}  // namespace

cbessfm_status fail(cbessfm_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

cbessfm_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? CBESSFM_ERR_OOM : CBESSFM_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

void clear_error() { g_last_error[0] = '\0'; }
const char* last_error_text() { return g_last_error; }

namespace {


bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// exp(j ang) rounded to a float pair whose norm stays as close to 1 as float spacing allows.
// The nearest floats to (cos, sin) can miss |w| = 1 by 6e-8; the chain multiplies by the same
// table entries in every step, so that gain error adds up coherently over the steps (an FP32
// emulation of a 15-step chain of 1024-point transforms: rel-L2 7.3e-6 with nearest-rounded
// constants, 2.8e-6 with norm-preserving ones).  Candidates within 3 float steps of the nearest
// pair; the norm error is weighed against one tenth of the phase error.
float2 unit_f32(double ang) {
    const double c = std::cos(ang), s = std::sin(ang);
    const float c0 = (float)c, s0 = (float)s;
    float bc = c0, bs = s0;
    double best = -1.0;
    float ci = c0;
    for (int i = 0; i < 3; ++i) ci = std::nextafter(ci, -2.0f);
    for (int i = -3; i <= 3; ++i, ci = std::nextafter(ci, 2.0f)) {
        float sj = s0;
        for (int j = 0; j < 3; ++j) sj = std::nextafter(sj, -2.0f);
        for (int j = -3; j <= 3; ++j, sj = std::nextafter(sj, 2.0f)) {
            const double dc = ci, ds = sj;
            const double norm_err = std::fabs(dc * dc + ds * ds - 1.0);
            const double phase_err = std::fabs(ds * c - dc * s);   // sin of the angle error
            const double key = norm_err + 0.1 * phase_err;
            if (best < 0.0 || key < best) {
                best = key;
                bc = ci;
                bs = sj;
            }
        }
    }
    return make_float2(bc, bs);
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

void free_plan(PlanImpl& p) {
    cudaFree(p.d_gvd);
    cudaFree(p.d_gvd_half);
    cudaFree(p.d_mix_tw);
    if (p.d_fft_tw_cl != p.d_fft_tw) cudaFree(p.d_fft_tw_cl);
    cudaFree(p.d_fft_tw);
    cudaFree(p.d_taps);
    cudaFree(p.d_rot);
    cudaFree(p.d_taps_t);
    cudaFree(p.d_status);
    p.d_gvd = nullptr;
    p.d_gvd_half = nullptr;
    p.d_mix_tw = nullptr;
    p.d_fft_tw = nullptr;
    p.d_fft_tw_cl = nullptr;
    p.d_taps = nullptr;
    p.d_rot = nullptr;
    p.d_taps_t = nullptr;
    p.d_status = nullptr;
}

// [n_st][n_sb][n_sb][ntaps] -> [n_st][n_sb][n_sb][ntaps_pad] with zero padding at the end
std::vector<float> pack_taps(const PlanImpl& p, const float* coeffs) {
    const size_t rows = (size_t)p.n_st * p.n_sb * p.n_sb;
    std::vector<float> out(rows * p.ntaps_pad, 0.f);
    for (size_t r = 0; r < rows; ++r)
        for (int m = 0; m < p.ntaps; ++m) out[r * p.ntaps_pad + m] = coeffs[r * p.ntaps + m];
    return out;
}

}  // namespace

int choose_blocks_per_cta(int tb, int region_bytes, int tpf, int bands, int extra_bytes,
                          int max_threads, int min_ctas) {
    // about 256 threads, whole warps (G * tb multiple of 32), shared memory (a share of the SM
    // when the kernel is built for several CTAs per SM) and named-barrier ids
    // (1 + g * bands + i <= 15 when groups span more than one warp)
    int granule = 1;
    while ((granule * tb) % 32 != 0) granule *= 2;
    int G = std::max(granule, (256 / tb) / granule * granule);
    G = std::min(G, kMaxG);
    const int smem_cap = min_ctas > 1 ? (228 * 1024) / min_ctas - 1024 - 4096 : kMaxDynSmem;
    auto fits = [&](int g) {
        return g * region_bytes + extra_bytes <= smem_cap && g * tb <= max_threads &&
               !(2 * tpf > 32 && g * bands > 15);
    };
    while (G > granule && !fits(G)) G -= granule;
    return fits(G) ? G : 0;
}

// OLS blocks resident per SM for G blocks of `tb` threads per CTA and `region` bytes each: the
// forward kernels are compiled for `max_threads` threads and `min_ctas` CTAs per SM, which sets
// their registers per thread (96 for 640 x 1 and 320 x 2), so registers bound the CTAs too.
int resident_blocks(int G, int tb, int region, int tables, int max_threads, int min_ctas) {
    if (G < 1) return 0;
    const int smem_per_cta = G * region + tables + 4096 + 1024;  // + static and reserved
    const int by_smem = (228 * 1024) / smem_per_cta;
    const int regs = std::min(255, 65536 / (max_threads * min_ctas)) / 8 * 8;
    const int by_regs = 65536 / (G * tb * regs);
    return G * std::min(by_smem, by_regs);
}

bool choose_layout(PlanImpl& p, int tb, int tpf) {
    const int bands = p.n_sb, n_fft = p.n_fft;
    const bool per_pol = p.per_pol != 0;
    const int E = chain_slots(n_fft, per_pol);
    const int max_threads = chain_max_threads(n_fft, per_pol);
    const int min_ctas = chain_min_ctas(n_fft, per_pol);
    // per-CTA tables: FFT twiddles always, one step's taps (double-buffered) for 9 to 12 taps
    const int tw = chain_tw_bytes(fft_tw_size(n_fft, E));
    const int tw_taps = tw + (p.nchunks == 3 ? chain_taps_bytes(bands) : 0);
    if (chain_packed(n_fft, per_pol)) {
        // one exchange array per group; its intensity row, (cos, sin) row (one spare per 16) and
        // the parked slots fit inside it
        // the array grows past its exchange size when long filters need longer intensity rows
        const int rows_bytes = 4 * p.pstride + 8 * (n_fft + n_fft / 16) + 8 * kParkSlots * 2 * tpf;
        const int xl_bytes = round_up(std::max(16 * xpad_len_s(n_fft, fft_xsh(n_fft, E)), rows_bytes), 128);
        const int region = round_up(bands * xl_bytes, 128);
        int tbl = tw_taps;
        int G = choose_blocks_per_cta(tb, region, tpf, bands, tbl, max_threads, min_ctas);
        if (G < 1 && tbl != tw) {
            tbl = tw;
            G = choose_blocks_per_cta(tb, region, tpf, bands, tbl, max_threads, min_ctas);
        }
        if (G < 1) return false;
        p.tbl_bytes = tbl;
        p.taps_smem = tbl != tw ? 1 : 0;
        p.layout = kLayoutPacked;
        p.region_bytes = region;
        p.nlpr_off = 0;
        p.exb_off = 0;
        p.pbuf_bytes = 0;
        p.G = G;
        p.threads = G * tb;
        return true;
    }
    const int exch = round_up(std::max(16 * p.N, 16 * xpad_len(p.N)), 128);  // staging fits too
    const int prow = round_up(4 * bands * p.pstride, 128);
    const int csr = round_up(8 * bands * xpad_len(n_fft), 128);
    struct Cand {
        int layout, region, nlpr_off, exb_off, pbuf;
    };
    // in order of preference; index k is the layout the override name names[k] selects
    Cand cands[4];
    if (p.per_pol) {
        // the Px - Py rows take the second intensity buffer (one intensity buffer, so the
        // barrier after the FIR spans the CTA); there is no one-buffer ping-pong form, so
        // "pingpong1" selects the same layout as "pingpong2"
        cands[0] = {kLayoutPingPong, 2 * exch + 2 * prow, 2 * exch, exch, 0};
        cands[1] = cands[0];
        cands[2] = {kLayoutSeparate, exch + 2 * prow + csr, exch, 0, 0};
        cands[3] = {kLayoutAlias, round_up(std::max(exch, 2 * prow + csr), 128), 0, 0, 0};
    } else {
        // ping-pong exchange arrays with two intensity buffers, then with one
        cands[0] = {kLayoutPingPong, 2 * exch + 2 * prow, 2 * exch, exch, prow};
        cands[1] = {kLayoutPingPong, 2 * exch + prow, 2 * exch, exch, 0};
        cands[2] = {kLayoutSeparate, exch + prow + csr, exch, 0, 0};
        cands[3] = {kLayoutAlias, round_up(std::max(exch, prow + csr), 128), 0, 0, 0};
    }
    // Optional override of the automatic choice (tuning): CBESSFM_SMEM_LAYOUT = pingpong2 |
    // pingpong1 | separate | alias.  A layout that does not fit falls back to the automatic one.
    int forced = -1;
    if (const char* env = std::getenv("CBESSFM_SMEM_LAYOUT")) {
        const char* names[4] = {"pingpong2", "pingpong1", "separate", "alias"};
        for (int k = 0; k < 4; ++k)
            if (std::strcmp(env, names[k]) == 0) forced = k;
    }
    int best = -1, best_res = 0, best_G = 0, best_tbl = 0;
    for (int k = 0; k < 4; ++k) {
        const Cand& c = cands[k];
        int tbl = tw_taps;
        int G = choose_blocks_per_cta(tb, c.region, tpf, bands, tbl, max_threads, min_ctas);
        if (G < 1 && tbl != tw) {
            tbl = tw;
            G = choose_blocks_per_cta(tb, c.region, tpf, bands, tbl, max_threads, min_ctas);
        }
        if (G < 1) continue;
        const int res = resident_blocks(G, tb, c.region, tbl, max_threads, min_ctas);
        if (k == forced) {
            best = k;
            best_G = G;
            best_tbl = tbl;
            break;
        }
        // candidates are in order of preference: a later one wins only with more resident blocks
        if (best < 0 || res > best_res) {
            best = k;
            best_res = res;
            best_G = G;
            best_tbl = tbl;
        }
    }
    if (best < 0) return false;
    const Cand& c = cands[best];
    p.tbl_bytes = best_tbl;
    p.taps_smem = best_tbl != tw ? 1 : 0;
    p.layout = c.layout;
    p.region_bytes = c.region;
    p.nlpr_off = c.nlpr_off;
    p.exb_off = c.exb_off;
    p.pbuf_bytes = c.pbuf;
    p.G = best_G;
    p.threads = best_G * tb;
    return true;
}

ChainArgs make_chain_args(const PlanImpl& p) {
    ChainArgs a{};
    a.n_sb = p.n_sb;
    a.n_st = p.n_st;
    a.N = p.N;
    a.n_ov = p.n_ov;
    a.V = p.V;
    a.G = p.G;
    a.nc = p.nc;
    a.ntaps_pad = p.ntaps_pad;
    a.nchunks = p.nchunks;
    a.H = p.H;
    a.p_off = p.p_off;
    a.pstride = p.pstride;
    a.region_bytes = p.region_bytes;
    a.nlpr_off = p.nlpr_off;
    a.layout = p.layout;
    a.exb_off = p.exb_off;
    a.pbuf_bytes = p.pbuf_bytes;
    a.tbl_bytes = p.tbl_bytes;
    a.taps_smem = p.taps_smem;
    a.per_pol = p.per_pol;
    a.gvd = p.d_gvd;
    a.gvd_half = p.d_gvd_half;
    a.gvd_first = p.d_gvd_half;
    a.gvd_last = p.d_gvd_half + 2 * (p.N / 2 + 1);
    a.mix_tw = p.d_mix_tw;
    {
        const int ef = chain_slots(p.n_fft, false);
        a.mix_td = p.d_mix_tw + (size_t)p.n_sb * p.N;
        a.mix_tm = a.mix_td + (size_t)p.n_sb * ef;
        a.fft_tw = p.d_fft_tw;
    }
    a.taps = p.d_taps;
    a.rot_tbl = p.d_rot;
    a.status = p.d_status;
    a.wait_cycles = p.wait_cycles;
    if (p.per_pol) classic_tables(p, a);
    return a;
}

void classic_tables(const PlanImpl& p, ChainArgs& a) {
    const int ef = chain_slots(p.n_fft, false), ec = fft_slots(p.n_fft);
    a.mix_td = p.d_mix_tw + (size_t)p.n_sb * p.N + 2 * (size_t)p.n_sb * ef;
    a.mix_tm = a.mix_td + (size_t)p.n_sb * ec;
    a.fft_tw = p.d_fft_tw_cl;
}

const PlanImpl* plan_impl(const cbessfm_plan* plan) { return plan ? &plan->impl : nullptr; }

}  // namespace cbessfm

using namespace cbessfm;

namespace cbessfm {

cbessfm_status forward_range(const cbessfm_plan* plan, const void* in, void* out,
                             int64_t n_samples, int batch, int cta0, int n_ctas,
                             cbessfm_stream stream) {
    if (plan == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "plan is NULL");
    if (in == nullptr || out == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "in/out is NULL");
    if (n_samples < 1) return fail(CBESSFM_ERR_INVALID_ARG, "n_samples must be >= 1");
    if (batch < 1) return fail(CBESSFM_ERR_INVALID_ARG, "batch must be >= 1");
    const PlanImpl& p = plan->impl;
    const unsigned long long sample_bytes = p.storage == CBESSFM_C64 ? 16ull : 8ull;
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u)
        return fail(CBESSFM_ERR_INVALID_ARG, "in/out must be 16-byte aligned");
    const long long n_blocks = blocks_for(n_samples, p.V);
    if (too_many_blocks(n_blocks, batch))
        return fail(CBESSFM_ERR_UNSUPPORTED, "too many blocks in one call");
    const unsigned long long bytes = (unsigned long long)n_samples * batch * sample_bytes;
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(in), o0 = reinterpret_cast<uintptr_t>(out);
    if (i0 < o0 + bytes && o0 < i0 + bytes) return fail(CBESSFM_ERR_ALIAS, "out overlaps in");
    const long long ctas = (n_blocks * batch + p.G - 1) / p.G;
    if (cta0 < 0 || n_ctas < 0 || cta0 > ctas)
        return fail(CBESSFM_ERR_INVALID_ARG, "CTA range %d + %d outside the batch's %lld", cta0,
                    n_ctas, ctas);
    if (cta0 == ctas) return CBESSFM_OK;
    ChainArgs a = make_chain_args(p);
    a.in = in;
    a.out = out;
    a.L = n_samples;
    a.batch = batch;
    a.n_blocks = (int)n_blocks;
    a.cta0 = cta0;
    a.n_ctas = n_ctas;
    const cudaError_t e = launch_forward(p, a, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "forward launch");
    return CBESSFM_OK;
}

}  // namespace cbessfm

extern "C" {

const char* cbessfm_last_error(void) { return cbessfm::last_error_text(); }

const char* cbessfm_version(void) { return "cbessfm-gb300 0.1 (sm_103a)"; }

static cbessfm_status plan_create_body(const cbessfm_link* link, int bands, int steps,
                                       double ratio, const float* coeffs, int ntaps, int n_fft,
                                       int overlap, cbessfm_storage storage, cbessfm_plan** out) {
    if (out == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (link == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "link is NULL");
    if (!(link->sample_rate > 0.0) || !std::isfinite(link->sample_rate))
        return fail(CBESSFM_ERR_INVALID_ARG, "sample_rate must be positive and finite");
    if (!(link->span_length > 0.0) || link->n_spans < 1)
        return fail(CBESSFM_ERR_INVALID_ARG, "span_length must be > 0 and n_spans >= 1");
    if (!std::isfinite(link->beta2)) return fail(CBESSFM_ERR_INVALID_ARG, "beta2 not finite");
    if (bands < 1 || bands > 16) return fail(CBESSFM_ERR_INVALID_ARG, "bands must be in [1, 16]");
    if (steps < 0 || steps > 4096) return fail(CBESSFM_ERR_INVALID_ARG, "steps must be in [0, 4096]");
    if (!(ratio >= 0.0 && ratio <= 1.0)) return fail(CBESSFM_ERR_INVALID_ARG, "ratio must be in [0, 1]");
    if (!is_pow2(n_fft) || n_fft < 16 || n_fft > 2048)
        return fail(CBESSFM_ERR_INVALID_ARG, "n_fft must be a power of two in [16, 2048]");
    if (ntaps < 1 || (ntaps & 1) == 0 || ntaps > n_fft / 2)
        return fail(CBESSFM_ERR_INVALID_ARG, "ntaps must be odd and in [1, n_fft/2]");
    if (overlap < 0 || (overlap & 1) || overlap >= n_fft)
        return fail(CBESSFM_ERR_INVALID_ARG, "overlap must be even and in [0, n_fft)");
    if (steps > 0 && coeffs == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "coeffs is NULL");
    if (storage != CBESSFM_C64 && storage != CBESSFM_F16x4 && storage != CBESSFM_BF16x4)
        return fail(CBESSFM_ERR_INVALID_ARG, "unknown storage type");

    PlanImpl p;
    p.link = *link;
    p.n_sb = bands;
    p.n_st = steps;
    p.ratio = ratio;
    p.ntaps = ntaps;
    p.n_fft = n_fft;
    p.overlap = overlap;
    p.storage = storage;
    p.N = bands * n_fft;
    p.n_ov = bands * overlap;
    p.V = p.N - p.n_ov;
    p.step_length = steps > 0 ? link->span_length * link->n_spans / steps : 0.0;
    p.nc = (ntaps - 1) / 2;
    p.nchunks = (ntaps + 3) / 4;
    p.ntaps_pad = 4 * p.nchunks;
    p.H = round_up(p.nc + 4, 4);
    p.p_off = ((3 - p.nc) % 4 + 4) % 4;
    p.pstride = round_up(n_fft + 2 * p.H + 8, 32);   // rows start on 128-byte boundaries

    const int tpf = n_fft / chain_slots(n_fft, false);
    const int tb = 2 * bands * tpf;                 // one polarization per thread
    if (tb > chain_max_threads(n_fft, false))
        return fail(CBESSFM_ERR_UNSUPPORTED, "%d threads per block exceed %d", tb,
                    chain_max_threads(n_fft, false));
    if (!choose_layout(p, tb, tpf))
        return fail(CBESSFM_ERR_UNSUPPORTED, "no shared-memory layout fits bands = %d, n_fft = %d",
                    bands, n_fft);

    cudaError_t e = cudaGetDevice(&p.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");

    // ---- FP64 tables on the host: FFT pass twiddles and DEMUX/MUX twiddles -------------------
    // FFT pass twiddles of the plan of (n_fft, E): the Manakov forward chain's E and fft_slots
    const double two_pi = 6.283185307179586476925286766559;
    auto pass_twiddles = [&](int E) {
        std::vector<float2> tw(std::max(1, fft_tw_size(n_fft, E)));
        for (int pass = 1; pass < fft_npasses(n_fft, E); ++pass) {
            const int R = fft_radix(n_fft, E, pass), NS = fft_ns(n_fft, E, pass);
            const int off = fft_tw_offset(n_fft, E, pass);
            for (int r = 1; r < R; ++r)
                for (int a = 0; a < NS; ++a) {
                    const long long num = (long long)a * r;           // < NS R
                    const double ang = -two_pi * (double)num / (double)(NS * R);
                    tw[off + (r - 1) * NS + a] = unit_f32(ang);
                }
        }
        return tw;
    };
    const int Ef = chain_slots(n_fft, false), Ec = fft_slots(n_fft);
    const bool same_plan = Ef == Ec;
    const std::vector<float2> fft_tw = pass_twiddles(Ef);
    const std::vector<float2> fft_tw_cl = same_plan ? std::vector<float2>() : pass_twiddles(Ec);
    // [bands][N] W_N^(K r), then the per-slot factors of the chain's DEMUX and MUX for the
    // forward chain's E, then for fft_slots' E:
    // [bands][E] W_N^(r (N'/E) t) times W_N^(-r N') for t >= E/2 (DEMUX), [bands][E] W_N^(r (N'/E) t)
    std::vector<float2> mix_tw((size_t)bands * p.N + 2 * (size_t)bands * (Ef + Ec));
    auto w_n = [&](long long num) {                  // W_N^num, exponent reduced exactly mod N
        num %= p.N;
        if (num < 0) num += p.N;
        return unit_f32(-two_pi * (double)num / (double)p.N);
    };
    for (int r = 0; r < bands; ++r)
        for (int K = 0; K < p.N; ++K) mix_tw[(size_t)r * p.N + K] = w_n((long long)K * r);
    auto slot_factors = [&](float2* mix_td, int E) {
        const int TPF = n_fft / E;
        float2* const mix_tm = mix_td + (size_t)bands * E;
        for (int r = 0; r < bands; ++r)
            for (int t = 0; t < E; ++t) {
                mix_td[r * E + t] = w_n((long long)r * (TPF * t - (t >= E / 2 ? n_fft : 0)));
                mix_tm[r * E + t] = w_n((long long)r * TPF * t);
            }
    };
    slot_factors(mix_tw.data() + (size_t)bands * p.N, Ef);
    slot_factors(mix_tw.data() + (size_t)bands * p.N + 2 * (size_t)bands * Ef, Ec);

    std::vector<float2> rot(256);
    for (int k = 0; k < 256; ++k) {
        rot[k] = unit_f32(two_pi * k / 256.0);
    }
    // every host container exists before the first device allocation (see abi_guard.h)
    const std::vector<float> packed = steps > 0 ? pack_taps(p, coeffs) : std::vector<float>();

    const size_t n_taps_dev = std::max<size_t>(1, (size_t)steps * bands * bands * p.ntaps_pad);
#define CB_TRY(call, what)                    \
    do {                                      \
        cudaError_t _e = (call);              \
        if (_e != cudaSuccess) {              \
            free_plan(p);                     \
            return cuda_fail(_e, what);       \
        }                                     \
    } while (0)
    CB_TRY(cudaMalloc(&p.d_gvd, sizeof(float2) * 3 * bands * n_fft), "cudaMalloc(gvd)");
    CB_TRY(cudaMalloc(&p.d_gvd_half, sizeof(float2) * 4 * (p.N / 2 + 1)), "cudaMalloc(gvd half)");
    CB_TRY(cudaMalloc(&p.d_mix_tw, sizeof(float2) * mix_tw.size()), "cudaMalloc(mix)");
    CB_TRY(cudaMalloc(&p.d_fft_tw, sizeof(float2) * fft_tw.size()), "cudaMalloc(fft tw)");
    if (same_plan) {
        p.d_fft_tw_cl = p.d_fft_tw;
    } else {
        CB_TRY(cudaMalloc(&p.d_fft_tw_cl, sizeof(float2) * fft_tw_cl.size()), "cudaMalloc(fft tw)");
        CB_TRY(cudaMemcpy(p.d_fft_tw_cl, fft_tw_cl.data(), sizeof(float2) * fft_tw_cl.size(),
                          cudaMemcpyHostToDevice), "copy fft twiddles");
    }
    CB_TRY(cudaMalloc(&p.d_taps, sizeof(float) * n_taps_dev), "cudaMalloc(taps)");
    CB_TRY(cudaMalloc(&p.d_taps_t, sizeof(float) * n_taps_dev), "cudaMalloc(transposed taps)");
    CB_TRY(cudaMalloc(&p.d_status, sizeof(unsigned int)), "cudaMalloc(status)");
    CB_TRY(cudaMalloc(&p.d_rot, sizeof(float2) * rot.size()), "cudaMalloc(rot)");
    CB_TRY(cudaMemcpy(p.d_rot, rot.data(), sizeof(float2) * rot.size(), cudaMemcpyHostToDevice),
           "copy rotation table");
    CB_TRY(cudaMemset(p.d_status, 0, sizeof(unsigned int)), "cudaMemset(status)");
    CB_TRY(cudaMemcpy(p.d_fft_tw, fft_tw.data(), sizeof(float2) * fft_tw.size(),
                      cudaMemcpyHostToDevice), "copy fft twiddles");
    CB_TRY(cudaMemcpy(p.d_mix_tw, mix_tw.data(), sizeof(float2) * mix_tw.size(),
                      cudaMemcpyHostToDevice), "copy mix twiddles");
    CB_TRY(cudaMemset(p.d_taps, 0, sizeof(float) * n_taps_dev), "cudaMemset(taps)");
    if (steps > 0)
        CB_TRY(cudaMemcpy(p.d_taps, packed.data(), sizeof(float) * packed.size(),
                          cudaMemcpyHostToDevice), "copy taps");
    CB_TRY(launch_build_gvd(p, nullptr), "build GVD tables");
    CB_TRY(launch_transpose_taps(p, nullptr), "transpose taps");
    CB_TRY(prepare_forward(n_fft, (int)storage, kMaxDynSmem), "set shared-memory limit");
    if (storage != CBESSFM_C64)      // the streamed passes of a 16-bit plan run complex64 kernels
        CB_TRY(prepare_forward(n_fft, (int)CBESSFM_C64, kMaxDynSmem), "set shared-memory limit");
    CB_TRY(cudaDeviceSynchronize(), "plan tables");
#undef CB_TRY

    cbessfm_plan* plan = new (std::nothrow) cbessfm_plan;
    if (plan == nullptr) {
        free_plan(p);
        return fail(CBESSFM_ERR_OOM, "host allocation of the plan failed");
    }
    plan->impl = p;
    *out = plan;
    return CBESSFM_OK;
}

cbessfm_status cbessfm_plan_create(const cbessfm_link* link, int bands, int steps, double ratio,
                                   const float* coeffs, int ntaps, int n_fft, int overlap,
                                   cbessfm_storage storage, cbessfm_plan** out) {
    TraceRange trace_range("cbessfm:plan_create");
    clear_error();
    return abi_guard([&] {
        return plan_create_body(link, bands, steps, ratio, coeffs, ntaps, n_fft, overlap, storage,
                                out);
    });
}

cbessfm_status cbessfm_plan_destroy(cbessfm_plan* plan) {
    clear_error();
    if (plan == nullptr) return CBESSFM_OK;
    cudaDeviceSynchronize();
    free_plan(plan->impl);
    destroy_host_pipeline(plan->pipe);
    delete plan;
    return CBESSFM_OK;
}

static cbessfm_status set_coeffs_body(cbessfm_plan* plan, const float* coeffs, int on_device,
                                      cbessfm_stream stream) {
    if (plan == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "plan is NULL");
    PlanImpl& p = plan->impl;
    if (p.n_st == 0) return CBESSFM_OK;
    if (coeffs == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "coeffs is NULL");
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (!on_device) {
        const std::vector<float> packed = pack_taps(p, coeffs);
        e = cudaMemcpyAsync(p.d_taps, packed.data(), sizeof(float) * packed.size(),
                            cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    } else {
        // row-wise copies of [ntaps] into [ntaps_pad] (padding stays zero)
        e = cudaMemcpy2DAsync(p.d_taps, sizeof(float) * p.ntaps_pad, coeffs,
                              sizeof(float) * p.ntaps, sizeof(float) * p.ntaps,
                              (size_t)p.n_st * p.n_sb * p.n_sb, cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess) e = launch_transpose_taps(p, st);
    if (e != cudaSuccess) return cuda_fail(e, "set_coeffs");
    return CBESSFM_OK;
}

cbessfm_status cbessfm_set_coeffs(cbessfm_plan* plan, const float* coeffs, int on_device,
                                  cbessfm_stream stream) {
    TraceRange trace_range("cbessfm:set_coeffs");
    clear_error();
    return abi_guard([&] { return set_coeffs_body(plan, coeffs, on_device, stream); });
}

cbessfm_status cbessfm_set_ratio(cbessfm_plan* plan, double ratio, cbessfm_stream stream) {
    TraceRange trace_range("cbessfm:set_ratio");
    clear_error();
    if (plan == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "plan is NULL");
    if (!(ratio >= 0.0 && ratio <= 1.0)) return fail(CBESSFM_ERR_INVALID_ARG, "ratio must be in [0, 1]");
    plan->impl.ratio = ratio;
    const cudaError_t e = launch_build_gvd(plan->impl, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "set_ratio");
    return CBESSFM_OK;
}

cbessfm_status cbessfm_backpropagate(const cbessfm_plan* plan, const void* in, void* out,
                                     int64_t n_samples, int batch, cbessfm_stream stream) {
    TraceRange trace_range("cbessfm:backpropagate");
    clear_error();
    return forward_range(plan, in, out, n_samples, batch, 0, 0, stream);
}

// Streamed form: one launch of the chain per step, each with one NLPR step and its own
// overlap-and-save; pass s applies the first GVD ((1 - rho) L_step) only when s = 0 and ends
// with L_step, or rho L_step for the last step.  Intermediate fields alternate between the
// workspace's two buffers.
namespace {

// complex64 fields of the streamed form's workspace: ping-pong between passes (one for two
// steps); a 16-bit plan's passes start from a widened copy of the input and end in a field
// that is narrowed into the output, which takes both fields from two steps on.
size_t streamed_buffers(const PlanImpl& p) {
    if (p.storage != CBESSFM_C64) return p.n_st >= 2 ? 2 : 0;
    return p.n_st >= 3 ? 2 : (p.n_st == 2 ? 1 : 0);
}

}  // namespace

cbessfm_status cbessfm_streamed_workspace_size(const cbessfm_plan* plan, int64_t n_samples,
                                               int batch, size_t* bytes) {
    clear_error();
    if (plan == nullptr || bytes == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "plan/bytes is NULL");
    if (n_samples < 1 || batch < 1) return fail(CBESSFM_ERR_INVALID_ARG, "n_samples and batch must be >= 1");
    if (too_many_blocks(blocks_for(n_samples, plan->impl.V), batch))
        return fail(CBESSFM_ERR_UNSUPPORTED, "too many blocks in one call");
    const size_t one = ((size_t)n_samples * batch * 16 + 255) / 256 * 256;
    *bytes = streamed_buffers(plan->impl) * one;
    return CBESSFM_OK;
}

cbessfm_status cbessfm_backpropagate_streamed(const cbessfm_plan* plan, const void* in, void* out,
                                              void* workspace, size_t ws_bytes, int64_t n_samples,
                                              int batch, cbessfm_stream stream) {
    TraceRange trace_range("cbessfm:backpropagate_streamed");
    clear_error();
    if (plan == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "plan is NULL");
    const PlanImpl& p = plan->impl;
    if (p.n_st <= 1) return cbessfm_backpropagate(plan, in, out, n_samples, batch, stream);
    if (in == nullptr || out == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "in/out is NULL");
    if (n_samples < 1 || batch < 1) return fail(CBESSFM_ERR_INVALID_ARG, "n_samples and batch must be >= 1");
    const long long n_blocks = blocks_for(n_samples, p.V);
    if (too_many_blocks(n_blocks, batch))
        return fail(CBESSFM_ERR_UNSUPPORTED, "too many blocks in one call");
    const size_t one = ((size_t)n_samples * batch * 16 + 255) / 256 * 256;
    if (workspace == nullptr || ws_bytes < streamed_buffers(p) * one)
        return fail(CBESSFM_ERR_INVALID_ARG, "workspace of %zu bytes is smaller than %zu", ws_bytes,
                    streamed_buffers(p) * one);
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out) |
         reinterpret_cast<uintptr_t>(workspace)) & 15u)
        return fail(CBESSFM_ERR_INVALID_ARG, "in/out/workspace must be 16-byte aligned");
    const bool wide = p.storage != CBESSFM_C64;   // 16-bit fields around complex64 passes
    const unsigned long long bytes = (unsigned long long)n_samples * batch * (wide ? 8ull : 16ull);
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(in), o0 = reinterpret_cast<uintptr_t>(out);
    const uintptr_t w0 = reinterpret_cast<uintptr_t>(workspace), w1 = w0 + streamed_buffers(p) * one;
    if (i0 < o0 + bytes && o0 < i0 + bytes) return fail(CBESSFM_ERR_ALIAS, "out overlaps in");
    if ((i0 < w1 && w0 < i0 + bytes) || (o0 < w1 && w0 < o0 + bytes))
        return fail(CBESSFM_ERR_ALIAS, "workspace overlaps in or out");
    unsigned char* buf[2] = {static_cast<unsigned char*>(workspace),
                             static_cast<unsigned char*>(workspace) + one};
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long n_all = (long long)n_samples * batch;
    if (wide) {                                   // widened input in buf[1]; pass s writes buf[s & 1]
        const cudaError_t e = launch_widen(p.storage, in, reinterpret_cast<float4*>(buf[1]), n_all, st);
        if (e != cudaSuccess) return cuda_fail(e, "streamed input widening");
    }
    for (int s = 0; s < p.n_st; ++s) {
        ChainArgs a = make_chain_args(p);
        if (wide) {
            a.in = s == 0 ? buf[1] : buf[(s - 1) & 1];
            a.out = buf[s & 1];
        } else {
            a.in = s == 0 ? in : buf[(s - 1) & 1];
            a.out = s == p.n_st - 1 ? out : buf[s & 1];
        }
        a.L = n_samples;
        a.batch = batch;
        a.n_blocks = (int)n_blocks;
        a.n_st = 1;
        a.taps = p.d_taps + (size_t)s * p.n_sb * p.n_sb * p.ntaps_pad;
        const size_t half = (size_t)(p.N / 2 + 1);
        a.gvd_first = p.d_gvd_half + (s == 0 ? 0 : 3) * half;
        a.gvd_last = p.d_gvd_half + (s == p.n_st - 1 ? 2 : 1) * half;
        const cudaError_t e = wide ? launch_forward_c64(p, a, st) : launch_forward(p, a, st);
        if (e != cudaSuccess) return cuda_fail(e, "streamed pass launch");
    }
    if (wide) {
        const cudaError_t e = launch_narrow(p.storage, reinterpret_cast<const float4*>(buf[(p.n_st - 1) & 1]),
                                            out, n_all, st);
        if (e != cudaSuccess) return cuda_fail(e, "streamed output narrowing");
    }
    return CBESSFM_OK;
}

extern "C" cbessfm_status cbessfm_set_wait_limit(cbessfm_plan* plan, long long cycles) {
    clear_error();
    if (!plan) return fail(CBESSFM_ERR_INVALID_ARG, "set_wait_limit: NULL plan");
    plan->impl.wait_cycles = cycles < 0 ? kWaitCycles : cycles;
    return CBESSFM_OK;
}

static cbessfm_status set_nlpr_mode_body(cbessfm_plan* plan, int per_polarization) {
    if (plan == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "plan is NULL");
    if (per_polarization != 0 && per_polarization != 1)
        return fail(CBESSFM_ERR_INVALID_ARG, "per_polarization must be 0 or 1");
    PlanImpl& p = plan->impl;
    if (per_polarization && p.storage != CBESSFM_C64)
        return fail(CBESSFM_ERR_UNSUPPORTED, "the per-polarization NLPR needs complex64 storage");
    if (p.per_pol == per_polarization) return CBESSFM_OK;
    PlanImpl trial = p;
    trial.per_pol = per_polarization;
    const int tpf = p.n_fft / chain_slots(p.n_fft, per_polarization != 0);
    const int tb = 2 * p.n_sb * tpf;
    if (!choose_layout(trial, tb, tpf))
        return fail(CBESSFM_ERR_UNSUPPORTED,
                    "the per-polarization NLPR of %d bands at n_fft %d does not fit shared memory",
                    p.n_sb, p.n_fft);
    p = trial;
    return CBESSFM_OK;
}

cbessfm_status cbessfm_set_nlpr_mode(cbessfm_plan* plan, int per_polarization) {
    clear_error();
    return abi_guard([&] { return set_nlpr_mode_body(plan, per_polarization); });
}

cbessfm_status cbessfm_get_status(const cbessfm_plan* plan, cbessfm_stream stream) {
    clear_error();
    if (plan == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "plan is NULL");
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, plan->impl.d_status, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(plan->impl.d_status, 0, sizeof(h), st);
    if (e != cudaSuccess) return cuda_fail(e, "get_status");
    if (h & kStatusTimeout)
        return fail(CBESSFM_ERR_TIMEOUT, "a bounded device wait for a shared-memory copy gave up");
    return CBESSFM_OK;
}

}  // extern "C"
