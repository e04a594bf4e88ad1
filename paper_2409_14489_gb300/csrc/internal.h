// internal.h -- host-side plan layout and kernel launch interfaces (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/cbessfm.h"

namespace cbessfm {

// Shared-memory layouts of one OLS block's region in the forward chain.
//  kLayoutAlias:    one exchange array; the intensity and (cos, sin) rows alias it, so two more
//                   block-wide barriers per step guard the reuse.
//  kLayoutSeparate: one exchange array, then the intensity rows and the (cos, sin) rows.
//  kLayoutPingPong: two exchange arrays A and B used alternately by the FFT passes (no barrier
//                   before a store), the (cos, sin) rows inside the array the inverse FFT read
//                   last, then one or two intensity-row buffers.  With two buffers (pbuf_bytes >
//                   0) the barrier after the FIR covers only the subband group.
//  kLayoutPacked:   the two-pass plan's layout (N' = 1024, 32 slots): one exchange array per
//                   subband group, holding the group's intensity row (at its start) and its
//                   (cos, sin) row (after it) while the FFTs do not use it.
constexpr int kLayoutAlias = 0;
constexpr int kLayoutSeparate = 1;
constexpr int kLayoutPingPong = 2;
constexpr int kLayoutPacked = 3;
// Packed layout: complex slots per thread parked in shared memory during the FIR (the registers
// they free keep the FIR's window and accumulators out of local memory), after the group's
// (cos, sin) row: [kParkSlots][2 NP/E] complex.
constexpr int kParkSlots = 8;

// Default bound of the chain kernels' waits for their staging copies, in SM clock cycles
// (about 2 s at 2 GHz: never reached by a live copy).
constexpr long long kWaitCycles = 4000000000LL;

// Kernel arguments of the chain kernels (forward and adjoint share them).
struct ChainArgs {
    const void* in;              // [batch][L] samples (storage type of the plan)
    void* out;                   // [batch][L]
    long long L;                 // samples per sequence
    int batch;
    int n_sb, n_st;              // subbands, steps
    int N, n_ov, V, n_blocks;    // block size, total overlap, valid samples, blocks per sequence
    int G;                       // OLS blocks per CTA
    int nc, ntaps_pad, nchunks;  // FIR: N_c, taps per row (multiple of 4), chunks of 4 taps
    int H, p_off, pstride;       // FIR intensity buffer: halo, alignment offset, row stride
    int region_bytes;            // shared memory per OLS block
    int nlpr_off;                // byte offset of the intensity rows in the region
    int layout;                  // shared-memory layout of a block's region (kLayout*)
    int exb_off;                 // byte offset of the second exchange array (ping-pong layout)
    int pbuf_bytes;              // bytes from the first to the second intensity-row buffer, or 0
    int tbl_bytes;               // shared memory after the G regions: FFT twiddles (+ tap buffers)
    int taps_smem;               // 1: each step's taps are staged in shared memory (4-tap chunks = 3)
    int per_pol;                 // 1: per-polarization NLPR of Eqs. (NLPR_polx/poly); the
                                 //    Px - Py rows follow the intensity rows
    const float2* gvd;           // [3][n_sb][NP]: first (x 1/N), interior (x 1/NP), last (x 1/NP)
    const float2* gvd_half;      // [4][N/2 + 1]: the same factors by |centred bin|, and the
                                 // unit factor (x 1/N) as kind 3
    const float2* gvd_first;     // gvd_half kind of the first GVD (kind 0, or 3 in later passes)
    const float2* gvd_last;      // gvd_half kind of the last step's GVD (kind 2, or 1)
    const float2* mix_tw;        // [n_sb][N]: W_N^(K r)
    const float2* mix_td;        // [n_sb][E] DEMUX slot factors of the kernel's E (see the
    const float2* mix_tm;        // [n_sb][E] MUX slot factors      chain's DEMUX and MUX)
    const float2* fft_tw;        // FFT pass twiddles of the kernel's plan (fft_tw_size(NP, E))
    const float* taps;           // [n_st][n_sb][n_sb][ntaps_pad]
    const float2* rot_tbl;       // [256] exp(j 2 pi k / 256)
    unsigned int* status;        // device status word
    float2* ckpt;                // adjoint checkpoints (checkpointed forward only), else null
    const float* taps_t;         // [n_st][n_sb][n_sb][ntaps_pad] transposed, reversed taps (adjoint)
    const float2* gout;          // adjoint: dL/d(out) as (re, im) pairs, [batch][L][2]
    float2* gin;                 // adjoint: dL/d(in), accumulated, or null
    float* gpart;                // adjoint: per-block partial tap and ratio gradients
    float2* stash;               // adjoint: per-block scratch, two fields [2][gi][idx][p]
    int want_ratio;              // adjoint: 1 if dL/drho is requested
    float kd0;                   // adjoint: 2 pi^2 beta2 L_step (R/N)^2 (ratio-gradient weights)
    long long wait_cycles;       // bound of the waits for the staging copies (SM cycles; <= 0:
                                 // one non-blocking test)
    int cta0, n_ctas;            // forward launch over CTAs [cta0, cta0 + n_ctas) of the whole
                                 // batch's grid (n_ctas = 0: to the end); CTA c runs work items
                                 // c G .. c G + G - 1, item = seq * n_blocks + blk
};

struct PlanImpl {
    int device = 0;
    cbessfm_link link{};
    int n_sb = 1, n_st = 0, ntaps = 1, n_fft = 16, overlap = 0;
    double ratio = 0.5;
    cbessfm_storage storage = CBESSFM_C64;
    int N = 16, n_ov = 0, V = 16;
    int nc = 0, ntaps_pad = 4, nchunks = 1, H = 4, p_off = 3, pstride = 32;
    int region_bytes = 0, nlpr_off = 0, layout = 0, exb_off = 0, pbuf_bytes = 0, G = 1, threads = 0;
    int tbl_bytes = 0, taps_smem = 0, per_pol = 0;
    double step_length = 0.0;
    float2* d_gvd = nullptr;      // [3][n_sb][NP]
    float2* d_gvd_half = nullptr; // [4][N/2 + 1]
    float2* d_mix_tw = nullptr;   // [n_sb][N], then DEMUX and MUX slot factors [n_sb][E] of the
                                  // Manakov forward chain's E, then of fft_slots (classic)
    float2* d_fft_tw = nullptr;   // FFT twiddles of the Manakov forward chain's plan
    float2* d_fft_tw_cl = nullptr;// FFT twiddles of the fft_slots plan (adjoint, per-polarization
                                  // chain); the same table when both plans agree
    long long wait_cycles = kWaitCycles;
    float* d_taps = nullptr;      // [n_st][n_sb][n_sb][ntaps_pad]
    float2* d_rot = nullptr;      // [256] exp(j 2 pi k / 256) from FP64
    float* d_taps_t = nullptr;    // transposed, reversed taps for the adjoint's intensity gradient
    unsigned int* d_status = nullptr;
};

// FP64 kernel that fills the three GVD tables (and the ratio-derivative table) on `stream`.
cudaError_t launch_build_gvd(const PlanImpl& p, cudaStream_t stream);

// taps_t[s][l][i][q] = taps[s][i][l][ntaps - 1 - q]: the adjoint's intensity-gradient filter.
cudaError_t launch_transpose_taps(const PlanImpl& p, cudaStream_t stream);

// Forward chain kernel; returns cudaSuccess or the launch error.
cudaError_t launch_forward(const PlanImpl& p, const ChainArgs& a, cudaStream_t stream);
// Opt in to `smem_bytes` of dynamic shared memory for the forward kernel of (NP, storage).
cudaError_t prepare_forward(int np, int storage, int smem_bytes);

ChainArgs make_chain_args(const PlanImpl& p);
// The tables of the fft_slots (classic) plan: FFT twiddles and DEMUX/MUX slot factors, for the
// adjoint kernel and the per-polarization chain.
void classic_tables(const PlanImpl& p, ChainArgs& a);

// Launch-shape limits shared by the plan and batch builders.
constexpr int kMaxDynSmem = 224 * 1024;     // 227 KB per block minus room for static shared memory
constexpr int kMaxThreads = 640;
constexpr int kMaxG = 16;
// OLS blocks per CTA for a block of `tb` threads and `region_bytes` of shared memory, with
// `extra_bytes` more per CTA, in a kernel compiled for at most `max_threads` threads and at
// least `min_ctas` CTAs per SM (0 = none fits).
int choose_blocks_per_cta(int tb, int region_bytes, int tpf, int bands, int extra_bytes = 0,
                          int max_threads = kMaxThreads, int min_ctas = 1);

// Per-CTA shared tables of the forward chain, after the G block regions: the FFT pass twiddles of
// N' (rounded to 128 bytes), then, when taps are staged, two buffers of one step's taps
// ([bands][bands][12] floats each).
__host__ __device__ constexpr int chain_tw_bytes(int tw_entries) {
    return (8 * tw_entries + 127) / 128 * 128;
}
__host__ __device__ constexpr int chain_taps_bytes(int bands) { return 2 * bands * bands * 12 * 4; }

// Error reporting (thread-local message, see cbessfm_last_error).
cbessfm_status fail(cbessfm_status st, const char* fmt, ...);
cbessfm_status cuda_fail(cudaError_t e, const char* what);
void clear_error();
const char* last_error_text();

// The plan object behind the opaque C handle.
const PlanImpl* plan_impl(const cbessfm_plan* plan);

// OLS blocks resident per SM for G blocks of `tb` threads per CTA, `region` bytes each, and
// `tables` bytes of per-CTA tables, in a kernel compiled for `max_threads` threads and
// `min_ctas` CTAs per SM (which fixes its registers per thread).
int resident_blocks(int G, int tb, int region, int tables, int max_threads = kMaxThreads,
                    int min_ctas = 1);

// cbessfm_backpropagate restricted to the CTAs [cta0, cta0 + n_ctas) of the whole batch's grid
// (n_ctas = 0: to the end), i.e. the work items [cta0 G, (cta0 + n_ctas) G) of the flattened
// (sequence, block) list, item = seq * n_blocks + blk, with G = the plan's blocks per CTA.  The
// blocks of the range read their input (with its overlap, which wraps within the sequence) and
// write their valid samples only.
cbessfm_status forward_range(const cbessfm_plan* plan, const void* in, void* out,
                             int64_t n_samples, int batch, int cta0, int n_ctas,
                             cbessfm_stream stream);

// Streams and events of cbessfm_backpropagate_host, created on first use, owned by the plan.
struct HostPipeline;
void destroy_host_pipeline(HostPipeline* hp);

}  // namespace cbessfm

// The object behind the opaque C handle.
struct cbessfm_plan {
    cbessfm::PlanImpl impl;
    cbessfm::HostPipeline* pipe = nullptr;   // streams and events of the host-pipelined entry
};

namespace cbessfm {

// Persistent batched launch of the forward kernel for one (NP, storage) group.
cudaError_t launch_forward_persistent(int np, int storage, const ChainArgs* jobs, const int2* items,
                                      int n_items, unsigned int* counter, int n_sb, int G,
                                      int region_bytes, int tbl_bytes, int per_pol, int threads,
                                      int grid, cudaStream_t stream);
cudaError_t forward_persistent_occupancy(int np, int storage, int threads, int smem_bytes,
                                         int* ctas_per_sm);

}  // namespace cbessfm
