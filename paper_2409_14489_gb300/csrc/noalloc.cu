// noalloc.cu -- batched backpropagation that allocates no device memory.
//
// Some callers cannot allocate device memory at the time they need to run: a receiver's
// real-time DSP thread that must not take the allocator's lock or pay its latency in the middle
// of a frame, a process whose device memory is reserved up front by another allocator and is
// capped, or a plugin host that forbids allocation inside its processing callbacks.
// cbessfm_batch_run_noalloc serves them.  It runs the same per-block chain as the batched form
// (chain_block), but the work list lives in one file-scope static device array instead of
// buffers from cudaMalloc:
//
//   g_noalloc_scratch  [0, 256)                       work counter (zeroed by every call)
//                      [256, 256 + 64 * 256)          up to kNoallocMaxJobs job descriptors
//                      [16640, 16640 + 65 * 4)        prefix sums of the per-job work items
//
// Every GPU that loads the library holds this 17 KB until the process exits.  All calls share
// it and it keeps the last call's contents, so two calls whose work overlaps on the GPU (two
// streams, or two host threads) race on it: callers must order them.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "abi_guard.h"
#include "block_count.h"
#include "fwd_kernel.cuh"
#include "internal.h"

namespace cbessfm {
namespace {

constexpr int kNoallocMaxJobs = 64;
constexpr int kDescBytes = 320;
constexpr int kCounterOff = 0;
constexpr int kDescOff = 256;
constexpr int kPrefixOff = kDescOff + kNoallocMaxJobs * kDescBytes;
constexpr int kScratchBytes = kPrefixOff + 512;
static_assert(sizeof(ChainArgs) <= kDescBytes, "job descriptor slot too small");
static_assert((kNoallocMaxJobs + 1) * 4 <= 512, "prefix area too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Same work distribution as the batched persistent kernel, with the item list replaced by the
// prefix sums: item i belongs to the job k with prefix[k] <= i < prefix[k + 1] and covers blocks
// (i - prefix[k]) G .. + G - 1 of that job.  Jobs are ordered by decreasing cost on the host.
template <int NP>
__global__ void __launch_bounds__(chain_max_threads(NP, false), chain_min_ctas(NP, false))
    cbessfm_fwd_noalloc_kernel(
    const ChainArgs* __restrict__ jobs, const int* __restrict__ prefix, int njobs,
    unsigned int* __restrict__ counter, int n_sb, int G, int region_bytes) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[kMaxG];
    __shared__ float2 s_rot[kRotTable];
    __shared__ ChainArgs s_job;
    __shared__ int s_item;
    constexpr int E = chain_slots(NP, false);
    const ThreadPos tp = thread_pos<NP, E>(n_sb);
    float2* const s_tw = reinterpret_cast<float2*>(smem + (size_t)G * region_bytes);
    float4* const s_taps = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(s_tw) +
                                                     chain_tw_bytes(fft_tw_size(NP, E)));
    for (int k = tp.tid; k < fft_tw_size(NP, E); k += blockDim.x) s_tw[k] = __ldg(jobs[0].fft_tw + k);
    if (tp.tid < G) mbar_init(&bars[tp.tid], 1);
    mbar_fence_init();
    const int n_items = prefix[njobs];
    int rot_of = -1;
    for (uint32_t it = 0;; ++it) {
        if (tp.tid == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;
        int k = 0;
        while (k + 1 < njobs && prefix[k + 1] <= item) ++k;
        for (int w = tp.tid; w < (int)(sizeof(ChainArgs) / sizeof(int)); w += blockDim.x)
            reinterpret_cast<int*>(&s_job)[w] = reinterpret_cast<const int*>(jobs + k)[w];
        __syncthreads();
        if (rot_of != k) {
            for (int r = tp.tid; r < kRotTable; r += blockDim.x) s_rot[r] = __ldg(s_job.rot_tbl + r);
            rot_of = k;
            __syncthreads();
        }
        const int blk = (item - prefix[k]) * G + tp.g;
        const bool real = blk < s_job.n_blocks;
        if (!chain_block<NP, 0>(s_job, smem, region_bytes, &bars[tp.g], it & 1u, s_rot, s_tw,
                                s_taps, tp, real, 0, real ? blk : 0))
            return;
        __syncthreads();
    }
}

template <int NP>
cudaError_t noalloc_prepare() {
    return cudaFuncSetAttribute(cbessfm_fwd_noalloc_kernel<NP>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

cudaError_t noalloc_prepare_all() {
    const cudaError_t e[] = {noalloc_prepare<16>(), noalloc_prepare<32>(), noalloc_prepare<64>(),
                             noalloc_prepare<128>(), noalloc_prepare<256>(), noalloc_prepare<512>(),
                             noalloc_prepare<1024>(), noalloc_prepare<2048>()};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return x;
    return cudaSuccess;
}

cudaError_t noalloc_launch(int np, const ChainArgs* jobs, const int* prefix, int njobs,
                           unsigned int* counter, int n_sb, int G, int region_bytes, int tbl_bytes,
                           int threads, int grid, cudaStream_t st) {
    const size_t smem = (size_t)G * region_bytes + tbl_bytes;
#define CB_CASE(NP)                                                                           \
    case NP:                                                                                  \
        cbessfm_fwd_noalloc_kernel<NP><<<grid, threads, smem, st>>>(jobs, prefix, njobs, counter, \
                                                                   n_sb, G, region_bytes);  \
        return cudaGetLastError();
    switch (np) {
        CB_CASE(16) CB_CASE(32) CB_CASE(64) CB_CASE(128) CB_CASE(256) CB_CASE(512) CB_CASE(1024)
        CB_CASE(2048)
        default: return cudaErrorInvalidValue;
    }
#undef CB_CASE
}

template <int NP>
cudaError_t noalloc_occ(int threads, int smem, int* per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, cbessfm_fwd_noalloc_kernel<NP>,
                                                         threads, smem);
}

cudaError_t noalloc_occupancy(int np, int threads, int smem, int* per_sm) {
    switch (np) {
        case 16: return noalloc_occ<16>(threads, smem, per_sm);
        case 32: return noalloc_occ<32>(threads, smem, per_sm);
        case 64: return noalloc_occ<64>(threads, smem, per_sm);
        case 128: return noalloc_occ<128>(threads, smem, per_sm);
        case 256: return noalloc_occ<256>(threads, smem, per_sm);
        case 512: return noalloc_occ<512>(threads, smem, per_sm);
        case 1024: return noalloc_occ<1024>(threads, smem, per_sm);
        case 2048: return noalloc_occ<2048>(threads, smem, per_sm);
        default: return cudaErrorInvalidValue;
    }
}

// Per-device set-up: the device address of g_noalloc_scratch (a host-side name of the array
// is not a device address) and the kernels' shared-memory limit.  Done by the first call on
// each device, with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

cbessfm_status device_setup(int dev, unsigned char** ptr, int* n_sm) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        e = noalloc_prepare_all();
        if (e != cudaSuccess) return cuda_fail(e, "set shared-memory limit");
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "device query");
        g_sm_count[dev] = sms;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *ptr = g_scratch_ptr[dev];
    *n_sm = g_sm_count[dev];
    return CBESSFM_OK;
}

}  // namespace
}  // namespace cbessfm

using namespace cbessfm;

extern "C" cbessfm_status cbessfm_batch_run_noalloc(const cbessfm_job* jobs, int njobs,
                                                    cbessfm_stream stream) {
    clear_error();
    if (jobs == nullptr || njobs < 1) return fail(CBESSFM_ERR_INVALID_ARG, "no jobs");
    if (njobs > kNoallocMaxJobs)
        return fail(CBESSFM_ERR_UNSUPPORTED,
                    "%d jobs exceed the %d job descriptors of the static scratch array", njobs,
                    kNoallocMaxJobs);
    // descriptors and the work-item prefix are built on the host stack
    ChainArgs desc[kNoallocMaxJobs];
    int order[kNoallocMaxJobs];
    int prefix[kNoallocMaxJobs + 1];
    int np = 0, n_sb = 0, region = 0;
    bool any_taps = false;
    // the static array and the plans' tables must be on the same (current) device
    int dev = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < njobs; ++k) {
        const cbessfm_job& jb = jobs[k];
        const PlanImpl* p = plan_impl(jb.plan);
        if (p == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "job %d: plan is NULL", k);
        if (k == 0 && (e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
        if (p->device != dev)
            return fail(CBESSFM_ERR_INVALID_ARG,
                        "job %d: plan was created on device %d, the current device is %d", k,
                        p->device, dev);
        if (jb.in == nullptr || jb.out == nullptr)
            return fail(CBESSFM_ERR_INVALID_ARG, "job %d: in/out is NULL", k);
        if (jb.n_samples < 1) return fail(CBESSFM_ERR_INVALID_ARG, "job %d: n_samples < 1", k);
        if ((reinterpret_cast<uintptr_t>(jb.in) | reinterpret_cast<uintptr_t>(jb.out)) & 15u)
            return fail(CBESSFM_ERR_INVALID_ARG, "job %d: in/out must be 16-byte aligned", k);
        if (p->storage != CBESSFM_C64)
            return fail(CBESSFM_ERR_UNSUPPORTED, "job %d: only complex64 storage is supported", k);
        if (k == 0) {
            np = p->n_fft;
            n_sb = p->n_sb;
        } else if (p->n_fft != np || p->n_sb != n_sb) {
            return fail(CBESSFM_ERR_UNSUPPORTED, "job %d: all jobs must share n_fft and bands", k);
        }
        if (p->per_pol)
            return fail(CBESSFM_ERR_UNSUPPORTED, "job %d: the per-polarization NLPR is not supported here", k);
        const long long nb = blocks_for(jb.n_samples, p->V);
        if (nb > (1ll << 30)) return fail(CBESSFM_ERR_UNSUPPORTED, "job %d: too many blocks", k);
        const unsigned long long bytes = (unsigned long long)jb.n_samples * 16ull;
        const uintptr_t i0 = reinterpret_cast<uintptr_t>(jb.in), o0 = reinterpret_cast<uintptr_t>(jb.out);
        if (i0 < o0 + bytes && o0 < i0 + bytes) return fail(CBESSFM_ERR_ALIAS, "job %d: out overlaps in", k);
        desc[k] = make_chain_args(*p);
        desc[k].in = jb.in;
        desc[k].out = jb.out;
        desc[k].L = jb.n_samples;
        desc[k].batch = 1;
        desc[k].n_blocks = (int)nb;
        region = std::max(region, p->region_bytes);
        any_taps = any_taps || desc[k].taps_smem;
        order[k] = k;
    }
    const int E = chain_slots(np, false);
    const int tpf = np / E;
    const int tb = 2 * n_sb * tpf;
    const int max_threads = chain_max_threads(np, false), min_ctas = chain_min_ctas(np, false);
    // per-CTA tables after the block regions: twiddles, plus tap buffers when they fit
    const int tw = chain_tw_bytes(fft_tw_size(np, E));
    int tbl = tw + (any_taps ? chain_taps_bytes(n_sb) : 0);
    int G = choose_blocks_per_cta(tb, region, tpf, n_sb, tbl, max_threads, min_ctas);
    if (G < 1 && any_taps) {
        tbl = tw;
        G = choose_blocks_per_cta(tb, region, tpf, n_sb, tbl, max_threads, min_ctas);
    }
    if (G < 1) return fail(CBESSFM_ERR_UNSUPPORTED, "no CTA shape for n_fft %d, bands %d", np, n_sb);
    // longest processing time first: order jobs by decreasing cost per work item (insertion
    // sort, stable, no temporary buffer)
    for (int k = 1; k < njobs; ++k) {
        const int v = order[k];
        int m = k;
        while (m > 0 && desc[order[m - 1]].n_st < desc[v].n_st) {
            order[m] = order[m - 1];
            --m;
        }
        order[m] = v;
    }
    ChainArgs sorted[kNoallocMaxJobs];
    prefix[0] = 0;
    for (int k = 0; k < njobs; ++k) {
        sorted[k] = desc[order[k]];
        sorted[k].G = G;
        sorted[k].region_bytes = region;
        sorted[k].tbl_bytes = tbl;
        if (tbl == tw) sorted[k].taps_smem = 0;
        const long long n = prefix[k] + (long long)(sorted[k].n_blocks + G - 1) / G;
        if (n > (1ll << 30)) return fail(CBESSFM_ERR_UNSUPPORTED, "too many work items");
        prefix[k + 1] = (int)n;
    }

    if (dev < 0 || dev >= kMaxDevices) return fail(CBESSFM_ERR_UNSUPPORTED, "device index %d", dev);
    unsigned char* scratch = nullptr;
    int n_sm = 0;
    // the set-up's mutex is the one thing here that can throw
    const cbessfm_status st0 = abi_guard([&] { return device_setup(dev, &scratch, &n_sm); });
    if (st0 != CBESSFM_OK) return st0;
    int per_sm = 0;
    e = noalloc_occupancy(np, G * tb, G * region + tbl, &per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (per_sm < 1) return fail(CBESSFM_ERR_UNSUPPORTED, "kernel does not fit an SM");
    const int grid = (int)std::min<long long>((long long)per_sm * n_sm, prefix[njobs]);

    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ChainArgs* d_desc = reinterpret_cast<ChainArgs*>(scratch + kDescOff);
    int* d_prefix = reinterpret_cast<int*>(scratch + kPrefixOff);
    unsigned int* d_counter = reinterpret_cast<unsigned int*>(scratch + kCounterOff);
    // Host-to-device copies from this stack frame: from pageable memory cudaMemcpyAsync returns
    // only after the bytes have been taken, so the frame may end right after.
    e = cudaMemcpyAsync(d_desc, sorted, sizeof(ChainArgs) * njobs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_prefix, prefix, sizeof(int) * (njobs + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess)
        e = noalloc_launch(np, d_desc, d_prefix, njobs, d_counter, n_sb, G, region, tbl, G * tb,
                           grid, st);
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation batched launch");
    return CBESSFM_OK;
}
