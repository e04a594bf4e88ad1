// batch.cu -- batched form: many independent DBP jobs (own plan, length, taps, step count) in
// one persistent launch per (N', subband count, storage) group.
//
// cbessfm_batch_create groups the jobs, cuts every job into work items of G consecutive
// overlap-and-save blocks, orders each group's items by decreasing cost (longest processing
// time first: cost = steps + 2 for the entry/exit transforms) and uploads the per-job
// descriptors and the item lists once.  cbessfm_batch_run then only resets one counter per group
// and launches the persistent kernels, so the same batch can be captured in a CUDA graph and
// replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "abi_guard.h"
#include "block_count.h"
#include "device_common.cuh"
#include "internal.h"
#include "trace.h"

struct cbessfm_batch {
    struct Group {
        int np = 0, n_sb = 0, storage = 0;
        int G = 1, threads = 0, region_bytes = 0, tbl_bytes = 0, per_pol = 0, grid = 0;
        int item_off = 0, n_items = 0;
    };
    std::vector<Group> groups;
    // groups after the first run on their own streams, forked from and joined back into the
    // caller's stream, so one group's persistent CTAs take over the SMs that another group's
    // finished CTAs free (empty with CBESSFM_BATCH_SERIAL=1: one group after the other)
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cbessfm::ChainArgs* d_jobs = nullptr;
    int2* d_items = nullptr;
    unsigned int* d_counters = nullptr;
    int njobs = 0;
    long long total_items = 0;
};

namespace cbessfm {
namespace {

void free_batch(cbessfm_batch* b) {
    if (!b) return;
    for (cudaStream_t st : b->side)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->joins)
        if (ev) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->d_jobs);
    cudaFree(b->d_items);
    cudaFree(b->d_counters);
    delete b;
}

}  // namespace
}  // namespace cbessfm

using namespace cbessfm;

extern "C" {

static cbessfm_status batch_create_body(const cbessfm_job* jobs, int njobs, cbessfm_batch** out) {
    if (out == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (jobs == nullptr || njobs < 1) return fail(CBESSFM_ERR_INVALID_ARG, "no jobs");

    std::vector<ChainArgs> args(njobs);
    std::map<std::tuple<int, int, int, int>, std::vector<int>> by_shape;
    int dev = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < njobs; ++k) {
        const cbessfm_job& jb = jobs[k];
        const PlanImpl* p = plan_impl(jb.plan);
        if (p == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "job %d: plan is NULL", k);
        // every plan's tables must be on the current device, where the batch's launches run
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
        const long long nb = blocks_for(jb.n_samples, p->V);
        if (nb > (1ll << 30)) return fail(CBESSFM_ERR_UNSUPPORTED, "job %d: too many blocks", k);
        const unsigned long long sb = p->storage == CBESSFM_C64 ? 16ull : 8ull;
        const unsigned long long bytes = (unsigned long long)jb.n_samples * sb;
        const uintptr_t i0 = reinterpret_cast<uintptr_t>(jb.in), o0 = reinterpret_cast<uintptr_t>(jb.out);
        if (i0 < o0 + bytes && o0 < i0 + bytes) return fail(CBESSFM_ERR_ALIAS, "job %d: out overlaps in", k);
        ChainArgs a = make_chain_args(*p);
        a.in = jb.in;
        a.out = jb.out;
        a.L = jb.n_samples;
        a.batch = 1;
        a.n_blocks = (int)nb;
        args[k] = a;
        by_shape[std::make_tuple(p->n_fft, p->n_sb, (int)p->storage, p->per_pol)].push_back(k);
    }

    int n_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");

    // the groups and work items are built in host containers before the batch and its device
    // memory exist (see abi_guard.h)
    std::vector<cbessfm_batch::Group> groups;
    std::vector<int2> items;
    for (const auto& kv : by_shape) {
        cbessfm_batch::Group gr;
        gr.np = std::get<0>(kv.first);
        gr.n_sb = std::get<1>(kv.first);
        gr.storage = std::get<2>(kv.first);
        gr.per_pol = std::get<3>(kv.first);
        const bool pp = gr.per_pol != 0;
        const int E = chain_slots(gr.np, pp);
        const int tpf = gr.np / E;
        const int tb = 2 * gr.n_sb * tpf;
        const int max_threads = chain_max_threads(gr.np, pp), min_ctas = chain_min_ctas(gr.np, pp);
        bool any_taps = false;
        for (int k : kv.second) {
            gr.region_bytes = std::max(gr.region_bytes, args[k].region_bytes);
            any_taps = any_taps || args[k].taps_smem;
        }
        // per-CTA tables: twiddles, plus the tap buffers if a job stages its taps and they fit
        const int tw = chain_tw_bytes(fft_tw_size(gr.np, E));
        gr.tbl_bytes = tw + (any_taps ? chain_taps_bytes(gr.n_sb) : 0);
        gr.G = choose_blocks_per_cta(tb, gr.region_bytes, tpf, gr.n_sb, gr.tbl_bytes, max_threads,
                                     min_ctas);
        if (gr.G < 1 && any_taps) {
            gr.tbl_bytes = tw;
            gr.G = choose_blocks_per_cta(tb, gr.region_bytes, tpf, gr.n_sb, gr.tbl_bytes,
                                         max_threads, min_ctas);
        }
        if (gr.G < 1)
            return fail(CBESSFM_ERR_UNSUPPORTED, "no CTA shape for n_fft %d, bands %d", gr.np, gr.n_sb);
        gr.threads = gr.G * tb;
        // work items: G consecutive blocks of one job, longest processing time first
        std::vector<std::pair<int, int2>> its;
        for (int k : kv.second) {
            const int cost = args[k].n_st + 2;
            for (int fb = 0; fb < args[k].n_blocks; fb += gr.G) its.push_back({cost, make_int2(k, fb)});
        }
        std::stable_sort(its.begin(), its.end(),
                         [](const std::pair<int, int2>& x, const std::pair<int, int2>& y) { return x.first > y.first; });
        gr.item_off = (int)items.size();
        gr.n_items = (int)its.size();
        for (auto& it : its) items.push_back(it.second);
        for (int k : kv.second) {
            args[k].G = gr.G;                       // informational inside the persistent kernel
            args[k].region_bytes = gr.region_bytes;
            args[k].tbl_bytes = gr.tbl_bytes;
            if (gr.tbl_bytes == tw) args[k].taps_smem = 0;
        }
        int per_sm = 0;
        e = forward_persistent_occupancy(gr.np, gr.storage, gr.threads,
                                         gr.G * gr.region_bytes + gr.tbl_bytes, &per_sm);
        if (e != cudaSuccess || per_sm < 1)
            return e != cudaSuccess ? cuda_fail(e, "occupancy") : fail(CBESSFM_ERR_UNSUPPORTED, "persistent kernel does not fit an SM");
        gr.grid = (int)std::min<long long>((long long)per_sm * n_sm, gr.n_items);
        groups.push_back(gr);
    }

    cbessfm_batch* b = new (std::nothrow) cbessfm_batch;
    if (b == nullptr) return fail(CBESSFM_ERR_OOM, "host allocation of the batch failed");
    b->njobs = njobs;
    b->groups.swap(groups);
    b->total_items = (long long)items.size();

    e = cudaMalloc(&b->d_jobs, sizeof(ChainArgs) * args.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(int2) * std::max<size_t>(1, items.size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(unsigned int) * b->groups.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_jobs, args.data(), sizeof(ChainArgs) * args.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpy(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
    const char* serial = std::getenv("CBESSFM_BATCH_SERIAL");
    if (e == cudaSuccess && b->groups.size() > 1 && !(serial && std::strcmp(serial, "1") == 0)) {
        e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (size_t k = 1; k < b->groups.size() && e == cudaSuccess; ++k) {
            cudaStream_t st = nullptr;
            cudaEvent_t ev = nullptr;
            e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e == cudaSuccess) b->side.push_back(st);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) b->joins.push_back(ev);
        }
    }
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "batch descriptors");
    }
    *out = b;
    return CBESSFM_OK;
}

cbessfm_status cbessfm_batch_create(const cbessfm_job* jobs, int njobs, cbessfm_batch** out) {
    TraceRange trace_range("cbessfm:batch_create");
    clear_error();
    return abi_guard([&] { return batch_create_body(jobs, njobs, out); });
}

cbessfm_status cbessfm_batch_run(const cbessfm_batch* b, cbessfm_stream stream) {
    TraceRange trace_range("cbessfm:batch_run");
    clear_error();
    if (b == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "batch is NULL");
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool fan = !b->side.empty();
    // every group's work counter reset first, on the caller's stream
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned int) * b->groups.size(), st);
    if (e == cudaSuccess && fan) e = cudaEventRecord(b->fork, st);
    for (size_t k = 1; fan && k < b->groups.size() && e == cudaSuccess; ++k)
        e = cudaStreamWaitEvent(b->side[k - 1], b->fork, 0);
    for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
        const cbessfm_batch::Group& gr = b->groups[gi];
        const cudaStream_t gs = (fan && gi > 0) ? b->side[gi - 1] : st;
        e = launch_forward_persistent(gr.np, gr.storage, b->d_jobs, b->d_items + gr.item_off,
                                      gr.n_items, b->d_counters + gi, gr.n_sb, gr.G,
                                      gr.region_bytes, gr.tbl_bytes, gr.per_pol, gr.threads,
                                      gr.grid, gs);
    }
    for (size_t k = 1; fan && k < b->groups.size() && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->joins[k - 1], b->side[k - 1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->joins[k - 1], 0);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batched launch");
    return CBESSFM_OK;
}

cbessfm_status cbessfm_batch_info(const cbessfm_batch* b, int* n_groups, long long* n_items) {
    clear_error();
    if (b == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "batch is NULL");
    if (n_groups) *n_groups = (int)b->groups.size();
    if (n_items) *n_items = b->total_items;
    return CBESSFM_OK;
}

cbessfm_status cbessfm_batch_destroy(cbessfm_batch* b) {
    clear_error();
    if (b == nullptr) return CBESSFM_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    return CBESSFM_OK;
}

}  // extern "C"
