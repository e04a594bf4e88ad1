// host_pipeline.cu -- backpropagation of host-resident fields with the transfers overlapped.
//
// A receiver's samples usually arrive in host memory.  cbessfm_backpropagate_host copies the
// batch in by groups of realizations on one copy stream, runs the chain kernel in launches of
// OLS blocks that alternate between the caller's stream and a second compute stream, and copies
// each group out on a second copy stream as soon as the launches holding its last block have
// finished.  A launch waits only for the copies of the realizations its blocks read.  With two
// compute streams each launch is one CTA per SM, so two launches together fill the GPU and the
// last partial wave of one overlaps the next; with one stream, launches are whole waves of
// resident CTAs.  Launches are cut at CTA counts, not at realization boundaries: a launch of one
// realization's blocks would leave most SMs idle in its last wave.  The time approaches the
// kernel time plus one group's copy in and out.  The copy and compute streams and the events
// belong to the plan and are created at the first call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <mutex>
#include <new>

#include "abi_guard.h"
#include "block_count.h"
#include "device_common.cuh"
#include "internal.h"
#include "trace.h"

namespace cbessfm {

constexpr int kMaxCopyGroups = 64;

struct HostPipeline {
    std::mutex mu;                    // one pipelined call per plan at a time
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaStream_t comp2 = nullptr;     // second compute stream: consecutive launches alternate
    cudaEvent_t start = nullptr, end = nullptr;
    cudaEvent_t launched[2] = {};     // after the latest launch on the caller's stream / comp2
    cudaEvent_t copied[kMaxCopyGroups] = {};
    int n_sm = 0;                     // SM count of the plan's device
};

void destroy_host_pipeline(HostPipeline* hp) {
    if (hp == nullptr) return;
    if (hp->h2d) cudaStreamDestroy(hp->h2d);
    if (hp->d2h) cudaStreamDestroy(hp->d2h);
    if (hp->comp2) cudaStreamDestroy(hp->comp2);
    for (int k = 0; k < 2; ++k)
        if (hp->launched[k]) cudaEventDestroy(hp->launched[k]);
    if (hp->start) cudaEventDestroy(hp->start);
    if (hp->end) cudaEventDestroy(hp->end);
    for (int k = 0; k < kMaxCopyGroups; ++k)
        if (hp->copied[k]) cudaEventDestroy(hp->copied[k]);
    delete hp;
}

namespace {

std::mutex g_create_mu;

cudaError_t create_pipeline(HostPipeline* hp, int device) {
    const unsigned flags = cudaEventDisableTiming;
    cudaError_t e = cudaDeviceGetAttribute(&hp->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->d2h, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->comp2, cudaStreamNonBlocking);
    for (int k = 0; e == cudaSuccess && k < 2; ++k)
        e = cudaEventCreateWithFlags(&hp->launched[k], flags);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp->start, flags);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp->end, flags);
    for (int k = 0; e == cudaSuccess && k < kMaxCopyGroups; ++k)
        e = cudaEventCreateWithFlags(&hp->copied[k], flags);
    return e;
}

}  // namespace
}  // namespace cbessfm

using namespace cbessfm;

extern "C" {

static cbessfm_status backpropagate_host_body(cbessfm_plan* plan, const void* host_in,
                                              void* host_out, void* dev_in, void* dev_out,
                                              int64_t n_samples, int batch, int launch_blocks,
                                              cbessfm_stream stream) {
    if (plan == nullptr) return fail(CBESSFM_ERR_INVALID_ARG, "plan is NULL");
    if (!host_in || !host_out || !dev_in || !dev_out)
        return fail(CBESSFM_ERR_INVALID_ARG, "host_in/host_out/dev_in/dev_out is NULL");
    if (n_samples < 1 || batch < 1 || launch_blocks < 0)
        return fail(CBESSFM_ERR_INVALID_ARG, "n_samples and batch must be >= 1, launch_blocks >= 0");
    const PlanImpl& p = plan->impl;
    const size_t sample_bytes = p.storage == CBESSFM_C64 ? 16 : 8;
    const size_t per_seq = (size_t)n_samples * sample_bytes;
    if ((per_seq & 15) && batch > 1)
        return fail(CBESSFM_ERR_INVALID_ARG, "each realization must span a multiple of 16 bytes");
    const long long n_blocks = blocks_for(n_samples, p.V);
    if (too_many_blocks(n_blocks, batch))
        return fail(CBESSFM_ERR_UNSUPPORTED, "too many blocks in one call");
    const int total = (int)(n_blocks * batch);
    const uintptr_t di = reinterpret_cast<uintptr_t>(dev_in), dO = reinterpret_cast<uintptr_t>(dev_out);
    if ((di | dO) & 15u) return fail(CBESSFM_ERR_INVALID_ARG, "dev_in/dev_out must be 16-byte aligned");
    if (di < dO + per_seq * batch && dO < di + per_seq * batch)
        return fail(CBESSFM_ERR_ALIAS, "dev_out overlaps dev_in");
    {
        std::lock_guard<std::mutex> lk(g_create_mu);
        if (plan->pipe == nullptr) {
            HostPipeline* hp = new (std::nothrow) HostPipeline;
            if (hp == nullptr) return fail(CBESSFM_ERR_OOM, "host allocation of the pipeline failed");
            const cudaError_t e = create_pipeline(hp, p.device);
            if (e != cudaSuccess) {
                destroy_host_pipeline(hp);
                return cuda_fail(e, "pipeline streams/events");
            }
            plan->pipe = hp;
        }
    }
    HostPipeline& hp = *plan->pipe;
    std::lock_guard<std::mutex> call_lock(hp.mu);
    // CTAs per launch: one wave of resident CTAs unless the caller fixes the blocks per launch
    // (rounded up to whole CTAs of G blocks)
    int wave = hp.n_sm * (resident_blocks(p.G, p.threads / p.G, p.region_bytes, p.tbl_bytes,
                                          chain_max_threads(p.n_fft, p.per_pol != 0),
                                          chain_min_ctas(p.n_fft, p.per_pol != 0)) /
                          p.G);
    if (wave < 1) wave = 1;
    // consecutive launches alternate between the caller's stream and the pipeline's second
    // compute stream, so a launch's last partial wave overlaps the next launch instead of
    // draining the GPU (they write disjoint blocks); CBESSFM_PIPELINE_STREAMS=1 keeps one stream
    int n_comp = 2;
    if (const char* env = std::getenv("CBESSFM_PIPELINE_STREAMS")) n_comp = std::atoi(env) == 1 ? 1 : 2;
    // automatic sizing. Two compute streams: launches of one CTA per SM each (half a wave at two
    // resident CTAs per SM), so the two streams together keep one wave in flight and the copy
    // out of each finished group starts early; on the c2 workload 76, 114, 152, 190, 228 CTAs
    // per launch gave 1.557, 1.543, 1.176, 1.378, 1.261 ms per step (one stream with the sizing
    // below: 1.300 ms on the same GPU). One stream: one wave first (it waits only for the copies
    // of the blocks it reads), then two waves per launch (1, 2, 3 waves gave 1.217, 1.204,
    // 1.235 ms, everything after the first wave in one launch 1.669 ms); CBESSFM_PIPELINE_WAVES
    // overrides the later count (tuning)
    int later_waves = 2;
    if (const char* env = std::getenv("CBESSFM_PIPELINE_WAVES")) later_waves = std::max(1, std::atoi(env));
    const int auto_first = n_comp == 2 ? hp.n_sm : wave;
    const int auto_later = n_comp == 2 ? hp.n_sm : later_waves * wave;
    const int first_launch = launch_blocks > 0 ? (launch_blocks + p.G - 1) / p.G : auto_first;
    const int per_launch = launch_blocks > 0 ? first_launch : auto_later;
    const int n_ctas = (total + p.G - 1) / p.G;
    // copy groups of `cg` realizations (at most kMaxCopyGroups groups)
    const int cg = (batch + kMaxCopyGroups - 1) / kMaxCopyGroups;
    const int n_groups = (batch + cg - 1) / cg;

    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const cudaStream_t comp[2] = {st, hp.comp2};
    cudaError_t e = cudaEventRecord(hp.start, st);              // after the caller's earlier work
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.h2d, hp.start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.d2h, hp.start, 0);
    if (e == cudaSuccess && n_comp == 2) e = cudaStreamWaitEvent(hp.comp2, hp.start, 0);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline start");
    const unsigned char* hin = static_cast<const unsigned char*>(host_in);
    unsigned char* hout = static_cast<unsigned char*>(host_out);
    unsigned char* din = static_cast<unsigned char*>(dev_in);
    unsigned char* dout = static_cast<unsigned char*>(dev_out);
    auto group_span = [&](int g, size_t* off, size_t* bytes) {
        const int r0 = g * cg, r1 = r0 + cg < batch ? r0 + cg : batch;
        *off = (size_t)r0 * per_seq;
        *bytes = (size_t)(r1 - r0) * per_seq;
        return r1;                                              // one past the group's last realization
    };
    for (int g = 0; g < n_groups; ++g) {                        // the copy engine runs them in order
        size_t off, bytes;
        group_span(g, &off, &bytes);
        e = cudaMemcpyAsync(din + off, hin + off, bytes, cudaMemcpyHostToDevice, hp.h2d);
        if (e == cudaSuccess) e = cudaEventRecord(hp.copied[g], hp.h2d);
        if (e != cudaSuccess) return cuda_fail(e, "pipeline copy in");
    }
    int waited[2] = {-1, -1}, out_next = 0;     // groups waited for per compute stream / copied out
    bool used2 = false;
    for (int c0 = 0, li = 0; c0 < n_ctas; ++li) {
        const int want = c0 == 0 ? first_launch : per_launch;
        const int nc = n_ctas - c0 > want ? want : n_ctas - c0;
        const int i1 = (c0 + nc) * p.G < total ? (c0 + nc) * p.G : total;   // items [c0 G, i1)
        const int g_in = (int)((i1 - 1) / n_blocks) / cg;       // last group the launch reads
        const int cs = n_comp == 2 ? (li & 1) : 0;
        used2 = used2 || cs == 1;
        if (g_in > waited[cs]) {
            e = cudaStreamWaitEvent(comp[cs], hp.copied[g_in], 0);
            if (e != cudaSuccess) return cuda_fail(e, "pipeline wait for copy in");
            waited[cs] = g_in;
        }
        const cbessfm_status s = forward_range(plan, din, dout, n_samples, batch, c0, nc,
                                               reinterpret_cast<cbessfm_stream>(comp[cs]));
        if (s != CBESSFM_OK) return s;
        e = cudaEventRecord(hp.launched[cs], comp[cs]);
        if (e != cudaSuccess) return cuda_fail(e, "pipeline launch event");
        // groups whose every block is now computed go out in one copy
        int g_end = out_next;
        while (g_end < n_groups) {
            size_t off, bytes;
            const int r1 = group_span(g_end, &off, &bytes);
            if ((long long)r1 * n_blocks > i1) break;
            ++g_end;
        }
        if (g_end > out_next) {
            size_t off0, b0, off1, b1;
            group_span(out_next, &off0, &b0);
            group_span(g_end - 1, &off1, &b1);
            // every launch so far is complete once the latest launch on each compute stream is
            // (each stream runs its own launches in order); a wait binds to the current record
            e = cudaStreamWaitEvent(hp.d2h, hp.launched[0], 0);
            if (e == cudaSuccess && used2) e = cudaStreamWaitEvent(hp.d2h, hp.launched[1], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hout + off0, dout + off0, off1 + b1 - off0,
                                    cudaMemcpyDeviceToHost, hp.d2h);
            if (e != cudaSuccess) return cuda_fail(e, "pipeline copy out");
            out_next = g_end;
        }
        c0 += nc;
    }
    e = cudaEventRecord(hp.end, hp.d2h);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, hp.end, 0);   // completion on `stream`
    if (e != cudaSuccess) return cuda_fail(e, "pipeline end");
    return CBESSFM_OK;
}

cbessfm_status cbessfm_backpropagate_host(cbessfm_plan* plan, const void* host_in, void* host_out,
                                          void* dev_in, void* dev_out, int64_t n_samples,
                                          int batch, int launch_blocks, cbessfm_stream stream) {
    TraceRange trace_range("cbessfm:backpropagate_host");
    clear_error();
    // the pipeline's mutexes are the one thing here that can throw
    return abi_guard([&] {
        return backpropagate_host_body(plan, host_in, host_out, dev_in, dev_out, n_samples, batch,
                                       launch_blocks, stream);
    });
}

}  // extern "C"
