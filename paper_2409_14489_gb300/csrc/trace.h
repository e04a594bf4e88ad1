// trace.h -- NVTX ranges around the C-ABI entry points, so a profiler's timeline (ncu with
// --nvtx, or any NVTX-aware tool) shows which library call issued which kernels.  Header-only
// NVTX v3: without an attached tool each range costs one call into an empty stub.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace cbessfm {

// Scoped range named "cbessfm:<call>"; the name must be a string literal.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace cbessfm
