// NVTX ranges around the library's host-level calls and serving batches, so
// that a profiler's timeline shows them (header-only NVTX 3: without a
// profiler attached a range costs a few nanoseconds).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace amc {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace amc
