// NVTX ranges around the library's entry points, so that a profiler's
// timeline (nsys, or ncu with --nvtx) shows which call a kernel belongs to.
// NVTX v3 is header-only; with no tool attached a range costs a few
// nanoseconds.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace ts {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace ts
