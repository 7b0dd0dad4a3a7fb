// Named NVTX ranges around the library's entry points, so that a profiler's
// timeline shows each call by name (the calls are no-ops when no tool is
// attached).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace bf {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace bf

#define BF_TRACE(name) ::bf::TraceRange bf_trace_range_(name)
