// pcs_trace.h -- NVTX ranges around the library's public entry points, so that a
// profiler's timeline shows which call a kernel belongs to.  NVTX3 is header-only
// and its calls return at once when no tool is attached.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace pcs {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace pcs

#define PCS_TRACE(name) ::pcs::TraceRange pcs_trace_range_(name)
