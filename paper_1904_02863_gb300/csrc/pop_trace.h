// NVTX ranges around the C-ABI calls, so that a profiler can attribute kernels to the call that
// launched them (for instance ncu --nvtx --nvtx-include "pop_loglik/").  NVTX3 is header-only;
// with no tool attached a range costs a few nanoseconds.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace pop {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace pop
