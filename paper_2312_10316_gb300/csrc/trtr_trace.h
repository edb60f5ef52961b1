// trtr_trace.h -- NVTX ranges around the library's host calls (step, moments, reductions,
// adjoint, batch step), so that a timeline tool shows which call enqueued which kernels.  NVTX
// v3 is header-only: without a tool attached every range is a no-op.  Not part of the ABI.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace trtr {

// Pushes a named range for the lifetime of the object.
class TraceRange {
   public:
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace trtr
