// NVTX ranges around the C-ABI calls that launch kernels, named after the call, so that a
// profiler timeline (or ncu --nvtx --nvtx-include "fastfca_iterate/") shows which library call
// issued which kernels.  NVTX v3 is header-only: with no tool attached a range costs a branch.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace ffca {

class TraceRange {
 public:
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace ffca

#define FFCA_TRACE(name) const ::ffca::TraceRange ffca_trace_range_(name)
