// trace.h -- NVTX ranges around the library's entry points. The NVTX3 headers
// are header-only: without an attached tool (a timeline profiler, or Nsight
// Compute's --nvtx include filters) a range costs a call and a branch; with one,
// every ABI call of a market or batch shows up as a named range on the calling
// thread, around the kernels it enqueued.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace tu {

class TraceRange {
 public:
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace tu

#define TU_TRACE(name) ::tu::TraceRange tu_trace_range_(name)
