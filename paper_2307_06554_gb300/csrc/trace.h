// NVTX ranges around the library's entry points (plan creation, launches,
// tuning, serving), visible to profilers that record NVTX.  NVTX 3 is
// header-only and costs a few instructions when no tool is attached.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace pm {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace pm
