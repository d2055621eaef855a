// NVTX ranges around the stages of a likelihood call (host side, at enqueue):
// a profiler attached to the process sees which stage launched each kernel
// (ncu: --nvtx --nvtx-include "lisa_td/tdi/").  NVTX 3 is header-only; with
// no tool attached a push or pop tests one function pointer and returns.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lisa {

// names of the LISA_TD_NSTAGE stages of lisa_td_loglike_batch and of
// lisa_td_het_loglike, in stage order
extern const char* const kStageRange[7];
extern const char* const kHetStageRange[7];

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace lisa
