// NVTX ranges named after the C-ABI entry points, so that a profiler's timeline, or
// `ncu --nvtx --nvtx-include "darb_bin_sort/"`, can pick out the kernels of one call.  The NVTX3
// headers are header-only: with no tool attached a range costs two calls into empty stubs.
// Building with -DDARB_NVTX=0 compiles the ranges out.
#pragma once

#ifndef DARB_NVTX
#define DARB_NVTX 1
#endif

#if DARB_NVTX
#include <nvtx3/nvToolsExt.h>

namespace darb {

class TraceRange {
  public:
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace darb

#define DARB_TRACE(name) const ::darb::TraceRange darb_trace_range_(name)
#else
#define DARB_TRACE(name) ((void)0)
#endif
