// NVTX ranges around the library's entry points, so that a timeline tool
// (Nsight Systems, or ncu's --nvtx filters) shows every call by its C name.
// NVTX v3 is header-only: with no tool attached a range costs a few
// nanoseconds and loads nothing. Building with -DTVOLAP_NO_NVTX removes them.
#pragma once

#ifndef TVOLAP_NO_NVTX
#include <nvtx3/nvToolsExt.h>

class TraceRange {
public:
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

#define TVOLAP_TRACE() TraceRange tvolap_trace_range_(__func__)
#else
#define TVOLAP_TRACE() ((void)0)
#endif
