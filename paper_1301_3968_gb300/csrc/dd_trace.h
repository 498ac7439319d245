// Tracing and logging of the host side.
//
// DD_TRACE(name) opens an NVTX range named after the entry point for the rest of the
// scope, so a timeline tool (Nsight Systems, or ncu's NVTX filter) shows every library
// call around its kernels; with no tool attached an NVTX call is a cheap no-op.
//
// dd::log_msg(level, ...) writes one line "[dd] ..." to stderr when the DD_LOG environment
// variable (read once) is at least `level`: 1 = plan decisions (tap-sum method, CTA
// shape, stage size, staged row length, shared memory), autotuner results and batch
// bindings; 2 = also every device call with its sizes.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace dd {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

int log_level();
void log_msg(int level, const char* fmt, ...) __attribute__((format(printf, 2, 3)));

}  // namespace dd

#define DD_TRACE(name) ::dd::TraceRange dd_trace_range_(name)
