// ac_trace.h - NVTX ranges around the library's entry points, in the "acgpu"
// domain, so that a profiler (nsys, or ncu with --nvtx) can attribute kernels
// and copies to the call that issued them, e.g.
//   ncu --nvtx --nvtx-include "acgpu@ac_scan/" ...
// NVTX is header-only; with no tool attached a range costs a check of one
// function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

inline nvtxDomainHandle_t ac_trace_domain() {
    static nvtxDomainHandle_t d = nvtxDomainCreateA("acgpu");
    return d;
}

// Pushes a range named `name` (a string literal) for the lifetime of the object.
class AcRange {
   public:
    explicit AcRange(const char* name) {
        nvtxEventAttributes_t a{};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(ac_trace_domain(), &a);
    }
    ~AcRange() { nvtxDomainRangePop(ac_trace_domain()); }
    AcRange(const AcRange&) = delete;
    AcRange& operator=(const AcRange&) = delete;
};
