// NVTX ranges for timeline tools (nsys, ncu --nvtx): one around every call
// of the C ABI and, when kernels are launched directly instead of replayed
// from a captured graph (HVP_NO_GRAPH, hvp_profile), one around each pass,
// block or gate launch, named with its index. NVTX3 is header-only: with no
// tool attached, each push or pop only tests one function pointer.
#pragma once

#include <cstdio>

#include <nvtx3/nvToolsExt.h>

namespace hvp {

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    NvtxRange(const char* what, int index) {
        char buf[64];
        std::snprintf(buf, sizeof buf, "%s %d", what, index);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace hvp
