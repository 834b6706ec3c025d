// nvtx_range.h -- named host-side ranges around the library's stages (advance,
// particle segments, compaction, planet chunks, read, checkpoint), for
// profilers that read NVTX (Nsight Systems timelines, ncu --nvtx filters).
// NVTX3 is header-only: without an attached tool each range costs a few
// nanoseconds and nothing else.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace glisse {
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace glisse
