// NVTX ranges around the library's stages (expansion, propagation, host
// pipeline chunks, serving batches, surrogate steps), so that a timeline
// profiler shows them by name.  NVTX 3 is header-only; without an attached
// tool a range costs one check.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace ppk {

class NvtxRange {
 public:
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace ppk
