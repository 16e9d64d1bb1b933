// A named NVTX range for the extent of a library call, so that a timeline
// tool attached to the process shows the C-ABI calls beside the kernels they
// launch.  Without a tool the push and pop return at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lbmp {

struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace lbmp
