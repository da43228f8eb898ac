// nvtx_range.h -- named NVTX ranges around the public C-ABI calls, so that a
// profiler timeline shows which call issued which kernels.  NVTX v3 is
// header-only: with no tool attached a push/pop is one indirect call.
// Define PROXMF_NO_NVTX to compile the ranges out.
#pragma once

#ifndef PROXMF_NO_NVTX
#include <nvtx3/nvToolsExt.h>
#endif

namespace proxmf {

struct NvtxRange {
#ifndef PROXMF_NO_NVTX
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
#else
    explicit NvtxRange(const char *) {}
#endif
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace proxmf

#define PROXMF_RANGE(name) ::proxmf::NvtxRange proxmf_nvtx_range_(name)
