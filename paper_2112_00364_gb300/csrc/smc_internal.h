// smc_internal.h -- host-side helpers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "../../include/smc.h"

namespace smc {

// Record a thread-local error message and return `status`.
smc_status set_error(smc_status status, const char* fmt, ...);

// Map a CUDA error to SMC_ECUDA with a message naming the failed call.
inline smc_status cuda_fail(cudaError_t e, const char* what) {
  return set_error(SMC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SMC_CUDA_TRY(call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return ::smc::cuda_fail(e_, #call); \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// An NVTX range around a host phase of a call (shown by Nsight Systems and
// other NVTX tools; without one attached the calls do nothing).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace smc
