// Error plumbing shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/cluster.h"

namespace fc {

void set_error(const char* fmt, ...);
void clear_error();

// Launch options of an iteration kernel.  win_bytes > 0: a persisting L2
// access window over [win, win + win_bytes) for the launch.
struct LaunchOpt {
  void* win = nullptr;
  size_t win_bytes = 0;
};

template <typename... P, typename... A>
inline void launch_ex(void (*fn)(P...), int grid, int block, size_t smem, cudaStream_t s, const LaunchOpt& o,
                      A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  int na = 0;
  if (o.win_bytes > 0) {
    at[na].id = cudaLaunchAttributeAccessPolicyWindow;
    at[na].val.accessPolicyWindow.base_ptr = o.win;
    at[na].val.accessPolicyWindow.num_bytes = o.win_bytes;
    at[na].val.accessPolicyWindow.hitRatio = 1.0f;
    at[na].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    at[na].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    ++na;
  }
  cfg.attrs = na > 0 ? at : nullptr;
  cfg.numAttrs = na;
  cudaLaunchKernelEx(&cfg, fn, static_cast<A&&>(args)...);
}

}  // namespace fc

#define FC_CUDA(expr)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      fc::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                    __LINE__);                                                        \
      return e_ == cudaErrorMemoryAllocation ? CLUSTER_ENOMEM : CLUSTER_ECUDA;        \
    }                                                                                 \
  } while (0)

#define FC_TRY(expr)                 \
  do {                               \
    cluster_status s_ = (expr);      \
    if (s_ != CLUSTER_OK) return s_; \
  } while (0)

#define FC_EINVAL(...)          \
  do {                          \
    fc::set_error(__VA_ARGS__); \
    return CLUSTER_EINVAL;      \
  } while (0)
