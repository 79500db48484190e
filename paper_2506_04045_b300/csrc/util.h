// Error plumbing shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/cluster.h"

namespace fc {

void set_error(const char* fmt, ...);
void clear_error();

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
