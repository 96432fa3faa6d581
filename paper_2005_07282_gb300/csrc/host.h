// Host-side helpers shared by the library's translation units: error
// reporting for rpcg_last_error(), CUDA call checking, device attributes.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>

#include "rpcg.h"

namespace rpcg {

// Record a message for rpcg_last_error() on this host thread.
void set_error(const char* fmt, ...);
void clear_error();

// Number of SMs of the current device (cached per device).
int sm_count();

}  // namespace rpcg

#define RPCG_CUDA_TRY(call)                                                                          \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) {                                                                         \
      rpcg::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);  \
      return RPCG_ERR_CUDA;                                                                          \
    }                                                                                                \
  } while (0)

#define RPCG_CHECK_ARG(cond, msg)         \
  do {                                    \
    if (!(cond)) {                        \
      rpcg::set_error("%s", msg);         \
      return RPCG_ERR_INVALID;            \
    }                                     \
  } while (0)
