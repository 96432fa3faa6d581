// The cluster-resident small-system solver (small.cu): its per-handle plan
// and the entry points the solve path calls.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

#include "rpcg.h"

namespace rpcg {

constexpr int kSmallMaxCtas = 16;                 // CTAs of the cluster (16 needs the non-portable size)
constexpr int kSmallMaxR = 1024;                  // rows per CTA
constexpr size_t kSmallMaxSmem = 200 * 1024;      // shared memory per CTA

// How a handle is split over the cluster (ok = 0: the system is too large
// for the cluster path).  checked: 0 not yet tried, 1 the cluster fits on
// this GPU, -1 it does not.
struct SmallPlan {
  int ok = 0;
  int R = 0, log2R = 0, nct = 0, emax = 0;
  size_t smem = 0;
  int checked = 0;
};

// Plan from the host copy of the SELL-32 slice offsets (nslices + 1 values).
void small_plan(rpcg_matrix_s* A, const long long* hsptr, int n);

// 1 if rpcg_solve runs (A, v, o) on the cluster path.
int small_path(rpcg_matrix_s* A, int v, const rpcg_opts& o);

// Run the solve as one cluster launch if the handle and variant allow it
// (*used = true); otherwise leave *used false and launch nothing.
rpcg_status small_solve(rpcg_matrix_s* A, const double* b, double* x, int v, const rpcg_opts& o, cudaStream_t s,
                        bool* used);

}  // namespace rpcg
