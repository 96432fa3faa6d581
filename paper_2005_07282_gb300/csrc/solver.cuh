// Internal definitions shared by the solver translation units (not part of
// the C ABI): the device matrix in SELL-32 form and its row kernel, the
// per-solve argument and state records, and the matrix handle.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <tuple>

#include "device.cuh"
#include "small.h"
#include "rpcg.h"

namespace rpcg {

struct PassScratch;  // grid-reduction scratch of the single-system passes (pcg.cu)

// Per-solve arguments, written by the host before every launch of the graph.
struct SolveArgs {
  const double* b;
  double* x;
  double* history;
  double tol;
  int max_iter;
  int fpe_size;
  int fpe_strict;
  int variant;
  int use_cond;  // 1: running inside the graph (set the while node's condition)
};

// Solver state, device resident.
struct SolveState {
  double rho, beta, beta_old, tau, gamma, bnorm, rel;
  int iter, status, bad_row, bzero, redo, fpe_inexact, active, fpe_p;  // fpe_p: expansion size in use
  double zr;    // fpe variant, multi-pass path: <z,r> of pass B1, finished with <r,r> in pass B2
  int zr_lost;  // and whether its expansions lost bits (or met a non-finite operand)
  int pad;
};

// Device matrix.  The handle stores A in SELL-32 form: rows are grouped
// in slices of 32 consecutive rows, and slice s keeps the k-th entry of its
// 32 rows contiguously at sptr[s] + 32 k + lane, for k below the longest row
// of the slice (shorter rows are padded; padded entries are never used).
// Each row keeps its CSR storage order, so the k-th FMA of a row is the
// same as in CSR.  A warp (32 consecutive rows) then reads 256 contiguous
// bytes of values and 128 of columns per step, straight from HBM.
struct MatDev {
  int n, nnz;
  const int* rowptr;     // CSR row pointers (row lengths), n + 1
  const long long* sptr; // slice offsets, n / 32 + 1 (rounded up)
  const double* val;     // SELL-32 values
  const int* col;        // SELL-32 columns
};

__device__ __forceinline__ long long sell_index(const MatDev& m, int row, int k) {
  return __ldg(m.sptr + (row >> 5)) + 32ll * k + (row & 31);
}

// ---- SpMV: y = A x, each row summed left to right with fma from +0 (Sec. 4.3).
//
// One thread per row, a warp per 32-row slice, CTAs persistent over the
// slices.  The matrix stream is read with coalesced streaming loads; the
// gathers x[col] go through L1/L2 (stencil locality).  The loads of the
// next 8 entries are issued before the FMAs of the current 8.
//
// The loads run over the slice's length (its longest row, from the slice
// offsets), not the row's own: padding entries hold column 0 and value 0,
// so every load stays in range, and the loads need not wait for the row
// pointers.  Only entries k < len (the row's length) enter the fma chain.
// The row whose entry k sits at base + 32 k, of length len, in a slice of
// length slen >= len.
__device__ __forceinline__ double sell_row_at(const MatDev& m, long long base, int len, int slen,
                                              const double* __restrict__ x) {
  constexpr int U = 8;
  const double* __restrict__ vp = m.val + base;
  const int* __restrict__ cp = m.col + base;
  double acc = 0.0;
  double xa[U], va[U];
#pragma unroll
  for (int j = 0; j < U; j++) {
    xa[j] = 0.0;
    va[j] = 0.0;
    if (j < slen) {
      va[j] = __ldcs(vp + 32 * j);
      xa[j] = __ldg(x + __ldcs(cp + 32 * j));
    }
  }
  for (int k = 0; k < slen; k += U) {
    double xb[U], vb[U];
#pragma unroll
    for (int j = 0; j < U; j++) {
      const int kk = k + U + j;
      xb[j] = 0.0;
      vb[j] = 0.0;
      if (kk < slen) {
        vb[j] = __ldcs(vp + 32ll * kk);
        xb[j] = __ldg(x + __ldcs(cp + 32ll * kk));
      }
    }
#pragma unroll
    for (int j = 0; j < U; j++)
      if (k + j < len) acc = __fma_rn(va[j], xa[j], acc);
#pragma unroll
    for (int j = 0; j < U; j++) {
      xa[j] = xb[j];
      va[j] = vb[j];
    }
  }
  return acc;
}

// Slice offset of `row`'s slice and that slice's length (entries per row).
__device__ __forceinline__ long long sell_slice(const MatDev& m, int row, int& slen) {
  const long long s0 = __ldg(m.sptr + (row >> 5)), s1 = __ldg(m.sptr + (row >> 5) + 1);
  slen = (int)((s1 - s0) >> 5);
  return s0;
}

__device__ __forceinline__ double sell_row(const MatDev& m, int row, const double* __restrict__ x) {
  int slen;
  const long long s0 = sell_slice(m, row, slen);
  const int len = __ldg(m.rowptr + row + 1) - __ldg(m.rowptr + row);
  return sell_row_at(m, s0 + (row & 31), len, slen, x);
}

// Two rows at once (ya = row ra of A x, yb = row rb): when both slices have
// at most 8 entries per row, the loads of both rows are issued together, so
// a thread keeps two rows' memory chains in flight with the registers
// sell_row spends on prefetching a row's next 8 entries.  Longer rows take
// sell_row.  Each row's fma chain is the one of sell_row.
__device__ __forceinline__ void sell_rows2(const MatDev& m, int ra, int rb, const double* __restrict__ x, double& ya,
                                           double& yb) {
  constexpr int U = 8;
  int sa, sb;
  const long long ba = sell_slice(m, ra, sa) + (ra & 31), bb = sell_slice(m, rb, sb) + (rb & 31);
  if (sa > U || sb > U) {
    ya = sell_row(m, ra, x);
    yb = sell_row(m, rb, x);
    return;
  }
  const int la = __ldg(m.rowptr + ra + 1) - __ldg(m.rowptr + ra);
  const int lb = __ldg(m.rowptr + rb + 1) - __ldg(m.rowptr + rb);
  double va[U], xa[U], vb[U], xb[U];
#pragma unroll
  for (int j = 0; j < U; j++) {
    va[j] = 0.0;
    xa[j] = 0.0;
    vb[j] = 0.0;
    xb[j] = 0.0;
    if (j < sa) {
      va[j] = __ldcs(m.val + ba + 32 * j);
      xa[j] = __ldg(x + __ldcs(m.col + ba + 32 * j));
    }
    if (j < sb) {
      vb[j] = __ldcs(m.val + bb + 32 * j);
      xb[j] = __ldg(x + __ldcs(m.col + bb + 32 * j));
    }
  }
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int j = 0; j < U; j++) {
    if (j < la) a = __fma_rn(va[j], xa[j], a);
    if (j < lb) b = __fma_rn(vb[j], xb[j], b);
  }
  ya = a;
  yb = b;
}

struct GraphKey {
  int variant, block, grid;
  bool operator<(const GraphKey& o) const {
    return std::tie(variant, block, grid) < std::tie(o.variant, o.block, o.grid);
  }
};

}  // namespace rpcg

struct rpcg_matrix_s {
  rpcg::MatDev m{};
  int* rowptr = nullptr;
  long long* sptr = nullptr;  // SELL-32 slice offsets
  int* col = nullptr;         // SELL-32 columns
  double* val = nullptr;      // SELL-32 values
  double* inv = nullptr;
  double* r = nullptr;
  double* d = nullptr;
  double* w = nullptr;
  double* bx = nullptr;  // staging for rpcg_solve_host: b then x
  rpcg::SolveArgs* args = nullptr;
  rpcg::SolveState* state = nullptr;
  rpcg::PassScratch* scratch = nullptr;
  rpcg::SolveArgs* h_args = nullptr;    // pinned
  rpcg::SolveState* h_state = nullptr;  // pinned
  std::map<rpcg::GraphKey, cudaGraphExec_t> graphs;
  std::map<rpcg::GraphKey, cudaGraph_t> graph_defs;
  std::map<rpcg::GraphKey, cudaGraphNode_t> x0_nodes;
  rpcg::SmallPlan small;  // the cluster-resident path for small systems
  int device = 0;
};

