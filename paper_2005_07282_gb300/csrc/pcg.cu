// Jacobi-PCG on one GPU: matrix handle, SpMV, the fused passes of one
// iteration and the CUDA graph that runs the whole loop on the device.
//
// One iteration of Fig. 2 (S8 next to S6) is three streaming passes over
// the vectors, each ending in a grid-wide reduction finished by the last
// CTA to arrive (the single-GPU form of the paper's Reduce + Round + Bcast,
// Listing 3 / Listing 4):
//   pass A  S1 + S2   w = A d (rows summed left to right with fma) and the
//                     dot <d, w> deposited from registers; last CTA: rho.
//   pass B  S3-S6,S8  x = fma(rho, d, x), r = fma(-rho, w, r), z = inv .* r
//                     (z is not stored), <z, r> and <r, r> deposited; last
//                     CTA: beta, tau, gamma = beta / beta', relres, the loop
//                     condition (cudaGraphSetConditional).
//   pass C  S7        d = fma(gamma, d, inv .* r).
// This merges S1 with S2 and S4 with S5 and S6 -- the task overlap of
// Sec. 3.3 turned into kernel fusion.  The loop body is the child graph of a
// conditional while node, so no host round trip happens per iteration.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "device.cuh"
#include "host.h"
#include "solver.cuh"

namespace rpcg {

constexpr int kMaxPassGrid = 4096;
constexpr int kMaxRows = (1 << 30) + ((1 << 30) - (1 << 25));  // 2^31 - 2^25

// Grid-reduction scratch of one pass: up to three simultaneous dots.
struct PassScratch {
  unsigned long long digits[3][kNDig];  // exact: global accumulators (cleared by the last CTA)
  unsigned int counter;                 // CTAs arrived (reset by the last CTA)
  unsigned int flags;                   // bit 0: non-finite operand; bit 1 + j: dot j lost bits (fpe)
  double partials[3][kMaxPassGrid];     // plain: CTA partial sums
};

// ------------------------------------------------------------------ reducers

struct FinalScratch {  // shared memory of the CTA and grid reductions
  long long dig[kNDig];
  uint32_t D[kNDig];
  double sw[32];
  double value[3];
  int lost[3];
  int slost;
  int range[2];
  bool last;
};


// Per-thread state of NACC simultaneous dot products for variant V.
template <int V, int NACC>
struct Reducer {
  Window win[NACC];          // exact
  double res[NACC][kFpeMax]; // fpe
  double err[NACC][kFpeMax];
  double acc[NACC];          // plain
  bool lost[NACC];
  bool bad;
};

template <int V, int NACC>
__device__ __forceinline__ void red_init(Reducer<V, NACC>& R) {
#pragma unroll
  for (int j = 0; j < NACC; j++) {
    if constexpr (V == RPCG_EXBLAS) window_init(R.win[j]);
    if constexpr (V == RPCG_FPE) {
#pragma unroll
      for (int i = 0; i < kFpeMax; i++) R.res[j][i] = R.err[j][i] = 0.0;
    }
    if constexpr (V == RPCG_PLAIN) R.acc[j] = 0.0;
    R.lost[j] = false;
  }
  R.bad = false;
}

// shared memory of the reducers: exact and fpe need NACC long accumulators
// with copies (fpe: the threads' expansions meet there)
template <int V, int NACC>
__host__ __device__ constexpr size_t red_smem_bytes() {
  return V != RPCG_PLAIN ? (size_t)NACC * kNDig * kCopies * sizeof(unsigned long long) : 0;
}

// Carve the reducer's shared memory: [long accumulators] then FinalScratch.
template <int V, int NACC>
__device__ __forceinline__ FinalScratch* red_carve(unsigned char* base, unsigned long long*& sacc) {
  sacc = reinterpret_cast<unsigned long long*>(base);
  FinalScratch* fs = reinterpret_cast<FinalScratch*>(base + red_smem_bytes<V, NACC>());
  return fs;
}

// fpe: fpe_dot_step (twoprod on the integer pipe, the Accumulate cascades
// with two_sum_fast in the result and two_sum_split in the error expansion).
template <int V, int NACC>
__device__ __forceinline__ void red_add(Reducer<V, NACC>& R, unsigned long long* sacc, int j, double a, double b,
                                        int p) {
  if constexpr (V == RPCG_EXBLAS) {
    const ExactProd e = exact_product(a, b);
    R.bad |= e.bad;
    exact_deposit(R.win[j], sacc + j * kNDig * kCopies, threadIdx.x & (kCopies - 1), e);
  } else if constexpr (V == RPCG_FPE) {
    if (!is_finite_bits(a) || !is_finite_bits(b)) R.bad = true;
    else R.lost[j] |= fpe_dot_step(R.res[j], R.err[j], p, a, b, R.bad);
  } else {
    R.acc[j] = __fma_rn(a, b, R.acc[j]);
  }
}

// CTA part of the reduction (all threads), then the grid part by the last
// CTA.  Returns true in every thread of the last CTA; fs->value[j] then
// holds the dot values and fs->lost[j] whether an expansion lost bits (fpe)
// or an operand was non-finite (all variants report NaN for those).
template <int V, int NACC, int BLOCK>
__device__ bool red_finish(Reducer<V, NACC>& R, unsigned long long* sacc, PassScratch* ws, FinalScratch* fs, int p) {
  const int copy = threadIdx.x & (kCopies - 1);
  if constexpr (V == RPCG_EXBLAS) {
#pragma unroll
    for (int j = 0; j < NACC; j++) window_flush(R.win[j], sacc + j * kNDig * kCopies, copy);
    if (R.bad) atomicOr(&ws->flags, 1u);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NACC; j++) smem_to_global(sacc + j * kNDig * kCopies, ws->digits[j]);
  } else if constexpr (V == RPCG_FPE) {
    // each thread merges its error expansion into its result expansion
    // (Alg. 3); the threads' expansions then meet exactly in the long
    // accumulator, so the merge loses nothing and the flag reports what the
    // threads' own expansions lost
    bool bad = R.bad;
#pragma unroll  // constant indices keep the expansions in registers
    for (int j = 0; j < NACC; j++) {
      R.lost[j] |= fpe_sum(R.res[j], R.err[j], p, bad);
      if (R.lost[j]) atomicOr(&ws->flags, 2u << j);
      window_init(R.win[j]);
#pragma unroll
      for (int i = 0; i < kFpeMax; i++) {
        if (i < p && !is_zero_bits(R.res[j][i])) {
          const ExactProd e = exact_product(R.res[j][i], 1.0);
          bad |= e.bad;
          exact_deposit(R.win[j], sacc + j * kNDig * kCopies, copy, e);
        }
      }
      window_flush(R.win[j], sacc + j * kNDig * kCopies, copy);
    }
    if (bad) atomicOr(&ws->flags, 1u);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NACC; j++) smem_to_global(sacc + j * kNDig * kCopies, ws->digits[j]);
  } else {
#pragma unroll
    for (int j = 0; j < NACC; j++) {
      const double s = block_sum_fixed<BLOCK>(R.acc[j], fs->sw);
      if (threadIdx.x == 0) ws->partials[j][blockIdx.x] = s;
    }
  }
  // arrival
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(&ws->counter, 1u);
    fs->last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!fs->last) return false;
  __threadfence();
  if constexpr (V == RPCG_EXBLAS) {
    for (int j = 0; j < NACC; j++) {
      const double v = take_and_round(ws->digits[j], fs->dig, fs->D, fs->range);
      if (threadIdx.x == 0) fs->value[j] = v;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const unsigned int f = atomicExch(&ws->flags, 0u);
      for (int j = 0; j < NACC; j++) {
        fs->lost[j] = (f & 1u) ? 1 : 0;
        if (f & 1u) fs->value[j] = __longlong_as_double(0x7FF8000000000000ll);
      }
    }
  } else if constexpr (V == RPCG_FPE) {
    for (int j = 0; j < NACC; j++) {
      const double v = take_and_round(ws->digits[j], fs->dig, fs->D, fs->range);
      if (threadIdx.x == 0) fs->value[j] = v;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const unsigned int f = atomicExch(&ws->flags, 0u);
      for (int j = 0; j < NACC; j++) {
        fs->lost[j] = (f & (2u << j)) ? 1 : 0;
        if (f & 1u) {  // a non-finite operand (or expansion term)
          fs->lost[j] = 1;
          fs->value[j] = __longlong_as_double(0x7FF8000000000000ll);
        }
      }
    }
  } else {
    for (int j = 0; j < NACC; j++) {
      double v = 0.0;
      for (int t = threadIdx.x; t < (int)gridDim.x; t += BLOCK) v = __dadd_rn(v, __ldcg(&ws->partials[j][t]));
      const double s = block_sum_fixed<BLOCK>(v, fs->sw);
      if (threadIdx.x == 0) {
        fs->value[j] = s;
        fs->lost[j] = 0;
      }
    }
  }
  if (threadIdx.x == 0) ws->counter = 0;
  __syncthreads();
  return true;
}

// ------------------------------------------------------------------ scalar steps (one thread)

__device__ __forceinline__ void set_cond(const SolveArgs* args, cudaGraphConditionalHandle cond, bool go) {
  if (args->use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
}

__device__ void stop_loop(SolveState* st, const SolveArgs* args, cudaGraphConditionalHandle cond) {
  st->active = 0;
  set_cond(args, cond, false);
}

// S2: rho = beta / <d, w> (with the breakdown checks).
__device__ void finalize_a(double dw, SolveState* st, const SolveArgs* args, cudaGraphConditionalHandle cond) {
  if (!isfinite(dw)) {
    st->status = RPCG_ERR_NONFINITE;
    stop_loop(st, args, cond);
    return;
  }
  if (!(dw > 0.0)) {
    st->status = RPCG_ERR_NOT_SPD;
    stop_loop(st, args, cond);
    return;
  }
  st->beta_old = st->beta;
  st->rho = __ddiv_rn(st->beta, dw);
}

// After S6 and S8: gamma for S7, the iteration count, relres and the loop test.
__device__ void finalize_b(double beta, double tau, SolveState* st, const SolveArgs* args,
                           cudaGraphConditionalHandle cond) {
  st->beta = beta;
  st->tau = tau;
  if (!isfinite(beta) || !isfinite(tau)) {
    st->status = RPCG_ERR_NONFINITE;
    st->iter += 1;
    stop_loop(st, args, cond);
    return;
  }
  st->gamma = __ddiv_rn(beta, st->beta_old);
  st->iter += 1;
  st->rel = __ddiv_rn(__dsqrt_rn(tau), st->bnorm);
  if (args->history) args->history[st->iter] = st->rel;
  if (tau > 0.0 && !(beta > 0.0)) {
    st->status = RPCG_ERR_NOT_SPD;
    stop_loop(st, args, cond);
    return;
  }
  const bool go = (st->rel >= args->tol) && (st->iter < args->max_iter);
  st->active = go;
  set_cond(args, cond, go);
}

// ------------------------------------------------------------------ kernels

__global__ void k_init_state(SolveState* st, const SolveArgs* args) {
  st->rho = st->beta = st->beta_old = st->gamma = st->bnorm = 0.0;
  st->tau = st->rel = __longlong_as_double(0x7FF8000000000000ll);
  st->iter = 0;
  st->status = 0;
  st->bad_row = INT_MAX;
  st->bzero = 0;
  st->redo = 0;
  st->fpe_inexact = 0;
  st->active = 0;
  // adaptive expansion size starts at 3, the size Sec. 4.3 finds enough for Poisson
  st->fpe_p = args->fpe_size > 0 ? args->fpe_size : 3;
}

// Adaptive expansion size (fpe_size = 0): after a dot that lost bits, the
// following dots use one more term (up to 8).
__device__ __forceinline__ void fpe_grow(SolveState* st, const SolveArgs* args) {
  if (args->fpe_size == 0 && st->fpe_p < kFpeMax) st->fpe_p += 1;
}

// Jacobi preconditioner (Sec. 3.1, Sec. 4.3): inv_i = RN(1 / a_ii).  Rows
// without a positive finite diagonal are recorded (lowest index wins).
__global__ void k_inv_diag(MatDev m, double* inv, SolveState* st) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.n; i += gridDim.x * blockDim.x) {
    double aii = 0.0;
    bool found = false;
    const int len = m.rowptr[i + 1] - m.rowptr[i];
    const long long base = sell_index(m, i, 0);
    for (int k = 0; k < len; k++) {
      if (m.col[base + 32ll * k] == i) {
        aii = m.val[base + 32ll * k];
        found = true;
      }
    }
    if (!found || !(aii > 0.0)) {
      atomicMin(&st->bad_row, i);
      inv[i] = 0.0;
    } else {
      inv[i] = __drcp_rn(aii);
    }
  }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_spmv(MatDev m, const double* __restrict__ x, double* __restrict__ y) {
  for (int row = blockIdx.x * BLOCK + threadIdx.x; row < m.n; row += gridDim.x * BLOCK) y[row] = sell_row(m, row, x);
}

// Pass A: S1 + S2 (the fpe variant uses k_spmv + k_pass_a_dot instead).
// The compiler keeps its own register choice (minimum blocks 0: an explicit
// 1 let the exact pass A grow to 110 registers and fall from 1.01 to 1.51 ms
// at 256^3); the fpe instance is capped at 64 registers (32 warps per SM).
template <int V, int BLOCK>
__global__ void __launch_bounds__(BLOCK, V == RPCG_FPE ? 1024 / BLOCK : 0)
    k_pass_a(MatDev m, const double* __restrict__ d, double* __restrict__ w, PassScratch* ws, SolveState* st,
             const SolveArgs* args, cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* sacc;
  FinalScratch* fs = red_carve<V, 1>(smem, sacc);
  if (st->status != 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) stop_loop(st, args, cond);
    return;
  }
  const int p = st->fpe_p;
  if constexpr (V != RPCG_PLAIN) smem_acc_zero(sacc);
  __syncthreads();
  Reducer<V, 1> R;
  red_init(R);
  for (int row = blockIdx.x * BLOCK + threadIdx.x; row < m.n; row += gridDim.x * BLOCK) {
    const double v = sell_row(m, row, d);
    w[row] = v;
    red_add<V, 1>(R, sacc, 0, __ldg(d + row), v, p);
  }
  if (red_finish<V, 1, BLOCK>(R, sacc, ws, fs, p) && threadIdx.x == 0) {
    if (st->status != 0) {
      stop_loop(st, args, cond);
      return;
    }
    if (V == RPCG_FPE && fs->lost[0]) {
      st->fpe_inexact += 1;
      fpe_grow(st, args);
      if (!args->fpe_strict) {
        st->redo = 1;  // recompute this dot exactly (k_redo_a)
        return;
      }
    }
    finalize_a(fs->value[0], st, args, cond);
  }
}

// FPE variant, pass A as two kernels: k_spmv writes w = A d (S1), then
// this kernel streams d and w (16 bytes a row more than a fused pass) and
// forms the FPE dot <d, w> (S2) with the finalisation of k_pass_a.  Each
// kernel fits 64 registers without spilling (the fused pass spilled ~0.8 KB
// per thread at that cap; both forms measured 1.55 ms per pass at 256^3).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_pass_a_dot(int n, const double* __restrict__ d,
                                                                    const double* __restrict__ w, PassScratch* ws,
                                                                    SolveState* st, const SolveArgs* args,
                                                                    cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* sacc;
  FinalScratch* fs = red_carve<RPCG_FPE, 1>(smem, sacc);
  if (st->status != 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) stop_loop(st, args, cond);
    return;
  }
  const int p = st->fpe_p;
  smem_acc_zero(sacc);
  __syncthreads();
  Reducer<RPCG_FPE, 1> R;
  red_init(R);
  for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK)
    red_add<RPCG_FPE, 1>(R, sacc, 0, __ldcs(d + i), __ldcs(w + i), p);
  if (red_finish<RPCG_FPE, 1, BLOCK>(R, sacc, ws, fs, p) && threadIdx.x == 0) {
    if (st->status != 0) {
      stop_loop(st, args, cond);
      return;
    }
    if (fs->lost[0]) {
      st->fpe_inexact += 1;
      fpe_grow(st, args);
      if (!args->fpe_strict) {
        st->redo = 1;  // recompute this dot exactly (k_redo_a)
        return;
      }
    }
    finalize_a(fs->value[0], st, args, cond);
  }
}

// Pass B: S3, S4, S5, S6 and S8.
template <int V, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_pass_b(int n, const double* __restrict__ d, const double* __restrict__ w,
                                                  const double* __restrict__ inv, double* __restrict__ r,
                                                  PassScratch* ws, SolveState* st, const SolveArgs* args,
                                                  cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* sacc;
  FinalScratch* fs = red_carve<V, 2>(smem, sacc);
  if (st->status != 0 || st->redo) {
    if (st->status != 0 && blockIdx.x == 0 && threadIdx.x == 0) stop_loop(st, args, cond);
    return;
  }
  const int p = st->fpe_p;
  double* __restrict__ x = args->x;
  const double rho = st->rho, nrho = -st->rho;
  if constexpr (V != RPCG_PLAIN) smem_acc_zero(sacc, 2);
  __syncthreads();
  Reducer<V, 2> R;
  red_init(R);
  auto elem = [&](double di, double wi, double ivi, double xi0, double ri0, double& xi, double& ri) {
    xi = __fma_rn(rho, di, xi0);
    ri = __fma_rn(nrho, wi, ri0);
    const double zi = __dmul_rn(ivi, ri);
    red_add(R, sacc, 0, zi, ri, p);
    red_add(R, sacc, 1, ri, ri, p);
  };
  if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
    // pairs of elements as double2 (d, w, inv, r are the handle's 256-byte
    // aligned vectors; x is the caller's, checked here): twice the bytes in
    // flight per thread
    const double2* __restrict__ d2 = reinterpret_cast<const double2*>(d);
    const double2* __restrict__ w2 = reinterpret_cast<const double2*>(w);
    const double2* __restrict__ v2 = reinterpret_cast<const double2*>(inv);
    double2* __restrict__ x2 = reinterpret_cast<double2*>(x);
    double2* __restrict__ r2 = reinterpret_cast<double2*>(r);
    const int n2 = n >> 1;
    for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n2; i += gridDim.x * BLOCK) {
      const double2 dv = __ldcs(d2 + i), wv = __ldcs(w2 + i), vv = __ldcs(v2 + i), xv = __ldcs(x2 + i),
                    rv = __ldcs(r2 + i);
      double2 xo, ro;
      elem(dv.x, wv.x, vv.x, xv.x, rv.x, xo.x, ro.x);
      elem(dv.y, wv.y, vv.y, xv.y, rv.y, xo.y, ro.y);
      __stcs(x2 + i, xo);
      __stcs(r2 + i, ro);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
      const int i = n - 1;
      double xi, ri;
      elem(d[i], w[i], inv[i], x[i], r[i], xi, ri);
      x[i] = xi;
      r[i] = ri;
    }
  } else {
    for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
      double xi, ri;
      elem(__ldcs(d + i), __ldcs(w + i), __ldcs(inv + i), __ldcs(x + i), __ldcs(r + i), xi, ri);
      __stcs(x + i, xi);
      __stcs(r + i, ri);
    }
  }
  if (red_finish<V, 2, BLOCK>(R, sacc, ws, fs, p) && threadIdx.x == 0) {
    if (V == RPCG_FPE && (fs->lost[0] || fs->lost[1])) {
      st->fpe_inexact += (fs->lost[0] ? 1 : 0) + (fs->lost[1] ? 1 : 0);
      fpe_grow(st, args);
      if (!args->fpe_strict) {
        st->redo = 2;  // recompute both dots exactly (k_redo_b)
        return;
      }
    }
    finalize_b(fs->value[0], fs->value[1], st, args, cond);
  }
}

// FPE variant: pass B as two kernels, so that each thread holds one pair of
// expansions instead of two and 64 registers (32 warps per SM) suffice.  B1: S3,
// S4, S5 and S6 (<z,r>, kept in the state); B2: S8 (<r,r> of the new r)
// and the finalisation of both dots, with the counting and recompute rules
// of pass B.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_pass_b1(int n, const double* __restrict__ d,
                                                                 const double* __restrict__ w,
                                                                 const double* __restrict__ inv, double* __restrict__ r,
                                                                 PassScratch* ws, SolveState* st, const SolveArgs* args,
                                                                 cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* sacc;
  FinalScratch* fs = red_carve<RPCG_FPE, 1>(smem, sacc);
  if (st->status != 0 || st->redo) {
    if (st->status != 0 && blockIdx.x == 0 && threadIdx.x == 0) stop_loop(st, args, cond);
    return;
  }
  const int p = st->fpe_p;
  double* __restrict__ x = args->x;
  const double rho = st->rho, nrho = -st->rho;
  smem_acc_zero(sacc);
  __syncthreads();
  Reducer<RPCG_FPE, 1> R;
  red_init(R);
  for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
    const double xi = __fma_rn(rho, __ldcs(d + i), __ldcs(x + i));
    const double ri = __fma_rn(nrho, __ldcs(w + i), __ldcs(r + i));
    const double zi = __dmul_rn(__ldcs(inv + i), ri);
    __stcs(x + i, xi);
    r[i] = ri;  // read again by B2
    red_add<RPCG_FPE, 1>(R, sacc, 0, zi, ri, p);
  }
  if (red_finish<RPCG_FPE, 1, BLOCK>(R, sacc, ws, fs, p) && threadIdx.x == 0) {
    st->zr = fs->value[0];
    st->zr_lost = fs->lost[0];
  }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_pass_b2(int n, const double* __restrict__ r, PassScratch* ws,
                                                                 SolveState* st, const SolveArgs* args,
                                                                 cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* sacc;
  FinalScratch* fs = red_carve<RPCG_FPE, 1>(smem, sacc);
  if (st->status != 0 || st->redo) return;  // B1 has stopped the loop
  const int p = st->fpe_p;
  smem_acc_zero(sacc);
  __syncthreads();
  Reducer<RPCG_FPE, 1> R;
  red_init(R);
  for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
    const double ri = __ldcs(r + i);
    red_add<RPCG_FPE, 1>(R, sacc, 0, ri, ri, p);
  }
  if (red_finish<RPCG_FPE, 1, BLOCK>(R, sacc, ws, fs, p) && threadIdx.x == 0) {
    const bool lost0 = st->zr_lost != 0, lost1 = fs->lost[0] != 0;
    if (lost0 || lost1) {
      st->fpe_inexact += (lost0 ? 1 : 0) + (lost1 ? 1 : 0);
      fpe_grow(st, args);
      if (!args->fpe_strict) {
        st->redo = 2;  // recompute both dots exactly (k_redo_b)
        return;
      }
    }
    finalize_b(st->zr, fs->value[0], st, args, cond);
  }
}

// Pass C: S7.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_pass_c(int n, double* __restrict__ d, const double* __restrict__ inv,
                                                  const double* __restrict__ r, const SolveState* st) {
  if (st->status != 0) return;
  const double g = st->gamma;
  // pairs as double2 (the handle's vectors are 256-byte aligned)
  const double2* __restrict__ v2 = reinterpret_cast<const double2*>(inv);
  const double2* __restrict__ r2 = reinterpret_cast<const double2*>(r);
  double2* __restrict__ d2 = reinterpret_cast<double2*>(d);
  const int n2 = n >> 1;
  for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n2; i += gridDim.x * BLOCK) {
    const double2 vv = __ldcs(v2 + i), rv = __ldcs(r2 + i), dv = d2[i];
    double2 o;
    o.x = __fma_rn(g, dv.x, __dmul_rn(vv.x, rv.x));
    o.y = __fma_rn(g, dv.y, __dmul_rn(vv.y, rv.y));
    d2[i] = o;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int i = n - 1;
    d[i] = __fma_rn(g, d[i], __dmul_rn(inv[i], r[i]));
  }
}

// FPE variant with fpe_strict = 0: an inexact dot is recomputed exactly.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_redo_a(int n, const double* __restrict__ d, const double* __restrict__ w,
                                                  PassScratch* ws, SolveState* st, const SolveArgs* args,
                                                  cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* sacc;
  FinalScratch* fs = red_carve<RPCG_EXBLAS, 1>(smem, sacc);
  if (st->redo != 1) return;
  smem_acc_zero(sacc);
  Reducer<RPCG_EXBLAS, 1> R;
  red_init(R);
  __syncthreads();
  for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) red_add(R, sacc, 0, d[i], w[i], 0);
  if (red_finish<RPCG_EXBLAS, 1, BLOCK>(R, sacc, ws, fs, 0) && threadIdx.x == 0) {
    st->redo = 0;
    finalize_a(fs->value[0], st, args, cond);
  }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_redo_b(int n, const double* __restrict__ inv, const double* __restrict__ r,
                                                  PassScratch* ws, SolveState* st, const SolveArgs* args,
                                                  cudaGraphConditionalHandle cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* sacc;
  FinalScratch* fs = red_carve<RPCG_EXBLAS, 2>(smem, sacc);
  if (st->redo != 2) return;
  smem_acc_zero(sacc, 2);
  Reducer<RPCG_EXBLAS, 2> R;
  red_init(R);
  __syncthreads();
  for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
    const double ri = r[i];
    const double zi = __dmul_rn(inv[i], ri);
    red_add(R, sacc, 0, zi, ri, 0);
    red_add(R, sacc, 1, ri, ri, 0);
  }
  if (red_finish<RPCG_EXBLAS, 2, BLOCK>(R, sacc, ws, fs, 0) && threadIdx.x == 0) {
    st->redo = 0;
    finalize_b(fs->value[0], fs->value[1], st, args, cond);
  }
}

// Set-up: r0 = b - A x0 (A x0 already in w), z0 = inv .* r0, d0 = z0,
// beta0 = <z0, r0>, tau0 = <r0, r0>, ||b||^2 = <b, b>; last CTA: checks,
// relres0 and the initial loop condition.  The set-up dots are always exact
// (plain for the plain variant).
template <int V, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_setup(MatDev m, const double* __restrict__ q, const double* __restrict__ inv,
                                                 double* __restrict__ r, double* __restrict__ d, PassScratch* ws,
                                                 SolveState* st, const SolveArgs* args,
                                                 cudaGraphConditionalHandle cond) {
  // the set-up dots are exact for both reproducible variants
  constexpr int VS = (V == RPCG_PLAIN) ? RPCG_PLAIN : RPCG_EXBLAS;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* sacc;
  FinalScratch* fs = red_carve<VS, 3>(smem, sacc);
  const int n = m.n;
  const double* __restrict__ b = args->b;
  if constexpr (VS == RPCG_EXBLAS) smem_acc_zero(sacc, 3);
  Reducer<VS, 3> R;
  red_init(R);
  __syncthreads();
  for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
    const double bi = b[i];
    const double ri = __dsub_rn(bi, q[i]);
    const double zi = __dmul_rn(inv[i], ri);
    r[i] = ri;
    d[i] = zi;
    red_add(R, sacc, 0, zi, ri, 0);
    red_add(R, sacc, 1, ri, ri, 0);
    red_add(R, sacc, 2, bi, bi, 0);
  }
  if (red_finish<VS, 3, BLOCK>(R, sacc, ws, fs, 0) && threadIdx.x == 0) {
    if (st->bad_row < n) {
      // the lowest-index row without a positive finite diagonal decides
      const int i = st->bad_row;
      double aii = 0.0;
      const int len = m.rowptr[i + 1] - m.rowptr[i];
      const long long base = sell_index(m, i, 0);
      for (int k = 0; k < len; k++)
        if (m.col[base + 32ll * k] == i) aii = m.val[base + 32ll * k];
      st->status = isfinite(aii) ? RPCG_ERR_NOT_SPD : RPCG_ERR_NONFINITE;
      stop_loop(st, args, cond);
      return;
    }
    const double beta = fs->value[0], tau = fs->value[1], bb = fs->value[2];
    if (!isfinite(beta) || !isfinite(tau) || !isfinite(bb)) {
      st->status = RPCG_ERR_NONFINITE;
      stop_loop(st, args, cond);
      return;
    }
    st->beta = beta;
    const double bnorm = __dsqrt_rn(bb);
    st->bnorm = bnorm;
    if (bnorm == 0.0) {
      st->bzero = 1;
      st->rel = 0.0;
      st->tau = 0.0;
      if (args->history) args->history[0] = 0.0;
      stop_loop(st, args, cond);
      return;
    }
    st->tau = tau;
    st->rel = __ddiv_rn(__dsqrt_rn(tau), bnorm);
    if (args->history) args->history[0] = st->rel;
    const bool go = (st->rel >= args->tol) && (0 < args->max_iter);
    st->active = go;
    set_cond(args, cond, go);
  }
}

// ------------------------------------------------------------------ handle

static int pick_block(int b) { return (b == 128 || b == 256 || b == 512) ? b : 256; }

template <int BLOCK>
static size_t spmv_smem() {
  return 0;
}

template <int V, int NACC>
static size_t pass_smem() {
  return red_smem_bytes<V, NACC>() + sizeof(FinalScratch) + 16;
}

static cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* deps, int ndeps,
                              const void* func, int grid, int block, size_t smem, void** args) {
  cudaKernelNodeParams p{};
  p.func = const_cast<void*>(func);
  p.gridDim = dim3(grid);
  p.blockDim = dim3(block);
  p.sharedMemBytes = (unsigned)smem;
  p.kernelParams = args;
  p.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &p);
}

template <typename F>
static cudaError_t set_smem(F* f, size_t bytes) {
  return cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Grid sizes and shared memory of every kernel of a solve.
struct LaunchCfg {
  int grid_stream, grid_tiles, grid_small;
  size_t smem_spmv, smem_a, smem_b, smem_s, smem_ra, smem_rb;
};

template <int V, int BLOCK>
static rpcg_status launch_cfg(int n, int grid, LaunchCfg* c) {
  const int sms = sm_count();
  const int ntiles = (n + BLOCK - 1) / BLOCK;
  int grid_stream = grid > 0 ? grid : sms * (BLOCK >= 512 ? 2 : 4);
  // persistent tile grid: as many CTAs as can be resident at once
  int occ = 1;
  {
    const size_t sm_a = pass_smem<V, 1>();
    RPCG_CUDA_TRY(set_smem(k_pass_a<V, BLOCK>, sm_a));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pass_a<V, BLOCK>, BLOCK, sm_a) != cudaSuccess || occ < 1)
      occ = 1;
  }
  int grid_tiles = grid > 0 ? grid : sms * occ;
  if (grid_stream > kMaxPassGrid) grid_stream = kMaxPassGrid;
  if (grid_tiles > kMaxPassGrid) grid_tiles = kMaxPassGrid;
  if (grid_tiles > ntiles) grid_tiles = ntiles > 0 ? ntiles : 1;  // ntiles: CTAs of BLOCK rows
  const int grid_elem_cap = (n + BLOCK - 1) / BLOCK;
  if (grid_stream > grid_elem_cap) grid_stream = grid_elem_cap > 0 ? grid_elem_cap : 1;
  const int grid_small = (n + BLOCK - 1) / BLOCK > 0 ? ((n + BLOCK - 1) / BLOCK < sms * 8 ? (n + BLOCK - 1) / BLOCK : sms * 8) : 1;
  c->grid_stream = grid_stream;
  c->grid_tiles = grid_tiles;
  c->grid_small = grid_small;
  c->smem_spmv = spmv_smem<BLOCK>();
  c->smem_a = pass_smem<V, 1>();
  c->smem_b = pass_smem<V, 2>();
  c->smem_s = pass_smem<(V == RPCG_PLAIN ? RPCG_PLAIN : RPCG_EXBLAS), 3>();
  c->smem_ra = pass_smem<RPCG_EXBLAS, 1>();
  c->smem_rb = pass_smem<RPCG_EXBLAS, 2>();
  RPCG_CUDA_TRY(set_smem(k_spmv<BLOCK>, c->smem_spmv));
  RPCG_CUDA_TRY(set_smem(k_pass_a<V, BLOCK>, c->smem_a));
  if constexpr (V == RPCG_FPE) {
    RPCG_CUDA_TRY(set_smem(k_pass_a_dot<BLOCK>, c->smem_a));
    RPCG_CUDA_TRY(set_smem(k_pass_b1<BLOCK>, c->smem_a));  // one FPE dot each, as pass A
    RPCG_CUDA_TRY(set_smem(k_pass_b2<BLOCK>, c->smem_a));
  } else {
    RPCG_CUDA_TRY(set_smem(k_pass_b<V, BLOCK>, c->smem_b));
  }
  RPCG_CUDA_TRY(set_smem(k_setup<V, BLOCK>, c->smem_s));
  RPCG_CUDA_TRY(set_smem(k_redo_a<BLOCK>, c->smem_ra));
  RPCG_CUDA_TRY(set_smem(k_redo_b<BLOCK>, c->smem_rb));
  return RPCG_OK;
}

// Build the solve graph for one (variant, block, grid).
template <int V, int BLOCK>
static rpcg_status build_graph(rpcg_matrix_t A, int grid, cudaGraph_t* out_graph, cudaGraphExec_t* out_exec,
                               cudaGraphNode_t* out_x0_node) {
  MatDev m = A->m;
  int n = m.n;
  LaunchCfg c;
  rpcg_status cs = launch_cfg<V, BLOCK>(n, grid, &c);
  if (cs != RPCG_OK) return cs;
  const int grid_stream = c.grid_stream, grid_tiles = c.grid_tiles, grid_small = c.grid_small;
  const size_t smem_spmv = c.smem_spmv, smem_a = c.smem_a, smem_b = c.smem_b, smem_s = c.smem_s;
  const size_t smem_ra = c.smem_ra, smem_rb = c.smem_rb;
  cudaGraph_t g = nullptr;
  RPCG_CUDA_TRY(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond;
  RPCG_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
  SolveState* st = A->state;
  SolveArgs* args = A->args;
  PassScratch* ws = A->scratch;
  double *inv = A->inv, *r = A->r, *d = A->d, *w = A->w;

  cudaGraphNode_t n_init, n_inv, n_spmv, n_setup, n_loop;
  {
    void* a[] = {&st, &args};
    RPCG_CUDA_TRY(add_kernel(g, &n_init, nullptr, 0, (const void*)k_init_state, 1, 1, 0, a));
  }
  {
    void* a[] = {&m, &inv, &st};
    RPCG_CUDA_TRY(add_kernel(g, &n_inv, &n_init, 1, (const void*)k_inv_diag, grid_small, BLOCK, 0, a));
  }
  // q = A x0 into w.  The kernel reads x0 through its parameter, which
  // set_x0() points at the caller's x before every launch.
  {
    const double* x0 = nullptr;
    void* a[] = {&m, &x0, &w};
    RPCG_CUDA_TRY(add_kernel(g, &n_spmv, &n_inv, 1, (const void*)k_spmv<BLOCK>, grid_tiles, BLOCK, smem_spmv, a));
  }
  {
    void* a[] = {&m, &w, &inv, &r, &d, &ws, &st, &args, &cond};
    RPCG_CUDA_TRY(add_kernel(g, &n_setup, &n_spmv, 1, (const void*)k_setup<V, BLOCK>, grid_stream, BLOCK, smem_s, a));
  }
  // the while loop
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  RPCG_CUDA_TRY(cudaGraphAddNode(&n_loop, g, &n_setup, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaGraphNode_t b_a, b_ra, b_b, b_rb, b_c;
  if (V == RPCG_FPE) {
    cudaGraphNode_t b_s;
    void* as[] = {&m, &d, &w};
    RPCG_CUDA_TRY(add_kernel(body, &b_s, nullptr, 0, (const void*)k_spmv<BLOCK>, grid_tiles, BLOCK, smem_spmv, as));
    void* a[] = {&n, &d, &w, &ws, &st, &args, &cond};
    RPCG_CUDA_TRY(add_kernel(body, &b_a, &b_s, 1, (const void*)k_pass_a_dot<BLOCK>, grid_stream, BLOCK, smem_a, a));
  } else {
    void* a[] = {&m, &d, &w, &ws, &st, &args, &cond};
    RPCG_CUDA_TRY(add_kernel(body, &b_a, nullptr, 0, (const void*)k_pass_a<V, BLOCK>, grid_tiles, BLOCK, smem_a, a));
  }
  cudaGraphNode_t prev = b_a;
  if (V == RPCG_FPE) {
    void* a[] = {&n, &d, &w, &ws, &st, &args, &cond};
    RPCG_CUDA_TRY(add_kernel(body, &b_ra, &prev, 1, (const void*)k_redo_a<BLOCK>, grid_stream, BLOCK, smem_ra, a));
    prev = b_ra;
  }
  if constexpr (V == RPCG_FPE) {
    void* a1[] = {&n, &d, &w, &inv, &r, &ws, &st, &args, &cond};
    RPCG_CUDA_TRY(add_kernel(body, &b_b, &prev, 1, (const void*)k_pass_b1<BLOCK>, grid_stream, BLOCK, smem_a, a1));
    prev = b_b;
    void* a2[] = {&n, &r, &ws, &st, &args, &cond};
    RPCG_CUDA_TRY(add_kernel(body, &b_b, &prev, 1, (const void*)k_pass_b2<BLOCK>, grid_stream, BLOCK, smem_a, a2));
    prev = b_b;
  } else {
    void* a[] = {&n, &d, &w, &inv, &r, &ws, &st, &args, &cond};
    RPCG_CUDA_TRY(add_kernel(body, &b_b, &prev, 1, (const void*)k_pass_b<V, BLOCK>, grid_stream, BLOCK, smem_b, a));
    prev = b_b;
  }
  if (V == RPCG_FPE) {
    void* a[] = {&n, &inv, &r, &ws, &st, &args, &cond};
    RPCG_CUDA_TRY(add_kernel(body, &b_rb, &prev, 1, (const void*)k_redo_b<BLOCK>, grid_stream, BLOCK, smem_rb, a));
    prev = b_rb;
  }
  {
    void* a[] = {&n, &d, &inv, &r, &st};
    RPCG_CUDA_TRY(add_kernel(body, &b_c, &prev, 1, (const void*)k_pass_c<BLOCK>, grid_stream, BLOCK, 0, a));
  }
  cudaGraphExec_t exec = nullptr;
  RPCG_CUDA_TRY(cudaGraphInstantiate(&exec, g, 0));
  *out_graph = g;
  *out_exec = exec;
  *out_x0_node = n_spmv;
  return RPCG_OK;
}

template <int BLOCK>
static rpcg_status build_graph_v(rpcg_matrix_t A, int v, int grid, cudaGraph_t* g, cudaGraphExec_t* e,
                                 cudaGraphNode_t* x0) {
  if (v == RPCG_PLAIN) return build_graph<RPCG_PLAIN, BLOCK>(A, grid, g, e, x0);
  if (v == RPCG_EXBLAS) return build_graph<RPCG_EXBLAS, BLOCK>(A, grid, g, e, x0);
  return build_graph<RPCG_FPE, BLOCK>(A, grid, g, e, x0);
}

static rpcg_status get_graph(rpcg_matrix_t A, int v, int block, int grid, cudaGraphExec_t* exec) {
  GraphKey key{v, block, grid};
  auto it = A->graphs.find(key);
  if (it != A->graphs.end()) {
    *exec = it->second;
    return RPCG_OK;
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  cudaGraphNode_t x0 = nullptr;
  rpcg_status s;
  if (block == 128) s = build_graph_v<128>(A, v, grid, &g, &e, &x0);
  else if (block == 512) s = build_graph_v<512>(A, v, grid, &g, &e, &x0);
  else s = build_graph_v<256>(A, v, grid, &g, &e, &x0);
  if (s != RPCG_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  A->graphs[key] = e;
  A->graph_defs[key] = g;
  A->x0_nodes[key] = x0;
  *exec = e;
  return RPCG_OK;
}

// The same kernels launched one by one, with CUDA events around each pass
// (pass_ms: set-up, A, B, C totals in milliseconds; launches: counts).
template <int V, int BLOCK>
static rpcg_status run_eager(rpcg_matrix_t A, int grid, const double* x0, cudaStream_t s, float* pass_ms,
                             int* launches) {
  MatDev m = A->m;
  const int n = m.n;
  LaunchCfg c;
  rpcg_status cs = launch_cfg<V, BLOCK>(n, grid, &c);
  if (cs != RPCG_OK) return cs;
  SolveState* st = A->state;
  SolveArgs* args = A->args;
  PassScratch* ws = A->scratch;
  double *inv = A->inv, *r = A->r, *d = A->d, *w = A->w;
  const cudaGraphConditionalHandle cond = 0;
  cudaEvent_t ev[8];
  for (auto& e : ev) RPCG_CUDA_TRY(cudaEventCreate(&e));
  float acc[4] = {0, 0, 0, 0};
  int cnt[4] = {0, 0, 0, 0};
  auto fail = [&](cudaError_t e) {
    for (auto& x : ev) cudaEventDestroy(x);
    set_error("eager solve: %s", cudaGetErrorString(e));
    return RPCG_ERR_CUDA;
  };
  cudaError_t e;
  e = cudaEventRecord(ev[0], s);
  k_init_state<<<1, 1, 0, s>>>(st, args);
  k_inv_diag<<<c.grid_small, BLOCK, 0, s>>>(m, inv, st);
  k_spmv<BLOCK><<<c.grid_tiles, BLOCK, c.smem_spmv, s>>>(m, x0, w);
  k_setup<V, BLOCK><<<c.grid_stream, BLOCK, c.smem_s, s>>>(m, w, inv, r, d, ws, st, args, cond);
  cudaEventRecord(ev[1], s);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(A->h_state, st, sizeof(SolveState), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
  float t;
  cudaEventElapsedTime(&t, ev[0], ev[1]);
  acc[0] += t;
  cnt[0] += 1;
  while (A->h_state->active) {
    cudaEventRecord(ev[2], s);
    if (V == RPCG_FPE) {
      k_spmv<BLOCK><<<c.grid_tiles, BLOCK, c.smem_spmv, s>>>(m, d, w);
      k_pass_a_dot<BLOCK><<<c.grid_stream, BLOCK, c.smem_a, s>>>(n, d, w, ws, st, args, cond);
    } else {
      k_pass_a<V, BLOCK><<<c.grid_tiles, BLOCK, c.smem_a, s>>>(m, d, w, ws, st, args, cond);
    }
    cudaEventRecord(ev[3], s);
    if (V == RPCG_FPE) k_redo_a<BLOCK><<<c.grid_stream, BLOCK, c.smem_ra, s>>>(n, d, w, ws, st, args, cond);
    cudaEventRecord(ev[4], s);
    if constexpr (V == RPCG_FPE) {
      k_pass_b1<BLOCK><<<c.grid_stream, BLOCK, c.smem_a, s>>>(n, d, w, inv, r, ws, st, args, cond);
      k_pass_b2<BLOCK><<<c.grid_stream, BLOCK, c.smem_a, s>>>(n, r, ws, st, args, cond);
    } else {
      k_pass_b<V, BLOCK><<<c.grid_stream, BLOCK, c.smem_b, s>>>(n, d, w, inv, r, ws, st, args, cond);
    }
    cudaEventRecord(ev[5], s);
    if (V == RPCG_FPE) k_redo_b<BLOCK><<<c.grid_stream, BLOCK, c.smem_rb, s>>>(n, inv, r, ws, st, args, cond);
    cudaEventRecord(ev[6], s);
    k_pass_c<BLOCK><<<c.grid_stream, BLOCK, 0, s>>>(n, d, inv, r, st);
    cudaEventRecord(ev[7], s);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(A->h_state, st, sizeof(SolveState), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return fail(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
    cudaEventElapsedTime(&t, ev[2], ev[3]);
    acc[1] += t;
    cudaEventElapsedTime(&t, ev[4], ev[5]);
    acc[2] += t;
    cudaEventElapsedTime(&t, ev[6], ev[7]);
    acc[3] += t;
    cnt[1] += 1;
    cnt[2] += 1;
    cnt[3] += 1;
    if (A->h_state->status != 0) break;
  }
  for (auto& x : ev) cudaEventDestroy(x);
  for (int i = 0; i < 4; i++) {
    if (pass_ms) pass_ms[i] = acc[i];
    if (launches) launches[i] = cnt[i];
  }
  return RPCG_OK;
}

// Point the set-up SpMV node at x0 for this call.
// Asynchronous solves: the arguments reach the device as kernel parameters
// (captured at launch), so two solves enqueued back to back cannot race on
// a host staging buffer; the result struct is written by a kernel at the end.
__global__ void k_set_args(SolveArgs* dst, SolveArgs a) { *dst = a; }
__global__ void k_set_state(SolveState* dst, SolveState a) { *dst = a; }

// The host-side result logic of rpcg_solve, on the device: status
// NOT_CONVERGED when the loop stopped at max_iter, FPE_INEXACT for strict fpe
// solves that saw an inexact dot, x = 0 when b = 0.  Every thread zeroes
// its part of x in that case; thread 0 of block 0 writes *out.
__global__ void k_finish_result(const SolveState* st, double tol, int variant, int fpe_strict, double* x, int n,
                                rpcg_result* out) {
  const SolveState s = *st;
  if (s.bzero)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int status = s.status;
    if (status == RPCG_OK) {
      if (!(s.rel < tol)) status = RPCG_NOT_CONVERGED;
      else if (variant == RPCG_FPE && fpe_strict && s.fpe_inexact > 0) status = RPCG_FPE_INEXACT;
    }
    rpcg_result r;
    r.iterations = s.iter;
    r.status = status;
    r.relres = s.rel;
    r.tau = s.tau;
    r.fpe_inexact_count = s.fpe_inexact;
    r.fpe_size_used = variant == RPCG_FPE ? s.fpe_p : 0;
    *out = r;
  }
}

static cudaError_t set_x0(rpcg_matrix_t A, cudaGraphNode_t nd, cudaGraphExec_t e, const double* x) {
  cudaKernelNodeParams p{};
  cudaError_t err = cudaGraphKernelNodeGetParams(nd, &p);
  if (err != cudaSuccess) return err;
  MatDev m = A->m;
  const double* x0 = x;
  double* w = A->w;
  void* a[] = {&m, &x0, &w};
  p.kernelParams = a;
  return cudaGraphExecKernelNodeSetParams(e, nd, &p);
}

static rpcg_status alloc_dev(void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes failed", bytes);
    return RPCG_ERR_OOM;
  }
  if (e != cudaSuccess) {
    set_error("cudaMalloc failed: %s", cudaGetErrorString(e));
    return RPCG_ERR_CUDA;
  }
  return RPCG_OK;
}

__global__ void k_check_csr(int n, int nnz, const int* rowptr, const int* col, int* bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
    const int v = rowptr[i];
    if (v < 0 || v > nnz || (i == 0 && v != 0) || (i == n && v != nnz) || (i < n && rowptr[i + 1] < v)) atomicOr(bad, 1);
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x) {
    const int c = col[k];
    if (c < 0 || c >= n) atomicOr(bad, 2);
  }
}

// The longest row of every 32-row slice (rows past n count as empty): one
// warp per slice, one lane per row.  Run after k_check_csr found the row
// pointers valid (the lengths are then non-negative).
__global__ void k_slice_len(int n, const int* __restrict__ rowptr, int* __restrict__ len) {
  const int nsl = (n + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < nsl; sl += warps) {
    const int row = 32 * sl + lane;
    const int l = row < n ? rowptr[row + 1] - rowptr[row] : 0;
    const int m = __reduce_max_sync(0xffffffffu, l);
    if (lane == 0) len[sl] = m;
  }
}

// Scatter CSR rows into the SELL-32 layout (entry k of row i at
// sptr[i / 32] + 32 k + i % 32), keeping each row's storage order.
__global__ void k_csr_to_sell(int n, const int* __restrict__ rowptr, const int* __restrict__ ccol,
                              const double* __restrict__ cval, const long long* __restrict__ sptr, int* scol,
                              double* sval) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int a = rowptr[i], e = rowptr[i + 1];
    const long long base = sptr[i >> 5] + (i & 31);
    for (int k = 0; k < e - a; k++) {
      scol[base + 32ll * k] = ccol[a + k];
      sval[base + 32ll * k] = cval[a + k];
    }
  }
}

static void destroy_handle(rpcg_matrix_t A) {
  if (!A) return;
  for (auto& kv : A->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : A->graph_defs) cudaGraphDestroy(kv.second);
  cudaFree(A->rowptr);
  cudaFree(A->sptr);
  cudaFree(A->col);
  cudaFree(A->val);
  cudaFree(A->inv);
  cudaFree(A->r);
  cudaFree(A->d);
  cudaFree(A->w);
  cudaFree(A->bx);
  cudaFree(A->args);
  cudaFree(A->state);
  cudaFree(A->scratch);
  cudaFreeHost(A->h_args);
  cudaFreeHost(A->h_state);
  delete A;
}

}  // namespace rpcg

using namespace rpcg;

extern "C" {

void rpcg_opts_default(rpcg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-8;
  o->max_iter = 1000;
  o->fpe_size = 8;
  o->fpe_strict = 0;
}

rpcg_status rpcg_create(rpcg_matrix_t* A_out, int32_t n, int32_t nnz, const int32_t* rowptr, const int32_t* col,
                        const double* val, int32_t ptr_kind, void* stream) {
  clear_error();
  RPCG_CHECK_ARG(A_out != nullptr, "A_out is NULL");
  *A_out = nullptr;
  RPCG_CHECK_ARG(n >= 0 && nnz >= 0, "n and nnz must be non-negative");
  // headroom for the 32-bit row indices of the grid-stride loops (strides up
  // to 2^21) and the batch's unit products (tiles up to 2^24)
  RPCG_CHECK_ARG(n <= kMaxRows, "n must be at most 2^31 - 2^25");
  RPCG_CHECK_ARG(rowptr != nullptr, "rowptr is NULL");
  RPCG_CHECK_ARG(nnz == 0 || (col != nullptr && val != nullptr), "col or val is NULL");
  RPCG_CHECK_ARG(ptr_kind == 0 || ptr_kind == 1, "ptr_kind must be 0 (host) or 1 (device)");
  cudaStream_t s = (cudaStream_t)stream;
  if (ptr_kind == 0 && (rowptr[0] != 0 || rowptr[n] != nnz)) {
    set_error("rowptr[0] must be 0 and rowptr[n] must be nnz");
    return RPCG_ERR_INVALID;
  }
  rpcg_matrix_t A = new rpcg_matrix_s();
  cudaGetDevice(&A->device);
  rpcg_status st = RPCG_OK;
  const size_t vec = (size_t)(n > 0 ? n : 1) * sizeof(double);
#define ALLOC(ptr, bytes)                                    \
  do {                                                       \
    st = alloc_dev((void**)&(ptr), (bytes));                 \
    if (st != RPCG_OK) {                                     \
      destroy_handle(A);                                     \
      return st;                                             \
    }                                                        \
  } while (0)
  ALLOC(A->rowptr, ((size_t)n + 1 + 8) * sizeof(int));
  ALLOC(A->inv, vec);
  ALLOC(A->r, vec);
  ALLOC(A->d, vec);
  ALLOC(A->w, vec);
  ALLOC(A->bx, 2 * vec);
  ALLOC(A->args, sizeof(SolveArgs));
  ALLOC(A->state, sizeof(SolveState));
  ALLOC(A->scratch, sizeof(PassScratch));
  if (cudaMallocHost((void**)&A->h_args, sizeof(SolveArgs)) != cudaSuccess ||
      cudaMallocHost((void**)&A->h_state, sizeof(SolveState)) != cudaSuccess) {
    cudaGetLastError();
    destroy_handle(A);
    set_error("pinned host allocation failed");
    return RPCG_ERR_OOM;
  }
  // 1. the CSR arrays into temporary device buffers
  int* ccol = nullptr;
  double* cval = nullptr;
  auto free_tmp = [&]() {
    cudaFree(ccol);
    cudaFree(cval);
  };
  st = alloc_dev((void**)&ccol, (size_t)(nnz > 0 ? nnz : 1) * sizeof(int));
  if (st == RPCG_OK) st = alloc_dev((void**)&cval, (size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
  if (st != RPCG_OK) {
    free_tmp();
    destroy_handle(A);
    return st;
  }
  const cudaMemcpyKind kind = ptr_kind == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaError_t e = cudaMemcpyAsync(A->rowptr, rowptr, ((size_t)n + 1) * sizeof(int), kind, s);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(ccol, col, (size_t)nnz * sizeof(int), kind, s);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(cval, val, (size_t)nnz * sizeof(double), kind, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(A->scratch, 0, offsetof(PassScratch, partials), s);
  // 2. validate on the device (monotone row pointers, columns in range) and
  // take every slice's longest row there
  const int nslices = (n + 31) / 32;
  std::vector<int> hlen((size_t)nslices);
  if (e == cudaSuccess) {
    int* bad = nullptr;
    e = cudaMallocAsync((void**)&bad, sizeof(int), s);
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e == cudaSuccess) {
      int g = sm_count() * 4;
      k_check_csr<<<g, 256, 0, s>>>(n, nnz, A->rowptr, ccol, bad);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && !hbad && nslices > 0) {
      // the lengths pass through the w vector, which is not in use yet
      // (n doubles hold the n / 32 + 1 ints)
      int* dlen = reinterpret_cast<int*>(A->w);
      k_slice_len<<<sm_count() * 4, 256, 0, s>>>(n, A->rowptr, dlen);
      e = cudaGetLastError();
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hlen.data(), dlen, (size_t)nslices * sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (bad) cudaFreeAsync(bad, s);
    if (e == cudaSuccess && hbad) {
      free_tmp();
      destroy_handle(A);
      set_error("invalid CSR (row pointers %s, column indices %s)", (hbad & 1) ? "bad" : "ok", (hbad & 2) ? "bad" : "ok");
      return RPCG_ERR_INVALID;
    }
  }
  // 3. SELL-32 slice offsets: 32 times the running sum of the longest rows
  std::vector<long long> hsptr((size_t)nslices + 1, 0);
  for (int sl = 0; sl < nslices && e == cudaSuccess; sl++) hsptr[sl + 1] = hsptr[sl] + 32ll * hlen[sl];
  const long long total = hsptr[nslices];
  if (e == cudaSuccess) {
    st = alloc_dev((void**)&A->sptr, ((size_t)nslices + 1) * sizeof(long long));
    if (st == RPCG_OK) st = alloc_dev((void**)&A->col, ((size_t)total + 32) * sizeof(int));
    if (st == RPCG_OK) st = alloc_dev((void**)&A->val, ((size_t)total + 32) * sizeof(double));
    if (st != RPCG_OK) {
      free_tmp();
      destroy_handle(A);
      return st;
    }
    e = cudaMemcpyAsync(A->sptr, hsptr.data(), ((size_t)nslices + 1) * sizeof(long long), cudaMemcpyHostToDevice, s);
  }
  // 4. scatter into SELL-32 (padding: column 0, value 0; never used)
  if (e == cudaSuccess) e = cudaMemsetAsync(A->col, 0, ((size_t)total + 32) * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(A->val, 0, ((size_t)total + 32) * sizeof(double), s);
  if (e == cudaSuccess && n > 0) {
    k_csr_to_sell<<<sm_count() * 8, 256, 0, s>>>(n, A->rowptr, ccol, cval, A->sptr, A->col, A->val);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  free_tmp();
  if (e != cudaSuccess) {
    set_error("rpcg_create: %s", cudaGetErrorString(e));
    destroy_handle(A);
    return RPCG_ERR_CUDA;
  }
  A->m.n = n;
  A->m.nnz = nnz;
  A->m.rowptr = A->rowptr;
  A->m.sptr = A->sptr;
  A->m.col = A->col;
  A->m.val = A->val;
  small_plan(A, hsptr.data(), n);
  *A_out = A;
  return RPCG_OK;
}

rpcg_status rpcg_destroy(rpcg_matrix_t A) {
  clear_error();
  if (!A) return RPCG_OK;
  cudaDeviceSynchronize();
  destroy_handle(A);
  return RPCG_OK;
}

rpcg_status rpcg_matrix_info(rpcg_matrix_t A, int32_t* n, int32_t* nnz) {
  RPCG_CHECK_ARG(A != nullptr, "A is NULL");
  if (n) *n = A->m.n;
  if (nnz) *nnz = A->m.nnz;
  return RPCG_OK;
}

rpcg_status rpcg_spmv(rpcg_matrix_t A, const double* x, double* y, void* stream) {
  clear_error();
  RPCG_CHECK_ARG(A != nullptr, "A is NULL");
  RPCG_CHECK_ARG(A->m.n == 0 || (x && y), "x or y is NULL");
  if (A->m.n == 0) return RPCG_OK;
  constexpr int B = 256;
  const size_t smem = spmv_smem<B>();
  RPCG_CUDA_TRY(set_smem(k_spmv<B>, smem));
  const int ntiles = (A->m.n + B - 1) / B;
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv<B>, B, smem) != cudaSuccess || occ < 1) occ = 1;
  int g = sm_count() * occ;
  if (g > ntiles) g = ntiles;
  k_spmv<B><<<g, B, smem, (cudaStream_t)stream>>>(A->m, x, y);
  RPCG_CUDA_TRY(cudaGetLastError());
  return RPCG_OK;
}

// async: enqueue only; *res is written on the device (device or pinned host
// memory) by k_finish_result and the stream is not synchronised.
static rpcg_status solve_impl(rpcg_matrix_t A, const double* b, double* x, int32_t v, const rpcg_opts* o,
                              rpcg_result* res, cudaStream_t s, float* pass_ms = nullptr, int* launches = nullptr,
                              bool async = false) {
  rpcg_opts opt;
  if (o) opt = *o;
  else rpcg_opts_default(&opt);
  RPCG_CHECK_ARG(v == RPCG_PLAIN || v == RPCG_EXBLAS || v == RPCG_FPE, "unknown variant");
  RPCG_CHECK_ARG(opt.max_iter >= 0, "max_iter must be >= 0");
  RPCG_CHECK_ARG(!(opt.tol < 0.0) && !std::isnan(opt.tol), "tol must be >= 0");
  RPCG_CHECK_ARG(opt.fpe_size >= 0 && opt.fpe_size <= kFpeMax, "fpe_size must be 0 (adaptive) or 1..8");
  RPCG_CHECK_ARG(opt.grid >= 0 && opt.grid <= kMaxPassGrid, "grid must be 0..4096");
  const int block = pick_block(opt.block);
  RPCG_CHECK_ARG(opt.block == 0 || opt.block == block, "block must be 0, 128, 256 or 512");
  const int n = A->m.n;
  if (n == 0 && async) {
    // nothing to solve: the result of an empty system, written in stream order
    SolveState zero{};
    zero.status = RPCG_OK;
    k_set_state<<<1, 1, 0, s>>>(A->state, zero);
    if (opt.history) RPCG_CUDA_TRY(cudaMemsetAsync(opt.history, 0, sizeof(double), s));
    k_finish_result<<<1, 32, 0, s>>>(A->state, INFINITY, v, 0, x, 0, res);
    RPCG_CUDA_TRY(cudaGetLastError());
    return RPCG_OK;
  }
  if (n == 0) {
    res->iterations = 0;
    res->status = RPCG_OK;
    res->relres = 0.0;
    res->tau = 0.0;
    res->fpe_inexact_count = 0;
    if (opt.history) RPCG_CUDA_TRY(cudaMemsetAsync(opt.history, 0, sizeof(double), s));
    RPCG_CUDA_TRY(cudaStreamSynchronize(s));
    return RPCG_OK;
  }
  const bool eager = pass_ms != nullptr;
  // small systems with the default launch shape: one cluster-resident launch
  bool small = false;
  if (!eager && opt.block == 0 && opt.grid == 0) {
    rpcg_status st = small_solve(A, b, x, v, opt, s, &small);
    if (st != RPCG_OK) return st;
  }
  cudaGraphExec_t exec = nullptr;
  if (!eager && !small) {
    rpcg_status st = get_graph(A, v, block, opt.grid, &exec);
    if (st != RPCG_OK) return st;
    RPCG_CUDA_TRY(set_x0(A, A->x0_nodes[GraphKey{v, block, opt.grid}], exec, x));
  }
  SolveArgs* ha = A->h_args;
  if (!small) {
  SolveArgs av{};
  av.b = b;
  av.x = x;
  av.history = opt.history;
  av.tol = opt.tol;
  av.max_iter = opt.max_iter;
  av.fpe_size = opt.fpe_size;
  av.fpe_strict = opt.fpe_strict;
  av.variant = v;
  av.use_cond = eager ? 0 : 1;
  if (async) {
    k_set_args<<<1, 1, 0, s>>>(A->args, av);
    RPCG_CUDA_TRY(cudaGetLastError());
  } else {
    *ha = av;
    RPCG_CUDA_TRY(cudaMemcpyAsync(A->args, ha, sizeof(SolveArgs), cudaMemcpyHostToDevice, s));
  }
  if (eager) {
    rpcg_status st;
#define RPCG_EAGER(VV, BB) st = run_eager<VV, BB>(A, opt.grid, x, s, pass_ms, launches)
    if (block == 128) {
      if (v == RPCG_PLAIN) RPCG_EAGER(RPCG_PLAIN, 128); else if (v == RPCG_EXBLAS) RPCG_EAGER(RPCG_EXBLAS, 128); else RPCG_EAGER(RPCG_FPE, 128);
    } else if (block == 512) {
      if (v == RPCG_PLAIN) RPCG_EAGER(RPCG_PLAIN, 512); else if (v == RPCG_EXBLAS) RPCG_EAGER(RPCG_EXBLAS, 512); else RPCG_EAGER(RPCG_FPE, 512);
    } else {
      if (v == RPCG_PLAIN) RPCG_EAGER(RPCG_PLAIN, 256); else if (v == RPCG_EXBLAS) RPCG_EAGER(RPCG_EXBLAS, 256); else RPCG_EAGER(RPCG_FPE, 256);
    }
#undef RPCG_EAGER
    if (st != RPCG_OK) return st;
  } else {
    RPCG_CUDA_TRY(cudaGraphLaunch(exec, s));
  }
  }
  if (async) {
    const int g = std::max(1, std::min((n + 255) / 256, sm_count() * 4));
    k_finish_result<<<g, 256, 0, s>>>(A->state, opt.tol, v, opt.fpe_strict, x, n, res);
    RPCG_CUDA_TRY(cudaGetLastError());
    return RPCG_OK;
  }
  RPCG_CUDA_TRY(cudaMemcpyAsync(A->h_state, A->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  RPCG_CUDA_TRY(cudaStreamSynchronize(s));
  const SolveState& hs = *A->h_state;
  if (hs.bzero) {
    RPCG_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)n * sizeof(double), s));
    RPCG_CUDA_TRY(cudaStreamSynchronize(s));
  }
  int status = hs.status;
  if (status == RPCG_OK) {
    if (!(hs.rel < opt.tol)) status = RPCG_NOT_CONVERGED;
    else if (v == RPCG_FPE && opt.fpe_strict && hs.fpe_inexact > 0) status = RPCG_FPE_INEXACT;
  }
  res->iterations = hs.iter;
  res->status = status;
  res->relres = hs.rel;
  res->tau = hs.tau;
  res->fpe_inexact_count = hs.fpe_inexact;
  res->fpe_size_used = v == RPCG_FPE ? hs.fpe_p : 0;
  return (rpcg_status)status;
}

rpcg_status rpcg_solve(rpcg_matrix_t A, const double* b, double* x, int32_t v, const rpcg_opts* o, rpcg_result* res,
                       void* stream) {
  clear_error();
  RPCG_CHECK_ARG(A != nullptr, "A is NULL");
  RPCG_CHECK_ARG(res != nullptr, "res is NULL");
  RPCG_CHECK_ARG(A->m.n == 0 || (b && x), "b or x is NULL");
  return solve_impl(A, b, x, v, o, res, (cudaStream_t)stream);
}

rpcg_status rpcg_solve_profiled(rpcg_matrix_t A, const double* b, double* x, int32_t v, const rpcg_opts* o,
                                rpcg_result* res, float* pass_ms, int32_t* launches, void* stream) {
  clear_error();
  RPCG_CHECK_ARG(A != nullptr, "A is NULL");
  RPCG_CHECK_ARG(res != nullptr && pass_ms != nullptr, "res or pass_ms is NULL");
  RPCG_CHECK_ARG(A->m.n == 0 || (b && x), "b or x is NULL");
  for (int i = 0; i < 4; i++) {
    pass_ms[i] = 0.f;
    if (launches) launches[i] = 0;
  }
  return solve_impl(A, b, x, v, o, res, (cudaStream_t)stream, pass_ms, launches);
}

rpcg_status rpcg_solve_async(rpcg_matrix_t A, const double* b, double* x, int32_t v, const rpcg_opts* o,
                             rpcg_result* res, void* stream) {
  clear_error();
  RPCG_CHECK_ARG(A != nullptr, "A is NULL");
  RPCG_CHECK_ARG(res != nullptr, "res is NULL");
  RPCG_CHECK_ARG(A->m.n == 0 || (b && x), "b or x is NULL");
  return solve_impl(A, b, x, v, o, res, (cudaStream_t)stream, nullptr, nullptr, true);
}

rpcg_status rpcg_solve_path(rpcg_matrix_t A, int32_t v, const rpcg_opts* o, int32_t* path) {
  clear_error();
  RPCG_CHECK_ARG(A != nullptr && path != nullptr, "A or path is NULL");
  rpcg_opts opt;
  if (o) opt = *o;
  else rpcg_opts_default(&opt);
  *path = small_path(A, v, opt);
  return RPCG_OK;
}

rpcg_status rpcg_solve_host(rpcg_matrix_t A, const double* b_host, double* x_host, int32_t v, const rpcg_opts* o,
                            rpcg_result* res, void* stream) {
  clear_error();
  RPCG_CHECK_ARG(A != nullptr, "A is NULL");
  RPCG_CHECK_ARG(res != nullptr, "res is NULL");
  RPCG_CHECK_ARG(A->m.n == 0 || (b_host && x_host), "b or x is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)A->m.n * sizeof(double);
  double* db = A->bx;
  double* dx = A->bx + (A->m.n > 0 ? A->m.n : 1);
  if (bytes) {
    RPCG_CUDA_TRY(cudaMemcpyAsync(db, b_host, bytes, cudaMemcpyHostToDevice, s));
    RPCG_CUDA_TRY(cudaMemcpyAsync(dx, x_host, bytes, cudaMemcpyHostToDevice, s));
  }
  rpcg_status st = solve_impl(A, db, dx, v, o, res, s);
  if (st < 0 && st != RPCG_ERR_NOT_SPD && st != RPCG_ERR_NONFINITE) return st;
  if (bytes) {
    RPCG_CUDA_TRY(cudaMemcpyAsync(x_host, dx, bytes, cudaMemcpyDeviceToHost, s));
    RPCG_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return st;
}

}  // extern "C"
