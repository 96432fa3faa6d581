// Device side of the batched solver, shared by the batch API (batch.cu) and
// the serving loop (server.cu): per-system records, the work-unit driver and
// the pass kernels.  See batch.cu for the scheme.
//
// Work units are ranges of `tile` rows of one system (unit k of system s is
// rows [k tile, min(n_s, (k+1) tile))).  After the set-up pass and after
// every iteration a one-block kernel lists the units of the systems still
// iterating as a prefix over systems (aprefix[s] = index of system s's
// first unit among the listed ones).  CTAs take chunks of listed units
// (up to kChunkUnits, one when few are listed) from an atomic work counter,
// so the work of the systems still iterating is spread over the whole GPU
// however few they are.  Inside a chunk the consecutive units of one
// system share the CTA's register windows and shared accumulator; the CTA
// flushes them once per system and adds the number of units it did to that
// system's arrival counter; the CTA whose addition completes the system
// finishes it.
#pragma once
#include <climits>
#include <type_traits>

#include "device.cuh"
#include "solver.cuh"

namespace rpcg {

// One system of a batch: its matrix, vectors and stopping rule.
struct SysDev {
  MatDev m;
  const double* b;
  double* x;
  double *r, *d, *w, *inv;
  double* history;  // max_iter + 1 relres values, or null
  double tol;
  int max_iter;
  int fpe_size, fpe_strict;  // fpe variant: expansion size (0: adaptive), 1: report inexact dots
  int pad;
};

struct SysState {
  double rho, beta, beta_old, tau, gamma, bnorm, rel;
  int iter, status, bad_row, bzero, active, pad;
  int fpe_p, fpe_inexact;  // fpe variant: expansion size in use, inexact dots seen
  int redo, pad2;          // fpe variant: 1 / 2 = pass A's / pass B's dots to recompute exactly
  double zr;               // fpe variant: <z,r> of pass B1, finished with <r,r> in pass B2
  int zr_lost, pad3;
};

// per-system reduction scratch (digits, arrival counter, flags)
struct SysRed {
  unsigned long long digits[3][kNDig];
  unsigned int counter;
  unsigned int flags;
};

constexpr int kChunkUnits = 4;  // listed units a CTA takes at a time
enum { kWorkSetup = 0, kWorkA = 1, kWorkB = 2, kWorkRA = 3, kWorkRB = 4, kWorkB2 = 5, kWorkCounters = 6 };

struct BatchHead {
  int active_count;  // systems still iterating
  int redo_any;      // fpe variant: bit 0 / 1 = some system recomputes pass A's / pass B's dots
  unsigned int work[kWorkCounters];  // work counters of the reducing passes
};

// Everything the kernels need about a batch (passed by value).
struct BatchDesc {
  const SysDev* sys;
  SysState* st;
  SysRed* red;
  BatchHead* head;
  int* aprefix;        // [count + 1] listed units of the iterating systems
  const int* nunits;   // [count] units of each system
  const int* uprefix;  // [count + 1] first unit of each system among all units (plain partials), or null
  double* partials;    // plain variant: per unit, 3 values
  int count;
  int tile;
};

static __device__ __forceinline__ void b_stop(SysState* st, BatchHead* head) {
  if (st->active) {
    st->active = 0;
    atomicSub(&head->active_count, 1);
  }
}

// the system of listed unit a: the largest s with prefix[s] <= a (systems
// with no listed units have prefix[s] == prefix[s + 1] and are skipped)
__device__ __forceinline__ int unit_system(const int* prefix, int count, int a) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= a) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Block-wide exclusive scan (blockDim.x a multiple of 32, at most 1024);
// *total receives the sum over the block.
static __device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;  // inclusive sums of the warp totals
  }
  __syncthreads();
  const int excl = x - v + (wid ? wsum[wid - 1] : 0);
  *total = wsum[nw - 1];
  __syncthreads();  // wsum may be reused
  return excl;
}

// One block: list the units of the systems that take part (every system
// with rows when `setup`, else the systems still iterating) as a prefix
// over systems.  Systems are split into contiguous per-thread ranges so the
// listing keeps system order.
static __device__ void build_prefix(const BatchDesc& B, bool setup) {
  const int T = blockDim.x;
  const int per = (B.count + T - 1) / T;
  const int lo = min(B.count, (int)threadIdx.x * per), hi = min(B.count, lo + per);
  auto units_of = [&](int s) { return (setup ? B.sys[s].m.n > 0 : B.st[s].active != 0) ? B.nunits[s] : 0; };
  int sum = 0;
  for (int s = lo; s < hi; s++) sum += units_of(s);
  int total = 0;
  int run = block_exclusive_scan(sum, &total);
  for (int s = lo; s < hi; s++) {
    B.aprefix[s] = run;
    run += units_of(s);
  }
  if (threadIdx.x == 0) B.aprefix[B.count] = total;
}

// ------------------------------------------------------------------ L2 prefetch
//
// Each warp of a reducing pass works on 32 consecutive rows per step; its
// lane 0 asks the copy engine to bring the rows of kPfSteps steps later
// into L2 (cp.async.bulk.prefetch: a hint that changes no value), so the
// DRAM stream does not wait for the threads' own loads to be issued.

constexpr int kPfSteps = 2;

__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(bytes) : "memory");
}

// the SELL-32 slab (values and columns) of the slice holding `row`
__device__ __forceinline__ void l2_prefetch_slice(const MatDev& m, int row) {
  const int sl = row >> 5;
  const long long so = __ldg(m.sptr + sl), se = __ldg(m.sptr + sl + 1);
  if (se > so) {
    l2_prefetch(m.val + so, (unsigned)((se - so) * 8));
    l2_prefetch(m.col + so, (unsigned)((se - so) * 4));
  }
}

// ------------------------------------------------------------------ unit driver

struct UnitSmem {
  double sw[32];
  long long dig[kNDig];
  uint32_t D[kNDig];
  double value[3];
  int range[2];
  int base;
  unsigned int lost;  // fpe: bit j = dot j inexact (an expansion lost bits, or a non-finite operand)
  bool last;
};

// the unit prefix is copied to shared memory for batches of up to
// kPrefixSmem - 1 systems; larger ones search it in global memory
constexpr int kPrefixSmem = 1024;

template <int V>
__host__ __device__ constexpr size_t b_smem(int nacc, int count) {
  return (V != RPCG_PLAIN ? (size_t)nacc * kNDig * kCopies * 8 : 0) + sizeof(UnitSmem) +
         (size_t)(count + 1 <= kPrefixSmem ? count + 1 : 0) * 4 + 16;
}

// Process the listed units of `prefix`, taking chunks from *work.
// row_fn(sys, row, dep) deposits dep(j, a, b) into dot j; fin_fn(sys,
// values, lost) runs in thread 0 of the CTA that completes a system (lost:
// the fpe variant's inexact-dot bits, 0 otherwise).
// row2_fn(ctx, ra, rb, dep) does rows ra and rb together (both in range);
// pass a NullRow2 to process rows one at a time.  skip_fn(sys) == true
// skips a system's units altogether (no deposit, no arrival, no fin_fn).
// fpe: fpe_dot_step (twoprod on the integer pipe, the Accumulate cascades
// with two_sum_fast in the result and two_sum_split in the error expansion).
struct NullRow2 {};
struct NoSkip {
  __device__ bool operator()(int) const { return false; }
};

template <int V, int NACC, int BLOCK, class CtxFn, class PfFn, class RowFn, class FinFn,
          class Row2Fn = NullRow2, class SkipFn = NoSkip>
__device__ __forceinline__ void for_units(const BatchDesc& B, const int* __restrict__ prefix, unsigned int* work,
                                          unsigned char* smem, CtxFn ctx_fn, PfFn pf_fn, RowFn row_fn,
                                          FinFn fin_fn, Row2Fn row2_fn = NullRow2{}, SkipFn skip_fn = NoSkip{}) {
  constexpr bool kPair = !std::is_same<Row2Fn, NullRow2>::value;
  unsigned long long* sacc = reinterpret_cast<unsigned long long*>(smem);
  UnitSmem* us = reinterpret_cast<UnitSmem*>(smem + (V != RPCG_PLAIN ? NACC * kNDig * kCopies * 8 : 0));
  const int copy = threadIdx.x & (kCopies - 1);
  const int* sp = prefix;
  if (B.count + 1 <= kPrefixSmem) {
    int* cp = reinterpret_cast<int*>(us + 1);
    for (int i = threadIdx.x; i <= B.count; i += BLOCK) cp[i] = prefix[i];
    sp = cp;
  }
  __syncthreads();
  const int total = sp[B.count];
  // chunks of up to kChunkUnits units while there is plenty of work; single
  // units when few are listed, so they spread over every CTA
  const int chunk = max(1, min(kChunkUnits, total / (2 * (int)gridDim.x)));
  for (;;) {
    if (threadIdx.x == 0) us->base = (int)atomicAdd(work, (unsigned)chunk);
    __syncthreads();
    const int base = us->base;
    __syncthreads();  // everyone has read base
    if (base >= total) break;
    const int end = min(base + chunk, total);
    for (int a = base; a < end;) {
      const int s = unit_system(sp, B.count, a);
      const int run_end = min(end, sp[s + 1]);
      if (skip_fn(s)) {  // the same answer in every thread: a system's record is stable during the pass
        a = run_end;
        continue;
      }
      const int k0 = a - sp[s], k1 = k0 + (run_end - a);  // units [k0, k1) of system s
      const int n = B.sys[s].m.n;
      SysRed* R = B.red + s;
      // what the rows of this run need (pointers, scalars) in registers: the
      // row stores could alias the system table, so reading it per row would
      // reload it every time
      const auto ctx = ctx_fn(s);
      if constexpr (V == RPCG_EXBLAS) {
        Window win[NACC];
        bool bad = false;
#pragma unroll
        for (int j = 0; j < NACC; j++) window_init(win[j]);
        smem_acc_zero(sacc, NACC);
        __syncthreads();
        const int r0 = k0 * B.tile, r1 = min(n, k1 * B.tile);
        auto dep = [&](int j, double x, double y) {
          const ExactProd e = exact_product(x, y);
          bad |= e.bad;
          exact_deposit(win[j], sacc + j * kNDig * kCopies, copy, e);
        };
        for (int row = r0 + threadIdx.x; row < r1; row += (kPair ? 2 : 1) * BLOCK) {
          const int ahead = row + kPfSteps * BLOCK;
          if ((threadIdx.x & 31) == 0 && ahead < r1) pf_fn(ctx, ahead);
          if constexpr (kPair) {
            if (row + BLOCK < r1) row2_fn(ctx, row, row + BLOCK, dep);
            else row_fn(ctx, row, dep);
          } else {
            row_fn(ctx, row, dep);
          }
        }
#pragma unroll
        for (int j = 0; j < NACC; j++) window_flush(win[j], sacc + j * kNDig * kCopies, copy);
        if (bad) atomicOr(&R->flags, 1u);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NACC; j++) smem_to_global(sacc + j * kNDig * kCopies, R->digits[j]);
      } else if constexpr (V == RPCG_FPE) {
        // each thread's rows into its result and error expansions (Algs. 2
        // and 4), merged (Alg. 3) at the end of the run; the terms are then
        // deposited exactly into the system's long accumulator, as in the
        // single-system passes
        double res[NACC][kFpeMax], err[NACC][kFpeMax];
        bool lost[NACC];
        bool bad = false;
#pragma unroll
        for (int j = 0; j < NACC; j++) {
#pragma unroll
          for (int i = 0; i < kFpeMax; i++) res[j][i] = err[j][i] = 0.0;
          lost[j] = false;
        }
        const int p = B.st[s].fpe_p;
        smem_acc_zero(sacc, NACC);
        __syncthreads();
        const int r0 = k0 * B.tile, r1 = min(n, k1 * B.tile);
        auto dep = [&](int j, double x, double y) {
          if (!is_finite_bits(x) || !is_finite_bits(y)) bad = true;
          else lost[j] |= fpe_dot_step(res[j], err[j], p, x, y, bad);
        };
        for (int row = r0 + threadIdx.x; row < r1; row += (kPair ? 2 : 1) * BLOCK) {
          const int ahead = row + kPfSteps * BLOCK;
          if ((threadIdx.x & 31) == 0 && ahead < r1) pf_fn(ctx, ahead);
          if constexpr (kPair) {
            if (row + BLOCK < r1) row2_fn(ctx, row, row + BLOCK, dep);
            else row_fn(ctx, row, dep);
          } else {
            row_fn(ctx, row, dep);
          }
        }
#pragma unroll
        for (int j = 0; j < NACC; j++) {
          lost[j] |= fpe_sum(res[j], err[j], p, bad);
          if (lost[j]) atomicOr(&R->flags, 2u << j);
          Window win;
          window_init(win);
#pragma unroll 1
          for (int i = 0; i < p; i++) {
            double t = res[j][0];
#pragma unroll
            for (int k = 1; k < kFpeMax; k++)
              if (i == k) t = res[j][k];
            if (!is_zero_bits(t)) {
              const ExactProd e = exact_product(t, 1.0);
              bad |= e.bad;
              exact_deposit(win, sacc + j * kNDig * kCopies, copy, e);
            }
          }
          window_flush(win, sacc + j * kNDig * kCopies, copy);
        }
        if (bad) atomicOr(&R->flags, 1u);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NACC; j++) smem_to_global(sacc + j * kNDig * kCopies, R->digits[j]);
      } else {
        // plain: one fixed-order partial per unit, summed in unit order at the end
        for (int k = k0; k < k1; k++) {
          double acc[NACC];
#pragma unroll
          for (int j = 0; j < NACC; j++) acc[j] = 0.0;
          const int r0 = k * B.tile, r1 = min(n, (k + 1) * B.tile);
          auto dep = [&](int j, double x, double y) { acc[j] = __fma_rn(x, y, acc[j]); };
          for (int row = r0 + threadIdx.x; row < r1; row += BLOCK) {
            const int ahead = row + kPfSteps * BLOCK;
            if ((threadIdx.x & 31) == 0 && ahead < r1) pf_fn(ctx, ahead);
            row_fn(ctx, row, dep);
          }
#pragma unroll
          for (int j = 0; j < NACC; j++) {
            const double sblk = block_sum_fixed<BLOCK>(acc[j], us->sw);
            if (threadIdx.x == 0) B.partials[(size_t)(B.uprefix[s] + k) * 3 + j] = sblk;
          }
        }
        __threadfence();
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int cnt = (unsigned)(k1 - k0);
        const unsigned int prev = atomicAdd(&R->counter, cnt);
        us->last = (prev + cnt == (unsigned)B.nunits[s]);
      }
      __syncthreads();
      if (us->last) {
        __threadfence();
        if constexpr (V != RPCG_PLAIN) {
#pragma unroll
          for (int j = 0; j < NACC; j++) {
            const double v = take_and_round(R->digits[j], us->dig, us->D, us->range);
            if (threadIdx.x == 0) us->value[j] = v;
            __syncthreads();
          }
          if (threadIdx.x == 0) {
            const unsigned int f = atomicExch(&R->flags, 0u);
            // a non-finite operand makes every dot of the pass NaN (and, for
            // fpe, inexact); otherwise bit j + 1 flags dot j's lost bits
            us->lost = (f & 1u) ? (1u << NACC) - 1u : (f >> 1) & ((1u << NACC) - 1u);
            if (f & 1u)
              for (int j = 0; j < NACC; j++) us->value[j] = __longlong_as_double(0x7FF8000000000000ll);
          }
        } else {
          if (threadIdx.x == 0) {
            for (int j = 0; j < NACC; j++) {
              double v = 0.0;
              for (int k = 0; k < B.nunits[s]; k++) v = __dadd_rn(v, __ldcg(&B.partials[(size_t)(B.uprefix[s] + k) * 3 + j]));
              us->value[j] = v;
            }
          }
        }
        if (threadIdx.x == 0) {
          if constexpr (V == RPCG_PLAIN) us->lost = 0u;
          R->counter = 0;
          fin_fn(s, us->value, V == RPCG_FPE ? us->lost : 0u);
        }
      }
      __syncthreads();
      a = run_end;
    }
  }
}

// ------------------------------------------------------------------ scalar steps (one thread)

// S2: rho = beta / <d, w> (with the breakdown checks).
static __device__ void b_finalize_a(SysState* t, double dw, BatchHead* head) {
  if (!isfinite(dw)) {
    t->status = RPCG_ERR_NONFINITE;
    b_stop(t, head);
    return;
  }
  if (!(dw > 0.0)) {
    t->status = RPCG_ERR_NOT_SPD;
    b_stop(t, head);
    return;
  }
  t->beta_old = t->beta;
  t->rho = __ddiv_rn(t->beta, dw);
}

// After S6 and S8: gamma, the iteration count, relres and the system's own
// stopping test.
static __device__ void b_finalize_b(const BatchDesc& B, int s, double beta, double tau) {
  SysState* t = B.st + s;
  const SysDev& S = B.sys[s];
  t->beta = beta;
  t->tau = tau;
  if (!isfinite(beta) || !isfinite(tau)) {
    t->status = RPCG_ERR_NONFINITE;
    t->iter += 1;
    b_stop(t, B.head);
    return;
  }
  t->gamma = __ddiv_rn(beta, t->beta_old);
  t->iter += 1;
  t->rel = __ddiv_rn(__dsqrt_rn(tau), t->bnorm);
  if (S.history) S.history[t->iter] = t->rel;
  if (tau > 0.0 && !(beta > 0.0)) {
    t->status = RPCG_ERR_NOT_SPD;
    b_stop(t, B.head);
    return;
  }
  if (!((t->rel >= S.tol) && (t->iter < S.max_iter))) {
    t->active = 2;  // finished this iteration: pass C still updates d (unobservable), then it stops
  }
}

// FPE variant, after a pass whose dots `lost` flags: count the inexact dots,
// grow the adaptive size by one, and with fpe_strict = 0 mark the system
// for the exact recomputation of the pass's dots (phase 1: pass A, 2: pass
// B).  Returns true when the pass's finalisation waits for that.  The same
// rules as the single-system passes.
static __device__ bool b_fpe_inexact(const BatchDesc& B, int s, unsigned lost, int phase) {
  if (!lost) return false;
  SysState* t = B.st + s;
  t->fpe_inexact += __popc(lost);
  if (B.sys[s].fpe_size == 0 && t->fpe_p < kFpeMax) t->fpe_p += 1;
  if (B.sys[s].fpe_strict) return false;
  t->redo = phase;
  atomicOr(&B.head->redo_any, phase);
  return true;
}

// ------------------------------------------------------------------ kernels

// Per-run contexts of the reducing passes.
struct PassACtx {
  MatDev m;
  const double* __restrict__ d;
  double* __restrict__ w;
};

struct PassBCtx {
  double* __restrict__ x;
  double* __restrict__ r;
  const double* __restrict__ d;
  const double* __restrict__ w;
  const double* __restrict__ inv;
  double rho;
  bool stopped;
};

// Reset the states of every system with rows, list their units, clear the
// work counters (one block).
static __global__ void k_b_init(BatchDesc B) {
  for (int s = threadIdx.x; s < B.count; s += blockDim.x) {
    SysState& t = B.st[s];
    t.rho = t.beta = t.beta_old = t.gamma = t.bnorm = 0.0;
    t.tau = t.rel = __longlong_as_double(0x7FF8000000000000ll);
    t.iter = 0;
    t.status = 0;
    t.bad_row = INT_MAX;
    t.bzero = 0;
    t.active = B.sys[s].m.n > 0 ? 1 : 0;  // an empty system has no units: done at once
    t.pad = 0;
    // the adaptive expansion size starts at 3, the size Sec. 4.3 finds enough for Poisson
    t.fpe_p = B.sys[s].fpe_size > 0 ? B.sys[s].fpe_size : 3;
    t.fpe_inexact = 0;
    t.redo = 0;
    t.pad2 = 0;
  }
  __shared__ int nact;
  if (threadIdx.x == 0) nact = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < B.count; s += blockDim.x)
    if (B.sys[s].m.n > 0) atomicAdd(&nact, 1);
  build_prefix(B, true);
  __syncthreads();
  if (threadIdx.x == 0) {
    B.head->active_count = nact;
    B.head->redo_any = 0;
    for (int k = 0; k < kWorkCounters; k++) B.head->work[k] = 0u;
  }
}

// Reset the listed (newly admitted) systems' states (serving loop).
static __global__ void k_b_init_list(BatchDesc B, const int* __restrict__ list, int nlist) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nlist; k += gridDim.x * blockDim.x) {
    const int s = list[k];
    SysState& t = B.st[s];
    t.rho = t.beta = t.beta_old = t.gamma = t.bnorm = 0.0;
    t.tau = t.rel = __longlong_as_double(0x7FF8000000000000ll);
    t.iter = 0;
    t.status = 0;
    t.bad_row = INT_MAX;
    t.bzero = 0;
    t.active = B.sys[s].m.n > 0 ? 1 : 0;
    if (t.active) atomicAdd(&B.head->active_count, 1);
    t.pad = 0;
    t.fpe_p = B.sys[s].fpe_size > 0 ? B.sys[s].fpe_size : 3;
    t.fpe_inexact = 0;
    t.redo = 0;
    t.pad2 = 0;
  }
}

// Inverse diagonal and A x0 for the listed units (no reduction: static split).
static __global__ void k_b_inv_q(BatchDesc B, const int* __restrict__ prefix) {
  const int total = prefix[B.count];
  for (int a = blockIdx.x; a < total; a += gridDim.x) {
    const int s = unit_system(prefix, B.count, a);
    const SysDev& S = B.sys[s];
    const int k = a - prefix[s];
    const int r1 = min(S.m.n, (k + 1) * B.tile);
    for (int i = k * B.tile + threadIdx.x; i < r1; i += blockDim.x) {
      double aii = 0.0;
      bool found = false;
      const int len = S.m.rowptr[i + 1] - S.m.rowptr[i];
      const long long base = sell_index(S.m, i, 0);
      for (int q = 0; q < len; q++) {
        if (S.m.col[base + 32ll * q] == i) {
          aii = S.m.val[base + 32ll * q];
          found = true;
        }
      }
      if (!found || !(aii > 0.0)) {
        atomicMin(&B.st[s].bad_row, i);
        S.inv[i] = 0.0;
      } else {
        S.inv[i] = __drcp_rn(aii);
      }
      S.w[i] = sell_row(S.m, i, S.x);
    }
  }
}

template <int V, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_b_setup(BatchDesc B, const int* __restrict__ prefix) {
  extern __shared__ __align__(16) unsigned char smem[];
  for_units<V, 3, BLOCK>(
      B, prefix, &B.head->work[kWorkSetup], smem, [&](int s) { return B.sys[s]; }, [](const SysDev&, int) {},
      [&](const SysDev& S, int i, auto dep) {
        const double bi = S.b[i];
        const double ri = __dsub_rn(bi, S.w[i]);
        const double zi = __dmul_rn(S.inv[i], ri);
        S.r[i] = ri;
        S.d[i] = zi;
        dep(0, zi, ri);
        dep(1, ri, ri);
        dep(2, bi, bi);
      },
      [&](int s, const double* v, unsigned) {
        SysState* t = B.st + s;
        const SysDev& S = B.sys[s];
        if (t->bad_row < S.m.n) {
          const int i = t->bad_row;
          double aii = 0.0;
          const int len = S.m.rowptr[i + 1] - S.m.rowptr[i];
          const long long base = sell_index(S.m, i, 0);
          for (int k = 0; k < len; k++)
            if (S.m.col[base + 32ll * k] == i) aii = S.m.val[base + 32ll * k];
          t->status = isfinite(aii) ? RPCG_ERR_NOT_SPD : RPCG_ERR_NONFINITE;
          b_stop(t, B.head);
          return;
        }
        if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])) {
          t->status = RPCG_ERR_NONFINITE;
          b_stop(t, B.head);
          return;
        }
        t->beta = v[0];
        const double bnorm = __dsqrt_rn(v[2]);
        t->bnorm = bnorm;
        double* hist = S.history;
        if (bnorm == 0.0) {
          t->bzero = 1;
          t->rel = 0.0;
          t->tau = 0.0;
          if (hist) hist[0] = 0.0;
          b_stop(t, B.head);
          return;
        }
        t->tau = v[1];
        t->rel = __ddiv_rn(__dsqrt_rn(v[1]), bnorm);
        if (hist) hist[0] = t->rel;
        if (!((t->rel >= S.tol) && (0 < S.max_iter))) b_stop(t, B.head);
      });
}

template <int V, int BLOCK>
__global__ void __launch_bounds__(BLOCK, V == RPCG_FPE ? 512 / BLOCK : 768 / BLOCK) k_b_pass_a(BatchDesc B) {
  extern __shared__ __align__(16) unsigned char smem[];
  for_units<V, 1, BLOCK>(
      B, B.aprefix, &B.head->work[kWorkA], smem,
      [&](int s) {
        const SysDev& S = B.sys[s];
        return PassACtx{S.m, S.d, S.w};
      },
      [](const PassACtx& c, int i) { l2_prefetch_slice(c.m, i); },
      [&](const PassACtx& c, int i, auto dep) {
        const double v = sell_row(c.m, i, c.d);
        c.w[i] = v;
        dep(0, __ldg(c.d + i), v);
      },
      [&](int s, const double* v, unsigned lost) {
        SysState* t = B.st + s;
        if (V == RPCG_FPE && b_fpe_inexact(B, s, lost, 1)) return;  // recomputed by k_b_redo_a
        b_finalize_a(t, v[0], B.head);
      },
      [&](const PassACtx& c, int ia, int ib, auto dep) {
        double va, vb;
        sell_rows2(c.m, ia, ib, c.d, va, vb);
        c.w[ia] = va;
        c.w[ib] = vb;
        dep(0, __ldg(c.d + ia), va);
        dep(0, __ldg(c.d + ib), vb);
      });
}

template <int V, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_b_pass_b(BatchDesc B) {
  extern __shared__ __align__(16) unsigned char smem[];
  for_units<V, 2, BLOCK>(
      B, B.aprefix, &B.head->work[kWorkB], smem,
      [&](int s) {
        const SysDev& S = B.sys[s];
        const SysState& t = B.st[s];
        return PassBCtx{S.x, S.r, S.d, S.w, S.inv, t.rho, t.status != 0};
      },
      [](const PassBCtx&, int) {},
      [&](const PassBCtx& c, int i, auto dep) {
        if (c.stopped) return;  // stopped in pass A of this iteration
        const double di = c.d[i], wi = c.w[i];
        const double xi = __fma_rn(c.rho, di, c.x[i]);
        const double ri = __fma_rn(-c.rho, wi, c.r[i]);
        const double zi = __dmul_rn(c.inv[i], ri);
        c.x[i] = xi;
        c.r[i] = ri;
        dep(0, zi, ri);
        dep(1, ri, ri);
      },
      [&](int s, const double* v, unsigned lost) {
        if (B.st[s].status != 0) return;
        if (V == RPCG_FPE && b_fpe_inexact(B, s, lost, 2)) return;  // recomputed by k_b_redo_b
        b_finalize_b(B, s, v[0], v[1]);
      },
      [&](const PassBCtx& c, int ia, int ib, auto dep) {
        if (c.stopped) return;
        // both rows' loads first, then the arithmetic of each row as in the single-row form
        const double da = c.d[ia], wa = c.w[ia], xa0 = c.x[ia], ra0 = c.r[ia], va = c.inv[ia];
        const double db = c.d[ib], wb = c.w[ib], xb0 = c.x[ib], rb0 = c.r[ib], vb = c.inv[ib];
        const double xa = __fma_rn(c.rho, da, xa0), ra = __fma_rn(-c.rho, wa, ra0), za = __dmul_rn(va, ra);
        const double xb = __fma_rn(c.rho, db, xb0), rb = __fma_rn(-c.rho, wb, rb0), zb = __dmul_rn(vb, rb);
        c.x[ia] = xa;
        c.r[ia] = ra;
        c.x[ib] = xb;
        c.r[ib] = rb;
        dep(0, za, ra);
        dep(1, ra, ra);
        dep(0, zb, rb);
        dep(1, rb, rb);
      });
}

// FPE variant: pass B as two passes, so that each thread holds one pair of
// expansions (64 registers), as in the single-system solve.  B1: S3-S6 (<z,r>, kept in the system's
// state); B2: S8 (<r,r> of the new r) and the finalisation of both dots.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_b_pass_b1(BatchDesc B) {
  extern __shared__ __align__(16) unsigned char smem[];
  for_units<RPCG_FPE, 1, BLOCK>(
      B, B.aprefix, &B.head->work[kWorkB], smem,
      [&](int s) {
        const SysDev& S = B.sys[s];
        const SysState& t = B.st[s];
        return PassBCtx{S.x, S.r, S.d, S.w, S.inv, t.rho, t.status != 0};
      },
      [](const PassBCtx&, int) {},
      [&](const PassBCtx& c, int i, auto dep) {
        if (c.stopped) return;  // stopped in pass A of this iteration
        const double xi = __fma_rn(c.rho, c.d[i], c.x[i]);
        const double ri = __fma_rn(-c.rho, c.w[i], c.r[i]);
        const double zi = __dmul_rn(c.inv[i], ri);
        c.x[i] = xi;
        c.r[i] = ri;
        dep(0, zi, ri);
      },
      [&](int s, const double* v, unsigned lost) {
        SysState* t = B.st + s;
        t->zr = v[0];
        t->zr_lost = (int)(lost & 1u);
      });
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_b_pass_b2(BatchDesc B) {
  extern __shared__ __align__(16) unsigned char smem[];
  for_units<RPCG_FPE, 1, BLOCK>(
      B, B.aprefix, &B.head->work[kWorkB2], smem,
      [&](int s) {
        const SysDev& S = B.sys[s];
        return PassBCtx{S.x, S.r, S.d, S.w, S.inv, 0.0, B.st[s].status != 0};
      },
      [](const PassBCtx&, int) {},
      [&](const PassBCtx& c, int i, auto dep) {
        if (c.stopped) return;
        const double ri = c.r[i];
        dep(0, ri, ri);
      },
      [&](int s, const double* v, unsigned lost) {
        SysState* t = B.st + s;
        if (t->status != 0) return;
        const unsigned both = (t->zr_lost ? 1u : 0u) | ((lost & 1u) << 1);
        if (b_fpe_inexact(B, s, both, 2)) return;  // recomputed by k_b_redo_b
        b_finalize_b(B, s, t->zr, v[0]);
      });
}

// FPE variant with fpe_strict = 0: the systems whose pass A (or pass B) dots
// were inexact recompute them exactly and take the pass's scalar step; the
// other systems' units are skipped.  Nothing to do (and every CTA returns at
// once) when no system asked.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_b_redo_a(BatchDesc B) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (!(*(volatile int*)&B.head->redo_any & 1)) return;
  for_units<RPCG_EXBLAS, 1, BLOCK>(
      B, B.aprefix, &B.head->work[kWorkRA], smem,
      [&](int s) {
        const SysDev& S = B.sys[s];
        return PassACtx{S.m, S.d, S.w};
      },
      [](const PassACtx&, int) {},
      [&](const PassACtx& c, int i, auto dep) { dep(0, c.d[i], c.w[i]); },
      [&](int s, const double* v, unsigned) {
        SysState* t = B.st + s;
        t->redo = 0;
        b_finalize_a(t, v[0], B.head);
      },
      NullRow2{}, [&](int s) { return B.st[s].redo != 1; });
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_b_redo_b(BatchDesc B) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (!(*(volatile int*)&B.head->redo_any & 2)) return;
  for_units<RPCG_EXBLAS, 2, BLOCK>(
      B, B.aprefix, &B.head->work[kWorkRB], smem,
      [&](int s) {
        const SysDev& S = B.sys[s];
        return PassBCtx{S.x, S.r, S.d, S.w, S.inv, 0.0, false};
      },
      [](const PassBCtx&, int) {},
      [&](const PassBCtx& c, int i, auto dep) {
        const double ri = c.r[i];
        const double zi = __dmul_rn(c.inv[i], ri);
        dep(0, zi, ri);
        dep(1, ri, ri);
      },
      [&](int s, const double* v, unsigned) {
        B.st[s].redo = 0;
        b_finalize_b(B, s, v[0], v[1]);
      },
      NullRow2{}, [&](int s) { return B.st[s].redo != 2; });
}

// S7 for every listed system that is still running (no reduction: static split).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_b_pass_c(BatchDesc B) {
  const int* prefix = B.aprefix;
  const int total = prefix[B.count];
  for (int a = blockIdx.x; a < total; a += gridDim.x) {
    const int s = unit_system(prefix, B.count, a);
    const SysState& t = B.st[s];
    if (!t.active || t.status != 0) continue;
    const SysDev& S = B.sys[s];
    const double g = t.gamma;
    const int k = a - prefix[s];
    const int r1 = min(S.m.n, (k + 1) * B.tile);
    for (int i = k * B.tile + threadIdx.x; i < r1; i += BLOCK) {
      const double zi = __dmul_rn(S.inv[i], S.r[i]);
      S.d[i] = __fma_rn(g, S.d[i], zi);
    }
  }
}

// One block, after pass C: retire the systems that finished in pass B, list
// the units of the systems still iterating, clear the work counters; with a
// graph conditional handle, set the while node's condition.
static __device__ void retire_and_list(BatchDesc B) {
  for (int s = threadIdx.x; s < B.count; s += blockDim.x) {
    if (B.st[s].active == 2 || (B.st[s].active && B.st[s].status != 0)) b_stop(B.st + s, B.head);
  }
  __syncthreads();
  build_prefix(B, false);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < kWorkCounters; k++) B.head->work[k] = 0u;
    B.head->redo_any = 0;
    __threadfence();
  }
}

static __global__ void k_b_cond(BatchDesc B, cudaGraphConditionalHandle cond) {
  retire_and_list(B);
  if (threadIdx.x == 0) cudaGraphSetConditional(cond, atomicAdd(&B.head->active_count, 0) > 0 ? 1u : 0u);
}

// The serving loop's form (the host reads the states between chunks).
static __global__ void k_b_retire(BatchDesc B) { retire_and_list(B); }

}  // namespace rpcg
