// Device side of the batched solver, shared by the batch API (batch.cu) and
// the serving loop (server.cu): per-system records, the work-unit driver and
// the pass kernels.  See batch.cu for the scheme.
#pragma once
#include <climits>

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
  int pad;
};

struct SysState {
  double rho, beta, beta_old, tau, gamma, bnorm, rel;
  int iter, status, bad_row, bzero, active, pad;
};

struct Unit {
  int sys, r0, r1;
};

struct BatchScratchHead {
  int active_count;
  int pad;
};

// per-system reduction scratch (digits, arrival counter, flags)
struct SysRed {
  unsigned long long digits[3][kNDig];
  unsigned int counter;
  unsigned int flags;
};

static __device__ __forceinline__ void b_stop(SysState* st, BatchScratchHead* head) {
  if (st->active) {
    st->active = 0;
    atomicSub(&head->active_count, 1);
  }
}

// ------------------------------------------------------------------ unit driver

struct UnitSmem {
  double sw[32];
  long long dig[kNDig];
  uint32_t D[kNDig];
  double value[3];
  bool last;
};

// Process every unit of the active systems.  row_fn(sys, row, R, sacc)
// deposits into the reducer; fin_fn(sys, values) runs in thread 0 of the
// CTA that completes a system.  `need_active` = 0 processes every system
// (the set-up pass).
template <int V, int NACC, int BLOCK, class RowFn, class FinFn>
__device__ __forceinline__ void for_units(const Unit* __restrict__ units, const int* __restrict__ nunits_p,
                                          const int* __restrict__ unit_count,
                                          SysState* states, SysRed* red, double* unit_partials, bool need_active,
                                          unsigned char* smem, RowFn row_fn, FinFn fin_fn) {
  unsigned long long* sacc = reinterpret_cast<unsigned long long*>(smem);
  UnitSmem* us = reinterpret_cast<UnitSmem*>(smem + (V == RPCG_EXBLAS ? NACC * kNDig * kCopies * 8 : 0));
  const int copy = threadIdx.x & (kCopies - 1);
  const int nunits = *nunits_p;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const Unit U = units[u];
    if (need_active && !states[U.sys].active) continue;  // uniform over the CTA
    Window win[NACC];
    double acc[NACC];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < NACC; j++) {
      window_init(win[j]);
      acc[j] = 0.0;
    }
    if constexpr (V == RPCG_EXBLAS) smem_acc_zero(sacc, NACC);
    __syncthreads();
    for (int row = U.r0 + threadIdx.x; row < U.r1; row += BLOCK) {
      row_fn(U.sys, row, [&](int j, double a, double b) {
        if constexpr (V == RPCG_EXBLAS) {
          const ExactProd e = exact_product(a, b);
          bad |= e.bad;
          exact_deposit(win[j], sacc + j * kNDig * kCopies, copy, e);
        } else {
          acc[j] = __fma_rn(a, b, acc[j]);
        }
      });
    }
    SysRed* R = red + U.sys;
    if constexpr (V == RPCG_EXBLAS) {
#pragma unroll
      for (int j = 0; j < NACC; j++) window_flush(win[j], sacc + j * kNDig * kCopies, copy);
      if (bad) atomicOr(&R->flags, 1u);
      __syncthreads();
      for (int j = 0; j < NACC; j++) smem_to_global(sacc + j * kNDig * kCopies, R->digits[j]);
    } else {
      for (int j = 0; j < NACC; j++) {
        const double sblk = block_sum_fixed<BLOCK>(acc[j], us->sw);
        if (threadIdx.x == 0) unit_partials[(size_t)u * 3 + j] = sblk;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned int prev = atomicAdd(&R->counter, 1u);
      us->last = (prev == (unsigned)unit_count[U.sys] - 1u);
    }
    __syncthreads();
    if (us->last) {
      __threadfence();
      if constexpr (V == RPCG_EXBLAS) {
        for (int j = 0; j < NACC; j++) {
          for (int k = threadIdx.x; k < kNDig; k += BLOCK) us->dig[k] = (long long)atomicExch(&R->digits[j][k], 0ull);
          __syncthreads();
          if (threadIdx.x == 0) us->value[j] = round_digits(us->dig, us->D);
          __syncthreads();
        }
        if (threadIdx.x == 0) {
          const unsigned int f = atomicExch(&R->flags, 0u);
          if (f & 1u)
            for (int j = 0; j < NACC; j++) us->value[j] = __longlong_as_double(0x7FF8000000000000ll);
        }
      } else {
        if (threadIdx.x == 0) {
          // the system's units are contiguous: sum their partials in unit order
          int first = u;
          while (first > 0 && units[first - 1].sys == U.sys) first--;
          for (int j = 0; j < NACC; j++) {
            double v = 0.0;
            for (int k = 0; k < unit_count[U.sys]; k++) v = __dadd_rn(v, __ldcg(&unit_partials[(size_t)(first + k) * 3 + j]));
            us->value[j] = v;
          }
        }
      }
      if (threadIdx.x == 0) {
        R->counter = 0;
        fin_fn(U.sys, us->value);
      }
    }
    __syncthreads();
  }
}

template <int V>
__host__ __device__ constexpr size_t b_smem(int nacc) {
  return (V == RPCG_EXBLAS ? (size_t)nacc * kNDig * kCopies * 8 : 0) + sizeof(UnitSmem) + 16;
}

// ------------------------------------------------------------------ kernels

static __global__ void k_b_init(const SysDev* __restrict__ sys, SysState* st, BatchScratchHead* head, int count,
                                int nactive) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
    SysState& t = st[s];
    t.rho = t.beta = t.beta_old = t.gamma = t.bnorm = 0.0;
    t.tau = t.rel = __longlong_as_double(0x7FF8000000000000ll);
    t.iter = 0;
    t.status = 0;
    t.bad_row = INT_MAX;
    t.bzero = 0;
    t.active = sys[s].m.n > 0 ? 1 : 0;  // an empty system has no units: done at once
    t.pad = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) head->active_count = nactive;
}

// inverse diagonal and A x0 for every unit
static __global__ void k_b_inv_q(const SysDev* __restrict__ sys, const Unit* __restrict__ units,
                                 const int* __restrict__ nunits_p, SysState* st) {
  const int nunits = *nunits_p;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const Unit U = units[u];
    const SysDev& S = sys[U.sys];
    for (int i = U.r0 + threadIdx.x; i < U.r1; i += blockDim.x) {
      double aii = 0.0;
      bool found = false;
      const int len = S.m.rowptr[i + 1] - S.m.rowptr[i];
      const long long base = sell_index(S.m, i, 0);
      for (int k = 0; k < len; k++) {
        if (S.m.col[base + 32ll * k] == i) {
          aii = S.m.val[base + 32ll * k];
          found = true;
        }
      }
      if (!found || !(aii > 0.0)) {
        atomicMin(&st[U.sys].bad_row, i);
        S.inv[i] = 0.0;
      } else {
        S.inv[i] = __drcp_rn(aii);
      }
      S.w[i] = sell_row(S.m, i, S.x);
    }
  }
}

template <int V, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_b_setup(const SysDev* __restrict__ sys, const Unit* __restrict__ units,
                                                   const int* __restrict__ nunits, const int* __restrict__ unit_count,
                                                   SysState* st, SysRed* red, double* unit_partials,
                                                   BatchScratchHead* head) {
  extern __shared__ __align__(16) unsigned char smem[];
  for_units<V, 3, BLOCK>(
      units, nunits, unit_count, st, red, unit_partials, false, smem,
      [&](int s, int i, auto dep) {
        const SysDev& S = sys[s];
        const double bi = S.b[i];
        const double ri = __dsub_rn(bi, S.w[i]);
        const double zi = __dmul_rn(S.inv[i], ri);
        S.r[i] = ri;
        S.d[i] = zi;
        dep(0, zi, ri);
        dep(1, ri, ri);
        dep(2, bi, bi);
      },
      [&](int s, const double* v) {
        SysState* t = st + s;
        const SysDev& S = sys[s];
        if (t->bad_row < S.m.n) {
          const int i = t->bad_row;
          double aii = 0.0;
          const int len = S.m.rowptr[i + 1] - S.m.rowptr[i];
          const long long base = sell_index(S.m, i, 0);
          for (int k = 0; k < len; k++)
            if (S.m.col[base + 32ll * k] == i) aii = S.m.val[base + 32ll * k];
          t->status = isfinite(aii) ? RPCG_ERR_NOT_SPD : RPCG_ERR_NONFINITE;
          b_stop(t, head);
          return;
        }
        if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])) {
          t->status = RPCG_ERR_NONFINITE;
          b_stop(t, head);
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
          b_stop(t, head);
          return;
        }
        t->tau = v[1];
        t->rel = __ddiv_rn(__dsqrt_rn(v[1]), bnorm);
        if (hist) hist[0] = t->rel;
        if (!((t->rel >= S.tol) && (0 < S.max_iter))) b_stop(t, head);
      });
}

template <int V, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_b_pass_a(const SysDev* __restrict__ sys, const Unit* __restrict__ units,
                                                    const int* __restrict__ nunits, const int* __restrict__ unit_count,
                                                    SysState* st, SysRed* red, double* unit_partials,
                                                    BatchScratchHead* head) {
  extern __shared__ __align__(16) unsigned char smem[];
  for_units<V, 1, BLOCK>(
      units, nunits, unit_count, st, red, unit_partials, true, smem,
      [&](int s, int i, auto dep) {
        const SysDev& S = sys[s];
        const double v = sell_row(S.m, i, S.d);
        S.w[i] = v;
        dep(0, __ldg(S.d + i), v);
      },
      [&](int s, const double* v) {
        SysState* t = st + s;
        const double dw = v[0];
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
      });
}

template <int V, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_b_pass_b(const SysDev* __restrict__ sys, const Unit* __restrict__ units,
                                                    const int* __restrict__ nunits, const int* __restrict__ unit_count,
                                                    SysState* st, SysRed* red, double* unit_partials,
                                                    BatchScratchHead* head) {
  extern __shared__ __align__(16) unsigned char smem[];
  for_units<V, 2, BLOCK>(
      units, nunits, unit_count, st, red, unit_partials, true, smem,
      [&](int s, int i, auto dep) {
        const SysDev& S = sys[s];
        const double rho = st[s].rho;
        const double di = S.d[i], wi = S.w[i];
        const double xi = __fma_rn(rho, di, S.x[i]);
        const double ri = __fma_rn(-rho, wi, S.r[i]);
        const double zi = __dmul_rn(S.inv[i], ri);
        S.x[i] = xi;
        S.r[i] = ri;
        dep(0, zi, ri);
        dep(1, ri, ri);
      },
      [&](int s, const double* v) {
        SysState* t = st + s;
        const SysDev& S = sys[s];
        const double beta = v[0], tau = v[1];
        t->beta = beta;
        t->tau = tau;
        if (!isfinite(beta) || !isfinite(tau)) {
          t->status = RPCG_ERR_NONFINITE;
          t->iter += 1;
          b_stop(t, head);
          return;
        }
        t->gamma = __ddiv_rn(beta, t->beta_old);
        t->iter += 1;
        t->rel = __ddiv_rn(__dsqrt_rn(tau), t->bnorm);
        if (S.history) S.history[t->iter] = t->rel;
        if (tau > 0.0 && !(beta > 0.0)) {
          t->status = RPCG_ERR_NOT_SPD;
          b_stop(t, head);
          return;
        }
        if (!((t->rel >= S.tol) && (t->iter < S.max_iter))) {
          t->active = 2;  // finished this iteration: pass C still updates d (unobservable), then it stops
        }
      });
}

// S7 for every system that ran pass B this iteration; systems that finished
// in pass B leave the active set here.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_b_pass_c(const SysDev* __restrict__ sys, const Unit* __restrict__ units,
                                                    const int* __restrict__ nunits_p, SysState* st) {
  const int nunits = *nunits_p;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const Unit U = units[u];
    const SysState& t = st[U.sys];
    if (!t.active || t.status != 0) continue;
    const SysDev& S = sys[U.sys];
    const double g = t.gamma;
    for (int i = U.r0 + threadIdx.x; i < U.r1; i += BLOCK) {
      const double zi = __dmul_rn(S.inv[i], S.r[i]);
      S.d[i] = __fma_rn(g, S.d[i], zi);
    }
  }
}

// Retire the systems that finished in pass B and set the loop condition.
static __global__ void k_b_cond(SysState* st, int count, BatchScratchHead* head, cudaGraphConditionalHandle cond) {
  for (int s = threadIdx.x; s < count; s += blockDim.x) {
    if (st[s].active == 2) b_stop(st + s, head);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    cudaGraphSetConditional(cond, atomicAdd(&head->active_count, 0) > 0 ? 1u : 0u);
  }
}

// Retire the systems that finished in pass B (the serving loop's form of
// k_b_cond: the host reads the states between chunks of iterations).
static __global__ void k_b_retire(SysState* st, int count, BatchScratchHead* head) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
    if (st[s].active == 2) b_stop(st + s, head);
  }
}

// Reset the states of the listed systems (newly admitted ones).
static __global__ void k_b_init_list(const int* __restrict__ list, int nlist, const SysDev* __restrict__ sys,
                                     SysState* st, BatchScratchHead* head) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nlist; k += gridDim.x * blockDim.x) {
    const int s = list[k];
    SysState& t = st[s];
    t.rho = t.beta = t.beta_old = t.gamma = t.bnorm = 0.0;
    t.tau = t.rel = __longlong_as_double(0x7FF8000000000000ll);
    t.iter = 0;
    t.status = 0;
    t.bad_row = INT_MAX;
    t.bzero = 0;
    t.active = sys[s].m.n > 0 ? 1 : 0;
    if (t.active) atomicAdd(&head->active_count, 1);
    t.pad = 0;
  }
}

}  // namespace rpcg
