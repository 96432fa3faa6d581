// Batched Jacobi-PCG: many independent SPD systems in one launch sequence.
//
// The systems keep their own matrix handles (SELL-32 copy, r, d, w, inv);
// the batch adds per-system scalars, per-system long accumulators and a list
// of work units -- ranges of at most `tile` rows of one system.  Each pass
// (set-up, A, B, C of Fig. 2) is one persistent kernel over all units of the
// systems still iterating; every unit deposits its dot products into its
// system's accumulators, and the CTA that completes a system's last unit
// finishes that system's reduction and scalar step (rho, or beta, tau,
// gamma, relres and its own convergence test).  Systems that have converged
// drop out of later passes.  A one-thread kernel sets the while node's
// condition from the count of systems still active.
//
// Every row, element and scalar operation is the one rpcg_solve performs
// and exact dots do not depend on how the work is split, so each system's
// iterates, residuals and iteration count are bit-identical to solving it
// alone (with RPCG_EXBLAS).  The plain variant sums unit partials in unit
// order: deterministic for a given tile size, not reproducible across tiles.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <tuple>
#include <vector>

#include "device.cuh"
#include "host.h"
#include "solver.cuh"

namespace rpcg {

struct SysDev {
  MatDev m;
  const double* b;
  double* x;
  double *r, *d, *w, *inv;
};

struct SysState {
  double rho, beta, beta_old, tau, gamma, bnorm, rel;
  int iter, status, bad_row, bzero, active, pad;
};

struct Unit {
  int sys, r0, r1;
};

struct BatchArgs {
  double* history;  // count x (max_iter + 1), or null
  double tol;
  int max_iter;
  int count;
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

__device__ __forceinline__ void b_stop(SysState* st, BatchScratchHead* head) {
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
__device__ __forceinline__ void for_units(const Unit* __restrict__ units, int nunits, const int* __restrict__ unit_count,
                                          SysState* states, SysRed* red, double* unit_partials, bool need_active,
                                          unsigned char* smem, RowFn row_fn, FinFn fin_fn) {
  unsigned long long* sacc = reinterpret_cast<unsigned long long*>(smem);
  UnitSmem* us = reinterpret_cast<UnitSmem*>(smem + (V == RPCG_EXBLAS ? NACC * kNDig * kCopies * 8 : 0));
  const int copy = threadIdx.x & (kCopies - 1);
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

__global__ void k_b_init(const SysDev* __restrict__ sys, SysState* st, BatchScratchHead* head, int count,
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
__global__ void k_b_inv_q(const SysDev* __restrict__ sys, const Unit* __restrict__ units, int nunits, SysState* st) {
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
                                                   int nunits, const int* __restrict__ unit_count, SysState* st,
                                                   SysRed* red, double* unit_partials, BatchScratchHead* head,
                                                   const BatchArgs* args) {
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
        double* hist = args->history ? args->history + (size_t)s * (args->max_iter + 1) : nullptr;
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
        if (!((t->rel >= args->tol) && (0 < args->max_iter))) b_stop(t, head);
      });
}

template <int V, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_b_pass_a(const SysDev* __restrict__ sys, const Unit* __restrict__ units,
                                                    int nunits, const int* __restrict__ unit_count, SysState* st,
                                                    SysRed* red, double* unit_partials, BatchScratchHead* head) {
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
                                                    int nunits, const int* __restrict__ unit_count, SysState* st,
                                                    SysRed* red, double* unit_partials, BatchScratchHead* head,
                                                    const BatchArgs* args) {
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
        if (args->history) args->history[(size_t)s * (args->max_iter + 1) + t->iter] = t->rel;
        if (tau > 0.0 && !(beta > 0.0)) {
          t->status = RPCG_ERR_NOT_SPD;
          b_stop(t, head);
          return;
        }
        if (!((t->rel >= args->tol) && (t->iter < args->max_iter))) {
          t->active = 2;  // finished this iteration: pass C still updates d (unobservable), then it stops
        }
      });
}

// S7 for every system that ran pass B this iteration; systems that finished
// in pass B leave the active set here.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_b_pass_c(const SysDev* __restrict__ sys, const Unit* __restrict__ units,
                                                    int nunits, SysState* st) {
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
__global__ void k_b_cond(SysState* st, int count, BatchScratchHead* head, cudaGraphConditionalHandle cond) {
  for (int s = threadIdx.x; s < count; s += blockDim.x) {
    if (st[s].active == 2) b_stop(st + s, head);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    cudaGraphSetConditional(cond, atomicAdd(&head->active_count, 0) > 0 ? 1u : 0u);
  }
}

}  // namespace rpcg

struct rpcg_batch_s {
  int count = 0;
  int nactive0 = 0;  // systems with at least one row
  std::vector<rpcg_matrix_t> mats;
  rpcg::SysDev* d_sys = nullptr;
  rpcg::SysDev* h_sys = nullptr;  // pinned
  rpcg::SysState* d_state = nullptr;
  rpcg::SysState* h_state = nullptr;  // pinned
  rpcg::SysRed* d_red = nullptr;
  rpcg::BatchScratchHead* d_head = nullptr;
  rpcg::BatchArgs* d_args = nullptr;
  rpcg::BatchArgs* h_args = nullptr;  // pinned
  // per tile size: units, unit counts, partials
  struct Layout {
    rpcg::Unit* units = nullptr;
    int* unit_count = nullptr;
    double* partials = nullptr;
    int nunits = 0;
  };
  std::map<int, Layout> layouts;
  std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;  // (variant, block, tile)
  std::map<std::tuple<int, int, int>, cudaGraph_t> graph_defs;
  int tuned_block = 0, tuned_tile = 0;
};

namespace rpcg {

static rpcg_status batch_layout(rpcg_batch_t B, int tile, rpcg_batch_s::Layout** out) {
  auto it = B->layouts.find(tile);
  if (it != B->layouts.end()) {
    *out = &it->second;
    return RPCG_OK;
  }
  std::vector<Unit> units;
  std::vector<int> counts(B->count, 0);
  for (int s = 0; s < B->count; s++) {
    const int n = B->mats[s]->m.n;
    for (int r0 = 0; r0 < n; r0 += tile) {
      units.push_back(Unit{s, r0, std::min(n, r0 + tile)});
      counts[s]++;
    }
    if (n == 0) counts[s] = 0;
  }
  rpcg_batch_s::Layout L;
  L.nunits = (int)units.size();
  RPCG_CUDA_TRY(cudaMalloc(&L.units, std::max<size_t>(1, units.size()) * sizeof(Unit)));
  RPCG_CUDA_TRY(cudaMalloc(&L.unit_count, std::max<size_t>(1, counts.size()) * sizeof(int)));
  RPCG_CUDA_TRY(cudaMalloc(&L.partials, std::max<size_t>(1, units.size()) * 3 * sizeof(double)));
  if (!units.empty()) RPCG_CUDA_TRY(cudaMemcpy(L.units, units.data(), units.size() * sizeof(Unit), cudaMemcpyHostToDevice));
  RPCG_CUDA_TRY(cudaMemcpy(L.unit_count, counts.data(), counts.size() * sizeof(int), cudaMemcpyHostToDevice));
  B->layouts[tile] = L;
  *out = &B->layouts[tile];
  return RPCG_OK;
}

static cudaError_t add_node(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* deps, int ndeps,
                            const void* func, int grid, int block, size_t smem, void** args) {
  cudaKernelNodeParams p{};
  p.func = const_cast<void*>(func);
  p.gridDim = dim3(grid);
  p.blockDim = dim3(block);
  p.sharedMemBytes = (unsigned)smem;
  p.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &p);
}

template <int V, int BLOCK>
static rpcg_status batch_graph(rpcg_batch_t B, int tile, cudaGraph_t* out_g, cudaGraphExec_t* out_e) {
  rpcg_batch_s::Layout* L = nullptr;
  rpcg_status st = batch_layout(B, tile, &L);
  if (st != RPCG_OK) return st;
  const size_t sm1 = b_smem<V>(1), sm2 = b_smem<V>(2), sm3 = b_smem<V>(3);
  RPCG_CUDA_TRY(cudaFuncSetAttribute((const void*)k_b_setup<V, BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
  RPCG_CUDA_TRY(cudaFuncSetAttribute((const void*)k_b_pass_a<V, BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
  RPCG_CUDA_TRY(cudaFuncSetAttribute((const void*)k_b_pass_b<V, BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
  auto occ_grid = [&](const void* f, size_t smem) {
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, BLOCK, smem) != cudaSuccess || occ < 1) occ = 1;
    int g = sm_count() * occ;
    if (g > L->nunits) g = L->nunits > 0 ? L->nunits : 1;
    return g;
  };
  const int g_setup = occ_grid((const void*)k_b_setup<V, BLOCK>, sm3);
  const int g_a = occ_grid((const void*)k_b_pass_a<V, BLOCK>, sm1);
  const int g_b = occ_grid((const void*)k_b_pass_b<V, BLOCK>, sm2);
  const int g_c = occ_grid((const void*)k_b_pass_c<BLOCK>, 0);
  const int g_q = occ_grid((const void*)k_b_inv_q, 0);

  cudaGraph_t g = nullptr;
  RPCG_CUDA_TRY(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond;
  RPCG_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
  SysDev* sys = B->d_sys;
  SysState* sst = B->d_state;
  SysRed* red = B->d_red;
  BatchScratchHead* head = B->d_head;
  BatchArgs* args = B->d_args;
  Unit* units = L->units;
  int nunits = L->nunits;
  int* ucount = L->unit_count;
  double* partials = L->partials;
  int count = B->count;
  int nactive = B->nactive0;
  cudaGraphNode_t n_init, n_q, n_setup, n_c0, n_loop;
  {
    void* a[] = {&sys, &sst, &head, &count, &nactive};
    RPCG_CUDA_TRY(add_node(g, &n_init, nullptr, 0, (const void*)k_b_init, (count + 255) / 256, 256, 0, a));
  }
  {
    void* a[] = {&sys, &units, &nunits, &sst};
    RPCG_CUDA_TRY(add_node(g, &n_q, &n_init, 1, (const void*)k_b_inv_q, g_q, BLOCK, 0, a));
  }
  {
    void* a[] = {&sys, &units, &nunits, &ucount, &sst, &red, &partials, &head, &args};
    RPCG_CUDA_TRY(add_node(g, &n_setup, &n_q, 1, (const void*)k_b_setup<V, BLOCK>, g_setup, BLOCK, sm3, a));
  }
  {
    void* a[] = {&sst, &count, &head, &cond};
    RPCG_CUDA_TRY(add_node(g, &n_c0, &n_setup, 1, (const void*)k_b_cond, 1, 256, 0, a));
  }
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  RPCG_CUDA_TRY(cudaGraphAddNode(&n_loop, g, &n_c0, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaGraphNode_t b_a, b_b, b_c, b_cond;
  {
    void* a[] = {&sys, &units, &nunits, &ucount, &sst, &red, &partials, &head};
    RPCG_CUDA_TRY(add_node(body, &b_a, nullptr, 0, (const void*)k_b_pass_a<V, BLOCK>, g_a, BLOCK, sm1, a));
  }
  {
    void* a[] = {&sys, &units, &nunits, &ucount, &sst, &red, &partials, &head, &args};
    RPCG_CUDA_TRY(add_node(body, &b_b, &b_a, 1, (const void*)k_b_pass_b<V, BLOCK>, g_b, BLOCK, sm2, a));
  }
  {
    void* a[] = {&sys, &units, &nunits, &sst};
    RPCG_CUDA_TRY(add_node(body, &b_c, &b_b, 1, (const void*)k_b_pass_c<BLOCK>, g_c, BLOCK, 0, a));
  }
  {
    void* a[] = {&sst, &count, &head, &cond};
    RPCG_CUDA_TRY(add_node(body, &b_cond, &b_c, 1, (const void*)k_b_cond, 1, 256, 0, a));
  }
  cudaGraphExec_t e = nullptr;
  RPCG_CUDA_TRY(cudaGraphInstantiate(&e, g, 0));
  *out_g = g;
  *out_e = e;
  return RPCG_OK;
}

static rpcg_status batch_get_graph(rpcg_batch_t B, int v, int block, int tile, cudaGraphExec_t* e) {
  auto key = std::make_tuple(v, block, tile);
  auto it = B->graphs.find(key);
  if (it != B->graphs.end()) {
    *e = it->second;
    return RPCG_OK;
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  rpcg_status st;
  if (block == 128) st = v == RPCG_PLAIN ? batch_graph<RPCG_PLAIN, 128>(B, tile, &g, &ex) : batch_graph<RPCG_EXBLAS, 128>(B, tile, &g, &ex);
  else st = v == RPCG_PLAIN ? batch_graph<RPCG_PLAIN, 256>(B, tile, &g, &ex) : batch_graph<RPCG_EXBLAS, 256>(B, tile, &g, &ex);
  if (st != RPCG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  B->graphs[key] = ex;
  B->graph_defs[key] = g;
  *e = ex;
  return RPCG_OK;
}

static void batch_free(rpcg_batch_t B) {
  if (!B) return;
  for (auto& kv : B->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : B->graph_defs) cudaGraphDestroy(kv.second);
  for (auto& kv : B->layouts) {
    cudaFree(kv.second.units);
    cudaFree(kv.second.unit_count);
    cudaFree(kv.second.partials);
  }
  cudaFree(B->d_sys);
  cudaFree(B->d_state);
  cudaFree(B->d_red);
  cudaFree(B->d_head);
  cudaFree(B->d_args);
  cudaFreeHost(B->h_sys);
  cudaFreeHost(B->h_state);
  cudaFreeHost(B->h_args);
  delete B;
}

// One launch of the batch graph (set-up + loop) with the given b/x.
static rpcg_status batch_run(rpcg_batch_t B, const double* const* b, double* const* x, int v, const rpcg_opts& o,
                             int block, int tile, cudaStream_t s) {
  cudaGraphExec_t e = nullptr;
  rpcg_status st = batch_get_graph(B, v, block, tile, &e);
  if (st != RPCG_OK) return st;
  for (int i = 0; i < B->count; i++) {
    rpcg_matrix_t A = B->mats[i];
    B->h_sys[i] = SysDev{A->m, b[i], x[i], A->r, A->d, A->w, A->inv};
  }
  B->h_args->history = o.history;
  B->h_args->tol = o.tol;
  B->h_args->max_iter = o.max_iter;
  B->h_args->count = B->count;
  RPCG_CUDA_TRY(cudaMemcpyAsync(B->d_sys, B->h_sys, B->count * sizeof(SysDev), cudaMemcpyHostToDevice, s));
  RPCG_CUDA_TRY(cudaMemcpyAsync(B->d_args, B->h_args, sizeof(BatchArgs), cudaMemcpyHostToDevice, s));
  RPCG_CUDA_TRY(cudaGraphLaunch(e, s));
  return RPCG_OK;
}

}  // namespace rpcg

using namespace rpcg;

extern "C" {

rpcg_status rpcg_batch_create(rpcg_batch_t* out, int32_t count, const rpcg_matrix_t* A) {
  clear_error();
  RPCG_CHECK_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  RPCG_CHECK_ARG(count >= 1 && A != nullptr, "count must be >= 1 and A non-NULL");
  std::set<rpcg_matrix_t> seen;
  for (int i = 0; i < count; i++) {
    RPCG_CHECK_ARG(A[i] != nullptr, "a matrix handle is NULL");
    RPCG_CHECK_ARG(seen.insert(A[i]).second, "a matrix handle appears twice in the batch");
  }
  rpcg_batch_t B = new rpcg_batch_s();
  B->count = count;
  B->mats.assign(A, A + count);
  for (int i = 0; i < count; i++) B->nactive0 += A[i]->m.n > 0 ? 1 : 0;
  cudaError_t e = cudaMalloc(&B->d_sys, count * sizeof(SysDev));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_state, count * sizeof(SysState));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_red, count * sizeof(SysRed));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_head, sizeof(BatchScratchHead));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_args, sizeof(BatchArgs));
  if (e == cudaSuccess) e = cudaMallocHost(&B->h_sys, count * sizeof(SysDev));
  if (e == cudaSuccess) e = cudaMallocHost(&B->h_state, count * sizeof(SysState));
  if (e == cudaSuccess) e = cudaMallocHost(&B->h_args, sizeof(BatchArgs));
  if (e == cudaSuccess) e = cudaMemset(B->d_red, 0, count * sizeof(SysRed));
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_free(B);
    set_error("rpcg_batch_create: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RPCG_ERR_OOM : RPCG_ERR_CUDA;
  }
  *out = B;
  return RPCG_OK;
}

rpcg_status rpcg_batch_destroy(rpcg_batch_t B) {
  clear_error();
  if (!B) return RPCG_OK;
  cudaDeviceSynchronize();
  batch_free(B);
  return RPCG_OK;
}

rpcg_status rpcg_batch_solve(rpcg_batch_t B, const double* const* b, double* const* x, int32_t v, const rpcg_opts* o,
                             rpcg_result* res, void* stream) {
  clear_error();
  RPCG_CHECK_ARG(B != nullptr && b != nullptr && x != nullptr && res != nullptr, "NULL argument");
  RPCG_CHECK_ARG(v == RPCG_PLAIN || v == RPCG_EXBLAS, "batched solves support the plain and exblas variants");
  rpcg_opts opt;
  if (o) opt = *o;
  else rpcg_opts_default(&opt);
  RPCG_CHECK_ARG(opt.max_iter >= 0 && !(opt.tol < 0.0) && !std::isnan(opt.tol), "bad tol or max_iter");
  RPCG_CHECK_ARG(opt.block == 0 || opt.block == 128 || opt.block == 256, "block must be 0, 128 or 256 here");
  RPCG_CHECK_ARG(opt.tile >= 0, "tile must be >= 0");
  for (int i = 0; i < B->count; i++) RPCG_CHECK_ARG(B->mats[i]->m.n == 0 || (b[i] && x[i]), "b[i] or x[i] is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int block = opt.block, tile = opt.tile;
  if (block == 0 || tile == 0) {
    if (!B->tuned_block) {
      // autotune: time a short run of every candidate (set-up + 8 iterations), keep the fastest.
      // The runs iterate on the handles' staging buffers (zeroed), never on the caller's x.
      rpcg_opts t = opt;
      t.max_iter = 8;
      t.history = nullptr;
      std::vector<double*> xt(B->count);
      for (int i = 0; i < B->count; i++) {
        rpcg_matrix_t Ai = B->mats[i];
        const int ni = Ai->m.n;
        xt[i] = Ai->bx + (ni > 0 ? ni : 1);
        if (ni) RPCG_CUDA_TRY(cudaMemsetAsync(xt[i], 0, (size_t)ni * sizeof(double), s));
      }
      cudaEvent_t e0, e1;
      RPCG_CUDA_TRY(cudaEventCreate(&e0));
      RPCG_CUDA_TRY(cudaEventCreate(&e1));
      float best = 1e30f;
      for (int cb : {128, 256}) {
        for (int ct : {2048, 8192, 32768}) {
          rpcg_status st = batch_run(B, b, xt.data(), RPCG_EXBLAS, t, cb, ct, s);  // builds the graph (untimed)
          if (st != RPCG_OK) return st;
          RPCG_CUDA_TRY(cudaEventRecord(e0, s));
          st = batch_run(B, b, xt.data(), RPCG_EXBLAS, t, cb, ct, s);
          if (st != RPCG_OK) return st;
          RPCG_CUDA_TRY(cudaEventRecord(e1, s));
          RPCG_CUDA_TRY(cudaEventSynchronize(e1));
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best) {
            best = ms;
            B->tuned_block = cb;
            B->tuned_tile = ct;
          }
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    if (block == 0) block = B->tuned_block;
    if (tile == 0) tile = B->tuned_tile;
  }
  rpcg_status st = batch_run(B, b, x, v, opt, block, tile, s);
  if (st != RPCG_OK) return st;
  RPCG_CUDA_TRY(cudaMemcpyAsync(B->h_state, B->d_state, B->count * sizeof(SysState), cudaMemcpyDeviceToHost, s));
  RPCG_CUDA_TRY(cudaStreamSynchronize(s));
  rpcg_status worst = RPCG_OK;
  for (int i = 0; i < B->count; i++) {
    const SysState& h = B->h_state[i];
    const int n = B->mats[i]->m.n;
    if (n == 0) {
      res[i] = rpcg_result{0, RPCG_OK, 0.0, 0.0, 0, 0};
      continue;
    }
    if (h.bzero) RPCG_CUDA_TRY(cudaMemsetAsync(x[i], 0, (size_t)n * sizeof(double), s));
    int status = h.status;
    if (status == RPCG_OK && !(h.rel < opt.tol)) status = RPCG_NOT_CONVERGED;
    res[i] = rpcg_result{h.iter, status, h.rel, h.tau, 0, 0};
    if (status < 0 && (worst >= 0 || status < worst)) worst = (rpcg_status)status;
    else if (status > 0 && worst == RPCG_OK) worst = (rpcg_status)status;
  }
  RPCG_CUDA_TRY(cudaStreamSynchronize(s));
  return worst;
}

rpcg_status rpcg_batch_tuned(rpcg_batch_t B, int32_t* block, int32_t* tile) {
  RPCG_CHECK_ARG(B != nullptr, "B is NULL");
  if (block) *block = B->tuned_block;
  if (tile) *tile = B->tuned_tile;
  return RPCG_OK;
}

rpcg_status rpcg_solve_batched(int32_t count, const rpcg_matrix_t* A, const double* const* b, double* const* x,
                               int32_t v, const rpcg_opts* o, rpcg_result* res, void* stream) {
  rpcg_batch_t B = nullptr;
  rpcg_status st = rpcg_batch_create(&B, count, A);
  if (st != RPCG_OK) return st;
  st = rpcg_batch_solve(B, b, x, v, o, res, stream);
  rpcg_batch_destroy(B);
  return st;
}

}  // extern "C"
