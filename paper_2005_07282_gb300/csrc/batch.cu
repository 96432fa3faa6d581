// Batched Jacobi-PCG: many independent SPD systems in one launch sequence.
//
// The systems keep their own matrix handles (SELL-32 copy, r, d, w, inv);
// the batch adds per-system scalars and per-system long accumulators, and
// cuts every system into work units of `tile` rows.  Each pass (set-up, A,
// B, C of Fig. 2) is one persistent kernel over the units of the systems
// still iterating, which CTAs take in chunks from a work counter; every unit
// deposits its dot products into its system's accumulators, and the CTA that
// completes a system's last unit finishes that system's reduction and
// scalar step (rho, or beta, tau, gamma, relres and its own convergence
// test).  After every iteration a one-block kernel retires the systems that
// stopped, lists the units of the others for the next iteration and sets
// the while node's condition, so converged systems cost nothing afterwards
// and the last few systems still iterating are spread over all SMs.
//
// Every row, element and scalar operation is the one rpcg_solve performs
// and exact dots do not depend on how the work is split, so each system's
// iterates, residuals and iteration count are bit-identical to solving it
// alone (with RPCG_EXBLAS, and with RPCG_FPE, whose inexact dots are
// recomputed exactly by two extra passes that skip the other systems).  The
// plain variant sums unit partials in unit order: deterministic for a given
// tile size, not reproducible across tiles.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <tuple>
#include <vector>

#include "batch.cuh"
#include "host.h"

struct rpcg_batch_s {
  int count = 0;
  std::vector<rpcg_matrix_t> mats;
  rpcg::SysDev* d_sys = nullptr;
  rpcg::SysDev* h_sys = nullptr;  // pinned
  rpcg::SysState* d_state = nullptr;
  rpcg::SysState* h_state = nullptr;  // pinned
  rpcg::SysRed* d_red = nullptr;
  rpcg::BatchHead* d_head = nullptr;
  int* d_aprefix = nullptr;  // [count + 1] listed units, rebuilt by the kernels
  // per tile size: units per system, their prefix, plain partials
  struct Layout {
    int* nunits = nullptr;   // [count]
    int* uprefix = nullptr;  // [count + 1]
    double* partials = nullptr;
    int total = 0;  // units of all systems
  };
  std::map<int, Layout> layouts;
  std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;  // (variant, block, tile)
  std::map<std::tuple<int, int, int>, cudaGraph_t> graph_defs;
  int tuned_block = 0, tuned_tile = 0;
  cudaEvent_t uploaded = nullptr;  // the last upload of h_sys (rewritten only after it ran)
};

namespace rpcg {

static rpcg_status batch_layout(rpcg_batch_t B, int tile, rpcg_batch_s::Layout** out) {
  auto it = B->layouts.find(tile);
  if (it != B->layouts.end()) {
    *out = &it->second;
    return RPCG_OK;
  }
  std::vector<int> counts(B->count, 0), prefix(B->count + 1, 0);
  for (int s = 0; s < B->count; s++) {
    const int n = B->mats[s]->m.n;
    counts[s] = (int)(((long long)n + tile - 1) / tile);
    prefix[s + 1] = prefix[s] + counts[s];
  }
  rpcg_batch_s::Layout L;
  L.total = prefix[B->count];
  RPCG_CUDA_TRY(cudaMalloc(&L.nunits, counts.size() * sizeof(int)));
  RPCG_CUDA_TRY(cudaMalloc(&L.uprefix, prefix.size() * sizeof(int)));
  RPCG_CUDA_TRY(cudaMalloc(&L.partials, std::max<size_t>(1, (size_t)L.total) * 3 * sizeof(double)));
  RPCG_CUDA_TRY(cudaMemcpy(L.nunits, counts.data(), counts.size() * sizeof(int), cudaMemcpyHostToDevice));
  RPCG_CUDA_TRY(cudaMemcpy(L.uprefix, prefix.data(), prefix.size() * sizeof(int), cudaMemcpyHostToDevice));
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

// Grid sizes and dynamic shared memory of the batch kernels for one
// (variant, block, tile): persistent grids of the occupancy limit.
struct BatchPlan {
  int g_setup, g_a, g_b, g_c, g_q, g_ra, g_rb;
  size_t sm1, sm2, sm3, smr1, smr2;
};

// the set-up dots of the fpe variant are exact (the single-system rule)
template <int V>
constexpr int setup_variant() {
  return V == RPCG_FPE ? RPCG_EXBLAS : V;
}

template <int V, int BLOCK>
static rpcg_status batch_plan(rpcg_batch_t B, const rpcg_batch_s::Layout* L, BatchPlan* P) {
  const int count = B->count;
  constexpr int VS = setup_variant<V>();
  P->sm1 = b_smem<V>(1, count);
  P->sm2 = b_smem<V>(2, count);
  P->sm3 = b_smem<VS>(3, count);
  P->smr1 = b_smem<RPCG_EXBLAS>(1, count);
  P->smr2 = b_smem<RPCG_EXBLAS>(2, count);
  RPCG_CUDA_TRY(cudaFuncSetAttribute((const void*)k_b_setup<VS, BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->sm3));
  RPCG_CUDA_TRY(cudaFuncSetAttribute((const void*)k_b_pass_a<V, BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->sm1));
  if constexpr (V != RPCG_FPE)  // the fpe variant's pass B is k_b_pass_b1 + k_b_pass_b2 (below)
    RPCG_CUDA_TRY(cudaFuncSetAttribute((const void*)k_b_pass_b<V, BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->sm2));
  auto occ_grid = [&](const void* f, size_t smem) {
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, BLOCK, smem) != cudaSuccess || occ < 1) occ = 1;
    int g = sm_count() * occ;
    if (g > L->total) g = L->total > 0 ? L->total : 1;
    return g;
  };
  P->g_setup = occ_grid((const void*)k_b_setup<VS, BLOCK>, P->sm3);
  P->g_a = occ_grid((const void*)k_b_pass_a<V, BLOCK>, P->sm1);
  if constexpr (V != RPCG_FPE) P->g_b = occ_grid((const void*)k_b_pass_b<V, BLOCK>, P->sm2);
  P->g_c = occ_grid((const void*)k_b_pass_c<BLOCK>, 0);
  P->g_q = occ_grid((const void*)k_b_inv_q, 0);
  P->g_ra = P->g_rb = 1;
  if constexpr (V == RPCG_FPE) {
    // pass B runs as B1 + B2 (one FPE dot each, the shared memory of pass A)
    RPCG_CUDA_TRY(cudaFuncSetAttribute((const void*)k_b_pass_b1<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->sm1));
    RPCG_CUDA_TRY(cudaFuncSetAttribute((const void*)k_b_pass_b2<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->sm1));
    P->g_b = occ_grid((const void*)k_b_pass_b1<BLOCK>, P->sm1);
    RPCG_CUDA_TRY(cudaFuncSetAttribute((const void*)k_b_redo_a<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->smr1));
    RPCG_CUDA_TRY(cudaFuncSetAttribute((const void*)k_b_redo_b<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->smr2));
    P->g_ra = occ_grid((const void*)k_b_redo_a<BLOCK>, P->smr1);
    P->g_rb = occ_grid((const void*)k_b_redo_b<BLOCK>, P->smr2);
  }
  return RPCG_OK;
}

template <int V, int BLOCK>
static rpcg_status batch_graph(rpcg_batch_t B, int tile, cudaGraph_t* out_g, cudaGraphExec_t* out_e) {
  rpcg_batch_s::Layout* L = nullptr;
  rpcg_status st = batch_layout(B, tile, &L);
  if (st != RPCG_OK) return st;
  BatchPlan P;
  st = batch_plan<V, BLOCK>(B, L, &P);
  if (st != RPCG_OK) return st;
  const int count = B->count;
  const int g_setup = P.g_setup, g_a = P.g_a, g_b = P.g_b, g_c = P.g_c, g_q = P.g_q;
  const size_t sm1 = P.sm1, sm2 = P.sm2, sm3 = P.sm3;
  constexpr int VS = setup_variant<V>();

  cudaGraph_t g = nullptr;
  RPCG_CUDA_TRY(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond;
  RPCG_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
  BatchDesc D{B->d_sys, B->d_state, B->d_red, B->d_head, B->d_aprefix, L->nunits, L->uprefix, L->partials, count, tile};
  int* aprefix = B->d_aprefix;
  cudaGraphNode_t n_init, n_q, n_setup, n_c0, n_loop;
  {
    void* a[] = {&D};
    RPCG_CUDA_TRY(add_node(g, &n_init, nullptr, 0, (const void*)k_b_init, 1, 256, 0, a));
  }
  {
    void* a[] = {&D, &aprefix};
    RPCG_CUDA_TRY(add_node(g, &n_q, &n_init, 1, (const void*)k_b_inv_q, g_q, BLOCK, 0, a));
    RPCG_CUDA_TRY(add_node(g, &n_setup, &n_q, 1, (const void*)k_b_setup<VS, BLOCK>, g_setup, BLOCK, sm3, a));
  }
  {
    void* a[] = {&D, &cond};
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
    void* a[] = {&D};
    RPCG_CUDA_TRY(add_node(body, &b_a, nullptr, 0, (const void*)k_b_pass_a<V, BLOCK>, g_a, BLOCK, sm1, a));
    if constexpr (V == RPCG_FPE) {  // the exact recomputations follow their passes
      cudaGraphNode_t b_ra;
      RPCG_CUDA_TRY(add_node(body, &b_ra, &b_a, 1, (const void*)k_b_redo_a<BLOCK>, P.g_ra, BLOCK, P.smr1, a));
      b_a = b_ra;
    }
    if constexpr (V == RPCG_FPE) {
      cudaGraphNode_t b_b1;
      RPCG_CUDA_TRY(add_node(body, &b_b1, &b_a, 1, (const void*)k_b_pass_b1<BLOCK>, P.g_b, BLOCK, sm1, a));
      RPCG_CUDA_TRY(add_node(body, &b_b, &b_b1, 1, (const void*)k_b_pass_b2<BLOCK>, P.g_b, BLOCK, sm1, a));
    } else {
      RPCG_CUDA_TRY(add_node(body, &b_b, &b_a, 1, (const void*)k_b_pass_b<V, BLOCK>, g_b, BLOCK, sm2, a));
    }
    if constexpr (V == RPCG_FPE) {
      cudaGraphNode_t b_rb;
      RPCG_CUDA_TRY(add_node(body, &b_rb, &b_b, 1, (const void*)k_b_redo_b<BLOCK>, P.g_rb, BLOCK, P.smr2, a));
      b_b = b_rb;
    }
    RPCG_CUDA_TRY(add_node(body, &b_c, &b_b, 1, (const void*)k_b_pass_c<BLOCK>, g_c, BLOCK, 0, a));
  }
  {
    void* a[] = {&D, &cond};
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
  if (block == 128) {
    if (v == RPCG_PLAIN) st = batch_graph<RPCG_PLAIN, 128>(B, tile, &g, &ex);
    else if (v == RPCG_FPE) st = batch_graph<RPCG_FPE, 128>(B, tile, &g, &ex);
    else st = batch_graph<RPCG_EXBLAS, 128>(B, tile, &g, &ex);
  } else {
    if (v == RPCG_PLAIN) st = batch_graph<RPCG_PLAIN, 256>(B, tile, &g, &ex);
    else if (v == RPCG_FPE) st = batch_graph<RPCG_FPE, 256>(B, tile, &g, &ex);
    else st = batch_graph<RPCG_EXBLAS, 256>(B, tile, &g, &ex);
  }
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
    cudaFree(kv.second.nunits);
    cudaFree(kv.second.uprefix);
    cudaFree(kv.second.partials);
  }
  cudaFree(B->d_aprefix);
  if (B->uploaded) cudaEventDestroy(B->uploaded);
  cudaFree(B->d_sys);
  cudaFree(B->d_state);
  cudaFree(B->d_red);
  cudaFree(B->d_head);
  cudaFreeHost(B->h_sys);
  cudaFreeHost(B->h_state);
  delete B;
}

static void batch_upload(rpcg_batch_t B, const double* const* b, double* const* x, const rpcg_opts& o) {
  for (int i = 0; i < B->count; i++) {
    rpcg_matrix_t A = B->mats[i];
    double* hist = o.history ? o.history + (size_t)i * (o.max_iter + 1) : nullptr;
    B->h_sys[i] = SysDev{A->m, b[i], x[i], A->r, A->d, A->w, A->inv, hist, o.tol, o.max_iter, o.fpe_size,
                         o.fpe_strict ? 1 : 0, 0};
  }
}

// One launch of the batch graph (set-up + loop) with the given b/x.
static rpcg_status batch_run(rpcg_batch_t B, const double* const* b, double* const* x, int v, const rpcg_opts& o,
                             int block, int tile, cudaStream_t s) {
  cudaGraphExec_t e = nullptr;
  rpcg_status st = batch_get_graph(B, v, block, tile, &e);
  if (st != RPCG_OK) return st;
  // the pinned table is read by the copy when it runs: wait for the previous
  // copy (usually long done) before rewriting it
  if (B->uploaded) RPCG_CUDA_TRY(cudaEventSynchronize(B->uploaded));
  batch_upload(B, b, x, o);
  RPCG_CUDA_TRY(cudaMemcpyAsync(B->d_sys, B->h_sys, B->count * sizeof(SysDev), cudaMemcpyHostToDevice, s));
  if (!B->uploaded) RPCG_CUDA_TRY(cudaEventCreateWithFlags(&B->uploaded, cudaEventDisableTiming));
  RPCG_CUDA_TRY(cudaEventRecord(B->uploaded, s));
  RPCG_CUDA_TRY(cudaGraphLaunch(e, s));
  return RPCG_OK;
}

// The per-system results of a batch run, on the device (the host logic of
// batch_results): NOT_CONVERGED when a system stopped at max_iter, x = 0
// for b = 0, an empty system OK with nothing done.  One block per system.
static __global__ void k_b_results(const SysDev* __restrict__ sys, const SysState* __restrict__ st, int count,
                                   int variant, rpcg_result* out) {
  for (int s = blockIdx.x; s < count; s += gridDim.x) {
    const SysState t = st[s];
    const int n = sys[s].m.n;
    if (n > 0 && t.bzero)
      for (int i = threadIdx.x; i < n; i += blockDim.x) sys[s].x[i] = 0.0;
    if (threadIdx.x == 0) {
      rpcg_result r{0, RPCG_OK, 0.0, 0.0, 0, 0};
      if (n > 0) {
        int status = t.status;
        if (status == RPCG_OK) {
          if (!(t.rel < sys[s].tol)) status = RPCG_NOT_CONVERGED;
          else if (variant == RPCG_FPE && sys[s].fpe_strict && t.fpe_inexact > 0) status = RPCG_FPE_INEXACT;
        }
        r.iterations = t.iter;
        r.status = status;
        r.relres = t.rel;
        r.tau = t.tau;
        r.fpe_inexact_count = t.fpe_inexact;
        r.fpe_size_used = variant == RPCG_FPE ? t.fpe_p : 0;
      }
      out[s] = r;
    }
  }
}

// The batch loop launched kernel by kernel from the host, with events
// around each kind of pass (set-up, A, B, C, retire/list): a measurement
// tool.  Same kernels, same order, same results as the graph.
template <int V, int BLOCK>
static rpcg_status batch_eager(rpcg_batch_t B, int tile, cudaStream_t s, float* pass_ms, int32_t* launches) {
  rpcg_batch_s::Layout* L = nullptr;
  rpcg_status st = batch_layout(B, tile, &L);
  if (st != RPCG_OK) return st;
  BatchPlan P;
  st = batch_plan<V, BLOCK>(B, L, &P);
  if (st != RPCG_OK) return st;
  const BatchDesc D{B->d_sys, B->d_state, B->d_red, B->d_head, B->d_aprefix, L->nunits, L->uprefix, L->partials,
                    B->count, tile};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RPCG_CUDA_TRY(cudaEventCreate(&e0));
  RPCG_CUDA_TRY(cudaEventCreate(&e1));
  int* h_active = nullptr;
  cudaError_t err = cudaMallocHost(&h_active, sizeof(int));
  auto timed = [&](int k, int nl, auto launch) {
    if (err != cudaSuccess) return;
    err = cudaEventRecord(e0, s);
    if (err == cudaSuccess) launch();
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    pass_ms[k] += ms;
    if (launches) launches[k] += nl;
  };
  auto active = [&]() {
    if (err == cudaSuccess) err = cudaMemcpyAsync(h_active, &B->d_head->active_count, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    return err == cudaSuccess ? *h_active : 0;
  };
  const int* ap = B->d_aprefix;
  constexpr int VS = setup_variant<V>();
  timed(0, 3, [&] {
    k_b_init<<<1, 256, 0, s>>>(D);
    k_b_inv_q<<<P.g_q, BLOCK, 0, s>>>(D, ap);
    k_b_setup<VS, BLOCK><<<P.g_setup, BLOCK, P.sm3, s>>>(D, ap);
  });
  timed(4, 1, [&] { k_b_retire<<<1, 256, 0, s>>>(D); });
  while (active() > 0) {
    // the fpe variant's exact recomputations count with their passes
    timed(1, 1, [&] {
      k_b_pass_a<V, BLOCK><<<P.g_a, BLOCK, P.sm1, s>>>(D);
      if (V == RPCG_FPE) k_b_redo_a<BLOCK><<<P.g_ra, BLOCK, P.smr1, s>>>(D);
    });
    timed(2, 1, [&] {
      if constexpr (V == RPCG_FPE) {
        k_b_pass_b1<BLOCK><<<P.g_b, BLOCK, P.sm1, s>>>(D);
        k_b_pass_b2<BLOCK><<<P.g_b, BLOCK, P.sm1, s>>>(D);
        k_b_redo_b<BLOCK><<<P.g_rb, BLOCK, P.smr2, s>>>(D);
      } else {
        k_b_pass_b<V, BLOCK><<<P.g_b, BLOCK, P.sm2, s>>>(D);
      }
    });
    timed(3, 1, [&] { k_b_pass_c<BLOCK><<<P.g_c, BLOCK, 0, s>>>(D); });
    timed(4, 1, [&] { k_b_retire<<<1, 256, 0, s>>>(D); });
  }
  if (h_active) cudaFreeHost(h_active);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    set_error("batch_eager: %s", cudaGetErrorString(err));
    return RPCG_ERR_CUDA;
  }
  return RPCG_OK;
}

// Read the per-system states after a run and fill `res`; returns the worst status.
static rpcg_status batch_results(rpcg_batch_t B, double* const* x, int v, const rpcg_opts& opt, rpcg_result* res,
                                 cudaStream_t s) {
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
    if (status == RPCG_OK) {
      if (!(h.rel < opt.tol)) status = RPCG_NOT_CONVERGED;
      else if (v == RPCG_FPE && opt.fpe_strict && h.fpe_inexact > 0) status = RPCG_FPE_INEXACT;
    }
    res[i] = rpcg_result{h.iter, status, h.rel, h.tau, h.fpe_inexact, v == RPCG_FPE ? h.fpe_p : 0};
    if (status < 0 && (worst >= 0 || status < worst)) worst = (rpcg_status)status;
    else if (status > 0 && worst == RPCG_OK) worst = (rpcg_status)status;
  }
  RPCG_CUDA_TRY(cudaStreamSynchronize(s));
  return worst;
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
  cudaError_t e = cudaMalloc(&B->d_sys, count * sizeof(SysDev));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_state, count * sizeof(SysState));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_red, count * sizeof(SysRed));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_head, sizeof(BatchHead));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_aprefix, ((size_t)count + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&B->h_sys, count * sizeof(SysDev));
  if (e == cudaSuccess) e = cudaMallocHost(&B->h_state, count * sizeof(SysState));
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
  RPCG_CHECK_ARG(v == RPCG_PLAIN || v == RPCG_EXBLAS || v == RPCG_FPE, "unknown variant");
  rpcg_opts opt;
  if (o) opt = *o;
  else rpcg_opts_default(&opt);
  RPCG_CHECK_ARG(opt.max_iter >= 0 && !(opt.tol < 0.0) && !std::isnan(opt.tol), "bad tol or max_iter");
  RPCG_CHECK_ARG(opt.fpe_size >= 0 && opt.fpe_size <= kFpeMax, "fpe_size must be 0 (adaptive) or 1..8");
  RPCG_CHECK_ARG(opt.block == 0 || opt.block == 128 || opt.block == 256, "block must be 0, 128 or 256 here");
  RPCG_CHECK_ARG(opt.tile >= 0 && opt.tile <= (1 << 24), "tile must be 0 (autotuned) or 1..2^24 rows");
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
        for (int ct : {1024, 4096, 16384}) {
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
  return batch_results(B, x, v, opt, res, s);
}

rpcg_status rpcg_batch_solve_profiled(rpcg_batch_t B, const double* const* b, double* const* x, int32_t v,
                                      const rpcg_opts* o, rpcg_result* res, float* pass_ms, int32_t* launches,
                                      void* stream) {
  clear_error();
  RPCG_CHECK_ARG(B != nullptr && b != nullptr && x != nullptr && res != nullptr && pass_ms != nullptr,
                 "NULL argument");
  RPCG_CHECK_ARG(v == RPCG_PLAIN || v == RPCG_EXBLAS || v == RPCG_FPE, "unknown variant");
  rpcg_opts opt;
  if (o) opt = *o;
  else rpcg_opts_default(&opt);
  RPCG_CHECK_ARG(opt.max_iter >= 0 && !(opt.tol < 0.0) && !std::isnan(opt.tol), "bad tol or max_iter");
  RPCG_CHECK_ARG(opt.fpe_size >= 0 && opt.fpe_size <= kFpeMax, "fpe_size must be 0 (adaptive) or 1..8");
  RPCG_CHECK_ARG(opt.block == 0 || opt.block == 128 || opt.block == 256, "block must be 0, 128 or 256 here");
  RPCG_CHECK_ARG(opt.tile >= 0 && opt.tile <= (1 << 24), "tile must be 0 (autotuned) or 1..2^24 rows");
  for (int i = 0; i < B->count; i++) RPCG_CHECK_ARG(B->mats[i]->m.n == 0 || (b[i] && x[i]), "b[i] or x[i] is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const int block = opt.block ? opt.block : (B->tuned_block ? B->tuned_block : 128);
  const int tile = opt.tile ? opt.tile : (B->tuned_tile ? B->tuned_tile : 4096);
  for (int k = 0; k < 5; k++) pass_ms[k] = 0.f;
  if (launches)
    for (int k = 0; k < 5; k++) launches[k] = 0;
  batch_upload(B, b, x, opt);
  RPCG_CUDA_TRY(cudaMemcpyAsync(B->d_sys, B->h_sys, B->count * sizeof(SysDev), cudaMemcpyHostToDevice, s));
  rpcg_status st;
  if (block == 128) {
    if (v == RPCG_PLAIN) st = batch_eager<RPCG_PLAIN, 128>(B, tile, s, pass_ms, launches);
    else if (v == RPCG_FPE) st = batch_eager<RPCG_FPE, 128>(B, tile, s, pass_ms, launches);
    else st = batch_eager<RPCG_EXBLAS, 128>(B, tile, s, pass_ms, launches);
  } else {
    if (v == RPCG_PLAIN) st = batch_eager<RPCG_PLAIN, 256>(B, tile, s, pass_ms, launches);
    else if (v == RPCG_FPE) st = batch_eager<RPCG_FPE, 256>(B, tile, s, pass_ms, launches);
    else st = batch_eager<RPCG_EXBLAS, 256>(B, tile, s, pass_ms, launches);
  }
  if (st != RPCG_OK) return st;
  return batch_results(B, x, v, opt, res, s);
}

rpcg_status rpcg_batch_solve_async(rpcg_batch_t B, const double* const* b, double* const* x, int32_t v,
                                   const rpcg_opts* o, rpcg_result* res, void* stream) {
  clear_error();
  RPCG_CHECK_ARG(B != nullptr && b != nullptr && x != nullptr && res != nullptr, "NULL argument");
  RPCG_CHECK_ARG(v == RPCG_PLAIN || v == RPCG_EXBLAS || v == RPCG_FPE, "unknown variant");
  rpcg_opts opt;
  if (o) opt = *o;
  else rpcg_opts_default(&opt);
  RPCG_CHECK_ARG(opt.max_iter >= 0 && !(opt.tol < 0.0) && !std::isnan(opt.tol), "bad tol or max_iter");
  RPCG_CHECK_ARG(opt.fpe_size >= 0 && opt.fpe_size <= kFpeMax, "fpe_size must be 0 (adaptive) or 1..8");
  RPCG_CHECK_ARG(opt.block == 0 || opt.block == 128 || opt.block == 256, "block must be 0, 128 or 256 here");
  RPCG_CHECK_ARG(opt.tile >= 0 && opt.tile <= (1 << 24), "tile must be 0 (autotuned) or 1..2^24 rows");
  for (int i = 0; i < B->count; i++) RPCG_CHECK_ARG(B->mats[i]->m.n == 0 || (b[i] && x[i]), "b[i] or x[i] is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  // no autotuning here (it times runs): the tuned shape if there is one, else 128 x 1024
  const int block = opt.block ? opt.block : (B->tuned_block ? B->tuned_block : 128);
  const int tile = opt.tile ? opt.tile : (B->tuned_tile ? B->tuned_tile : 1024);
  rpcg_status st = batch_run(B, b, x, v, opt, block, tile, s);
  if (st != RPCG_OK) return st;
  k_b_results<<<std::max(1, std::min(B->count, sm_count() * 8)), 256, 0, s>>>(B->d_sys, B->d_state, B->count, v, res);
  RPCG_CUDA_TRY(cudaGetLastError());
  return RPCG_OK;
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
