// Serving loop: continuous batching of PCG solve requests on one GPU.
//
// Requests (CSR + b in host memory) enter a FIFO queue.  A scheduler thread
// owns the GPU side: it admits requests into a fixed table of slots while a
// slot is free and the device bytes in use stay within the HBM budget,
// keeps matrices on the device in an LRU cache (requests on the same matrix
// share one device copy; each slot has its own b, x and Krylov vectors),
// runs the set-up pass for newly admitted systems, and then a chunk of
// kChunk iterations of the batched passes over every system still
// iterating.  Between chunks it retires the systems that stopped (copying x
// back to the host) and admits new requests, so work that arrives while
// others run joins the batch at the next chunk boundary.
//
// A cached device copy is only ever reused for a request whose matrix is
// known to have the same contents.  Every request names a "generation": a
// matrix registered with rpcg_server_register (the server keeps its own
// host copy, so its contents cannot change), or host arrays passed to
// rpcg_server_submit.  Arrays passed to submit must stay unchanged until
// that ticket is collected, so a request submitted while an earlier request
// on the same addresses is still uncollected sees the same contents and
// joins its generation; once every ticket of a generation has been
// collected the caller may have reused the memory, the addresses stop
// naming it, and its device copy is freed.
//
// Each system goes through exactly the arithmetic of rpcg_solve with the
// exact dots, so its result is bit-identical to solving it alone, whatever
// else shares the GPU with it.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <set>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "host.h"

namespace rpcg {

constexpr int kChunk = 16;          // iterations between scheduling decisions
constexpr int kServeTile = 1024;    // rows per work unit (the batch autotuner's choice on stencil systems)
constexpr int kServeBlock = 128;

static double now_us() {
  using namespace std::chrono;
  return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

}  // namespace rpcg

struct rpcg_server_s {
  struct Req {
    uint64_t ticket;
    int n, nnz;
    const int* rowptr;
    const int* col;
    const double* val;
    const double* b;
    const double* x0;
    double tol;
    int max_iter;
    double t_submit;
    uint64_t gen;  // the matrix generation this request solves with
  };
  struct Done {
    rpcg_result res;
    std::vector<double> x;
    double queue_us, service_us;
  };
  // host arrays of a submit request, and the generation they name while
  // some request on them is uncollected
  using AddrKey = std::tuple<const void*, const void*, const void*, int, int>;
  struct Gen {
    int holders = 0;      // uncollected tickets, plus one while registered
    bool has_addr = false;
    bool registered = false;  // held by rpcg_server_register until rpcg_server_unregister
    AddrKey addr{};
    // a registered matrix: the server's own copy of the CSR arrays
    std::vector<int> rowptr, col;
    std::vector<double> val;
  };
  using MatKey = uint64_t;  // generation id
  struct Mat {
    rpcg_matrix_t h = nullptr;
    size_t bytes = 0;
    int users = 0;
    uint64_t last_use = 0;
  };
  struct Slot {
    bool used = false;
    Req req{};
    double t_admit = 0;
    MatKey key{};
    double* buf = nullptr;  // b, x, r, d, w, inv (6 n doubles)
    size_t bytes = 0;
  };

  int device = 0;
  size_t budget = 0;
  int max_slots = 0;
  cudaStream_t stream = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<Req> queue;
  std::unordered_map<uint64_t, Done> done;
  std::map<uint64_t, int> pending;  // tickets not yet completed (queued or running)
  std::unordered_map<uint64_t, uint64_t> ticket_gen;  // uncollected ticket -> generation
  std::unordered_map<uint64_t, Gen> gens;             // live generations
  std::map<AddrKey, uint64_t> addr_gen;              // submit arrays -> their live generation
  std::vector<uint64_t> dead_gens;                    // no ticket can name these again
  uint64_t next_gen = 1;

  // device cache and byte count (read by rpcg_server_stats; guarded by mu)
  std::map<MatKey, Mat> mats;
  size_t used_bytes = 0;

  // scheduler thread only
  std::vector<Slot> slots;
  uint64_t clock = 0;
  rpcg::SysDev* d_sys = nullptr;
  rpcg::SysDev* h_sys = nullptr;
  rpcg::SysState* d_state = nullptr;
  rpcg::SysState* h_state = nullptr;
  rpcg::SysRed* d_red = nullptr;
  rpcg::BatchHead* d_head = nullptr;
  int* d_aprefix = nullptr;  // [max_slots + 1] units of the iterating systems (built on the device)
  int* d_sprefix = nullptr;  // [max_slots + 1] units of the newly admitted systems (built here)
  int* h_sprefix = nullptr;
  int* d_nunits = nullptr;  // [max_slots]
  int* h_nunits = nullptr;
  int* d_list = nullptr;
  int grid_setup = 1, grid_a = 1, grid_b = 1, grid_c = 1, grid_q = 1;

  // statistics
  uint64_t n_completed = 0, n_failed = 0, n_chunks = 0;
};

namespace rpcg {

static size_t slot_bytes(int n) { return (size_t)6 * (size_t)(n > 0 ? n : 1) * sizeof(double); }

// device bytes of a matrix handle built from (n, nnz): SELL-32 values and
// columns (with slice padding, estimated at 5%), row pointers, slice
// offsets, its own vectors (6 n doubles) and reduction scratch
static size_t mat_bytes(int n, int nnz) {
  return (size_t)((double)nnz * 12.0 * 1.05) + (size_t)4 * (n + 1) + (size_t)8 * (n / 32 + 2) + slot_bytes(n) +
         (size_t)(256 << 10);
}

// Drop one hold on a generation (S->mu held).  At zero no ticket names it
// and none can again: its addresses are forgotten, a registered copy is
// freed, and the scheduler frees the device copy.
static void release_gen(rpcg_server_t S, uint64_t g) {
  auto it = S->gens.find(g);
  if (it == S->gens.end()) return;
  if (--it->second.holders > 0) return;
  if (it->second.has_addr) {
    auto a = S->addr_gen.find(it->second.addr);
    if (a != S->addr_gen.end() && a->second == g) S->addr_gen.erase(a);
  }
  S->gens.erase(it);
  S->dead_gens.push_back(g);
  S->cv_work.notify_one();
}

static void complete(rpcg_server_t S, uint64_t ticket, const rpcg_result& res, std::vector<double>&& x, double qus,
                     double sus) {
  std::lock_guard<std::mutex> lock(S->mu);
  auto& d = S->done[ticket];
  d.res = res;
  d.x = std::move(x);
  d.queue_us = qus;
  d.service_us = sus;
  S->pending.erase(ticket);
  if (res.status < 0) S->n_failed++;
  S->n_completed++;
  S->cv_done.notify_all();
}

static void fail_req(rpcg_server_t S, const rpcg_server_s::Req& r, int status, double t_admit) {
  rpcg_result res{0, status, 0.0, 0.0, 0, 0};
  complete(S, r.ticket, res, {}, t_admit - r.t_submit, now_us() - t_admit);
}

// Evict cached matrices nobody uses, least recently used first, until
// `need` more bytes fit.  Returns whether they fit; the evicted handles are
// appended to `victims` (destroyed by the caller outside the queue lock).
static bool make_room(rpcg_server_t S, size_t need, std::vector<rpcg_matrix_t>& victims) {
  while (S->used_bytes + need > S->budget) {
    auto victim = S->mats.end();
    for (auto it = S->mats.begin(); it != S->mats.end(); ++it) {
      if (it->second.users == 0 && (victim == S->mats.end() || it->second.last_use < victim->second.last_use)) victim = it;
    }
    if (victim == S->mats.end()) return false;
    victims.push_back(victim->second.h);
    S->used_bytes -= victim->second.bytes;
    S->mats.erase(victim);
  }
  return true;
}

template <class F>
static cudaError_t launch_check(F f) {
  f();
  return cudaGetLastError();
}

static void serve_loop(rpcg_server_t S) {
  cudaSetDevice(S->device);
  cudaStream_t s = S->stream;
  SysDev* sys = S->d_sys;
  SysState* sst = S->d_state;
  SysRed* red = S->d_red;
  BatchHead* head = S->d_head;
  std::vector<int> running;  // slots being iterated
  for (;;) {
    // ---- admission (FIFO: stop at the first request that does not fit yet).
    // A cached matrix is pinned (users + 1) as soon as a request naming it is
    // admitted; a matrix still to be created is reserved once per admission pass.
    std::vector<std::pair<int, rpcg_server_s::Req>> admitted;
    std::vector<rpcg_matrix_t> victims;
    std::set<rpcg_server_s::MatKey> creating;  // matrix bytes reserved in this pass, not created yet
    std::set<rpcg_server_s::MatKey> created;   // created in this pass
    {
      std::unique_lock<std::mutex> lock(S->mu);
      // device copies of generations no ticket can name again
      for (const uint64_t g : S->dead_gens) {
        auto it = S->mats.find(g);
        if (it != S->mats.end() && it->second.users == 0) {
          victims.push_back(it->second.h);
          S->used_bytes -= it->second.bytes;
          S->mats.erase(it);
        }
      }
      S->dead_gens.clear();
      if (running.empty() && S->queue.empty()) {
        if (S->stop) break;
        if (victims.empty()) S->cv_work.wait_for(lock, std::chrono::milliseconds(50));
        if (S->queue.empty()) {
          lock.unlock();
          for (rpcg_matrix_t h : victims) rpcg_destroy(h);
          continue;
        }
      }
      while (!S->queue.empty()) {
        int free_slot = -1;
        for (int i = 0; i < S->max_slots; i++) {
          bool taken = S->slots[i].used;
          for (auto& a : admitted) taken |= a.first == i;
          if (!taken) {
            free_slot = i;
            break;
          }
        }
        if (free_slot < 0) break;
        const rpcg_server_s::Req r = S->queue.front();
        const rpcg_server_s::MatKey key = r.gen;
        const bool cached = S->mats.count(key) > 0;
        const bool known = cached || creating.count(key) > 0;
        const size_t need = slot_bytes(r.n) + (known ? 0 : mat_bytes(r.n, r.nnz));
        if (slot_bytes(r.n) + mat_bytes(r.n, r.nnz) > S->budget) {
          S->queue.pop_front();
          S->pending.erase(r.ticket);
          auto& d = S->done[r.ticket];
          d.res = rpcg_result{0, RPCG_ERR_OOM, 0.0, 0.0, 0, 0};
          d.queue_us = now_us() - r.t_submit;
          d.service_us = 0.0;
          S->n_failed++;
          S->n_completed++;
          S->cv_done.notify_all();
          continue;
        }
        if (cached) S->mats[key].users++;  // pinned from now on
        if (!make_room(S, need, victims)) {
          if (cached) S->mats[key].users--;
          break;
        }
        S->queue.pop_front();
        S->used_bytes += need;  // the slot, and the matrix when it is new
        if (!known) creating.insert(key);
        admitted.push_back({free_slot, r});
      }
    }
    for (rpcg_matrix_t h : victims) rpcg_destroy(h);
    // ---- set up the admitted requests
    std::vector<int> fresh;
    for (auto& a : admitted) {
      const int si = a.first;
      const rpcg_server_s::Req& r = a.second;
      const double t_admit = now_us();
      const rpcg_server_s::MatKey key = r.gen;
      rpcg_matrix_t h = nullptr;
      bool have = false;
      {
        std::lock_guard<std::mutex> lock(S->mu);
        auto it = S->mats.find(key);
        if (it != S->mats.end()) {
          // created earlier in this admission pass for another request; (a
          // matrix cached before this pass was pinned at admission)
          if (created.count(key)) it->second.users++;
          it->second.last_use = ++S->clock;
          h = it->second.h;
          have = true;
        }
      }
      if (!have) {
        // first request of this admission pass naming the matrix: create it
        // (its bytes were reserved at admission); the generation's arrays stay
        // unchanged while this request is uncollected
        const rpcg_status cs = rpcg_create(&h, r.n, r.nnz, r.rowptr, r.col, r.val, 0, s);
        {
          std::lock_guard<std::mutex> lock(S->mu);
          // the matrix bytes were reserved by the request that admitted the
          // generation in this pass; if that one failed, this one takes them
          const bool reserved = creating.erase(key) > 0;
          if (cs != RPCG_OK) {
            S->used_bytes -= slot_bytes(r.n) + (reserved ? mat_bytes(r.n, r.nnz) : 0);
          } else {
            if (!reserved) S->used_bytes += mat_bytes(r.n, r.nnz);
            created.insert(key);
            rpcg_server_s::Mat m;
            m.h = h;
            m.bytes = mat_bytes(r.n, r.nnz);
            m.users = 1;
            m.last_use = ++S->clock;
            S->mats.emplace(key, m);
          }
        }
        if (cs != RPCG_OK) {
          fail_req(S, r, cs, t_admit);
          continue;
        }
      }
      rpcg_server_s::Slot& sl = S->slots[si];
      sl.used = true;
      sl.req = r;
      sl.t_admit = t_admit;
      sl.key = key;
      sl.bytes = slot_bytes(r.n);
      const size_t nb = (size_t)(r.n > 0 ? r.n : 1) * sizeof(double);
      cudaError_t e = cudaMallocAsync((void**)&sl.buf, 6 * nb, s);
      double* B = sl.buf;
      const int n = r.n;
      if (e == cudaSuccess && n) e = cudaMemcpyAsync(B, r.b, nb, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess && n) {
        e = r.x0 ? cudaMemcpyAsync(B + n, r.x0, nb, cudaMemcpyHostToDevice, s) : cudaMemsetAsync(B + n, 0, nb, s);
      }
      if (e != cudaSuccess) {
        cudaGetLastError();
        if (sl.buf) cudaFreeAsync(sl.buf, s);
        sl.buf = nullptr;
        sl.used = false;
        {
          std::lock_guard<std::mutex> lock(S->mu);
          S->mats[key].users--;
          S->used_bytes -= sl.bytes;
        }
        fail_req(S, r, RPCG_ERR_CUDA, t_admit);
        continue;
      }
      S->h_sys[si] = SysDev{h->m, B, B + n, B + 2 * (size_t)n, B + 3 * (size_t)n, B + 4 * (size_t)n,
                            B + 5 * (size_t)n, nullptr, r.tol, r.max_iter, 0};
      fresh.push_back(si);
    }
    // ---- upload the new systems; run their set-up and a chunk of iterations
    bool ok = true;
    if (!fresh.empty() || !running.empty()) {
      cudaError_t e = cudaSuccess;
      const BatchDesc D{sys, sst, red, head, S->d_aprefix, S->d_nunits, nullptr, nullptr, S->max_slots, kServeTile};
      constexpr int B = kServeBlock;
      if (!fresh.empty()) {
        std::fill(S->h_sprefix, S->h_sprefix + S->max_slots + 1, 0);
        for (int si : fresh) {
          S->h_nunits[si] = (int)(((long long)S->slots[si].req.n + kServeTile - 1) / kServeTile);
          S->h_sprefix[si + 1] = S->h_nunits[si];
        }
        for (int i = 0; i < S->max_slots; i++) S->h_sprefix[i + 1] += S->h_sprefix[i];
        for (int si : fresh) {
          if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->d_sys + si, S->h_sys + si, sizeof(SysDev), cudaMemcpyHostToDevice, s);
          if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->d_nunits + si, S->h_nunits + si, sizeof(int), cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(S->d_list, fresh.data(), fresh.size() * sizeof(int), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(S->d_sprefix, S->h_sprefix, (S->max_slots + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
        const int* sp = S->d_sprefix;
        if (e == cudaSuccess) {
          e = launch_check([&] {
            k_b_init_list<<<1, 256, 0, s>>>(D, S->d_list, (int)fresh.size());
            k_b_inv_q<<<S->grid_q, B, 0, s>>>(D, sp);
            k_b_setup<RPCG_EXBLAS, B><<<S->grid_setup, B, b_smem<RPCG_EXBLAS>(3, S->max_slots), s>>>(D, sp);
            k_b_retire<<<1, 256, 0, s>>>(D);  // lists the units of every system now iterating
          });
        }
        for (int si : fresh) running.push_back(si);
      }
      if (e == cudaSuccess) {
        e = launch_check([&] {
          for (int k = 0; k < kChunk; k++) {
            k_b_pass_a<RPCG_EXBLAS, B><<<S->grid_a, B, b_smem<RPCG_EXBLAS>(1, S->max_slots), s>>>(D);
            k_b_pass_b<RPCG_EXBLAS, B><<<S->grid_b, B, b_smem<RPCG_EXBLAS>(2, S->max_slots), s>>>(D);
            k_b_pass_c<B><<<S->grid_c, B, 0, s>>>(D);
            k_b_retire<<<1, 256, 0, s>>>(D);
          }
        });
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->h_state, S->d_state, S->max_slots * sizeof(SysState), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        ok = false;
        cudaGetLastError();
        // every running request fails below; start the device records afresh
        cudaMemsetAsync(S->d_state, 0, S->max_slots * sizeof(SysState), s);
        cudaMemsetAsync(S->d_red, 0, S->max_slots * sizeof(SysRed), s);
        cudaMemsetAsync(S->d_head, 0, sizeof(BatchHead), s);
        cudaMemsetAsync(S->d_aprefix, 0, (S->max_slots + 1) * sizeof(int), s);
        cudaStreamSynchronize(s);
      }
      S->n_chunks++;
    }
    // ---- retire the systems that stopped (or everything, after an error)
    std::vector<int> still;
    for (int si : running) {
      rpcg_server_s::Slot& sl = S->slots[si];
      const SysState& h = S->h_state[si];
      if (ok && h.active) {
        still.push_back(si);
        continue;
      }
      const int n = sl.req.n;
      std::vector<double> x((size_t)n);
      rpcg_result res{h.iter, h.status, h.rel, h.tau, 0, 0};
      if (!ok) res.status = RPCG_ERR_CUDA;
      if (ok && h.bzero) std::fill(x.begin(), x.end(), 0.0);
      else if (n && cudaMemcpy(x.data(), sl.buf + n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        res.status = RPCG_ERR_CUDA;
      if (res.status == RPCG_OK && !(h.rel < sl.req.tol)) res.status = RPCG_NOT_CONVERGED;
      cudaFreeAsync(sl.buf, s);
      sl.buf = nullptr;
      sl.used = false;
      {
        std::lock_guard<std::mutex> lock(S->mu);
        S->mats[sl.key].users--;
        S->used_bytes -= sl.bytes;
      }
      complete(S, sl.req.ticket, res, std::move(x), sl.t_admit - sl.req.t_submit, now_us() - sl.t_admit);
    }
    running.swap(still);
  }
}

}  // namespace rpcg

using namespace rpcg;

extern "C" {

rpcg_status rpcg_server_create(rpcg_server_t* out, size_t hbm_budget_bytes, int32_t max_slots) {
  clear_error();
  RPCG_CHECK_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  RPCG_CHECK_ARG(max_slots >= 1 && max_slots <= 4096, "max_slots must be 1..4096");
  RPCG_CHECK_ARG(hbm_budget_bytes >= ((size_t)1 << 20), "the budget must be at least 1 MiB");
  rpcg_server_t S = new rpcg_server_s();
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  S->slots.resize(max_slots);
  cudaGetDevice(&S->device);
  cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&S->d_sys, max_slots * sizeof(SysDev));
  if (e == cudaSuccess) e = cudaMallocHost(&S->h_sys, max_slots * sizeof(SysDev));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_state, max_slots * sizeof(SysState));
  if (e == cudaSuccess) e = cudaMallocHost(&S->h_state, max_slots * sizeof(SysState));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_red, max_slots * sizeof(SysRed));
  if (e == cudaSuccess) e = cudaMemset(S->d_red, 0, max_slots * sizeof(SysRed));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_head, sizeof(BatchHead));
  if (e == cudaSuccess) e = cudaMemset(S->d_head, 0, sizeof(BatchHead));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_aprefix, ((size_t)max_slots + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(S->d_aprefix, 0, ((size_t)max_slots + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_sprefix, ((size_t)max_slots + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&S->h_sprefix, ((size_t)max_slots + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_nunits, max_slots * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(S->d_nunits, 0, max_slots * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&S->h_nunits, max_slots * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_list, max_slots * sizeof(int));
  if (e == cudaSuccess) {
    std::memset(S->h_state, 0, max_slots * sizeof(SysState));
    e = cudaMemset(S->d_state, 0, max_slots * sizeof(SysState));
  }
  constexpr int B = kServeBlock;
  auto occ = [&](const void* f, size_t smem) {
    int o = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, f, B, smem) != cudaSuccess || o < 1) o = 1;
    return sm_count() * o;
  };
  if (e == cudaSuccess) {
    const size_t sm1 = b_smem<RPCG_EXBLAS>(1, max_slots), sm2 = b_smem<RPCG_EXBLAS>(2, max_slots),
                 sm3 = b_smem<RPCG_EXBLAS>(3, max_slots);
    cudaFuncSetAttribute((const void*)k_b_setup<RPCG_EXBLAS, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
    cudaFuncSetAttribute((const void*)k_b_pass_a<RPCG_EXBLAS, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    cudaFuncSetAttribute((const void*)k_b_pass_b<RPCG_EXBLAS, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    S->grid_setup = occ((const void*)k_b_setup<RPCG_EXBLAS, B>, sm3);
    S->grid_a = occ((const void*)k_b_pass_a<RPCG_EXBLAS, B>, sm1);
    S->grid_b = occ((const void*)k_b_pass_b<RPCG_EXBLAS, B>, sm2);
    S->grid_c = occ((const void*)k_b_pass_c<B>, 0);
    S->grid_q = occ((const void*)k_b_inv_q, 0);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_error("rpcg_server_create: %s", cudaGetErrorString(e));
    rpcg_server_destroy(S);
    return e == cudaErrorMemoryAllocation ? RPCG_ERR_OOM : RPCG_ERR_CUDA;
  }
  S->worker = std::thread(serve_loop, S);
  *out = S;
  return RPCG_OK;
}

rpcg_status rpcg_server_submit(rpcg_server_t S, int32_t n, int32_t nnz, const int32_t* rowptr, const int32_t* col,
                               const double* val, const double* b, const double* x0, int32_t v, const rpcg_opts* o,
                               uint64_t* ticket) {
  clear_error();
  RPCG_CHECK_ARG(S != nullptr && ticket != nullptr, "server or ticket is NULL");
  RPCG_CHECK_ARG(v == RPCG_EXBLAS, "the serving loop runs the exblas variant");
  RPCG_CHECK_ARG(n >= 0 && nnz >= 0 && rowptr != nullptr && (n == 0 || b != nullptr), "bad request arrays");
  RPCG_CHECK_ARG(nnz == 0 || (col != nullptr && val != nullptr), "col or val is NULL");
  rpcg_opts opt;
  if (o) opt = *o;
  else rpcg_opts_default(&opt);
  RPCG_CHECK_ARG(opt.max_iter >= 0 && !(opt.tol < 0.0), "bad tol or max_iter");
  rpcg_server_s::Req r{};
  r.n = n;
  r.nnz = nnz;
  r.rowptr = rowptr;
  r.col = col;
  r.val = val;
  r.b = b;
  r.x0 = x0;
  r.tol = opt.tol;
  r.max_iter = opt.max_iter;
  r.t_submit = now_us();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    RPCG_CHECK_ARG(!S->stop, "server is shutting down");
    // the arrays name a live generation while a request on them is
    // uncollected (their contents are unchanged since it was submitted)
    const rpcg_server_s::AddrKey ak{rowptr, col, val, n, nnz};
    auto a = S->addr_gen.find(ak);
    if (a != S->addr_gen.end()) {
      r.gen = a->second;
    } else {
      r.gen = S->next_gen++;
      rpcg_server_s::Gen& G = S->gens[r.gen];
      G.has_addr = true;
      G.addr = ak;
      S->addr_gen[ak] = r.gen;
    }
    S->gens[r.gen].holders++;
    r.ticket = S->next_ticket++;
    S->queue.push_back(r);
    S->pending[r.ticket] = 1;
    S->ticket_gen[r.ticket] = r.gen;
    *ticket = r.ticket;
  }
  S->cv_work.notify_one();
  return RPCG_OK;
}

rpcg_status rpcg_server_register(rpcg_server_t S, int32_t n, int32_t nnz, const int32_t* rowptr, const int32_t* col,
                                 const double* val, uint64_t* matrix) {
  clear_error();
  RPCG_CHECK_ARG(S != nullptr && matrix != nullptr, "server or matrix is NULL");
  RPCG_CHECK_ARG(n >= 0 && nnz >= 0 && rowptr != nullptr, "bad matrix arrays");
  RPCG_CHECK_ARG(nnz == 0 || (col != nullptr && val != nullptr), "col or val is NULL");
  RPCG_CHECK_ARG(rowptr[0] == 0 && rowptr[n] == nnz, "rowptr[0] must be 0 and rowptr[n] must be nnz");
  rpcg_server_s::Gen G;
  G.registered = true;
  G.holders = 1;
  G.rowptr.assign(rowptr, rowptr + (size_t)n + 1);
  G.col.assign(col, col + (size_t)nnz);
  G.val.assign(val, val + (size_t)nnz);
  std::lock_guard<std::mutex> lock(S->mu);
  RPCG_CHECK_ARG(!S->stop, "server is shutting down");
  const uint64_t g = S->next_gen++;
  S->gens.emplace(g, std::move(G));
  *matrix = g;
  return RPCG_OK;
}

rpcg_status rpcg_server_submit_registered(rpcg_server_t S, uint64_t matrix, const double* b, const double* x0, int32_t v,
                                          const rpcg_opts* o, uint64_t* ticket) {
  clear_error();
  RPCG_CHECK_ARG(S != nullptr && ticket != nullptr, "server or ticket is NULL");
  RPCG_CHECK_ARG(v == RPCG_EXBLAS, "the serving loop runs the exblas variant");
  rpcg_opts opt;
  if (o) opt = *o;
  else rpcg_opts_default(&opt);
  RPCG_CHECK_ARG(opt.max_iter >= 0 && !(opt.tol < 0.0), "bad tol or max_iter");
  {
    std::lock_guard<std::mutex> lock(S->mu);
    RPCG_CHECK_ARG(!S->stop, "server is shutting down");
    auto it = S->gens.find(matrix);
    RPCG_CHECK_ARG(it != S->gens.end() && it->second.registered, "unknown or unregistered matrix id");
    rpcg_server_s::Gen& G = it->second;
    const int n = (int)G.rowptr.size() - 1;
    RPCG_CHECK_ARG(n == 0 || b != nullptr, "b is NULL");
    rpcg_server_s::Req r{};
    r.n = n;
    r.nnz = (int)G.val.size();
    r.rowptr = G.rowptr.data();
    r.col = G.col.data();
    r.val = G.val.data();
    r.b = b;
    r.x0 = x0;
    r.tol = opt.tol;
    r.max_iter = opt.max_iter;
    r.t_submit = now_us();
    r.gen = matrix;
    G.holders++;
    r.ticket = S->next_ticket++;
    S->queue.push_back(r);
    S->pending[r.ticket] = 1;
    S->ticket_gen[r.ticket] = matrix;
    *ticket = r.ticket;
  }
  S->cv_work.notify_one();
  return RPCG_OK;
}

rpcg_status rpcg_server_unregister(rpcg_server_t S, uint64_t matrix) {
  clear_error();
  RPCG_CHECK_ARG(S != nullptr, "server is NULL");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->gens.find(matrix);
  RPCG_CHECK_ARG(it != S->gens.end() && it->second.registered, "unknown or unregistered matrix id");
  it->second.registered = false;
  release_gen(S, matrix);
  return RPCG_OK;
}

rpcg_status rpcg_server_wait(rpcg_server_t S, uint64_t ticket, double* x_host, rpcg_result* res,
                             rpcg_server_timing* timing, int64_t timeout_us) {
  clear_error();
  RPCG_CHECK_ARG(S != nullptr && res != nullptr, "server or res is NULL");
  std::unique_lock<std::mutex> lock(S->mu);
  auto ready = [&] { return S->done.count(ticket) > 0 || (S->pending.count(ticket) == 0); };
  if (timeout_us < 0) S->cv_done.wait(lock, ready);
  else if (!S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), ready)) {
    set_error("rpcg_server_wait: ticket %llu not done within %lld us", (unsigned long long)ticket, (long long)timeout_us);
    return RPCG_ERR_TIMEOUT;
  }
  auto it = S->done.find(ticket);
  if (it == S->done.end()) {
    set_error("rpcg_server_wait: unknown ticket %llu", (unsigned long long)ticket);
    return RPCG_ERR_INVALID;
  }
  *res = it->second.res;
  if (x_host && !it->second.x.empty()) std::memcpy(x_host, it->second.x.data(), it->second.x.size() * sizeof(double));
  if (timing) {
    timing->queue_us = it->second.queue_us;
    timing->service_us = it->second.service_us;
  }
  S->done.erase(it);
  // the ticket is collected: its hold on the matrix generation ends (the
  // caller may now change or free the arrays it submitted)
  auto tg = S->ticket_gen.find(ticket);
  if (tg != S->ticket_gen.end()) {
    const uint64_t g = tg->second;
    S->ticket_gen.erase(tg);
    release_gen(S, g);
  }
  return (rpcg_status)res->status;
}

rpcg_status rpcg_server_stats(rpcg_server_t S, rpcg_server_stats_t* st) {
  RPCG_CHECK_ARG(S != nullptr && st != nullptr, "NULL argument");
  std::lock_guard<std::mutex> lock(S->mu);
  st->completed = S->n_completed;
  st->failed = S->n_failed;
  st->queued = S->queue.size();
  st->chunks = S->n_chunks;
  st->bytes_in_use = S->used_bytes;
  st->matrices_cached = S->mats.size();
  return RPCG_OK;
}

rpcg_status rpcg_server_destroy(rpcg_server_t S) {
  clear_error();
  if (!S) return RPCG_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  if (S->stream) cudaStreamSynchronize(S->stream);
  for (auto& sl : S->slots)
    if (sl.buf) cudaFree(sl.buf);
  for (auto& kv : S->mats) rpcg_destroy(kv.second.h);
  cudaFree(S->d_sys);
  cudaFreeHost(S->h_sys);
  cudaFree(S->d_state);
  cudaFreeHost(S->h_state);
  cudaFree(S->d_red);
  cudaFree(S->d_head);
  cudaFree(S->d_aprefix);
  cudaFree(S->d_sprefix);
  cudaFreeHost(S->h_sprefix);
  cudaFree(S->d_nunits);
  cudaFreeHost(S->h_nunits);
  cudaFree(S->d_list);
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
  return RPCG_OK;
}

}  // extern "C"
