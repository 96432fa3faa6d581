// Standalone dot products: exact (long accumulator), FPE with exactness
// flag, and the plain FP64 baseline; plus the library-wide host helpers.
#include <cuda.h>  // CUcontext and CUresult types only: driver entry points are fetched at run time

#include <cmath>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "device.cuh"
#include "host.h"

namespace rpcg {

// ------------------------------------------------------------------ host helpers
static thread_local char g_err[512];

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cache[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cache[dev] = v;
  }
  return cache[dev];
}

// ------------------------------------------------------------------ scratch
constexpr int kDotBlock = 256;
constexpr int kDotMaxGrid = 2048;

struct DotScratch {
  // zeroed before every launch (header)
  unsigned long long digits[kNDig];
  unsigned int counter;
  unsigned int flags;  // bit 0: non-finite input; bit 1: an expansion lost bits; bit 2: FPE non-finite
  // written before being read (no clearing needed)
  double partials[kDotMaxGrid];
};
constexpr size_t kDotScratchHeader = offsetof(DotScratch, partials);

// ------------------------------------------------------------------ exact dot
// The shared accumulator of k_dot_exact holds kNHalf digits of 16 bits
// (half digit h weighs 2^(16 h) units of the 32-bit digit grid), each a
// signed 32-bit word, in 32 copies: sacc[h * 32 + lane].  Native 32-bit
// shared atomics add to it (64-bit ones run about four times slower), and
// with one copy per lane a warp's atomics never share a bank.  Each add is
// at most 2^16 in magnitude; a word takes at most 3 adds per product from
// each of the BLOCK / 32 threads of its lane (the product's own chunk, and
// the flush of both register windows, whose digits overlap, when they
// move) and 2 more from each at the end, so spilling the words to the
// global digits every kSpillProducts products per thread keeps every word's
// sum below 2^31: (3 * 8 * 1024 + 16) * 2^16 < 2^31 at BLOCK = 256.
constexpr int kNHalf = 2 * kNDig;
constexpr int kSpillProducts = 1024;

// A product in complemented form: |a b| shifted left by its in-digit
// offset, in five words, all bits flipped when the product is negative.
// With m below and above them (bits shifted in and the sign extension) and
// a carry-in of m & 1, adding these words adds the signed product in two's
// complement; the flip is done on the four product words before the shift
// instead of on the six words of every window add.
struct WinProd {
  uint32_t w0, w1, w2, w3, w4;
  int q;       // digit index of w0
  uint32_t m;  // all ones for a negative product
  bool nz;     // false only for a non-finite operand
  bool bad;    // a or b is Inf or NaN
};

__device__ __forceinline__ WinProd win_product(double a, double b) {
  const uint32_t ah = (uint32_t)__double2hiint(a), al = (uint32_t)__double2loint(a);
  const uint32_t bh = (uint32_t)__double2hiint(b), bl = (uint32_t)__double2loint(b);
  const uint32_t fa = ah & 0x7ff00000u, fb = bh & 0x7ff00000u;
  WinProd p;
  // field 0 wraps to 0xfff00000, field 0x7ff to 0x7fe00000: both outside the normal range
  if ((fa - 0x00100000u) >= 0x7fe00000u || (fb - 0x00100000u) >= 0x7fe00000u) {
    const ExactProd e = exact_product_general(a, b);
    p.w0 = e.w0 ^ e.neg;
    p.w1 = e.w1 ^ e.neg;
    p.w2 = e.w2 ^ e.neg;
    p.w3 = e.w3 ^ e.neg;
    p.w4 = e.w4 ^ e.neg;
    p.q = e.q;
    p.m = e.neg;
    p.nz = e.nz;
    p.bad = e.bad;
    return p;
  }
  p.bad = false;
  p.nz = true;
  const uint32_t m = (uint32_t)((int32_t)(ah ^ bh) >> 31);
  const uint32_t mah = (ah & 0x000FFFFFu) | 0x00100000u;
  const uint32_t mbh = (bh & 0x000FFFFFu) | 0x00100000u;
  // offset of the product's lowest bit from 2^kE0 (28 .. 4118; fa + fb < 2^32);
  // the funnel shifts take it modulo 32
  const uint32_t o = ((fa + fb) >> 20) - (uint32_t)(2150 + kE0);
  p.q = (int)(o >> 5);
  const uint64_t p0 = (uint64_t)al * bl;
  const uint64_t p1 = (uint64_t)al * mbh + (uint64_t)mah * bl;  // < 2^54
  const uint64_t p2 = (uint64_t)mah * mbh;                      // < 2^42
  uint32_t v1, v2, v3;
  asm("add.cc.u32 %0, %3, %4;\n\t"
      "addc.cc.u32 %1, %5, %6;\n\t"
      "addc.u32 %2, %7, 0;"
      : "=r"(v1), "=r"(v2), "=r"(v3)
      : "r"((uint32_t)(p0 >> 32)), "r"((uint32_t)p1), "r"((uint32_t)(p1 >> 32)), "r"((uint32_t)p2),
        "r"((uint32_t)(p2 >> 32)));
  const uint32_t c0 = (uint32_t)p0 ^ m, c1 = v1 ^ m, c2 = v2 ^ m, c3 = v3 ^ m;
  p.w0 = __funnelshift_l(m, c0, o);
  p.w1 = __funnelshift_l(c0, c1, o);
  p.w2 = __funnelshift_l(c1, c2, o);
  p.w3 = __funnelshift_l(c2, c3, o);
  p.w4 = __funnelshift_l(c3, m, o);
  p.m = m;
  return p;
}

// W += a0..a5 (then m) with a carry-in of m & 1: a 224-bit add.
__device__ __forceinline__ void window_chain(Window& w, uint32_t m, uint32_t a0, uint32_t a1, uint32_t a2,
                                             uint32_t a3, uint32_t a4, uint32_t a5) {
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "add.cc.u32 t, %7, %7;\n\t"
      "addc.cc.u32 %0, %0, %8;\n\t"
      "addc.cc.u32 %1, %1, %9;\n\t"
      "addc.cc.u32 %2, %2, %10;\n\t"
      "addc.cc.u32 %3, %3, %11;\n\t"
      "addc.cc.u32 %4, %4, %12;\n\t"
      "addc.cc.u32 %5, %5, %13;\n\t"
      "addc.u32 %6, %6, %7;\n\t"
      "}"
      : "+r"(w.W[0]), "+r"(w.W[1]), "+r"(w.W[2]), "+r"(w.W[3]), "+r"(w.W[4]), "+r"(w.W[5]), "+r"(w.W[6])
      : "r"(m), "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(a4), "r"(a5));
}

// W += the signed product at word offset t1 (0 or 1) in the window, the
// words placed by six selects.  The main window instead branches on the
// offset (half_exact_deposit): when the lanes of a warp agree on it, as
// products that span a few bits of exponent do, one chain runs with the
// words already in place (on U[-1, 1] pairs 7% faster than selects); the
// low window, which only data with a wide exponent spread reaches, keeps
// the selects (a branch there was 6% slower on pairs of condition 1e32).
__device__ __forceinline__ void window_add_c(Window& w, const WinProd& p, bool t1) {
  window_chain(w, p.m, t1 ? p.m : p.w0, t1 ? p.w0 : p.w1, t1 ? p.w1 : p.w2, t1 ? p.w2 : p.w3, t1 ? p.w3 : p.w4,
               t1 ? p.w4 : p.m);
}

// A product that no register window takes: the ten 16-bit chunks of its
// five words at half digits 2q .. 2q + 9 (the lowest with the carry-in
// m & 1), and m at 2q + 10 for the all-ones bits above them.  No test for
// zero chunks: a predicate costs as much issue as the atomic it would skip.
__device__ __forceinline__ void half_deposit(uint32_t* sacc, const WinProd& p) {
  uint32_t* at = sacc + 2 * p.q * 32;
  atomicAdd(at + 0 * 32, (p.w0 & 0xffffu) + (p.m & 1u));
  atomicAdd(at + 1 * 32, p.w0 >> 16);
  atomicAdd(at + 2 * 32, p.w1 & 0xffffu);
  atomicAdd(at + 3 * 32, p.w1 >> 16);
  atomicAdd(at + 4 * 32, p.w2 & 0xffffu);
  atomicAdd(at + 5 * 32, p.w2 >> 16);
  atomicAdd(at + 6 * 32, p.w3 & 0xffffu);
  atomicAdd(at + 7 * 32, p.w3 >> 16);
  atomicAdd(at + 8 * 32, p.w4 & 0xffffu);
  atomicAdd(at + 9 * 32, p.w4 >> 16);
  atomicAdd(at + 10 * 32, p.m);
}

__device__ __forceinline__ void half_add(uint32_t* at, uint32_t v) {
  if (v) atomicAdd(at, v);
}

// Empty a register window into the half digits 2 qb .. 2 qb + 13: its six
// low words unsigned, the top word (the window's sign) as an unsigned low
// half and a signed high half.
__device__ __forceinline__ void half_flush(Window& w, uint32_t* sacc) {
  if (w.qb < 0) return;
  uint32_t* at = sacc + 2 * w.qb * 32;
#pragma unroll
  for (int k = 0; k < kWin - 1; k++) {
    half_add(at + (2 * k) * 32, w.W[k] & 0xffffu);
    half_add(at + (2 * k + 1) * 32, w.W[k] >> 16);
  }
  half_add(at + (2 * kWin - 2) * 32, w.W[kWin - 1] & 0xffffu);
  half_add(at + (2 * kWin - 1) * 32, (uint32_t)((int32_t)w.W[kWin - 1] >> 16));
#pragma unroll
  for (int k = 0; k < kWin; k++) w.W[k] = 0;
}

// Two register windows per thread: `w` over digits qb .. qb + 6 and `lo`
// two digits below it.  A product whose digit index is in {qb, qb + 1} goes
// to w, in {qb - 2, qb - 1} to lo, anything else to the shared half digits.
// A product above w also raises `qtop`; the windows move up to it only at
// the end of a round of products (half_reanchor), so that the flush code
// exists once in the loop instead of once per product of the round (inlined
// eight times it overflowed the instruction cache).
__device__ __forceinline__ void half_exact_deposit(Window& w, Window& lo, uint32_t* sacc, int& qtop,
                                                   const WinProd& p) {
  if (!p.nz) return;
  const int t = p.q - w.qb;
  if (t == 1) {  // the main window by branch, the common offset first
    window_chain(w, p.m, p.m, p.w0, p.w1, p.w2, p.w3, p.w4);
  } else if (t == 0) {
    window_chain(w, p.m, p.w0, p.w1, p.w2, p.w3, p.w4, p.m);
  } else if ((unsigned)(t + 2) < 2u) {
    window_add_c(lo, p, t == -1);
  } else {
    half_deposit(sacc, p);
    if (t > 1) qtop = max(qtop, p.q);
  }
}

// Move both windows up to the largest product seen above them (if any).
__device__ __forceinline__ void half_reanchor(Window& w, Window& lo, uint32_t* sacc, int& qtop) {
  if (qtop < 0) return;
  half_flush(w, sacc);
  half_flush(lo, sacc);
  // qb >= 2 keeps lo anchored at digit 0 or above; q <= kNDig - 5 for every
  // product, so q - qb stays in {0, 1} below the upper clamp too
  const int qb = min(max(qtop - 1, 2), kNDig - kWin);
  w.qb = qb;
  lo.qb = qb - 2;
  qtop = -1;
}

// Add the 32 copies of every half digit to the global 32-bit digits: digit
// k takes half digits 2k and 2k + 1 (the latter shifted up 16 bits) in one
// atomic; with `clear`, zero the copies for the next spill interval.  Needs
// a __syncthreads() before (deposits done) and, with `clear`, one after.
__device__ __forceinline__ void half_to_global(uint32_t* sacc, unsigned long long* gacc, bool clear) {
  for (int k = threadIdx.x; k < kNDig; k += blockDim.x) {
    long long s0 = 0, s1 = 0;
#pragma unroll 8
    for (int c = 0; c < 32; c++) {
      const int col = (c + k) & 31;  // staggered: the lanes of a warp read 32 different banks
      uint32_t* at0 = sacc + (2 * k) * 32 + col;
      uint32_t* at1 = sacc + (2 * k + 1) * 32 + col;
      s0 += (int32_t)*at0;
      s1 += (int32_t)*at1;
      if (clear) {
        *at0 = 0u;
        *at1 = 0u;
      }
    }
    const long long v = s0 + s1 * 65536ll;  // |v| < 2^53
    if (v) atomicAdd(gacc + k, (unsigned long long)v);
  }
  __threadfence();
}

__device__ __forceinline__ void exact_step(Window& win, Window& lo, uint32_t* sacc, int& qtop, bool& bad, double x,
                                           double y) {
  const WinProd p = win_product(x, y);
  bad |= p.bad;
  half_exact_deposit(win, lo, sacc, qtop, p);
}

// The last CTA: normalise, round once, publish, leave the scratch clean.
// Out of line so that its registers do not count against the main loop's.
static __device__ __noinline__ void dot_exact_finish(DotScratch* ws, double* out, long long* sdig, uint32_t* sD) {
  __shared__ int srange[2];
  const double v = take_and_round(ws->digits, sdig, sD, srange);
  if (threadIdx.x == 0) {
    const unsigned int f = atomicExch(&ws->flags, 0u);
    *out = (f & 1u) ? __longlong_as_double(0x7FF8000000000000ll) : v;
    ws->counter = 0;
  }
}

// ALIGNED: a and b start on 16-byte boundaries (pairs of elements are
// loaded as double2); the host picks the instance.  Each thread keeps two
// register windows of digits (half_exact_deposit), so products spread over
// up to four digit positions stay in registers: on U[-1, 1] pairs, whose
// products all fit the first window, the second one costs about 2% against
// a one-window kernel; on ill-conditioned pairs (cond 1e16 to 1e32) it
// halves the time.  The loops run the same number of times in every thread
// of a CTA, so that the spills' barriers are reached by all.
template <int BLOCK, bool ALIGNED>
__global__ void __launch_bounds__(BLOCK) k_dot_exact(int64_t n, const double* __restrict__ a,
                                                     const double* __restrict__ b, DotScratch* ws, double* out) {
  static_assert(BLOCK == 256, "the spill bound assumes 8 threads per lane copy");
  __shared__ __align__(16) uint32_t sacc[kNHalf * 32];
  __shared__ long long sdig[kNDig];
  __shared__ uint32_t sD[kNDig];
  for (int k = threadIdx.x; k < kNHalf * 8; k += BLOCK) reinterpret_cast<uint4*>(sacc)[k] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  Window win, lo;
  window_init(win);
  window_init(lo);
  uint32_t* sl = sacc + (threadIdx.x & 31);  // this lane's copy
  int qtop = -1;
  bool bad = false;
  const int64_t nthr = (int64_t)gridDim.x * BLOCK;
  int64_t i0 = (int64_t)blockIdx.x * BLOCK;  // the CTA's first index of the current round
  int since = 0;                             // products per thread since the last spill
  if constexpr (ALIGNED) {
    const double2* a2 = reinterpret_cast<const double2*>(a);
    const double2* b2 = reinterpret_cast<const double2*>(b);
    const int64_t n2 = n >> 1;
    // rounds of 8 products per thread, while every thread of the CTA has them
    for (; i0 + (BLOCK - 1) + 3 * nthr < n2; i0 += 4 * nthr) {
      const int64_t i = i0 + threadIdx.x;
      double2 x[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        x[u] = __ldcs(a2 + i + u * nthr);
        y[u] = __ldcs(b2 + i + u * nthr);
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        exact_step(win, lo, sl, qtop, bad, x[u].x, y[u].x);
        exact_step(win, lo, sl, qtop, bad, x[u].y, y[u].y);
      }
      half_reanchor(win, lo, sl, qtop);
      since += 8;
      // spill while there is room for one more round (8 products) and the
      // rest after the loop (at most 9), so no interval exceeds kSpillProducts
      if (since > kSpillProducts - 8 - 9) {
        __syncthreads();
        half_to_global(sacc, ws->digits, true);
        __syncthreads();
        since = 0;
      }
    }
    // the rest: at most 4 pairs per thread, and the odd last element
    for (int64_t i = i0 + threadIdx.x; i < n2; i += nthr) {
      const double2 x = __ldcs(a2 + i), y = __ldcs(b2 + i);
      exact_step(win, lo, sl, qtop, bad, x.x, y.x);
      exact_step(win, lo, sl, qtop, bad, x.y, y.y);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) exact_step(win, lo, sl, qtop, bad, a[n - 1], b[n - 1]);
  } else {
    for (; i0 < n; i0 += nthr) {
      const int64_t i = i0 + threadIdx.x;
      if (i < n) exact_step(win, lo, sl, qtop, bad, a[i], b[i]);
      half_reanchor(win, lo, sl, qtop);
      if (++since == kSpillProducts) {
        __syncthreads();
        half_to_global(sacc, ws->digits, true);
        __syncthreads();
        since = 0;
      }
    }
  }
  half_flush(win, sl);
  half_flush(lo, sl);
  if (bad) atomicOr(&ws->flags, 1u);
  __syncthreads();
  half_to_global(sacc, ws->digits, false);
  if (is_last_block(&ws->counter)) dot_exact_finish(ws, out, sdig, sD);
}

// ------------------------------------------------------------------ FPE dot
// Alg. 1 in FP64 for the elements two_sum_split does not cover (non-finite
// operands, sums that overflow).  Out of line, so that the compiler cannot
// turn this rare path into predicated FP64 work for every element.
static __device__ __noinline__ double2 eft_twosum_fp64(double x, double y) {
  double rr, ss;
  two_sum(x, y, rr, ss);
  return make_double2(rr, ss);
}

// Elementwise Alg. 1 (which = 0) or Alg. 2 (which = 1) as the FPE dot
// computes them: two_sum_split (one FP64 addition, the error on the integer
// pipe; non-finite elements and sums that overflow take the FP64 formulas)
// and two_prod_int (the FP64 formulas outside its range).
__global__ void k_eft(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ r,
                      double* __restrict__ s, int which) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = a[i], y = b[i];
    double rr, ss;
    if (which == 1) {
      if (!two_prod_int(x, y, rr, ss)) two_prod(x, y, rr, ss);
    } else {
      bool ovf = !is_finite_bits(x) || !is_finite_bits(y);
      if (!ovf) {
        two_sum_split(x, y, rr, ss, ovf);
      }
      if (ovf) {
        const double2 t = eft_twosum_fp64(x, y);
        rr = t.x;
        ss = t.y;
      }
    }
    r[i] = rr;
    s[i] = ss;
  }
}

// FPE dot (Sec. 4.2): each thread accumulates its products into a result
// and an error expansion (Algs. 2 and 4, early exit) and merges the two
// (Alg. 3); the threads' expansions then meet exactly in the long
// accumulator and are rounded once, so the merge loses nothing and *exact
// reports whether any thread's expansion lost bits (or a product fell below
// twoprod's exact range).  twoprod runs on the integer pipe
// (two_prod_int); the result expansion's twosums are Fast2Sum (three FP64
// additions) and the error expansion's take one FP64 addition with the
// error computed on the integer pipe (two_sum_split), which shares the
// work between GB300's scarce FP64 pipe and the integer pipes.
// PMAX: the expansions' array size, p <= PMAX.  The host launches PMAX = 4
// for p <= 4: the unused terms of 8-term arrays cost registers and code
// (at p = 4 on 2^24 U[-1, 1] pairs, 0.292 against 0.323 ms).
constexpr int kFpeDotWarps = 32;  // 64 registers (24 and 16 warps per SM measured slower; 48 no faster)
template <int BLOCK, int PMAX>
__global__ void __launch_bounds__(BLOCK, kFpeDotWarps * 32 / BLOCK) k_dot_fpe(int64_t n, const double* __restrict__ a,
                                                      const double* __restrict__ b, int p, DotScratch* ws, double* out,
                                                      int32_t* exact) {
  __shared__ unsigned long long sacc[kNDig * kCopies];
  __shared__ long long sdig[kNDig];
  __shared__ uint32_t sD[kNDig];
  smem_acc_zero(sacc);
  double res[PMAX], err[PMAX];
#pragma unroll
  for (int i = 0; i < PMAX; i++) res[i] = err[i] = 0.0;
  bool lost = false, nonfinite = false;
  const int64_t tid = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * BLOCK;
  // compute-bound: no loads run ahead, which keeps registers for more warps.
  // The loop runs the same number of times in every lane of a warp, and the
  // lanes meet again at the end of each element.
  const int64_t lane = threadIdx.x & 31;
  for (int64_t i0 = tid - lane; i0 < n; i0 += nthr) {
    const int64_t i = i0 + lane;
    if (i < n) {
      const double x = __ldcs(a + i), y = __ldcs(b + i);
      if (!is_finite_bits(x) || !is_finite_bits(y)) nonfinite = true;
      else lost |= fpe_dot_step(res, err, p, x, y, nonfinite);
    }
    __syncwarp();
  }
  bool ovf = false;
  lost |= fpe_sum(res, err, p, ovf);
  nonfinite |= ovf;
  Window win;
  window_init(win);
  const int copy = threadIdx.x & (kCopies - 1);
#pragma unroll
  for (int i = 0; i < PMAX; i++) {
    if (i < p && !is_zero_bits(res[i])) {
      const ExactProd e = exact_product(res[i], 1.0);
      nonfinite |= e.bad;
      exact_deposit(win, sacc, copy, e);
    }
  }
  window_flush(win, sacc, copy);
  if (nonfinite) atomicOr(&ws->flags, 4u);
  if (lost) atomicOr(&ws->flags, 2u);
  __syncthreads();
  smem_to_global(sacc, ws->digits);
  if (is_last_block(&ws->counter)) {
    __shared__ int srange[2];
    const double v = take_and_round(ws->digits, sdig, sD, srange);
    if (threadIdx.x == 0) {
      const unsigned int f = atomicExch(&ws->flags, 0u);
      const bool fin = !(f & 4u);
      *out = fin ? v : __longlong_as_double(0x7FF8000000000000ll);
      *exact = (fin && !(f & 2u)) ? 1 : 0;
      ws->counter = 0;
    }
  }
}

// ------------------------------------------------------------------ plain dot
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_dot_plain(int64_t n, const double* __restrict__ a,
                                                     const double* __restrict__ b, DotScratch* ws, double* out) {
  __shared__ double sw[32];
  double acc = 0.0;
  const int64_t tid = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * BLOCK;
  for (int64_t i = tid; i < n; i += nthr) acc = __fma_rn(__ldcs(a + i), __ldcs(b + i), acc);
  const double s = block_sum_fixed<BLOCK>(acc, sw);
  if (threadIdx.x == 0) ws->partials[blockIdx.x] = s;
  if (is_last_block(&ws->counter)) {
    double v = 0.0;
    for (int t = threadIdx.x; t < (int)gridDim.x; t += BLOCK) v = __dadd_rn(v, __ldcg(&ws->partials[t]));
    const double tot = block_sum_fixed<BLOCK>(v, sw);
    if (threadIdx.x == 0) {
      *out = tot;
      ws->counter = 0;
    }
  }
}

// CTAs of k_dot_exact resident per SM on the current device (3 of 256
// threads at its 80 registers; a grid of exactly that many leaves no
// partial second wave).  A 64-register cap (4 CTAs) spilled and measured
// no faster.
static int exact_resident() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dot_exact<kDotBlock, true>, kDotBlock, 0) != cudaSuccess ||
        occ < 1) {
      cudaGetLastError();
      occ = 3;
    }
    cache[dev] = occ;
  }
  return cache[dev];
}

static int dot_grid(int64_t n, int per_thread, int cap, int per_sm = 4) {
  int64_t want = (n + (int64_t)kDotBlock * per_thread - 1) / ((int64_t)kDotBlock * per_thread);
  int64_t g = (int64_t)sm_count() * per_sm;
  if (want < g) g = want;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

static void launch_dot_exact(int64_t n, const double* a, const double* b, DotScratch* ws, double* out,
                             cudaStream_t s) {
  const int g = dot_grid(n, 8, kDotMaxGrid, exact_resident());
  if ((((uintptr_t)a | (uintptr_t)b) & 15) == 0) k_dot_exact<kDotBlock, true><<<g, kDotBlock, 0, s>>>(n, a, b, ws, out);
  else k_dot_exact<kDotBlock, false><<<g, kDotBlock, 0, s>>>(n, a, b, ws, out);
}

}  // namespace rpcg

using namespace rpcg;

extern "C" {

const char* rpcg_last_error(void) { return g_err; }

const char* rpcg_status_string(int32_t s) {
  switch (s) {
    case RPCG_OK: return "ok";
    case RPCG_NOT_CONVERGED: return "not converged";
    case RPCG_FPE_INEXACT: return "floating-point expansion lost bits";
    case RPCG_ERR_INVALID: return "invalid argument";
    case RPCG_ERR_NOT_SPD: return "matrix not SPD (diagonal or curvature)";
    case RPCG_ERR_NONFINITE: return "non-finite value";
    case RPCG_ERR_OOM: return "out of device memory or budget";
    case RPCG_ERR_CUDA: return "CUDA error";
    case RPCG_ERR_TIMEOUT: return "timed out";
    default: return "unknown status";
  }
}

static rpcg_status dot_common(int kind, int64_t n, const double* a, const double* b, int32_t p, double* out,
                              int32_t* exact, void* stream) {
  clear_error();
  RPCG_CHECK_ARG(n >= 0 && n <= (int64_t(1) << 30), "n must be in [0, 2^30]");
  RPCG_CHECK_ARG(out != nullptr, "out is NULL");
  RPCG_CHECK_ARG(n == 0 || (a != nullptr && b != nullptr), "a or b is NULL");
  RPCG_CHECK_ARG(kind != 1 || (p >= 1 && p <= kFpeMax && exact != nullptr), "fpe: p must be 1..8 and exact non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  DotScratch* ws = nullptr;
  RPCG_CUDA_TRY(cudaMallocAsync((void**)&ws, sizeof(DotScratch), s));
  cudaError_t e = cudaMemsetAsync(ws, 0, kDotScratchHeader, s);
  if (e == cudaSuccess) {
    if (kind == 0) {
      launch_dot_exact(n, a, b, ws, out, s);
    } else if (kind == 1) {
      const int g = dot_grid(n, 16, kDotMaxGrid, kFpeDotWarps * 32 / kDotBlock);
      if (p <= 4) k_dot_fpe<kDotBlock, 4><<<g, kDotBlock, 0, s>>>(n, a, b, p, ws, out, exact);
      else k_dot_fpe<kDotBlock, kFpeMax><<<g, kDotBlock, 0, s>>>(n, a, b, p, ws, out, exact);
    } else {
      k_dot_plain<kDotBlock><<<dot_grid(n, 4, kDotMaxGrid), kDotBlock, 0, s>>>(n, a, b, ws, out);
    }
    e = cudaGetLastError();
  }
  cudaFreeAsync(ws, s);
  if (e != cudaSuccess) {
    set_error("dot launch failed: %s", cudaGetErrorString(e));
    return RPCG_ERR_CUDA;
  }
  return RPCG_OK;
}

rpcg_status rpcg_dot_exact(int64_t n, const double* a, const double* b, double* out, void* stream) {
  return dot_common(0, n, a, b, 0, out, nullptr, stream);
}

rpcg_status rpcg_dot_fpe(int64_t n, const double* a, const double* b, int32_t p, double* out, int32_t* exact,
                         void* stream) {
  return dot_common(1, n, a, b, p, out, exact, stream);
}

rpcg_status rpcg_dot_plain(int64_t n, const double* a, const double* b, double* out, void* stream) {
  return dot_common(2, n, a, b, 0, out, nullptr, stream);
}

static rpcg_status eft_common(int which, int64_t n, const double* a, const double* b, double* r, double* s,
                              void* stream) {
  clear_error();
  RPCG_CHECK_ARG(n >= 0, "n must be >= 0");
  RPCG_CHECK_ARG(n == 0 || (a && b && r && s), "NULL array");
  if (n == 0) return RPCG_OK;
  int64_t g = (n + 255) / 256;
  if (g > sm_count() * 8) g = sm_count() * 8;
  k_eft<<<(int)g, 256, 0, (cudaStream_t)stream>>>(n, a, b, r, s, which);
  RPCG_CUDA_TRY(cudaGetLastError());
  return RPCG_OK;
}

rpcg_status rpcg_eft_twosum(int64_t n, const double* a, const double* b, double* r, double* s, void* stream) {
  return eft_common(0, n, a, b, r, s, stream);
}

rpcg_status rpcg_eft_twoprod(int64_t n, const double* a, const double* b, double* r, double* s, void* stream) {
  return eft_common(1, n, a, b, r, s, stream);
}

}  // extern "C"

// ------------------------------------------------------------------ exact dot without allocation
//
// Some callers cannot let a library allocate device memory: for example a
// framework whose caching allocator has already reserved all of the GPU's
// memory for itself, or a time-critical loop where an allocation (and the
// device synchronisation that cudaMalloc may imply) is not acceptable.  For
// them rpcg_dot_exact_noalloc runs the same exact-dot kernel as
// rpcg_dot_exact, but its scratch is the fixed array below, which every GPU
// that loads this library holds until the process exits.

namespace rpcg {

// Capacity of the fixed scratch: room for one DotScratch (about 34 KiB).
constexpr size_t kNoAllocScratchBytes = 64 * 1024;
static_assert(sizeof(DotScratch) <= kNoAllocScratchBytes, "DotScratch must fit the fixed scratch array");

// Largest n accepted: the digit headroom of the long accumulator.
constexpr int64_t kNoAllocMaxN = int64_t(1) << 30;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// In host code the array's name is only a stand-in, not a device address:
// its address is looked up with cudaGetSymbolAddress, once per CUDA context
// (a device's primary context, or another one the caller made current), with
// that context current.  The cache is keyed by the driver's context ID, which
// is unique for the life of the process, so a context created after
// cudaDeviceReset (or a different context on the same device) gets its own
// lookup instead of a stale address.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

static std::mutex g_noalloc_mutex;
static std::vector<std::pair<unsigned long long, void*>> g_noalloc_addr;  // (context ID, device address)

// ID of the current context; false if there is none yet or the driver
// entry points are unavailable (then nothing is cached).
static bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();
  });
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

static rpcg_status noalloc_scratch(void** out) {
  int dev = 0;
  RPCG_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  if (have_id) {
    for (const auto& e : g_noalloc_addr) {
      if (e.first == id) {
        *out = e.second;
        return RPCG_OK;
      }
    }
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // with the caller's context current
  if (e != cudaSuccess || p == nullptr) {
    set_error("rpcg_dot_exact_noalloc: cudaGetSymbolAddress on device %d failed: %s", dev, cudaGetErrorString(e));
    return RPCG_ERR_CUDA;
  }
  // the lookup creates the primary context if none was current before it
  if (have_id || current_context_id(&id)) g_noalloc_addr.emplace_back(id, p);
  *out = p;
  return RPCG_OK;
}

}  // namespace rpcg

extern "C" rpcg_status rpcg_dot_exact_noalloc(int64_t n, const double* a, const double* b, double* out,
                                              void* stream) {
  clear_error();
  if (n < 0 || n > kNoAllocMaxN) {
    set_error("rpcg_dot_exact_noalloc: n = %lld is outside [0, 2^30], the largest size it accepts", (long long)n);
    return RPCG_ERR_INVALID;
  }
  RPCG_CHECK_ARG(out != nullptr, "out is NULL");
  RPCG_CHECK_ARG(n == 0 || (a != nullptr && b != nullptr), "a or b is NULL");
  void* scratch = nullptr;
  const rpcg_status st = noalloc_scratch(&scratch);
  if (st != RPCG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  DotScratch* ws = static_cast<DotScratch*>(scratch);
  // the array keeps the previous call's contents: clear the part the kernel
  // expects to start at zero (accumulator digits, arrival counter, flags)
  RPCG_CUDA_TRY(cudaMemsetAsync(ws, 0, kDotScratchHeader, s));
  launch_dot_exact(n, a, b, ws, out, s);
  RPCG_CUDA_TRY(cudaGetLastError());
  return RPCG_OK;
}
