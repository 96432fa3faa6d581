// Device primitives of the reproducible dot products.
//
// Exact dot (Sec. 2.1, Sec. 4.1).  A finite double is +-m 2^e with integer
// m < 2^53 and e >= -1074, so a product is +-M 2^E with M = m_a m_b < 2^106
// and E >= -2148.  The long accumulator is a fixed-point integer whose bit 0
// weighs 2^kE0; it is stored as kNDig signed 64-bit digits, digit k holding
// a sum of 32-bit chunks of weight 2^(32k + kE0).  A digit only ever
// receives values below 2^32 in magnitude, so 2^31 deposits fit in its 64
// bits without a carry (the paper's carry-safe headroom, Sec. 4.3; here
// 32 headroom bits instead of 12).
//
// GB300 has ~1.7 FP64 instructions per clock per SM against ~120 simple
// integer instructions, so the per-element work of the exact dot runs on
// the integer pipe: the 106-bit product is formed with 32x32-bit multiplies
// and added, shifted, into a 224-bit register window (a per-thread long
// accumulator segment, the role the FPE plays in ExBLAS); products outside
// the window go to a shared-memory accumulator with 64-bit atomics; the CTA
// accumulators meet in global memory with 64-bit atomics (exact and
// order-independent, the single-GPU form of Listing 3's MPI_Reduce); the
// last CTA normalises the carries and rounds once (Round in Listing 3).
//
// FPE dot (Sec. 4.2).  twosum (Alg. 1), twoprod (Alg. 2), Accumulate with
// early exit (Alg. 4) and fpesum (Alg. 3) in FP64.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rpcg {

constexpr int kE0 = -2176;            // weight exponent of accumulator bit 0
constexpr int kNDig = 136;            // 32-bit digits (4352 bits)
constexpr int kSubLsb = -1074 - kE0;  // bit index of 2^-1074 (1102)
constexpr int kCopies = 8;            // shared-memory accumulator copies (spread contention)
constexpr int kWin = 7;               // 32-bit words of the register window
constexpr int kFpeMax = 8;            // largest expansion size

// ------------------------------------------------------------------ exact products

// |a*b| as five 32-bit words already shifted by the in-digit offset, the
// digit index q of word 0, the sign as an all-ones mask, and flags.
struct ExactProd {
  uint32_t w0, w1, w2, w3, w4;
  int q;
  uint32_t neg;
  bool nz;
  bool bad;  // a or b is Inf or NaN
};

// General form: every finite, zero, subnormal, infinite or NaN operand.
__device__ __forceinline__ ExactProd exact_product_general(double a, double b) {
  // everything on 32-bit halves: exponent field, significand high part
  // with the hidden bit (normal numbers) or without it (subnormals, whose
  // exponent is that of field 1)
  const uint32_t ah = (uint32_t)__double2hiint(a), al = (uint32_t)__double2loint(a);
  const uint32_t bh = (uint32_t)__double2hiint(b), bl = (uint32_t)__double2loint(b);
  const uint32_t ea = (ah >> 20) & 0x7ffu, eb = (bh >> 20) & 0x7ffu;
  ExactProd p;
  p.bad = (ea == 0x7ffu) | (eb == 0x7ffu);
  const uint32_t mah = (ah & 0xFFFFFu) | (ea ? 0x100000u : 0u);
  const uint32_t mbh = (bh & 0xFFFFFu) | (eb ? 0x100000u : 0u);
  // product LSB weight 2^(max(ea,1) + max(eb,1) - 2150); offset from 2^kE0
  const int o = (int)(max(ea, 1u) + max(eb, 1u)) - 2150 - kE0;  // 28 .. 4118
  p.q = o >> 5;
  const uint32_t r = (uint32_t)o & 31u;
  // 106-bit significand product (mah:al) x (mbh:bl) from four 32x32 products
  const uint64_t p0 = (uint64_t)al * bl;
  const uint64_t p1 = (uint64_t)al * mbh + (uint64_t)mah * bl;  // < 2^54
  const uint64_t p2 = (uint64_t)mah * mbh;                      // < 2^42
  const uint32_t v0 = (uint32_t)p0;
  uint32_t v1, v2, v3;
  asm("add.cc.u32 %0, %3, %4;\n\t"
      "addc.cc.u32 %1, %5, %6;\n\t"
      "addc.u32 %2, %7, 0;"
      : "=r"(v1), "=r"(v2), "=r"(v3)
      : "r"((uint32_t)(p0 >> 32)), "r"((uint32_t)p1), "r"((uint32_t)(p1 >> 32)), "r"((uint32_t)p2),
        "r"((uint32_t)(p2 >> 32)));
  p.w0 = v0 << r;
  p.w1 = __funnelshift_l(v0, v1, r);
  p.w2 = __funnelshift_l(v1, v2, r);
  p.w3 = __funnelshift_l(v2, v3, r);
  p.w4 = __funnelshift_l(v3, 0u, r);
  p.neg = (uint32_t)((int32_t)(ah ^ bh) >> 31);
  // a zero product (either significand zero) yields five zero words: adding
  // it anywhere changes nothing, so no separate test is needed on the fast path
  p.nz = !p.bad;
  return p;
}

// Fast form for two normal operands (exponent field neither 0 nor all
// ones), the case of every product in practice; others take the general
// form (inlined: a call in the per-element loop costs more than it saves).
// Same fields, fewer ALU instructions: the exponent sum comes from the two
// exponent fields in place, with no subnormal clamps or hidden-bit selects.
__device__ __forceinline__ ExactProd exact_product(double a, double b) {
  const uint32_t ah = (uint32_t)__double2hiint(a), al = (uint32_t)__double2loint(a);
  const uint32_t bh = (uint32_t)__double2hiint(b), bl = (uint32_t)__double2loint(b);
  const uint32_t fa = ah & 0x7ff00000u, fb = bh & 0x7ff00000u;
  // field 0 wraps to 0xfff00000, field 0x7ff to 0x7fe00000: both outside the normal range
  if ((fa - 0x00100000u) >= 0x7fe00000u || (fb - 0x00100000u) >= 0x7fe00000u) return exact_product_general(a, b);
  ExactProd p;
  p.bad = false;
  p.nz = true;
  const uint32_t mah = (ah & 0x000FFFFFu) | 0x00100000u;
  const uint32_t mbh = (bh & 0x000FFFFFu) | 0x00100000u;
  const int o = (int)((fa + fb) >> 20) - 2150 - kE0;  // fa + fb < 2^32
  p.q = o >> 5;
  const uint32_t r = (uint32_t)o & 31u;
  const uint64_t p0 = (uint64_t)al * bl;
  const uint64_t p1 = (uint64_t)al * mbh + (uint64_t)mah * bl;  // < 2^54
  const uint64_t p2 = (uint64_t)mah * mbh;                      // < 2^42
  const uint32_t v0 = (uint32_t)p0;
  uint32_t v1, v2, v3;
  asm("add.cc.u32 %0, %3, %4;\n\t"
      "addc.cc.u32 %1, %5, %6;\n\t"
      "addc.u32 %2, %7, 0;"
      : "=r"(v1), "=r"(v2), "=r"(v3)
      : "r"((uint32_t)(p0 >> 32)), "r"((uint32_t)p1), "r"((uint32_t)(p1 >> 32)), "r"((uint32_t)p2),
        "r"((uint32_t)(p2 >> 32)));
  p.w0 = v0 << r;
  p.w1 = __funnelshift_l(v0, v1, r);
  p.w2 = __funnelshift_l(v1, v2, r);
  p.w3 = __funnelshift_l(v2, v3, r);
  p.w4 = __funnelshift_l(v3, 0u, r);
  p.neg = (uint32_t)((int32_t)(ah ^ bh) >> 31);
  return p;
}

// signed 64-bit contribution of an unsigned 32-bit chunk under a sign mask
__device__ __forceinline__ unsigned long long signed_chunk(uint32_t w, uint32_t neg) {
  const long long v = (long long)w;
  return (unsigned long long)(neg ? -v : v);
}

// Deposit a product into a shared-memory accumulator laid out as
// sacc[digit * kCopies + copy] (64-bit atomics; wrap-around addition of
// two's-complement values is exact while the true digit sum fits).
__device__ __forceinline__ void smem_deposit(unsigned long long* sacc, int copy, const ExactProd& p) {
  unsigned long long* base = sacc + p.q * kCopies + copy;
  if (p.w0) atomicAdd(base + 0 * kCopies, signed_chunk(p.w0, p.neg));
  if (p.w1) atomicAdd(base + 1 * kCopies, signed_chunk(p.w1, p.neg));
  if (p.w2) atomicAdd(base + 2 * kCopies, signed_chunk(p.w2, p.neg));
  if (p.w3) atomicAdd(base + 3 * kCopies, signed_chunk(p.w3, p.neg));
  if (p.w4) atomicAdd(base + 4 * kCopies, signed_chunk(p.w4, p.neg));
}

// Per-thread register window: a 224-bit two's-complement integer W whose
// word 0 has digit index qb.  Products whose digit index is qb or qb + 1
// are added with one carry chain; others go to shared memory.  When a
// larger product arrives the window is flushed and moved up so that it
// tracks the top of the magnitude range.
struct Window {
  uint32_t W[kWin];
  int qb;  // kUnanchored: not anchored yet
};

// Not anchored yet: qb far below every digit, so the first product moves
// the window up to itself (the flush of the empty window adds nothing).
constexpr int kUnanchored = -(1 << 20);

__device__ __forceinline__ void window_init(Window& w) {
#pragma unroll
  for (int k = 0; k < kWin; k++) w.W[k] = 0;
  w.qb = kUnanchored;
}

__device__ __forceinline__ void window_flush(Window& w, unsigned long long* sacc, int copy) {
  if (w.qb < 0) return;
  unsigned long long* base = sacc + w.qb * kCopies + copy;
#pragma unroll
  for (int k = 0; k < kWin - 1; k++) {
    if (w.W[k]) atomicAdd(base + k * kCopies, (unsigned long long)w.W[k]);
  }
  // the top word carries the sign of the whole window
  if (w.W[kWin - 1]) atomicAdd(base + (kWin - 1) * kCopies, (unsigned long long)(long long)(int)w.W[kWin - 1]);
#pragma unroll
  for (int k = 0; k < kWin; k++) w.W[k] = 0;
}

// W += (neg ? -1 : 1) * (p.w << 32 t), t in {0, 1}: the addend is formed
// as (chunk XOR mask) with carry-in (mask & 1) -- two's-complement negation
// folded into one add-with-carry chain.
__device__ __forceinline__ void window_add(Window& w, const ExactProd& p, bool t1) {
  const uint32_t m = p.neg;
  const uint32_t a0 = (t1 ? 0u : p.w0) ^ m;
  const uint32_t a1 = (t1 ? p.w0 : p.w1) ^ m;
  const uint32_t a2 = (t1 ? p.w1 : p.w2) ^ m;
  const uint32_t a3 = (t1 ? p.w2 : p.w3) ^ m;
  const uint32_t a4 = (t1 ? p.w3 : p.w4) ^ m;
  const uint32_t a5 = (t1 ? p.w4 : 0u) ^ m;
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

__device__ __forceinline__ void exact_deposit(Window& w, unsigned long long* sacc, int copy, const ExactProd& p) {
  if (!p.nz) return;
  const int t = p.q - w.qb;
  if ((unsigned)t < 2u) {
    window_add(w, p, t == 1);
  } else if (t > 1) {
    // a larger product (or the first one): move the window up to it.  q is at
    // most 128, so the clamped anchor keeps q - qb in {0, 1}.
    window_flush(w, sacc, copy);
    const int qb = min(max(p.q - 1, 0), kNDig - kWin);
    w.qb = qb;
    window_add(w, p, p.q - qb == 1);
  } else {
    smem_deposit(sacc, copy, p);
  }
}

// Sum the kCopies copies of each digit of a CTA's shared accumulator and add
// the non-zero digits to the global accumulator.  Needs a __syncthreads()
// before (all deposits done) -- the caller provides it.
__device__ __forceinline__ void smem_to_global(const unsigned long long* sacc, unsigned long long* gacc) {
  for (int k = threadIdx.x; k < kNDig; k += blockDim.x) {
    unsigned long long s = 0;
#pragma unroll
    for (int c = 0; c < kCopies; c++) s += sacc[k * kCopies + c];
    if (s) atomicAdd(gacc + k, s);
  }
  // make this thread's additions visible device-wide before the CTA announces
  // its arrival (the last CTA reads the digits right after)
  __threadfence();
}

// Zero `nacc` shared-memory accumulators (kNDig * kCopies words each).
__device__ __forceinline__ void smem_acc_zero(unsigned long long* sacc, int nacc = 1) {
  for (int k = threadIdx.x; k < nacc * kNDig * kCopies; k += blockDim.x) sacc[k] = 0ull;
}

// ------------------------------------------------------------------ rounding

// Normalise the carries of kNDig signed digits and round the value
// sum_k dig[k] 2^(32k + kE0) once to the nearest binary64, ties to even,
// with gradual underflow and overflow to +-inf.  An exact zero gives +0.
// dig[k] must be zero outside [lo, hi] (lo > hi: every digit is zero).
// Runs on one thread; D is kNDig words of scratch (shared memory), of which
// only [lo, hi + 1] is written.
//
// Below lo every normalised digit is 0.  After digit hi the carry is
// below 2^31 in magnitude, so digit hi + 1 takes it and every digit above
// is the sign extension (0, or all ones for a negative value).  The
// two's-complement negation of a negative value sends its +1 through the
// zero digits below lo and stops at lo (that digit is non-zero), so the
// magnitude lives in [lo, hi + 1] as well.
static __device__ __noinline__ double round_digits_range(const long long* dig, uint32_t* D, int lo, int hi) {
  if (lo > hi) return 0.0;
  const int top = hi + 1 < kNDig ? hi + 1 : kNDig - 1;
  long long c = 0;
  for (int k = lo; k <= top; k++) {
    const long long v = dig[k] + c;  // |dig| < 2^62, |c| < 2^31: no overflow
    D[k] = (uint32_t)v;
    c = v >> 32;  // arithmetic shift: floor division by 2^32
  }
  const bool negative = c < 0;
  if (negative) {
    unsigned long long carry = 1;
    for (int k = lo; k <= top; k++) {
      const unsigned long long t = (unsigned long long)(~D[k]) + carry;
      D[k] = (uint32_t)t;
      carry = t >> 32;
    }
  }
  auto digit = [&](int k) -> uint32_t { return (k >= lo && k <= top) ? D[k] : 0u; };
  int kt = -1;
  for (int k = top; k >= lo; k--) {
    if (D[k]) {
      kt = k;
      break;
    }
  }
  if (kt < 0) return 0.0;
  const int t = 32 * kt + 31 - __clz(D[kt]);  // index of the leading bit
  int lsb = t - 52;
  if (lsb < kSubLsb) lsb = kSubLsb;
  // 64 bits starting at lsb
  const int wi = lsb >> 5, bi = lsb & 31;
  const unsigned long long w_lo = (unsigned long long)digit(wi) | ((unsigned long long)digit(wi + 1) << 32);
  const unsigned long long w_hi = digit(wi + 2);
  unsigned long long mant = bi ? ((w_lo >> bi) | (w_hi << (64 - bi))) : w_lo;
  const int nbits = t - lsb + 1;  // 1 .. 53
  mant &= (nbits >= 64) ? ~0ull : ((1ull << nbits) - 1ull);
  // round bit and sticky bits below it
  const int rb_i = lsb - 1;
  const uint32_t rbit = (digit(rb_i >> 5) >> (rb_i & 31)) & 1u;
  bool sticky = (digit(rb_i >> 5) & ((1u << (rb_i & 31)) - 1u)) != 0u;
  for (int k = (rb_i >> 5) - 1; k >= lo && !sticky; k--) sticky = D[k] != 0u;
  if (rbit && (sticky || (mant & 1ull))) mant += 1ull;
  if (mant == (1ull << 53)) {
    mant >>= 1;
    lsb += 1;
  }
  unsigned long long bits;
  if (mant >= (1ull << 52)) {
    const int biased = lsb + kE0 + 1075;  // exponent field of mant * 2^(lsb + kE0)
    if (biased >= 2047) bits = 0x7FF0000000000000ull;
    else bits = ((unsigned long long)biased << 52) | (mant - (1ull << 52));
  } else {
    bits = mant;  // subnormal (lsb == kSubLsb)
  }
  if (negative) bits |= 0x8000000000000000ull;
  return __longlong_as_double((long long)bits);
}

// round_digits_range for the common case of at most kRegDigits digits in
// [lo, min(hi + 1, kNDig - 1)]: the same steps on an unrolled register copy
// (no shared-memory round trip per digit; digits are picked by compare and
// select, so nothing is indexed dynamically).  Callers check the width.
constexpr int kRegDigits = 8;

__device__ __forceinline__ uint32_t reg_digit(const uint32_t (&D)[kRegDigits], int k) {
  uint32_t v = 0u;
#pragma unroll
  for (int j = 0; j < kRegDigits; j++) v = (k == j) ? D[j] : v;
  return v;
}

__device__ __forceinline__ double round_digits_reg(const long long* dig, int lo, int hi) {
  if (lo > hi) return 0.0;
  const int top = hi + 1 < kNDig ? hi + 1 : kNDig - 1;
  const int cnt = top - lo + 1;  // <= kRegDigits
  uint32_t D[kRegDigits];
  long long c = 0;
#pragma unroll
  for (int k = 0; k < kRegDigits; k++) {
    const long long v = (k < cnt ? dig[lo + k] : 0ll) + c;
    D[k] = (uint32_t)v;
    c = k < cnt ? (v >> 32) : c;
  }
  const bool negative = c < 0;
  if (negative) {
    unsigned long long carry = 1;
#pragma unroll
    for (int k = 0; k < kRegDigits; k++) {
      const unsigned long long t = (unsigned long long)(~D[k]) + carry;
      D[k] = (uint32_t)t;
      carry = t >> 32;
    }
  }
#pragma unroll
  for (int k = 0; k < kRegDigits; k++) D[k] = k < cnt ? D[k] : 0u;  // above top: zero once negated
  int kt = -1;
#pragma unroll
  for (int k = 0; k < kRegDigits; k++) kt = D[k] ? k : kt;
  if (kt < 0) return 0.0;
  const int t = 32 * (lo + kt) + 31 - __clz(reg_digit(D, kt));  // index of the leading bit
  int lsb = t - 52;
  if (lsb < kSubLsb) lsb = kSubLsb;
  const int wi = (lsb >> 5) - lo, bi = lsb & 31;  // word index relative to lo (may be negative)
  const unsigned long long w_lo = (unsigned long long)reg_digit(D, wi) | ((unsigned long long)reg_digit(D, wi + 1) << 32);
  const unsigned long long w_hi = reg_digit(D, wi + 2);
  unsigned long long mant = bi ? ((w_lo >> bi) | (w_hi << (64 - bi))) : w_lo;
  const int nbits = t - lsb + 1;  // 1 .. 53
  mant &= (nbits >= 64) ? ~0ull : ((1ull << nbits) - 1ull);
  const int rb_i = lsb - 1;
  const int rw = (rb_i >> 5) - lo;  // word of the round bit, relative to lo
  const uint32_t rword = reg_digit(D, rw);
  const uint32_t rbit = (rword >> (rb_i & 31)) & 1u;
  bool sticky = (rword & ((1u << (rb_i & 31)) - 1u)) != 0u;
#pragma unroll
  for (int k = 0; k < kRegDigits; k++) sticky |= (k < rw) && D[k] != 0u;
  if (rbit && (sticky || (mant & 1ull))) mant += 1ull;
  if (mant == (1ull << 53)) {
    mant >>= 1;
    lsb += 1;
  }
  unsigned long long bits;
  if (mant >= (1ull << 52)) {
    const int biased = lsb + kE0 + 1075;
    if (biased >= 2047) bits = 0x7FF0000000000000ull;
    else bits = ((unsigned long long)biased << 52) | (mant - (1ull << 52));
  } else {
    bits = mant;
  }
  if (negative) bits |= 0x8000000000000000ull;
  return __longlong_as_double((long long)bits);
}

// Either form, by the width of the live range.
__device__ __forceinline__ double round_digits_fast(const long long* dig, uint32_t* D, int lo, int hi) {
  const int top = hi + 1 < kNDig ? hi + 1 : kNDig - 1;
  if (lo <= hi && top - lo + 1 <= kRegDigits) return round_digits_reg(dig, lo, hi);
  return round_digits_range(dig, D, lo, hi);
}

// round_digits_range over the non-zero digits of dig (found by a scan).
static __device__ __noinline__ double round_digits(const long long* dig, uint32_t* D) {
  int lo = kNDig, hi = -1;
  for (int k = 0; k < kNDig; k++) {
    if (dig[k]) {
      lo = k < lo ? k : lo;
      hi = k;
    }
  }
  return round_digits_range(dig, D, lo, hi);
}

// Block-parallel form: every thread of the block calls it; the digits are
// taken (and zeroed) from the global accumulator g into dig (shared), the
// non-zero range is found with shared atomics, and thread 0 returns the
// rounded value (the others return 0).  range is two ints of shared scratch.
__device__ __forceinline__ double take_and_round(unsigned long long* g, long long* dig, uint32_t* D, int* range) {
  if (threadIdx.x == 0) {
    range[0] = kNDig;
    range[1] = -1;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kNDig; k += blockDim.x) {
    const long long v = (long long)atomicExch(&g[k], 0ull);
    dig[k] = v;
    if (v) {
      atomicMin(&range[0], k);
      atomicMax(&range[1], k);
    }
  }
  __syncthreads();
  return threadIdx.x == 0 ? round_digits_fast(dig, D, range[0], range[1]) : 0.0;
}

// ------------------------------------------------------------------ EFTs and FPEs

// Alg. 1
__device__ __forceinline__ void two_sum(double a, double b, double& r, double& s) {
  r = __dadd_rn(a, b);
  const double z = __dsub_rn(r, a);
  s = __dadd_rn(__dsub_rn(a, __dsub_rn(r, z)), __dsub_rn(b, z));
}

// Alg. 1's result with half the FP64 work: order the operands by magnitude
// with an integer compare of their bit patterns, then Dekker's Fast2Sum
// (r = RN(a + b), z = RN(r - a), s = RN(b - z) is exact when |a| >= |b|).
// The pair (r, s) of an error-free addition is unique, so this gives the
// same values as Alg. 1.
__device__ __forceinline__ void two_sum_ordered(double a, double b, double& r, double& s) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b) & 0x7FFFFFFFFFFFFFFFull;
  const bool sw = ub > ua;
  const double big = sw ? b : a, small = sw ? a : b;
  r = __dadd_rn(big, small);
  const double z = __dsub_rn(r, big);
  s = __dsub_rn(small, z);
}

// Alg. 2
__device__ __forceinline__ void two_prod(double a, double b, double& r, double& s) {
  r = __dmul_rn(a, b);
  s = __fma_rn(a, b, -r);
}

// Tests on the bit pattern (integer pipe), keeping the scarce FP64 pipe for
// the arithmetic of the error-free transformations.
__device__ __forceinline__ bool is_zero_bits(double x) { return ((unsigned long long)__double_as_longlong(x) << 1) == 0ull; }
__device__ __forceinline__ bool is_finite_bits(double x) {
  return (((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffull) != 0x7ffull;
}

// Alg. 4 with the early exit of Sec. 4.2; returns the value carried out of
// the last of the p terms (0 when nothing was lost).
__device__ __forceinline__ double fpe_accumulate(double (&f)[kFpeMax], int p, double x) {
#pragma unroll
  for (int i = 0; i < kFpeMax; i++) {
    if (i < p) {
      double r, s;
      two_sum_ordered(f[i], x, r, s);
      f[i] = r;
      x = s;
      if (is_zero_bits(x)) break;
    }
  }
  return x;
}

// Alg. 3: a += b; returns true if a term was lost.
// The loop over b's terms is rolled (the term is picked by selects, so both
// expansions stay in registers): one copy of Alg. 4's loop instead of
// kFpeMax keeps the code small.
__device__ __forceinline__ bool fpe_sum(double (&a)[kFpeMax], const double (&b)[kFpeMax], int p) {
  bool lost = false;
#pragma unroll 1
  for (int i = 0; i < p; i++) {
    double bi = b[0];
#pragma unroll
    for (int k = 1; k < kFpeMax; k++)
      if (i == k) bi = b[k];
    if (!is_zero_bits(bi)) lost |= !is_zero_bits(fpe_accumulate(a, p, bi));
  }
  return lost;
}

constexpr double kTwoProdSafe = 0x1p-969;  // |a*b| >= this: twoprod's error term is exact

// One element of the FPE dot: product into the result expansion, its error
// into the error expansion.  Returns true if bits may have been lost.
__device__ __forceinline__ bool fpe_dot_step(double (&res)[kFpeMax], double (&err)[kFpeMax], int p, double a, double b) {
  if (is_zero_bits(a) || is_zero_bits(b)) return false;  // adds nothing
  double r, s;
  two_prod(a, b, r, s);
  // |r| < 2^-969 (exponent field below 54) or r not finite: bits may be lost
  const unsigned rexp = (unsigned)(((unsigned long long)__double_as_longlong(r) >> 52) & 0x7ffull);
  bool lost = (rexp < 54u) | (rexp == 0x7ffu);
  lost |= !is_zero_bits(fpe_accumulate(res, p, r));
  if (!is_zero_bits(s)) lost |= !is_zero_bits(fpe_accumulate(err, p, s));
  return lost;
}

// ------------------------------------------------------------------ misc

// Fixed-shape sum over a CTA (warp shuffles, then warp 0 over the warp
// sums); the result is valid in thread 0.  sw: 32 doubles of shared memory.
template <int BLOCK>
__device__ __forceinline__ double block_sum_fixed(double v, double* sw) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sw[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < BLOCK / 32 ? sw[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_down_sync(0xffffffffu, s, o));
  }
  return s;
}

__device__ __forceinline__ bool is_last_block(unsigned int* counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Exact sum of up to kFpeMax doubles (used to round a merged expansion):
// deposit each term into plain digits and round.  One thread.
static __device__ __noinline__ double exact_sum_terms(const double* terms, int p, long long* dig, uint32_t* D) {
  for (int k = 0; k < kNDig; k++) dig[k] = 0;
  for (int i = 0; i < p; i++) {
    const ExactProd e = exact_product(terms[i], 1.0);
    if (!e.nz) continue;
    const uint32_t w[5] = {e.w0, e.w1, e.w2, e.w3, e.w4};
    for (int k = 0; k < 5; k++) {
      const long long v = (long long)w[k];
      dig[e.q + k] += e.neg ? -v : v;
    }
  }
  return round_digits(dig, D);
}

}  // namespace rpcg
