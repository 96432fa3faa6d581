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
// FPE dot (Sec. 4.2).  twoprod (Alg. 2) in FP64; twosum (Alg. 1) in FP64
// or as exact integer arithmetic on the bit patterns; Accumulate with early
// exit (Alg. 4) and fpesum (Alg. 3) built on either twosum.
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
    for (int c = 0; c < kCopies; c++) s += sacc[k * kCopies + ((c + k) & (kCopies - 1))];  // staggered: fewer bank conflicts
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

// Binary64 bits (sign clear) of m * 2^lsb, for m < 2^56 exactly representable
// at or above 2^-1074 and lsb >= -1074: normalise m to 53 bits (right
// shifts drop only zero bits), or stop at 2^-1074 (subnormal).  Adding the
// shifted significand to (lsb' + 1074) << 52 lets its hidden bit carry into
// the exponent field, so normal and subnormal values take the same formula.
// ovf is set if the value is 2^1024 or more.  m = 0 gives +0.
__device__ __forceinline__ unsigned long long pack_bits(unsigned long long m, int lsb, bool& ovf) {
  const int nb = 64 - __clzll((long long)m);
  int shift = 53 - nb;
  int lsb2 = lsb - shift;
  if (lsb2 < -1074) {
    shift = lsb + 1074;
    lsb2 = -1074;
  }
  const unsigned long long mm = shift >= 0 ? (m << shift) : (m >> (-shift));
  ovf |= (m != 0ull) & (lsb2 >= 972);
  return m ? ((unsigned long long)(lsb2 + 1074) << 52) + mm : 0ull;
}

// Alg. 1 on the integer pipe, every case, for finite a and b: r = RN(a + b) and
// s = a + b - r, the same unique pair as the FP64 formulas (zero terms may
// differ in sign, which changes no sum).  Let |A| >= |B| be the operands
// ordered by magnitude, with significands mA, mB and last-bit exponents
// (B's is the unit below).  If their exponent fields differ by d > 54,
// |B| < ulp(A)/4: r = A, s = B.  Otherwise B is split at k = max(d - 3, 0)
// bits into a high part and a low part L < 2^k, so that
// |A + B| = Mh 2^k + Ml with Mh = mA 2^(d-k) +- high part (below 2^57, three
// guard bits) and 0 <= Ml < 2^k (a borrow turns a subtracted low part into
// a positive one): everything fits 64-bit integers.  Mh is rounded to 53
// bits, ties to even, with Ml as the sticky part; the dropped bits minus
// the rounding increment, times 2^k, plus Ml, are s.  ovf is set if |r|
// reaches 2^1024 (the FP64 formulas give a non-finite r there).
struct TwoSumOut {
  double r, s;
  bool ovf;
};

__device__ __forceinline__ TwoSumOut two_sum_int_general_body(double a, double b) {
  bool ovf = false;
  constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull, kM52 = 0xFFFFFFFFFFFFFull;
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  const bool sw = (ub & kAbs) > (ua & kAbs);
  const unsigned long long A = sw ? ub : ua, B = sw ? ua : ub;
  const unsigned long long xa = A & kAbs, xb = B & kAbs;
  const int EA = (int)(xa >> 52), EB = (int)(xb >> 52);
  const unsigned long long mA = (xa & kM52) | ((unsigned long long)(EA != 0) << 52);
  const unsigned long long mB = (xb & kM52) | ((unsigned long long)(EB != 0) << 52);
  const int eB = max(EB, 1);
  const int d = max(EA, 1) - eB;  // >= 0
  const bool opp = (long long)(A ^ B) < 0;
  const int k = min(max(d - 3, 0), 51);  // (clamped only on the d > 54 path, whose values are not used)
  const unsigned long long mBh = mB >> k, mBl = mB & ((1ull << k) - 1ull);
  const unsigned long long Ah = mA << min(d, 3);
  const unsigned long long br = (opp && mBl != 0ull) ? 1ull : 0ull;
  const unsigned long long Mh = opp ? Ah - mBh - br : Ah + mBh;
  const unsigned long long Ml = opp ? (br ? (1ull << k) - mBl : 0ull) : mBl;
  const int nb = 64 - __clzll((long long)Mh);
  const int sh = max(nb - 53, 0);
  const unsigned long long q0 = Mh >> sh;
  const unsigned long long low = Mh & ((1ull << sh) - 1ull);
  const unsigned long long half = (1ull << sh) >> 1;
  const bool up = sh != 0 && (low > half || (low == half && (Ml != 0ull || (q0 & 1ull))));
  const unsigned long long q = q0 + (up ? 1ull : 0ull);
  // s in units of B's last bit, as a two's-complement 64-bit value (|s| < 2^56)
  const unsigned long long sv = ((low - (up ? (1ull << sh) : 0ull)) << k) + Ml;
  const bool sneg = (long long)sv < 0;
  const unsigned long long smag = sneg ? 0ull - sv : sv;
  const unsigned long long signA = A & ~kAbs;
  bool o = false;
  const unsigned long long rb = q ? (pack_bits(q, eB - 1075 + k + sh, o) | signA) : 0ull;
  const unsigned long long sb = smag ? (pack_bits(smag, eB - 1075, o) | (sneg ? signA ^ ~kAbs : signA)) : 0ull;
  const bool trivial = xb == 0ull || d > 54;  // r = A, s = B (B may be zero)
  ovf |= o && !trivial;
  TwoSumOut out;
  out.r = __longlong_as_double((long long)(trivial ? A : rb));
  out.s = __longlong_as_double((long long)(trivial ? (xb ? B : 0ull) : sb));
  out.ovf = ovf;
  return out;
}

static __device__ __noinline__ TwoSumOut two_sum_int_general(double a, double b) {
  return two_sum_int_general_body(a, b);
}

// 64-bit integer arithmetic on 32-bit halves.  Written out with 32-bit
// instructions (add/sub with carry, clamped funnel shifts) so that it stays
// on the integer pipe.
__device__ __forceinline__ void add_u64(uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl, uint32_t& rh, uint32_t& rl) {
  asm("add.cc.u32 %1, %3, %5;\n\taddc.u32 %0, %2, %4;" : "=r"(rh), "=r"(rl) : "r"(ah), "r"(al), "r"(bh), "r"(bl));
}
__device__ __forceinline__ void sub_u64(uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl, uint32_t& rh, uint32_t& rl) {
  asm("sub.cc.u32 %1, %3, %5;\n\tsubc.u32 %0, %2, %4;" : "=r"(rh), "=r"(rl) : "r"(ah), "r"(al), "r"(bh), "r"(bl));
}
// (hi:lo) <<= n for n in [0, 63]: two clamped funnel-shift stages of at most 32
__device__ __forceinline__ void shl_u64(uint32_t& hi, uint32_t& lo, uint32_t n) {
  const uint32_t h1 = __funnelshift_lc(lo, hi, n), l1 = __funnelshift_lc(0u, lo, n);
  const uint32_t n2 = n > 32u ? n - 32u : 0u;
  hi = __funnelshift_lc(l1, h1, n2);
  lo = __funnelshift_lc(0u, l1, n2);
}

// Alg. 1 split between the pipes, for finite a and b: r = RN(a + b) is one
// FP64 addition; s = a + b - r is computed exactly on the integer pipe (GB300
// issues about 60 integer instructions in the time of one FP64 one).  With
// |A| >= |B| the operands ordered by magnitude, s = B - (r - A) (Fast2Sum,
// both subtractions exact):
//   * a zero operand, or a sum that cancels below half of A (|r| < |A|/2:
//     then a + b is exact), or a subnormal r (likewise exact): s = 0;
//   * B more than 54 exponent fields below A (B under a quarter ulp of A):
//     r = A, s = B;
//   * otherwise, with B's field >= 54 (so s is normal), in units of half of
//     B's last bit: r - A = |r| - |A| (same sign, r within a factor two of
//     A) is formed from the significands in units of half of A's last bit,
//     shifted up by the field difference d <= 54, and subtracted from (or,
//     for operands of opposite signs, added to) 2 m_B; the result has at
//     most 53 significant bits and is normalised into s's bits (the hidden
//     bit carries into the exponent field).  Everything fits 64 bits, held
//     as 32-bit halves.
// Other operands (B with field < 54) take two_sum_int_general out of line.
// ovf is set if r overflows (the FP64 formulas give a non-finite pair).
// The pair equals the FP64 algorithm's (zero terms may differ in sign,
// which changes no sum).
__device__ __forceinline__ void two_sum_split(double a, double b, double& r, double& s, bool& ovf) {
  r = __dadd_rn(a, b);
  const uint32_t ah = (uint32_t)__double2hiint(a), al = (uint32_t)__double2loint(a);
  const uint32_t bh = (uint32_t)__double2hiint(b), bl = (uint32_t)__double2loint(b);
  const uint32_t rh = (uint32_t)__double2hiint(r), rl = (uint32_t)__double2loint(r);
  const uint32_t xah = ah & 0x7FFFFFFFu, xbh = bh & 0x7FFFFFFFu;
  const bool sw = (xbh > xah) || (xbh == xah && bl > al);
  const uint32_t Ah = sw ? bh : ah, Al = sw ? bl : al, Bh = sw ? ah : bh, Bl = sw ? al : bl;
  const uint32_t EA = (Ah >> 20) & 0x7FFu, EB = (Bh >> 20) & 0x7FFu, ER = (rh >> 20) & 0x7FFu;
  const uint32_t d = EA - EB;
  if (ER == 0x7FFu) {
    ovf = true;
    s = 0.0;
    return;
  }
  if (((Bh & 0x7FFFFFFFu) | Bl) == 0u || ER + 1u < EA || ER == 0u) {
    s = 0.0;
    return;
  }
  if (d > 54u && EB != 0u) {
    s = __hiloint2double((int)Bh, (int)Bl);
    return;
  }
  if (EB >= 54u && d <= 54u) {
    // z = (m_r << (ER + 1 - EA)) - (m_A << 1): |r| - |A| in units of half A's last bit
    uint32_t zh = (rh & 0xFFFFFu) | 0x100000u, zl = rl;
    const uint32_t k1 = ER + 1u - EA;  // 0 .. 2
    zh = __funnelshift_lc(zl, zh, k1);
    zl = __funnelshift_lc(0u, zl, k1);
    const uint32_t mah = (Ah & 0xFFFFFu) | 0x100000u;
    uint32_t th, tl;
    add_u64(mah, Al, mah, Al, th, tl);
    sub_u64(zh, zl, th, tl, zh, zl);
    shl_u64(zh, zl, d);  // r - A in units of half B's last bit (two's complement)
    const uint32_t mbh = (Bh & 0xFFFFFu) | 0x100000u;
    uint32_t b2h, b2l;
    add_u64(mbh, Bl, mbh, Bl, b2h, b2l);  // 2 m_B
    // s / sign(A) = 2 m_B - z (same signs) or -(2 m_B + z) (opposite signs)
    const bool opp = (int32_t)(Ah ^ Bh) < 0;
    uint32_t vh, vl, wh, wl;
    add_u64(b2h, b2l, zh, zl, wh, wl);
    sub_u64(b2h, b2l, zh, zl, vh, vl);
    vh = opp ? wh : vh;
    vl = opp ? wl : vl;
    const uint32_t m = (uint32_t)((int32_t)vh >> 31);
    uint32_t mh, ml;
    sub_u64(vh ^ m, vl ^ m, m, m, mh, ml);  // |v|
    const uint32_t sneg = ((m != 0u) != opp) ? 0x80000000u : 0u;
    const uint32_t c = mh ? (uint32_t)__clz((int)mh) : 32u + (uint32_t)__clz((int)ml);  // 9 .. 64
    shl_u64(mh, ml, c - 9u);  // leading bit to bit 54 (c = 64 only for |v| = 0)
    ml = __funnelshift_rc(ml, mh, 2u);
    mh >>= 2;
    const uint32_t e = EB + 9u - c;  // exponent field of s minus one
    const uint32_t sh = (mh + (e << 20)) | ((Ah & 0x80000000u) ^ sneg);
    s = (mh | ml) ? __hiloint2double((int)sh, (int)ml) : 0.0;
    return;
  }
  const TwoSumOut o = two_sum_int_general(a, b);
  s = o.s;
  ovf |= o.ovf;
}

// Alg. 2
__device__ __forceinline__ void two_prod(double a, double b, double& r, double& s) {
  r = __dmul_rn(a, b);
  s = __fma_rn(a, b, -r);
}

// two_prod out of line, for the rare operands two_prod_int declines: a call
// is a real branch, where an inlined fallback could be turned into
// predicated instructions that take FP64-pipe slots for every element.
static __device__ __noinline__ void two_prod_rare(double a, double b, double& r, double& s) { two_prod(a, b, r, s); }

// Alg. 2 on the integer pipe for two normal operands whose product has an
// exponent field in [107, 2045] (|a b| from 2^-916 up, no overflow; s is
// then normal or zero); returns false for other operands, which take
// two_prod (FP64 multiply and fma use four FP64-pipe slots on GB300, a
// half-rate pipe).  The 106-bit product of the significands comes from
// four 32x32-bit multiplies; r keeps its top 53 bits rounded to nearest
// even (the bits below are the sticky part), and s = the dropped bits minus
// the rounding increment, normalised.  The same pair as Alg. 2 (checked
// elementwise against the FP64 formulas).
__device__ __forceinline__ bool two_prod_int(double a, double b, double& r, double& s) {
  const uint32_t ah = (uint32_t)__double2hiint(a), al = (uint32_t)__double2loint(a);
  const uint32_t bh = (uint32_t)__double2hiint(b), bl = (uint32_t)__double2loint(b);
  const uint32_t EA = (ah >> 20) & 0x7FFu, EB = (bh >> 20) & 0x7FFu;
  const int fr = (int)(EA + EB) - 1023;  // r's exponent field if the product has 105 bits (106: one more)
  if (EA == 0u || EB == 0u || EA == 0x7FFu || EB == 0x7FFu || fr < 107 || fr > 2045) return false;
  const uint32_t mah = (ah & 0xFFFFFu) | 0x100000u, mbh = (bh & 0xFFFFFu) | 0x100000u;
  // product (w3:w2:w1:w0) = (mah:al) (mbh:bl)
  const uint64_t p0 = (uint64_t)al * bl, p2 = (uint64_t)mah * mbh;
  const uint64_t p1 = (uint64_t)al * mbh + (uint64_t)mah * bl;  // < 2^54
  const uint32_t w0 = (uint32_t)p0;
  uint32_t w1, w2, w3;
  asm("add.cc.u32 %0, %3, %4;\n\t"
      "addc.cc.u32 %1, %5, %6;\n\t"
      "addc.u32 %2, %7, 0;"
      : "=r"(w1), "=r"(w2), "=r"(w3)
      : "r"((uint32_t)(p0 >> 32)), "r"((uint32_t)p1), "r"((uint32_t)(p1 >> 32)), "r"((uint32_t)p2),
        "r"((uint32_t)(p2 >> 32)));
  const uint32_t big = w3 >> 9;     // the product has 106 bits (top bit 105) or 105
  const uint32_t sh32 = 20u + big;  // bits dropped: 52 + big = 32 + sh32
  const uint32_t qh = __funnelshift_rc(w2, w3, sh32), ql = __funnelshift_rc(w1, w2, sh32);
  const uint32_t lowh = w1 & ((1u << sh32) - 1u), halfh = 1u << (sh32 - 1u);  // dropped bits (lowh:w0), half = halfh:0
  const bool up = lowh > halfh || (lowh == halfh && (w0 != 0u || (ql & 1u)));
  uint32_t rqh, rql;
  add_u64(qh, ql, 0u, up ? 1u : 0u, rqh, rql);
  const uint32_t sign = (ah ^ bh) & 0x80000000u;
  r = __hiloint2double((int)((rqh + ((uint32_t)(fr - 1 + (int)big) << 20)) | sign), (int)rql);
  // s = dropped bits - up 2^(52 + big), in units of the product's last bit
  uint32_t vh = lowh, vl = w0;
  if (up) sub_u64(lowh, w0, 1u << sh32, 0u, vh, vl);
  const uint32_t m = (uint32_t)((int32_t)vh >> 31);
  uint32_t mh, ml;
  sub_u64(vh ^ m, vl ^ m, m, m, mh, ml);
  const uint32_t c = mh ? (uint32_t)__clz((int)mh) : 32u + (uint32_t)__clz((int)ml);  // 11 .. 64
  shl_u64(mh, ml, c - 11u);  // leading bit to bit 52
  const uint32_t sb = (mh + ((EA + EB - 1065u - c) << 20)) | (sign ^ (m ? 0x80000000u : 0u));
  s = (mh | ml) ? __hiloint2double((int)sb, (int)ml) : 0.0;
  return true;
}

// Tests on the bit pattern (integer pipe), keeping the scarce FP64 pipe for
// the arithmetic of the error-free transformations.
// Both work on the 32-bit halves: written on the 64-bit pattern, the tests
// were turned into FP64 compares, which take FP64-pipe slots.
__device__ __forceinline__ bool is_zero_bits(double x) {
  return (((uint32_t)__double2hiint(x) << 1) | (uint32_t)__double2loint(x)) == 0u;
}
// the exponent field of x (bits 52..62)
__device__ __forceinline__ uint32_t exp_field(double x) { return ((uint32_t)__double2hiint(x) >> 20) & 0x7FFu; }
__device__ __forceinline__ bool is_finite_bits(double x) { return exp_field(x) != 0x7FFu; }

// Alg. 1 as Fast2Sum on the operand of larger magnitude: r = RN(A + B) and
// s = B - (r - A), both subtractions exact when |A| >= |B| (Dekker).  Three
// FP64 additions and an integer compare; the same (r, s) as two_sum_split.
// A sum that overflows sets ovf (s = 0).
__device__ __forceinline__ void two_sum_fast(double a, double b, double& r, double& s, bool& ovf) {
  const uint32_t xah = (uint32_t)__double2hiint(a) & 0x7FFFFFFFu, xbh = (uint32_t)__double2hiint(b) & 0x7FFFFFFFu;
  const bool sw = xbh > xah || (xbh == xah && (uint32_t)__double2loint(b) > (uint32_t)__double2loint(a));
  const double A = sw ? b : a, B = sw ? a : b;
  r = __dadd_rn(A, B);
  if (exp_field(r) == 0x7FFu) {
    ovf = true;
    s = 0.0;
    return;
  }
  s = __dsub_rn(B, __dsub_rn(r, A));
}

// One level of a cascade: twosum of term i with the carry x.  FAST = false:
// two_sum_split (one FP64 addition, the error on the integer pipe); true:
// two_sum_fast (three FP64 additions).
template <bool FAST = false>
__device__ __forceinline__ void fpe_level(double& fi, double& x, bool& ovf) {
  double r, s;
  if constexpr (FAST) two_sum_fast(fi, x, r, s, ovf);
  else two_sum_split(fi, x, r, s, ovf);
  fi = r;
  x = s;
}

// The helpers below take expansions as arrays of N terms (N = kFpeMax, or
// fewer in kernel instances built for small p), of which the first p are in
// use.

// Alg. 4 with the early exit of Sec. 4.2; returns the value carried out of
// the last of the p terms (0 when nothing was lost).  ovf is set if a term
// overflows.
template <int N>
__device__ __forceinline__ double fpe_accumulate(double (&f)[N], int p, double x, bool& ovf) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (i < p) {
      fpe_level(f[i], x, ovf);
      if (is_zero_bits(x)) break;
    }
  }
  return x;
}

// Alg. 3: a += b; returns true if a term was lost.
// The loop over b's terms is rolled (the term is picked by selects, so both
// expansions stay in registers): one copy of Alg. 4's loop instead of
// kFpeMax keeps the code small.
template <int N>
__device__ __forceinline__ bool fpe_sum(double (&a)[N], const double (&b)[N], int p, bool& ovf) {
  bool lost = false;
#pragma unroll 1
  for (int i = 0; i < p; i++) {
    double bi = b[0];
#pragma unroll
    for (int k = 1; k < N; k++)
      if (i == k) bi = b[k];
    if (!is_zero_bits(bi)) lost |= !is_zero_bits(fpe_accumulate(a, p, bi, ovf));
  }
  return lost;
}

// Alg. 4 from term 1 on, for a carry that term 0 has already produced.
// A lane whose carry became zero does nothing more (the early exit); the
// warp leaves the unrolled levels as soon as no lane here has a carry left.
// That exit is a vote, so the branch is the same in every lane and stays a
// branch: with per-lane exits alone the levels ran as predicated code, and
// every element issued the FP64 additions of all N - 1 levels.
template <bool FAST, int N>
__device__ __forceinline__ double fpe_accumulate_from1(double (&f)[N], int p, double x, bool& ovf) {
#pragma unroll
  for (int i = 1; i < N; i++) {
    if (i < p) {
      if (__all_sync(__activemask(), is_zero_bits(x))) break;
      if (!is_zero_bits(x)) fpe_level<FAST>(f[i], x, ovf);
    }
  }
  return x;
}

// Which twosum each expansion's cascades use.  The result expansion takes
// two_sum_fast (three FP64 additions, little integer work) and the error
// expansion two_sum_split (one FP64 addition, the error on the integer
// pipe), which balances the FP64 and ALU pipes: on 2^24 U[-1, 1] pairs the
// FPE dot takes 0.32 ms, against 0.40 ms with two_sum_split in both and
// 0.35 ms with two_sum_fast in both.
constexpr bool kFpeResFast = true;
constexpr bool kFpeErrFast = false;

// One element of the FPE dot: product into the result expansion, its error
// into the error expansion.  Returns true if bits may have been lost.
// twoprod (Alg. 2) is two_prod_int (FP64 only for out-of-range operands);
// the twosums of the Accumulate cascades (Alg. 4) are two_sum_fast in the
// result expansion and two_sum_split in the error expansion (kFpeResFast,
// kFpeErrFast; both give Alg. 1's exact pair).  The two expansions are independent,
// so term 0 of both (a level nearly every element reaches) is updated
// together: two independent dependency chains in flight.  Each expansion
// still sees exactly Alg. 4's sequence of twosums (twosum(e, 0) = (e, 0),
// so a zero error term changes nothing).  A product or a term that
// overflows sets `nonfinite` (the dot's value is then NaN, as the FP64
// formulas' non-finite terms would make it).
template <int N>
__device__ __forceinline__ bool fpe_dot_step(double (&res)[N], double (&err)[N], int p, double a, double b,
                                             bool& nonfinite) {
  if (is_zero_bits(a) || is_zero_bits(b)) return false;  // adds nothing
  double r, s;
  if (!two_prod_int(a, b, r, s)) two_prod_rare(a, b, r, s);
  // |r| < 2^-969 (exponent field below 54) or r not finite: bits may be lost
  const unsigned rexp = exp_field(r);
  if (rexp == 0x7ffu) {
    nonfinite = true;
    return true;
  }
  bool ovf = false;
  bool lost = rexp < 54u;
  fpe_level<kFpeResFast>(res[0], r, ovf);
  fpe_level<kFpeErrFast>(err[0], s, ovf);
  if (!is_zero_bits(r)) lost |= p < 2 || !is_zero_bits(fpe_accumulate_from1<kFpeResFast>(res, p, r, ovf));
  if (!is_zero_bits(s)) lost |= p < 2 || !is_zero_bits(fpe_accumulate_from1<kFpeErrFast>(err, p, s, ovf));
  nonfinite |= ovf;
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
