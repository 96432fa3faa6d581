// Error-free transformations (Alg. 1 twosum, Alg. 2 twoprod) computed on
// the integer pipe.
//
// GB300 issues about 1.9 FP64 instructions per clock per SM but ~120
// integer ones, so the FPE dot's twosums and twoprods run as exact integer
// arithmetic on binary64 values.  A value is kept unpacked as a signed
// significand and the exponent of its last bit: v = m * 2^e, normalised
// (m == 0, or 2^52 <= |m| < 2^53, or e == -1074 for subnormals).
//
// twosum(a, x): the exact sum S = a + x is formed as a 128-bit integer in
// units of the smaller last-bit exponent, rounded once to 53 bits with ties
// to even (r = RN(a + x)), and s = S - r is exact (the error of a
// round-to-nearest addition is always a binary64 number).  If the exponents
// differ by more than 54 the smaller operand is below a quarter ulp of the
// larger: r = the larger, s = the smaller.
// twoprod(a, b): the 106-bit product of the significands, rounded once (to
// 53 bits, or at 2^-1074 in the subnormal range) gives r = RN(a b); s is
// the exact remainder when it is representable (|r| >= 2^-969, which the
// FPE dot requires anyway).
//
// The values produced are exactly those of the FP64 formulas of Algs. 1-2
// (the signs of zero terms may differ, which changes no sum).  Overflow
// (|r| >= 2^1024) sets the `bad` flag.
#pragma once
#include <cstdint>

#include "device.cuh"

namespace rpcg {

struct SF {
  long long m;  // signed significand, |m| < 2^53
  int e;        // exponent of the last bit
};

__device__ __forceinline__ int bitlen128(unsigned __int128 v) {
  const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
  return hi ? 128 - __clzll(hi) : (lo ? 64 - __clzll(lo) : 0);
}

__device__ __forceinline__ int bitlen64(unsigned long long v) { return v ? 64 - __clzll(v) : 0; }

// Normalise an exactly representable value v * 2^e (|v| < 2^63): shift the
// significand to 53 bits, or as far as e allows towards -1074.  Sets `bad`
// if bits would be lost (not representable).
__device__ __forceinline__ SF sf_exact(long long v, int e, bool& bad) {
  if (v == 0) return SF{0, 0};
  const bool neg = v < 0;
  unsigned long long a = neg ? 0ull - (unsigned long long)v : (unsigned long long)v;
  int nb = bitlen64(a);
  if (nb > 53) {
    const int sh = nb - 53;
    bad |= (a & ((1ull << sh) - 1ull)) != 0ull;
    a >>= sh;
    e += sh;
    nb = 53;
  }
  if (e < -1074) {
    // below the last subnormal bit: representable only if those bits are zero
    const int sh = -1074 - e;
    if (sh >= 64) {
      bad |= a != 0ull;
      a = 0ull;
    } else {
      bad |= (a & ((1ull << sh) - 1ull)) != 0ull;
      a >>= sh;
    }
    e = -1074;
    if (a == 0ull) return SF{0, 0};
    nb = bitlen64(a);
  }
  int sh = 53 - nb;  // left-normalise, not below 2^-1074
  const int room = e + 1074;
  if (sh > room) sh = room;
  a <<= sh;
  e -= sh;
  if (e > 971) bad = true;  // |v| >= 2^1024
  return SF{neg ? -(long long)a : (long long)a, e};
}

// Round the magnitude M * 2^e (M < 2^117) to binary64, ties to even, with
// gradual underflow; returns the rounded significand/exponent and the exact
// remainder M * 2^e - R * 2^(e + sh) as (rem, e) with |rem| <= 2^(sh-1).
__device__ __forceinline__ void sf_round(unsigned __int128 M, int e, unsigned long long& R, int& re, long long& rem) {
  const int nb = bitlen128(M);
  int sh = nb - 53;
  if (e + sh < -1074) sh = -1074 - e;  // subnormal result: last bit at 2^-1074
  if (sh > 127) sh = 127;              // M < 2^117: any shift past 117 already rounds to zero
  if (sh <= 0) {
    // exact (the caller normalises)
    R = (unsigned long long)M;
    re = e;
    rem = 0;
    return;
  }
  const unsigned __int128 q = M >> sh;
  const unsigned __int128 low = M - (q << sh);
  const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
  unsigned __int128 r = q;
  if (low > half || (low == half && (q & 1))) r += 1;
  // remainder relative to 2^e: low - (r - q) * 2^sh, |.| <= 2^(sh-1)
  const __int128 d = (__int128)low - (__int128)((r - q) << sh);
  rem = (long long)d;  // |d| <= 2^(sh-1) <= 2^63 only when sh <= 64: callers guarantee sh <= 56
  R = (unsigned long long)r;
  re = e + sh;
  if (R == (1ull << 53)) {
    R >>= 1;
    re += 1;
  }
}

// Alg. 1 on unpacked values.
__device__ __forceinline__ void sf_twosum(SF a, SF x, SF& r, SF& s, bool& bad) {
  if (x.m == 0) {
    r = a;
    s = SF{0, 0};
    return;
  }
  if (a.m == 0) {
    r = x;
    s = SF{0, 0};
    return;
  }
  const bool a_hi = a.e >= x.e;
  const SF hi = a_hi ? a : x;
  const SF lo = a_hi ? x : a;
  const int d = hi.e - lo.e;
  if (d > 54) {  // |lo| < ulp(hi) / 4 (hi is normal: its exponent exceeds the subnormal one)
    r = hi;
    s = lo;
    return;
  }
  const __int128 S = ((__int128)hi.m << d) + (__int128)lo.m;  // exact, |S| < 2^108
  if (S == 0) {
    r = SF{0, 0};
    s = SF{0, 0};
    return;
  }
  const bool neg = S < 0;
  const unsigned __int128 M = neg ? (unsigned __int128)(-S) : (unsigned __int128)S;
  unsigned long long R;
  int re;
  long long rem;
  sf_round(M, lo.e, R, re, rem);
  r = sf_exact(neg ? -(long long)R : (long long)R, re, bad);
  s = sf_exact(neg ? -rem : rem, lo.e, bad);
}

// Unpack a finite double.
__device__ __forceinline__ SF sf_from(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7ff);
  long long m = (long long)(b & 0xFFFFFFFFFFFFFull);
  int e;
  if (E) {
    m |= 1ll << 52;
    e = E - 1075;
  } else {
    e = -1074;
  }
  if (b >> 63) m = -m;
  return SF{m, e};
}

// Pack (exact: a normalised value is a binary64 number unless e > 971).
__device__ __forceinline__ double sf_to_double(SF v) {
  if (v.m == 0) return 0.0;
  const bool neg = v.m < 0;
  const unsigned long long a = neg ? 0ull - (unsigned long long)v.m : (unsigned long long)v.m;
  unsigned long long bits;
  if (a >= (1ull << 52)) {
    const int biased = v.e + 1075;
    bits = biased >= 2047 ? 0x7FF0000000000000ull : (((unsigned long long)biased << 52) | (a - (1ull << 52)));
  } else {
    bits = a;  // subnormal (e == -1074)
  }
  if (neg) bits |= 0x8000000000000000ull;
  return __longlong_as_double((long long)bits);
}

// Alg. 2 on doubles (finite inputs; the caller checks finiteness).
__device__ __forceinline__ void sf_twoprod(double a, double b, SF& r, SF& s, bool& bad) {
  const SF A = sf_from(a), B = sf_from(b);
  if (A.m == 0 || B.m == 0) {
    r = SF{0, 0};
    s = SF{0, 0};
    return;
  }
  const bool neg = (A.m < 0) != (B.m < 0);
  const unsigned long long ma = (unsigned long long)(A.m < 0 ? -A.m : A.m);
  const unsigned long long mb = (unsigned long long)(B.m < 0 ? -B.m : B.m);
  const unsigned __int128 P = (unsigned __int128)ma * mb;  // < 2^106
  unsigned long long R;
  int re;
  long long rem;
  // the remainder fits 64 bits only if the rounding drops at most ~62 bits;
  // deeper subnormal rounding (|r| < 2^-969) is flagged by the FPE dot itself
  const int e = A.e + B.e;
  sf_round(P, e, R, re, rem);
  if (re - e > 56) {
    bad = true;  // the product's error is below the representable range
    rem = 0;
  }
  r = sf_exact(neg ? -(long long)R : (long long)R, re, bad);
  s = sf_exact(neg ? -rem : rem, e, bad);
}

// Accumulate (Alg. 4, early exit) of an unpacked carry into an expansion
// whose terms are stored as doubles; returns the carry out of the last term.
template <int PMAX>
__device__ __forceinline__ SF sf_accumulate(double (&f)[PMAX], int p, SF x, bool& bad) {
#pragma unroll
  for (int i = 0; i < PMAX; i++) {
    if (i < p && x.m != 0) {
      SF r, s;
      sf_twosum(sf_from(f[i]), x, r, s, bad);
      f[i] = sf_to_double(r);
      x = s;
    }
  }
  return x;
}

// |v| < 2^-969 (v != 0 or the operands were non-zero)
__device__ __forceinline__ bool sf_below_twoprod_safe(SF v) {
  if (v.m == 0) return true;
  const unsigned long long a = (unsigned long long)(v.m < 0 ? -v.m : v.m);
  return v.e + bitlen64(a) - 1 < -969;
}

// One element of the FPE dot on the integer pipe: twoprod, the product into
// the result expansion, its error into the error expansion.  Returns true if
// bits may have been lost; a, b must be finite.
template <int PMAX>
__device__ __forceinline__ bool sf_fpe_dot_step(double (&res)[PMAX], double (&err)[PMAX], int p, double a, double b) {
  if (a == 0.0 || b == 0.0) return false;  // adds nothing
  bool bad = false;
  SF r, s;
  sf_twoprod(a, b, r, s, bad);
  bool lost = sf_below_twoprod_safe(r);
  lost |= sf_accumulate(res, p, r, bad).m != 0;
  if (s.m != 0) lost |= sf_accumulate(err, p, s, bad).m != 0;
  return lost | bad;
}

// One element of the FPE dot on the integer pipe with the expansions and
// flag of fpe_dot_step: twoprod and Alg. 4's twosums as exact integer
// arithmetic.  A product whose error is not representable (|r| < 2^-969)
// or that overflows takes fpe_dot_step itself (both flag it as inexact).
// A sum that overflows sets `nonfinite` (fpe_dot_step leaves an infinite
// term there, which makes the dot NaN when the terms are deposited), so the
// results agree in that case too.  a, b finite.
__device__ __forceinline__ bool fpe_dot_step_int(double (&res)[kFpeMax], double (&err)[kFpeMax], int p, double a,
                                                 double b, bool& nonfinite) {
  if (is_zero_bits(a) || is_zero_bits(b)) return false;  // adds nothing
  bool bad = false;
  SF r, s;
  sf_twoprod(a, b, r, s, bad);
  if (bad || sf_below_twoprod_safe(r)) return fpe_dot_step(res, err, p, a, b);
  bool lost = sf_accumulate(res, p, r, bad).m != 0;
  if (s.m != 0) lost |= sf_accumulate(err, p, s, bad).m != 0;
  nonfinite |= bad;
  return lost | bad;
}

// GB300's FP64 pipe is its scarce unit: 3 of every 8 warps of a CTA run the
// FPE dot's element steps on the integer pipes instead (fpe_dot_step_int
// gives the same expansions), so both kinds of pipe work at once.
// Warp-uniform.
__device__ __forceinline__ bool fpe_int_warp() {
  const int nw = (int)(blockDim.x >> 5);
  return (int)(threadIdx.x >> 5) < (3 * nw + 4) / 8;
}

}  // namespace rpcg
