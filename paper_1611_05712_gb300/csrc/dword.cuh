// Double-word arithmetic: a float64-accurate number as an unevaluated sum of two floats.
//
// GB300 runs float64 at 1/64 of its float32 rate, and the FP64 form's row FFT was bound by
// the float64 unit.  Its butterflies run on the float32 units with each real number an
// unevaluated sum of two floats, hi + lo with |lo| <= ulp(hi)/2: about 48 significant bits
// (double-word arithmetic after Dekker, Numer. Math. 18, 1971, with error-free products
// from fused multiply-adds).  Sum: the exact sum of the high parts (Knuth's two-sum) plus
// the low parts, renormalised: error below 2u^2 (|x| + |y|), u = 2^-24, an absolute error
// of the kind an FFT's error bound is made of.  Product: the exact product of the high
// parts (one fma) plus the cross terms: error below a few u^2 |x y|.  Grids stay doubles
// in memory; the conversions use integer operations and, on the way out, one float64
// addition per value.
#pragma once

#include <stdint.h>

namespace pic {

struct dw {
  float hi, lo;
  dw() = default;
  __host__ __device__ constexpr dw(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit dw(int v) : hi((float)v), lo(0.f) {}
  dw(double) = delete;   // a double converts through dw_from_double, never through int
};
struct dw2 {
  dw x, y;
};

__device__ __forceinline__ float dw_neg_if(float v, bool neg) {
  return __int_as_float(__float_as_int(v) ^ (neg ? (int)0x80000000u : 0));
}
__device__ __forceinline__ dw neg_if(dw v, bool neg) { return dw(dw_neg_if(v.hi, neg), dw_neg_if(v.lo, neg)); }
__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {   // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return dw(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dw operator+(dw x, dw y) {
  const float s = __fadd_rn(x.hi, y.hi);
  const float bb = __fsub_rn(s, x.hi);
  const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));   // s + e = x.hi + y.hi
  return dw_fast_two_sum(s, __fadd_rn(e, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dw operator-(dw x) { return dw(-x.hi, -x.lo); }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }
__device__ __forceinline__ dw operator*(dw x, dw y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);   // p + e = x.hi y.hi exactly
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return dw_fast_two_sum(p, e);
}

// double -> double word: hi = x with its mantissa cut to 24 bits, lo = the remaining 29
// bits rounded to nearest (even) to a float, subnormal where it falls below the normal
// range, all in integer operations (a conversion instruction would run on the float64
// unit).  |x| >= 2^128 gives +-inf and |x| < 2^-126 +-0; in between the pair keeps about
// 48 bits while |x| >= 2^-74 and fewer below, losing at most 2^-150 of absolute value.
__device__ __forceinline__ dw dw_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < -126) return dw(__uint_as_float(sign), 0.f);
  if (e > 127) return dw(__uint_as_float(sign | 0x7f800000u), 0.f);
  const unsigned long long m = b & 0xfffffffffffffull;
  const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
  unsigned r = (unsigned)(m & 0x1fffffffull);   // the rest: r 2^(e - 52)
  if (r == 0u) return dw(hi, 0.f);
  int p = 31 - __clz(r);                           // leading bit of r, 0 .. 28
  int sh = p - 23;                                 // right shift to 24 significant bits
  if (p + e - 52 + 127 < 1) sh = -(e - 52 + 149);  // shift so that one unit is 2^-149
  unsigned q;
  if (sh > 0) {                                    // round to nearest, ties to even
    if (sh >= 32) return dw(hi, 0.f);
    const unsigned rem = r & ((1u << sh) - 1u), half = 1u << (sh - 1);
    q = r >> sh;
    if (rem > half || (rem == half && (q & 1u))) ++q;
  } else {
    q = r << (-sh);
  }
  unsigned lob;
  if (p + e - 52 + 127 < 1) {
    lob = q;                                       // subnormal (a carry into bit 23 is the smallest normal)
  } else {
    int pe = p;
    if (q == (1u << 24)) { q >>= 1; ++pe; }
    lob = ((unsigned)(pe + e - 52 + 127) << 23) | (q & 0x7fffffu);
  }
  return dw(hi, __uint_as_float(sign | lob));
}

// float -> double exactly, by the bits.
__device__ __forceinline__ double dw_widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xffu, mf = u & 0x7fffffu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long d;
  if (ef == 0u) {   // 0 or subnormal: mf 2^-149
    if (mf == 0u) {
      d = sgn;
    } else {
      const int p = 31 - __clz(mf);
      d = sgn | ((unsigned long long)(1023 - 149 + p) << 52) | (((unsigned long long)mf << (52 - p)) & 0xfffffffffffffull);
    }
  } else {
    d = sgn | ((unsigned long long)(ef == 0xffu ? 0x7ffu : ef - 127 + 1023) << 52) | ((unsigned long long)mf << 29);
  }
  return __longlong_as_double((long long)d);
}
__device__ __forceinline__ double dw_to_double(dw v) { return dw_widen(v.hi) + dw_widen(v.lo); }
__device__ __forceinline__ dw& operator+=(dw& x, dw y) { return x = x + y; }
__device__ __forceinline__ dw& operator-=(dw& x, dw y) { return x = x - y; }
__device__ __forceinline__ dw& operator*=(dw& x, dw y) { return x = x * y; }

}  // namespace pic
