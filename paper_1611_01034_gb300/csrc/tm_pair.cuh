// Arithmetic on unevaluated sums h + l of two FP32 numbers ("pairs").
//
// GB300 runs FP64 at 1/64 of its FP32 rate.  Where a result must be
// FP64-accurate but the arithmetic is heavy, every real is carried as a pair
// (Dekker's double-length arithmetic, Numer. Math. 18 (1971) 224, with
// Knuth's two-sum): the product a.h * b.h is made exact with an FMA, the cross
// terms and all rounding errors gather in l.  A pair holds about 47 bits of
// significand; products and sums lose a few bits more.
//
// Conversions go through integer operations on the bit patterns, so that no
// FP64 instruction is issued per element where it can be avoided:
//   d2pair: FP64 -> pair, h the FP64 value truncated to 24 significant bits, l
//           the remainder truncated to 24 bits (47 bits in all);
//   f2d_bits: FP32 -> FP64 exactly (normal numbers).
#pragma once
#include "tm_internal.cuh"

namespace tmamg {

// a value h + l
struct dfl {
  float h, l;
};

// error-free transforms (the _rn intrinsics are never contracted into FMAs)
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// acc += a * b, a a pair, b an exact FP32 number
__device__ __forceinline__ void fma_pf(dfl& acc, dfl a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = __fmaf_rn(a.h, b, -p);
  e = __fmaf_rn(a.l, b, e);
  const dfl s = two_sum(acc.h, p);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}
// acc += a * b, both pairs (the l * l term, 2^-48 relative, is dropped)
__device__ __forceinline__ void fma_pp(dfl& acc, dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const dfl s = two_sum(acc.h, p);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}
__device__ __forceinline__ dfl neg(dfl a) { return {-a.h, -a.l}; }
__device__ __forceinline__ void add_to(dfl& acc, dfl a) {
  const dfl s = two_sum(acc.h, a.h);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, a.l));
}

struct cdf {
  dfl r, i;
};

// acc += u * x (pairs)
__device__ __forceinline__ void cfma_pp(cdf& acc, cdf u, cdf x) {
  fma_pp(acc.r, u.r, x.r);
  fma_pp(acc.r, neg(u.i), x.i);
  fma_pp(acc.i, u.r, x.i);
  fma_pp(acc.i, u.i, x.r);
}
// acc += conj(u) * x (pairs)
__device__ __forceinline__ void cfmac_pp(cdf& acc, cdf u, cdf x) {
  fma_pp(acc.r, u.r, x.r);
  fma_pp(acc.r, u.i, x.i);
  fma_pp(acc.i, u.r, x.i);
  fma_pp(acc.i, neg(u.i), x.r);
}
// acc += u * x, x exact FP32
__device__ __forceinline__ void cfma_pf(cdf& acc, cdf u, cx<float> x) {
  fma_pf(acc.r, u.r, x.r);
  fma_pf(acc.r, neg(u.i), x.i);
  fma_pf(acc.i, u.r, x.i);
  fma_pf(acc.i, u.i, x.r);
}
__device__ __forceinline__ void cfmac_pf(cdf& acc, cdf u, cx<float> x) {
  fma_pf(acc.r, u.r, x.r);
  fma_pf(acc.r, u.i, x.i);
  fma_pf(acc.i, u.r, x.i);
  fma_pf(acc.i, neg(u.i), x.r);
}

// FP32 bits -> FP64 with integer operations (exact for normal numbers; FP32
// subnormals, below 1.2e-38, become zero)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned mag = u & 0x7fffffffu;
  if (mag < 0x00800000u) return __longlong_as_double((long long)sgn);
  if (mag >= 0x7f800000u) return (double)f;  // Inf, NaN
  const unsigned long long bits = sgn | (((unsigned long long)mag << 29) + (896ull << 52));
  return __longlong_as_double((long long)bits);
}

// FP64 -> pair by bit operations.  x = (-1)^s 2^E (1 + m / 2^52): h keeps the
// top 23 bits of m; the remaining 29 bits r give x - h = (-1)^s 2^(E-23) r / 2^29,
// formed exactly as the difference of the FP32 numbers 2^(E-23) (1 + (r >> 6) / 2^23)
// and 2^(E-23) (Sterbenz) after dropping r's lowest 6 bits.  Magnitudes below
// 2^-103 (where 2^(E-23) leaves the FP32 normal range) become 0; above the FP32
// range the ordinary conversion applies.
__device__ __forceinline__ dfl d2pair(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned top = (unsigned)(u >> 32);
  const unsigned sgn = top & 0x80000000u;
  const int e = (int)((top >> 20) & 0x7ffu) - 1023;  // unbiased exponent
  if (e < -103) return dfl{__uint_as_float(sgn), 0.f};
  if (e > 127) return dfl{__double2float_rn(x), 0.f};
  const unsigned E = (unsigned)(e + 127);
  const float h = __uint_as_float(sgn | (E << 23) | ((unsigned)(u >> 29) & 0x7fffffu));
  const unsigned r = (unsigned)u & 0x1fffffffu;
  const unsigned El = (E - 23u) << 23;
  const float l = __fsub_rn(__uint_as_float(El | (r >> 6)), __uint_as_float(El));
  return dfl{h, sgn ? -l : l};
}

// pair -> FP64 (one FP64 addition)
__device__ __forceinline__ double pair2d(dfl a) { return f2d_bits(a.h) + f2d_bits(a.l); }

__device__ __forceinline__ cdf cx2pair(double re, double im) { return cdf{d2pair(re), d2pair(im)}; }

}  // namespace tmamg
