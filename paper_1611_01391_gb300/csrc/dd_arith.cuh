// Double-float arithmetic: every value is an unevaluated pair hi + lo of
// FP32 numbers (Dekker, "A floating-point technique for extending the
// available precision", 1971; Knuth TAOCP vol. 2, 4.2.2; Hida, Li & Bailey,
// "Algorithms for quad-double precision", 2001), carrying about 48
// significant bits.  On this GPU the FP64 pipe issues 1/64 of the FP32 rate,
// so a double-float multiply-add (10 to 20 FP32 instructions) is several
// times cheaper than a native FP64 one.  The explicitly rounded intrinsics
// (__fadd_rn, __fmul_rn, ...) keep the compiler from contracting the
// error-free transformations into FMAs.
#pragma once

#include <cuda_runtime.h>

namespace lra {

struct __align__(8) dd {  // 8-byte aligned: one 64-bit access per pair
  float hi, lo;
};

__device__ __forceinline__ dd dd_make(float x) { return dd{x, 0.0f}; }

__device__ __forceinline__ dd dd_from_double(double x) {
  const float h = (float)x;
  return dd{h, (float)(x - (double)h)};
}

__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return dd{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}

// Dekker's FastTwoSum (|a| >= |b|): renormalise a pair.
__device__ __forceinline__ dd quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dd{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  const dd t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }

// TwoProduct through the FMA, plus the cross terms.
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}

__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) { return dd_add(dd_mul(a, b), c); }

// Compensated accumulator of a dot product of double-float vectors: the
// FP32 running sum s plus the FP32 sum c of every rounding error (the
// product errors come exactly from the FMA, the sum errors from TwoSum), so
// s + c carries about twice FP32 precision (Dot2 of Ogita, Rump & Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005, with the
// low parts of the operands folded into the product error).
struct dacc {
  float s, c;
};

__device__ __forceinline__ void acc_fma(dacc& a, dd x, dd y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  const dd t = two_sum(a.s, p);
  a.s = t.hi;
  a.c = __fadd_rn(a.c, __fadd_rn(t.lo, e));
}

__device__ __forceinline__ dacc acc_add(dacc a, dacc b) {
  const dd t = two_sum(a.s, b.s);
  return dacc{t.hi, __fadd_rn(__fadd_rn(a.c, b.c), t.lo)};
}

__device__ __forceinline__ dd acc_value(dacc a) { return two_sum(a.s, a.c); }

// Sum over the G consecutive lanes of a group (G a power of two <= 32);
// every lane of the warp must take part.
template <int G>
__device__ __forceinline__ dacc acc_group_sum(dacc a) {
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1)
    a = acc_add(a, dacc{__shfl_xor_sync(0xffffffffu, a.s, off), __shfl_xor_sync(0xffffffffu, a.c, off)});
  return a;
}

// x y + a for an FP32 x (exact, no low part) and a pair y.
__device__ __forceinline__ void acc_fma_f(dacc& a, float x, dd y) {
  const float p = __fmul_rn(x, y.hi);
  float e = fmaf(x, y.hi, -p);
  e = fmaf(x, y.lo, e);
  const dd t = two_sum(a.s, p);
  a.s = t.hi;
  a.c = __fadd_rn(a.c, __fadd_rn(t.lo, e));
}

// b - c r, renormalised: the product error comes exactly from the FMA (plus
// the cross terms of the low parts), the difference error from TwoSum.
__device__ __forceinline__ dd dd_fnma(dd c, dd r, dd b) {
  const float p = __fmul_rn(c.hi, r.hi);
  float e = fmaf(c.hi, r.hi, -p);
  e = fmaf(c.hi, r.lo, e);
  e = fmaf(c.lo, r.hi, e);
  const dd t = two_sum(b.hi, -p);
  return quick_two_sum(t.hi, __fadd_rn(t.lo, __fsub_rn(b.lo, e)));
}

// a / b: the FP32 quotient q1 of the high parts, corrected by the quotient
// of the remainder a - q1 b (formed exactly up to the low-part products)
// by b.hi (Dekker's division).
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const float p = __fmul_rn(q1, b.hi);
  float e = fmaf(q1, b.hi, -p);
  e = fmaf(q1, b.lo, e);
  const dd r = two_sum(a.hi, -p);
  const float rem = __fadd_rn(r.hi, __fadd_rn(r.lo, __fsub_rn(a.lo, e)));
  return quick_two_sum(q1, __fdiv_rn(rem, b.hi));
}

}  // namespace lra
