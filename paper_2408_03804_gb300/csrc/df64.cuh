// Double-float ("df64") arithmetic: a real number carried as an unevaluated
// sum hi + lo of two FP32 values with |lo| <= ulp(hi)/2, about 48 significant
// bits. On this GPU FP32 issues about 75 times faster than FP64, so a
// transform whose FP64 operations are the bound runs several times faster in
// df64 at a precision (2^-48 per operation) far below the CG tolerances.
//
// The operations are the classical error-free transformations: Knuth's
// TwoSum (the exact rounding error of a + b, any ordering), Dekker's
// FastTwoSum (|a| >= |b|), and the exact product error fma(a, b, -ab). The
// addition below keeps the error of the low parts at FP32 level relative to
// the operands (|error| <= about 2^-47 (|a| + |b|)), the bound the FFT's
// normwise error analysis needs; products keep about 2^-47 relative error.
#pragma once

#include <cuda_runtime.h>

namespace fh {

struct df64 {
  float hi, lo;
};

// complex df64, 16 bytes like a double2: (re.hi, re.lo, im.hi, im.lo)
struct __align__(16) dfc {
  df64 re, im;
};

__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df64{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
  const float s = a + b;
  return df64{s, b - (s - a)};
}

__device__ __forceinline__ df64 dd_add(df64 a, df64 b) {
  df64 s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df64 dd_neg(df64 a) { return df64{-a.hi, -a.lo}; }

__device__ __forceinline__ df64 dd_sub(df64 a, df64 b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ df64 dd_mul(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}

// a * b + c with a single renormalisation
__device__ __forceinline__ df64 dd_fma(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
  df64 s = two_sum(p, c.hi);
  s.lo += e + c.lo;
  return fast_two_sum(s.hi, s.lo);
}

// conversions (the FP64 side does them: one rounding to float each way)
__host__ __device__ __forceinline__ df64 to_df64(double x) {
  const float hi = (float)x;
  return df64{hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ double to_double(df64 a) { return (double)a.hi + (double)a.lo; }

// ---- complex df64 -----------------------------------------------------------
__device__ __forceinline__ dfc cadd(dfc a, dfc b) { return dfc{dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ dfc csub(dfc a, dfc b) { return dfc{dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
// a * w
__device__ __forceinline__ dfc cmul(dfc a, dfc w) {
  return dfc{dd_fma(a.re, w.re, dd_neg(dd_mul(a.im, w.im))), dd_fma(a.re, w.im, dd_mul(a.im, w.re))};
}
// a * conj(w)
__device__ __forceinline__ dfc cmulc(dfc a, dfc w) {
  return dfc{dd_fma(a.re, w.re, dd_mul(a.im, w.im)), dd_fma(a.im, w.re, dd_neg(dd_mul(a.re, w.im)))};
}
__device__ __forceinline__ dfc cscale(dfc a, df64 s) { return dfc{dd_mul(a.re, s), dd_mul(a.im, s)}; }
__device__ __forceinline__ dfc cscale(dfc a, double s) { return cscale(a, to_df64(s)); }

template <bool INV>
__device__ __forceinline__ dfc mul_mi(dfc a) {
  return INV ? dfc{dd_neg(a.im), a.re} : dfc{a.im, dd_neg(a.re)};
}

}  // namespace fh
