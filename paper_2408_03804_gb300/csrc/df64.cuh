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
static_assert(sizeof(dfc) == sizeof(double2), "a double-float entry takes the place of an FP64 one");

__host__ __device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df64{s, (a - (s - bb)) + (b - bb)};
}

__host__ __device__ __forceinline__ df64 fast_two_sum(float a, float b) {
  const float s = a + b;
  return df64{s, b - (s - a)};
}

__host__ __device__ __forceinline__ df64 dd_add(df64 a, df64 b) {
  df64 s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return fast_two_sum(s.hi, s.lo);
}

__host__ __device__ __forceinline__ df64 dd_neg(df64 a) { return df64{-a.hi, -a.lo}; }

__host__ __device__ __forceinline__ df64 dd_sub(df64 a, df64 b) { return dd_add(a, dd_neg(b)); }

__host__ __device__ __forceinline__ df64 dd_mul(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}

// a * b + c with a single renormalisation
__host__ __device__ __forceinline__ df64 dd_fma(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
  df64 s = two_sum(p, c.hi);
  s.lo += e + c.lo;
  return fast_two_sum(s.hi, s.lo);
}

// conversion through FP64 arithmetic (one rounding to float each way): for
// constants and per-thread scalars
__host__ __device__ __forceinline__ df64 to_df64(double x) {
  const float hi = (float)x;
  return df64{hi, (float)(x - (double)hi)};
}

// Conversions of field values on the integer pipe (FP64 issue is the
// scarce resource): split_double cuts the 52-bit significand of x after 23
// bits (hi, exact) and turns the remaining 29 bits into lo, truncated to 24
// significant bits, so that |x - hi - lo| < 2^-47 |x|. Values below the
// smallest normal float (2^-126) become 0, and a lo below it is dropped (an
// absolute error under 2^-125); infinities and NaN map to hi.
__device__ __forceinline__ df64 split_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);  // biased by 1023
  const unsigned long long m = b & 0xfffffffffffffull;
  if (e == 0x7ff) return df64{__uint_as_float(sign | 0x7f800000u | (unsigned)(m >> 29)), 0.f};
  const int ef = e - 1023 + 127;  // float exponent field of hi
  if (ef <= 0) return df64{__uint_as_float(sign), 0.f};
  if (ef >= 255) return df64{__uint_as_float(sign | 0x7f800000u), 0.f};
  const float hi = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)(m >> 29));
  const unsigned rem = (unsigned)(m & 0x1fffffffu);  // weight 2^(e - 1023 - 52) each
  if (rem == 0) return df64{hi, 0.f};
  const int top = 31 - __clz(rem);           // highest set bit of the 29-bit remainder
  const int el = ef - 52 + top;               // float exponent field of lo
  if (el <= 0) return df64{hi, 0.f};
  const unsigned frac = top >= 23 ? (rem >> (top - 23)) : (rem << (23 - top));
  return df64{hi, __uint_as_float(sign | ((unsigned)el << 23) | (frac & 0x7fffffu))};
}

// (double)f for a normal float or zero by bit operations (denormals give 0)
__device__ __forceinline__ double float_bits_to_double(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned ef = (u >> 23) & 0xffu;
  if (ef == 0) return __longlong_as_double((long long)sign);
  if (ef == 0xffu)
    return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | ((unsigned long long)(u & 0x7fffffu) << 29)));
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(ef + 1023 - 127) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// hi + lo with one FP64 addition
__device__ __forceinline__ double join_df64(df64 a) { return float_bits_to_double(a.hi) + float_bits_to_double(a.lo); }

// ---- complex df64 -----------------------------------------------------------
__host__ __device__ __forceinline__ dfc cadd(dfc a, dfc b) { return dfc{dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__host__ __device__ __forceinline__ dfc csub(dfc a, dfc b) { return dfc{dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
// a * w
__host__ __device__ __forceinline__ dfc cmul(dfc a, dfc w) {
  return dfc{dd_fma(a.re, w.re, dd_neg(dd_mul(a.im, w.im))), dd_fma(a.re, w.im, dd_mul(a.im, w.re))};
}
// a * conj(w)
__host__ __device__ __forceinline__ dfc cmulc(dfc a, dfc w) {
  return dfc{dd_fma(a.re, w.re, dd_mul(a.im, w.im)), dd_fma(a.im, w.re, dd_neg(dd_mul(a.re, w.im)))};
}
__host__ __device__ __forceinline__ dfc cscale(dfc a, df64 s) { return dfc{dd_mul(a.re, s), dd_mul(a.im, s)}; }
__host__ __device__ __forceinline__ dfc cscale(dfc a, double s) { return cscale(a, to_df64(s)); }

// s a + b, zero, the parts of a twiddle (cos, -sin), a Rader permutation entry (two indices)
__host__ __device__ __forceinline__ dfc caxpy(df64 s, dfc a, dfc b) { return dfc{dd_fma(s, a.re, b.re), dd_fma(s, a.im, b.im)}; }
__host__ __device__ __forceinline__ void czero(dfc& a) { a = dfc{df64{0.f, 0.f}, df64{0.f, 0.f}}; }
__host__ __device__ __forceinline__ df64 tw_cos(dfc w) { return w.re; }
__host__ __device__ __forceinline__ df64 tw_sin(dfc w) { return dd_neg(w.im); }
__host__ __device__ __forceinline__ int perm_first(dfc w) { return (int)w.re.hi; }
__host__ __device__ __forceinline__ int perm_second(dfc w) { return (int)w.im.hi; }

template <bool INV>
__host__ __device__ __forceinline__ dfc mul_mi(dfc a) {
  return INV ? dfc{dd_neg(a.im), a.re} : dfc{a.im, dd_neg(a.re)};
}

}  // namespace fh
