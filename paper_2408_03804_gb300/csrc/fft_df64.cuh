// R-point butterflies in double-float arithmetic (df64.cuh) for the Stockham
// stages of fft_core.cuh, which pick them by the element type: the same
// radix-2/3/4/8/16 factorisations as the FP64 butterflies, written with the
// complex df64 operations.
#pragma once

#include "df64.cuh"
#include "fft_core.cuh"

namespace fh {

__host__ __device__ __forceinline__ df64 dd_half(df64 a) { return df64{0.5f * a.hi, 0.5f * a.lo}; }  // exact

template <bool INV>
__host__ __device__ __forceinline__ void dft2(dfc* v) {
  const dfc a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

// X0 = a + t1, X1,2 = a - t1/2 +- sin(pi/3) (-+ i t2), t1 = b + c, t2 = b - c
template <bool INV>
__host__ __device__ __forceinline__ void dft3(dfc* v) {
  const dfc a = v[0];
  const dfc t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
  const dfc m = csub(a, dfc{dd_half(t1.re), dd_half(t1.im)});
  const dfc r = cscale(mul_mi<INV>(t2), to_df64(kS3));
  v[0] = cadd(a, t1);
  v[1] = cadd(m, r);
  v[2] = csub(m, r);
}

template <bool INV>
__host__ __device__ __forceinline__ void dft4(dfc& v0, dfc& v1, dfc& v2, dfc& v3) {
  const dfc t0 = cadd(v0, v2), t1 = csub(v0, v2);
  const dfc t2 = cadd(v1, v3), t3 = mul_mi<INV>(csub(v1, v3));
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = cadd(t1, t3);
  v3 = csub(t1, t3);
}

template <bool INV>
__host__ __device__ __forceinline__ void dft4(dfc* v) {
  dft4<INV>(v[0], v[1], v[2], v[3]);
}

// o times w8^m for m = 1, 3 (w8 = exp(-+ 2 pi i / 8)): (s + i t) cos(pi/4)
template <bool INV, int M>
__host__ __device__ __forceinline__ dfc rot8(dfc o) {
  df64 s, t;
  if constexpr (M == 1) {
    s = INV ? dd_sub(o.re, o.im) : dd_add(o.re, o.im);
    t = INV ? dd_add(o.re, o.im) : dd_sub(o.im, o.re);
  } else {
    s = INV ? dd_neg(dd_add(o.re, o.im)) : dd_sub(o.im, o.re);
    t = INV ? dd_sub(o.re, o.im) : dd_neg(dd_add(o.re, o.im));
  }
  const df64 c = to_df64(kC8);
  return dfc{dd_mul(s, c), dd_mul(t, c)};
}

template <bool INV>
__host__ __device__ __forceinline__ void dft8(dfc* v) {
  dfc e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  dfc o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  const dfc r1 = rot8<INV, 1>(o1);
  v[1] = cadd(e1, r1);
  v[5] = csub(e1, r1);
  const dfc r2 = mul_mi<INV>(o2);
  v[2] = cadd(e2, r2);
  v[6] = csub(e2, r2);
  const dfc r3 = rot8<INV, 3>(o3);
  v[3] = cadd(e3, r3);
  v[7] = csub(e3, r3);
}

// multiply by w16^m (forward exp(-2 pi i m/16), inverse its conjugate), m in 1..9
template <bool INV, int M>
__host__ __device__ __forceinline__ dfc rot16(dfc a) {
  if constexpr (M == 4) {
    return mul_mi<INV>(a);
  } else if constexpr (M == 2) {
    return rot8<INV, 1>(a);
  } else if constexpr (M == 6) {
    return rot8<INV, 3>(a);
  } else {
    constexpr double sg = INV ? 1.0 : -1.0;
    constexpr double wr = (M == 1) ? kC16 : (M == 3) ? kS16 : -kC16;
    constexpr double wi = sg * ((M == 1) ? kS16 : (M == 3) ? kC16 : -kS16);
    return cmul(a, dfc{to_df64(wr), to_df64(wi)});
  }
}

template <bool INV>
__host__ __device__ __forceinline__ void dft16(dfc* v) {
  // 16 = 4 x 4: DFT-4 over stride-4 inputs, twiddles w16^(j k1), DFT-4 across
  dfc a[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    a[j][0] = v[j];
    a[j][1] = v[j + 4];
    a[j][2] = v[j + 8];
    a[j][3] = v[j + 12];
    dft4<INV>(a[j][0], a[j][1], a[j][2], a[j][3]);
  }
  a[1][1] = rot16<INV, 1>(a[1][1]);
  a[1][2] = rot16<INV, 2>(a[1][2]);
  a[1][3] = rot16<INV, 3>(a[1][3]);
  a[2][1] = rot16<INV, 2>(a[2][1]);
  a[2][2] = rot16<INV, 4>(a[2][2]);
  a[2][3] = rot16<INV, 6>(a[2][3]);
  a[3][1] = rot16<INV, 3>(a[3][1]);
  a[3][2] = rot16<INV, 6>(a[3][2]);
  a[3][3] = rot16<INV, 9>(a[3][3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    dfc b0 = a[0][k1], b1 = a[1][k1], b2 = a[2][k1], b3 = a[3][k1];
    dft4<INV>(b0, b1, b2, b3);
    v[k1] = b0;
    v[k1 + 4] = b1;
    v[k1 + 8] = b2;
    v[k1 + 12] = b3;
  }
}

template <int R, bool INV>
__host__ __device__ __forceinline__ void dft_r(dfc* v) {
  if constexpr (R == 2) dft2<INV>(v);
  else if constexpr (R == 3) dft3<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
}

}  // namespace fh
