// Batched complex FFTs of power-of-two length on pencils held in shared
// memory: the building block of the 3D transforms of Eq. 1.
//
// Each length-L transform is a Stockham auto-sort sequence of radix-R stages
// (R in {2, 3, 4, 8, 16}) that ping-pongs between two shared-memory buffers. A
// stage with radix R and current sub-transform size Ns treats L/R butterflies;
// butterfly j reads the R inputs j + r L/R, multiplies input r by the twiddle
// w_L^(r (j mod Ns) L/(Ns R)), applies an R-point DFT in registers and writes
// output r to (j div Ns) Ns R + (j mod Ns) + r Ns. The first stage (Ns = 1)
// needs no twiddles. Twiddles w_L^m = exp(-2 pi i m / L) come from a table that
// each CTA first copies from global to shared memory (reading them through the
// texture path throttled the FP64 kernels); the inverse uses their conjugates.
// In FP64 the twiddled stages read them in a tangent form and fold them into
// their butterflies (6 FMAs per radix-2 butterfly, see below).
//
// The plans minimise FP64 instructions (FP64 issue is the bound of this path):
// 32 = 8x4, 64 = 8x8, 128 = 16x8, 256 = 16x16 (16x4x4 in FP64), smaller powers
// of two in one stage; lengths 3 * 2^a end with a radix-3 stage (48 = 16x3,
// 96 = 8x4x3).
// Per complex point a length-128 transform takes 18 FP64 operations (144 for
// the radix-16 butterfly, 72 for a twiddled radix-8 one).
#pragma once

#include <cstring>

#include "fh_common.cuh"

namespace fh {

constexpr double kC8 = 0.70710678118654752440;   // cos(pi/4)
constexpr double kS3 = 0.86602540378443864676;   // sin(pi/3)
constexpr double kC16 = 0.92387953251128675613;  // cos(pi/8)
constexpr double kS16 = 0.38268343236508977173;  // sin(pi/8)
constexpr double kT16 = 0.41421356237309504880;  // tan(pi/8) = sqrt(2) - 1

// multiply by -i (forward, INV = false) or +i (inverse)
template <bool INV>
__host__ __device__ __forceinline__ double2 mul_mi(double2 a) {
  return INV ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// scalar helpers shared with the double-float element type (df64.cuh has the
// dfc overloads): s a + b, zero, the cosine and minus-sine parts of a twiddle
// (cos, -sin), and the index pair stored in a Rader permutation entry
__host__ __device__ __forceinline__ double2 caxpy(double s, double2 a, double2 b) {
  return make_double2(fma(s, a.x, b.x), fma(s, a.y, b.y));
}
__host__ __device__ __forceinline__ void czero(double2& a) { a = make_double2(0.0, 0.0); }
__device__ __forceinline__ double tw_cos(double2 w) { return w.x; }
__device__ __forceinline__ double tw_sin(double2 w) { return -w.y; }
__device__ __forceinline__ int perm_first(double2 w) { return (int)w.x; }
__device__ __forceinline__ int perm_second(double2 w) { return (int)w.y; }

template <bool INV>
__host__ __device__ __forceinline__ void dft2(double2* v) {
  const double2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

// X0 = a + b + c, X1,2 = a - (b + c)/2 -+ i sin(pi/3) (b - c) (forward; signs
// of the sine term swap for the inverse)
template <bool INV>
__host__ __device__ __forceinline__ void dft3(double2* v) {
  const double2 a = v[0];
  const double2 t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
  const double2 m = make_double2(fma(-0.5, t1.x, a.x), fma(-0.5, t1.y, a.y));
  v[0] = cadd(a, t1);
  const double sx = INV ? -kS3 : kS3;
  v[1] = make_double2(fma(sx, t2.y, m.x), fma(-sx, t2.x, m.y));
  v[2] = make_double2(fma(-sx, t2.y, m.x), fma(sx, t2.x, m.y));
}

template <bool INV>
__host__ __device__ __forceinline__ void dft4(double2& v0, double2& v1, double2& v2, double2& v3) {
  const double2 t0 = cadd(v0, v2), t1 = csub(v0, v2);
  const double2 t2 = cadd(v1, v3), t3 = mul_mi<INV>(csub(v1, v3));
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = cadd(t1, t3);
  v3 = csub(t1, t3);
}

template <bool INV>
__host__ __device__ __forceinline__ void dft4(double2* v) {
  dft4<INV>(v[0], v[1], v[2], v[3]);
}

// e + w8^1 o and e - w8^1 o, fused (w8 = exp(-+ 2 pi i / 8))
template <bool INV>
__host__ __device__ __forceinline__ void bfly_w8_1(double2& e, double2& o) {
  // forward: o (1 - i)/sqrt2 = ((x + y) + i (y - x))/sqrt2 ; inverse: ((x - y) + i (x + y))/sqrt2
  const double s = INV ? o.x - o.y : o.x + o.y;
  const double t = INV ? o.x + o.y : o.y - o.x;
  const double2 a = e;
  e = make_double2(fma(kC8, s, a.x), fma(kC8, t, a.y));
  o = make_double2(fma(-kC8, s, a.x), fma(-kC8, t, a.y));
}
// e + w8^3 o and e - w8^3 o
template <bool INV>
__host__ __device__ __forceinline__ void bfly_w8_3(double2& e, double2& o) {
  // forward: o (-1 - i)/sqrt2 = ((y - x) - i (x + y))/sqrt2 ; inverse: (-(x + y) + i (x - y))/sqrt2
  const double s = INV ? -(o.x + o.y) : o.y - o.x;
  const double t = INV ? o.x - o.y : -(o.x + o.y);
  const double2 a = e;
  e = make_double2(fma(kC8, s, a.x), fma(kC8, t, a.y));
  o = make_double2(fma(-kC8, s, a.x), fma(-kC8, t, a.y));
}

template <bool INV>
__host__ __device__ __forceinline__ void dft8(double2* v) {
  double2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  double2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  bfly_w8_1<INV>(e1, o1);
  v[1] = e1;
  v[5] = o1;
  const double2 r2 = mul_mi<INV>(o2);
  v[2] = cadd(e2, r2);
  v[6] = csub(e2, r2);
  bfly_w8_3<INV>(e3, o3);
  v[3] = e3;
  v[7] = o3;
}

// a (1 + i sg), a (-1 + i sg) and a (1 + i sg t16), with sg = -1 forward and
// +1 inverse (the sign of the imaginary part of w16^1) and t16 = tan(pi/8)
template <bool INV>
__host__ __device__ __forceinline__ double2 mul_1pi(double2 a) {
  return INV ? make_double2(a.x - a.y, a.y + a.x) : make_double2(a.x + a.y, a.y - a.x);
}
template <bool INV>
__host__ __device__ __forceinline__ double2 mul_m1pi(double2 a) {
  return INV ? make_double2(-a.x - a.y, a.x - a.y) : make_double2(a.y - a.x, -a.y - a.x);
}
template <bool INV>
__host__ __device__ __forceinline__ double2 mul_1pit(double2 a) {
  return INV ? make_double2(fma(-kT16, a.y, a.x), fma(kT16, a.x, a.y))
             : make_double2(fma(kT16, a.y, a.x), fma(-kT16, a.x, a.y));
}

// 16 = 4 x 4: DFT-4 over the stride-4 inputs (column k1 of a[j] from inputs
// j + 4 n1), the twiddles w16^(j k1), DFT-4 across j. The twiddles of a
// column are written as a common real factor times values of the form
// 1 + i sg, -1 + i sg or (1 +- i sg t16) times a power of i: w16^1, w16^3 and
// w16^9 all equal c16 times such a value, w16^2 and w16^6 c8 times one. The
// factor then enters the DFT-4 as the multiplier of an FMA, so a twiddled
// column costs 22 (20 for k1 = 2) FP64 operations instead of 28 (24); the
// whole transform 144 instead of 160.
template <bool INV>
__host__ __device__ __forceinline__ void dft16(double2* v) {
  double2 a[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    a[j][0] = v[j];
    a[j][1] = v[j + 4];
    a[j][2] = v[j + 8];
    a[j][3] = v[j + 12];
    dft4<INV>(a[j][0], a[j][1], a[j][2], a[j][3]);
  }
  {  // k1 = 0: no twiddles
    double2 b0 = a[0][0], b1 = a[1][0], b2 = a[2][0], b3 = a[3][0];
    dft4<INV>(b0, b1, b2, b3);
    v[0] = b0;
    v[4] = b1;
    v[8] = b2;
    v[12] = b3;
  }
  {  // k1 = 1: w^1 = c16 (1 + i sg t16), w^2 = c8 (1 + i sg), w^3 = c16 i sg (1 - i sg t16)
    const double2 u1 = mul_1pit<INV>(a[1][1]);
    const double2 u3 = mul_mi<INV>(mul_1pit<!INV>(a[3][1]));
    const double2 s2 = mul_1pi<INV>(a[2][1]);
    const double2 t0 = caxpy(kC8, s2, a[0][1]), t1 = caxpy(-kC8, s2, a[0][1]);
    const double2 p = cadd(u1, u3), d = mul_mi<INV>(csub(u1, u3));
    v[1] = caxpy(kC16, p, t0);
    v[9] = caxpy(-kC16, p, t0);
    v[5] = caxpy(kC16, d, t1);
    v[13] = caxpy(-kC16, d, t1);
  }
  {  // k1 = 2: w^2 = c8 (1 + i sg), w^4 = i sg, w^6 = c8 (-1 + i sg)
    const double2 b2 = mul_mi<INV>(a[2][2]);
    const double2 t0 = cadd(a[0][2], b2), t1 = csub(a[0][2], b2);
    const double2 s1 = mul_1pi<INV>(a[1][2]), s3 = mul_m1pi<INV>(a[3][2]);
    const double2 p = cadd(s1, s3), d = mul_mi<INV>(csub(s1, s3));
    v[2] = caxpy(kC8, p, t0);
    v[10] = caxpy(-kC8, p, t0);
    v[6] = caxpy(kC8, d, t1);
    v[14] = caxpy(-kC8, d, t1);
  }
  {  // k1 = 3: w^3 = c16 i sg (1 - i sg t16), w^6 = c8 (-1 + i sg), w^9 = -c16 (1 + i sg t16)
    const double2 u1 = mul_mi<INV>(mul_1pit<!INV>(a[1][3]));
    const double2 z3 = mul_1pit<INV>(a[3][3]);  // b3 = -c16 z3
    const double2 s2 = mul_m1pi<INV>(a[2][3]);
    const double2 t0 = caxpy(kC8, s2, a[0][3]), t1 = caxpy(-kC8, s2, a[0][3]);
    const double2 p = csub(u1, z3), d = mul_mi<INV>(cadd(u1, z3));
    v[3] = caxpy(kC16, p, t0);
    v[11] = caxpy(-kC16, p, t0);
    v[7] = caxpy(kC16, d, t1);
    v[15] = caxpy(-kC16, d, t1);
  }
}

template <int R, bool INV>
__host__ __device__ __forceinline__ void dft_r(double2* v) {
  if constexpr (R == 2) dft2<INV>(v);
  else if constexpr (R == 3) dft3<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
}

// ---- plans: radix of each stage for a length L --------------------------------
template <int L>
struct Plan;
template <> struct Plan<1>   { static constexpr int n = 0; static constexpr int r[3] = {1, 1, 1}; };
template <> struct Plan<2>   { static constexpr int n = 1; static constexpr int r[3] = {2, 1, 1}; };
template <> struct Plan<3>   { static constexpr int n = 1; static constexpr int r[3] = {3, 1, 1}; };
template <> struct Plan<4>   { static constexpr int n = 1; static constexpr int r[3] = {4, 1, 1}; };
template <> struct Plan<6>   { static constexpr int n = 2; static constexpr int r[3] = {2, 3, 1}; };
template <> struct Plan<8>   { static constexpr int n = 1; static constexpr int r[3] = {8, 1, 1}; };
template <> struct Plan<12>  { static constexpr int n = 2; static constexpr int r[3] = {4, 3, 1}; };
template <> struct Plan<16>  { static constexpr int n = 1; static constexpr int r[3] = {16, 1, 1}; };
template <> struct Plan<24>  { static constexpr int n = 2; static constexpr int r[3] = {8, 3, 1}; };
template <> struct Plan<32>  { static constexpr int n = 2; static constexpr int r[3] = {8, 4, 1}; };
template <> struct Plan<48>  { static constexpr int n = 2; static constexpr int r[3] = {16, 3, 1}; };
template <> struct Plan<64>  { static constexpr int n = 2; static constexpr int r[3] = {8, 8, 1}; };
template <> struct Plan<96>  { static constexpr int n = 3; static constexpr int r[3] = {8, 4, 3}; };
template <> struct Plan<128> { static constexpr int n = 2; static constexpr int r[3] = {16, 8, 1}; };
template <> struct Plan<192> { static constexpr int n = 3; static constexpr int r[3] = {16, 4, 3}; };
template <> struct Plan<256> { static constexpr int n = 2; static constexpr int r[3] = {16, 16, 1}; };

// the plan of an element type: FP64 transforms of length 256 run 16 x 4 x 4,
// the same FP64 operations as 16 x 16 in the tangent form (9 + 6 + 6 per
// point) without the registers of a twiddled radix-16 butterfly, which spilled
template <int L, class C>
struct PlanFor : Plan<L> {};
template <>
struct PlanFor<256, double2> {
  static constexpr int n = 3;
  static constexpr int r[3] = {16, 4, 4};
};

// Pencil addressing inside a shared buffer: element j of pencil q lives at
// q_stride * q + j_stride * j (in double2 units). Pencils come in groups of
// `group`; only the first `valid` of each group hold data (the others pad a
// ragged last chunk of columns and are skipped). JFAST selects the mapping of
// threads to (pencil, butterfly): butterfly index fastest when pencils are
// contiguous (j_stride == 1), pencil index fastest otherwise, so that
// neighbouring threads touch neighbouring addresses.
struct PencilLayout {
  int np;        // number of pencils (a multiple of group)
  int q_stride;
  int j_stride;
  int group;
  int valid;     // 1 <= valid <= group
};

__device__ __forceinline__ int pencil_of(int qv, const PencilLayout& lay) {
  return lay.valid == lay.group ? qv : (qv / lay.valid) * lay.group + qv % lay.valid;
}

// copy the twiddle table of length L (first n entries) to shared memory;
// the caller synchronises before use. The element type C is double2, or dfc
// for the double-float transforms (same offsets, df64.cuh).
template <int L, class C>
__device__ __forceinline__ void stage_twiddles(C* dst, const C* __restrict__ table, int n) {
  constexpr int off = twiddle_offset(L);
  const C* src = table + off;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// ---- twiddled stages in the tangent form (FP64) ------------------------------
// A root of unity is stored as w = i^Q rho (1 + i tau) with |tau| <= 1: the
// tangent form of the twiddled FFT stages (the table at kTwiddleTotal +
// twiddle_offset(L) holds (rho, tau) of w_L^m; Q follows from m and L). Then
// x + w b and x - w b take 6 FMAs, u = b (1 + i tau) and x +- rho i^Q u, where
// the power of i only swaps the parts of u and flips the signs of rho (integer
// operations); the usual complex product and two additions take 8. This is
// the FMA butterfly of S. Goedecker (SIAM J. Sci. Comput. 18, 1997).

template <class C>
struct IsFp64Complex {
  static constexpr bool value = false;
};
template <>
struct IsFp64Complex<double2> {
  static constexpr bool value = true;
};

// the table of the FFT stages of length L: the tangent form for FP64, the
// (cos, -sin) form for double-float elements
template <int L, class C>
__device__ __forceinline__ void stage_fft_twiddles(C* dst, const C* __restrict__ table, int n) {
  constexpr int off = (IsFp64Complex<C>::value ? kTwiddleTotal : 0) + twiddle_offset(L);
  const C* src = table + off;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// x with its sign bit flipped when f is 1
__host__ __device__ __forceinline__ double flip_sign(double x, unsigned f) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(x) ^ ((unsigned long long)f << 63)));
#else
  unsigned long long b;
  memcpy(&b, &x, sizeof b);
  b ^= (unsigned long long)f << 63;
  memcpy(&x, &b, sizeof b);
  return x;
#endif
}

// w = i^Q rho (1 + i tau) as the multipliers of the butterfly: the real and
// imaginary parts of w b are rx p_x and ry p_y, (p_x, p_y) = u or u swapped
struct TanTw {
  double rx, ry, tau;
  bool swap;
};

// w_L^m (its conjugate for the inverse) from the tangent table t: with qr the
// nearest quarter turn of 2 pi m / L (halves rounded up), w_L^m = (-i)^qr
// rho (1 + i tau); the conjugate is i^qr rho (1 - i tau)
template <int L, bool INV>
__host__ __device__ __forceinline__ TanTw tan_twiddle(const double2* __restrict__ t, int m) {
  const double2 e = t[m];
  const int qr = (8 * m + L) / (2 * L);
  const unsigned Q = (unsigned)(INV ? qr : -qr) & 3u;
  // i^Q u: Q = 0 (u_x, u_y), 1 (-u_y, u_x), 2 (-u_x, -u_y), 3 (u_y, -u_x)
  return TanTw{flip_sign(e.x, ((Q + 1u) >> 1) & 1u), flip_sign(e.x, Q >> 1), INV ? -e.y : e.y, (Q & 1u) != 0};
}

// x + w b into x, x - w b into b (6 FMAs)
__host__ __device__ __forceinline__ void bfly_tan(double2& x, double2& b, const TanTw& w) {
  const double ux = fma(-w.tau, b.y, b.x), uy = fma(w.tau, b.x, b.y);
  const double px = w.swap ? uy : ux, py = w.swap ? ux : uy;
  const double2 a = x;
  x = make_double2(fma(w.rx, px, a.x), fma(w.ry, py, a.y));
  b = make_double2(fma(-w.rx, px, a.x), fma(-w.ry, py, a.y));
}

// w b (2 FMAs and 2 products)
__host__ __device__ __forceinline__ double2 mul_tan(double2 b, const TanTw& w) {
  const double ux = fma(-w.tau, b.y, b.x), uy = fma(w.tau, b.x, b.y);
  return make_double2(w.rx * (w.swap ? uy : ux), w.ry * (w.swap ? ux : uy));
}

// The pair steps of the real-to-complex transform along z (passes.cuh) in the
// tangent form, w = w_NZ^k: unpack (x_k, x_{M-k}) = (e + t, conj(e - t)) with
// t = -i w o, and pack (z_k, z_{M-k}) = (a + u, conj(a - u)) with u = i conj(w) b
// (wc: the conjugate's multipliers). 6 FMAs each against a complex product and
// two complex additions (8).
__host__ __device__ __forceinline__ void unpack_pair_tan(double2 e, double2 o, const TanTw& w, double2& xk,
                                                         double2& xm) {
  const double ux = fma(-w.tau, o.y, o.x), uy = fma(w.tau, o.x, o.y);
  const double px = w.swap ? uy : ux, py = w.swap ? ux : uy;  // w o = (rx px, ry py)
  xk = make_double2(fma(w.ry, py, e.x), fma(-w.rx, px, e.y));
  xm = make_double2(fma(-w.ry, py, e.x), fma(-w.rx, px, -e.y));
}
__host__ __device__ __forceinline__ void pack_pair_tan(double2 a, double2 b, const TanTw& wc, double2& zk,
                                                       double2& zm) {
  const double ux = fma(-wc.tau, b.y, b.x), uy = fma(wc.tau, b.x, b.y);
  const double px = wc.swap ? uy : ux, py = wc.swap ? ux : uy;  // conj(w) b = (rx px, ry py)
  zk = make_double2(fma(-wc.ry, py, a.x), fma(wc.rx, px, a.y));
  zm = make_double2(fma(wc.ry, py, a.x), fma(wc.rx, px, -a.y));
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
__host__ __device__ constexpr int bit_reverse(int r, int bits) {
  return bits == 0 ? 0 : ((r & 1) << (bits - 1)) | bit_reverse(r >> 1, bits - 1);
}

// layer LAYER of dft_pow2_twiddled, from the pair offset S on (every index a
// compile-time constant, so the R values stay in registers)
template <int L, int R, bool INV, int LAYER, int S>
__host__ __device__ __forceinline__ void tw_layer(double2 (&a)[R], const double2* __restrict__ t, int m1) {
  constexpr int half = 1 << (LAYER - 1);
  if constexpr (S < half) {
    const TanTw w = tan_twiddle<L, INV>(t, m1 * (R >> LAYER) + S * (L >> LAYER));
    if constexpr (S < R) bfly_tan(a[S], a[S + half], w);
    if constexpr (2 * half + S < R) bfly_tan(a[2 * half + S], a[3 * half + S], w);
    if constexpr (4 * half + S < R) bfly_tan(a[4 * half + S], a[5 * half + S], w);
    if constexpr (6 * half + S < R) bfly_tan(a[6 * half + S], a[7 * half + S], w);
    if constexpr (8 * half + S < R) bfly_tan(a[8 * half + S], a[9 * half + S], w);
    if constexpr (10 * half + S < R) bfly_tan(a[10 * half + S], a[11 * half + S], w);
    if constexpr (12 * half + S < R) bfly_tan(a[12 * half + S], a[13 * half + S], w);
    if constexpr (14 * half + S < R) bfly_tan(a[14 * half + S], a[15 * half + S], w);
    tw_layer<L, R, INV, LAYER, S + 1>(a, t, m1);
  }
}

template <int L, int R, bool INV, int LAYER>
__host__ __device__ __forceinline__ void tw_layers(double2 (&a)[R], const double2* __restrict__ t, int m1) {
  if constexpr ((1 << LAYER) <= R) {
    tw_layer<L, R, INV, LAYER, 0>(a, t, m1);
    tw_layers<L, R, INV, LAYER + 1>(a, t, m1);
  }
}

template <int R, int P, int I>
__host__ __device__ __forceinline__ void load_bit_reversed(double2 (&a)[R], const double2* v) {
  if constexpr (I < R) {
    constexpr int src = bit_reverse(I, P);
    a[I] = v[src];
    load_bit_reversed<R, P, I + 1>(a, v);
  }
}

// Y_s = sum_r v_r omega^r w_R^(r s), omega = w_L^m1, R = 2^P <= 16, in place:
// the DFT of a twiddled radix-R stage as P layers of radix-2 decimation in
// time on the bit-reversed inputs. Layer l combines pairs half = 2^(l-1)
// apart with the twiddle omega^(R / 2^l) w_(2^l)^s = w_L^(m1 R / 2^l + s L / 2^l)
// for the pair's offset s in its group; 3 P R FP64 operations (72 for R = 8
// against 80 for seven complex products and the radix-8 butterfly).
template <int L, int R, bool INV>
__host__ __device__ __forceinline__ void dft_pow2_twiddled(double2* v, const double2* __restrict__ t, int m1) {
  constexpr int P = ilog2(R);
  static_assert((1 << P) == R && R <= 16 && L % R == 0, "radix 2^P <= 16 dividing L");
  double2 a[R];
  load_bit_reversed<R, P, 0>(a, v);
  tw_layers<L, R, INV, 1>(a, t, m1);
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = a[r];
}

// the butterfly of a stage with sub-transform size NS > 1 of a compile-time
// plan: v_r times w_L^(r m1), then the R-point DFT. FP64 elements use the
// tangent table (radix 2^P as above; radix 3 by two products in the tangent
// form); double-float elements the (cos, -sin) table.
template <int L, int R, bool INV, class C>
__device__ __forceinline__ void twiddled_butterfly(C* v, const C* __restrict__ tw, int m1) {
  if constexpr (IsFp64Complex<C>::value) {
    if constexpr (R == 3) {
      v[1] = mul_tan(v[1], tan_twiddle<L, INV>(tw, m1));
      v[2] = mul_tan(v[2], tan_twiddle<L, INV>(tw, 2 * m1));
      dft3<INV>(v);
    } else {
      dft_pow2_twiddled<L, R, INV>(v, tw, m1);
    }
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const C w = tw[r * m1];
      v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
    }
    dft_r<R, INV>(v);
  }
}

template <int L, int R, int NS, bool INV, bool JFAST, class C>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ src, C* __restrict__ dst,
                                               const PencilLayout& lay, const C* __restrict__ tw) {
  constexpr int NB = L / R;  // butterflies per pencil
  const int nq = (lay.np / lay.group) * lay.valid;
  const int total = nq * NB;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int q = pencil_of(JFAST ? t / NB : t % nq, lay);
    const int j = JFAST ? t % NB : t / nq;
    const C* s = src + q * lay.q_stride;
    C* d = dst + q * lay.q_stride;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[(j + r * NB) * lay.j_stride];
    if constexpr (NS > 1) {
      constexpr int step = L / (NS * R);
      twiddled_butterfly<L, R, INV>(v, tw, (j % NS) * step);
    } else {
      dft_r<R, INV>(v);
    }
    const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
    for (int r = 0; r < R; ++r) d[(base + r * NS) * lay.j_stride] = v[r];
  }
}

template <int L, bool INV, bool JFAST, int S, int NS, class C>
__device__ __forceinline__ C* run_stages(C* a, C* b, const PencilLayout& lay, const C* tw) {
  if constexpr (S == PlanFor<L, C>::n) {
    return a;
  } else {
    constexpr int R = PlanFor<L, C>::r[S];
    __syncthreads();
    stockham_stage<L, R, NS, INV, JFAST>(a, b, lay, tw);
    return run_stages<L, INV, JFAST, S + 1, NS * R>(b, a, lay, tw);
  }
}

// Transform all pencils of `a` (length L). Uses `b` as the ping-pong partner;
// `tw` is the length-L table of the FFT stages (stage_fft_twiddles: the
// tangent form for FP64) in shared memory. Returns the buffer
// holding the result. Synchronises the CTA before each stage and after the
// last one.
template <int L, bool INV, bool JFAST, class C>
__device__ __forceinline__ C* fft_pencils(C* a, C* b, const PencilLayout& lay, const C* tw) {
  static_assert(L == 1 || Plan<L>::n > 0, "plan");
  C* out = run_stages<L, INV, JFAST, 0, 1>(a, b, lay, tw);
  __syncthreads();
  return out;
}

// ---- lengths without a compile-time plan ------------------------------------
// An axis whose length has no template plan (any length up to kMaxNAny, e.g.
// the odd grids 169, 199, 299 or 384, 512) runs a plan chosen at run time:
// radix-16/8/4/2 and radix-3 stages with the butterflies above, and every other
// prime factor p as one stage of a direct p-point DFT. Its twiddles
// w_L^m = exp(-2 pi i m / L), m < L, sit at `tw_off` of the context's table;
// the p-point roots of a direct stage are entries of the same table
// (w_p^e = w_L^(e L / p)).

template <int R, bool INV, bool JFAST, class C>
__device__ __forceinline__ void stockham_stage_rt(const C* __restrict__ src, C* __restrict__ dst,
                                                  const PencilLayout& lay, const C* __restrict__ tw, int L,
                                                  int NS) {
  const int NB = L / R;
  const int nq = (lay.np / lay.group) * lay.valid;
  const int total = nq * NB;
  const int step = L / (NS * R);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int q = pencil_of(JFAST ? t / NB : t % nq, lay);
    const int j = JFAST ? t % NB : t / nq;
    const C* s = src + q * lay.q_stride;
    C* d = dst + q * lay.q_stride;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[(j + r * NB) * lay.j_stride];
    const int k = j % NS;
    if (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const C w = tw[r * k * step];
        v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
      }
    }
    dft_r<R, INV>(v);
    const int base = (j / NS) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[(base + r * NS) * lay.j_stride] = v[r];
  }
}

// One stage of odd radix R (any R >= 5) as a direct DFT: with the inputs
// twiddled, S_m = v_m + v_{R-m} and D_m = v_m - v_{R-m} (m = 1 .. (R-1)/2).
// With P_r = sum_m S_m cos(2 pi r m / R) and Q_r = sum_m D_m sin(2 pi r m / R),
// X_r = v_0 + P_r -+ i Q_r and X_{R-r} = v_0 + P_r +- i Q_r (upper signs
// forward), so one pass over m gives a pair of outputs. Two phases, each
// spread over all threads: one (butterfly, m) pair per thread forms S_m and
// D_m and writes them back over the source entries (each butterfly owns its
// R entries; the source buffer is dead after the stage), then one
// (butterfly, r) per thread, r = 0 .. (R-1)/2, writes X_0 (r = 0) or the
// pair X_r, X_{R-r}.
template <bool INV, bool JFAST, class C>
__device__ __forceinline__ void stockham_stage_odd(C* __restrict__ src, C* __restrict__ dst, const PencilLayout& lay,
                                                   const C* __restrict__ tw, int L, int R, int NS) {
  const int NB = L / R;
  const int nq = (lay.np / lay.group) * lay.valid;
  const int step = L / (NS * R);
  const int H = (R - 1) / 2;
  // phase 1: twiddled pairs -> (S_m, D_m)
  for (int t = threadIdx.x; t < nq * NB * H; t += blockDim.x) {
    const int m = 1 + t % H, qj = t / H;
    const int q = pencil_of(JFAST ? qj / NB : qj % nq, lay);
    const int j = JFAST ? qj % NB : qj / nq;
    C* s = src + q * lay.q_stride;
    C a = s[(j + m * NB) * lay.j_stride];
    C b = s[(j + (R - m) * NB) * lay.j_stride];
    if (NS > 1) {
      const int k = j % NS;
      const C wa = tw[m * k * step], wb = tw[(R - m) * k * step];
      a = INV ? cmulc(a, wa) : cmul(a, wa);
      b = INV ? cmulc(b, wb) : cmul(b, wb);
    }
    s[(j + m * NB) * lay.j_stride] = cadd(a, b);
    s[(j + (R - m) * NB) * lay.j_stride] = csub(a, b);
  }
  __syncthreads();
  // phase 2: X_0, or the pair X_r, X_{R-r}
  const int H1 = H + 1;
  for (int t = threadIdx.x; t < nq * NB * H1; t += blockDim.x) {
    const int r = t % H1, qj = t / H1;
    const int q = pencil_of(JFAST ? qj / NB : qj % nq, lay);
    const int j = JFAST ? qj % NB : qj / nq;
    const C* s = src + q * lay.q_stride;
    const C v0 = s[j * lay.j_stride];
    const int base = (j / NS) * NS * R + j % NS;
    C* d = dst + q * lay.q_stride;
    if (r == 0) {
      C acc = v0;
      for (int m = 1; m <= H; ++m) acc = cadd(acc, s[(j + m * NB) * lay.j_stride]);
      d[base * lay.j_stride] = acc;
      continue;
    }
    C P, Q;
    czero(P);
    czero(Q);
    int e = 0;
    for (int m = 1; m <= H; ++m) {
      e += r;
      if (e >= R) e -= R;
      const C w = tw[e * NB];  // (cos, -sin) of 2 pi e / R
      P = caxpy(tw_cos(w), s[(j + m * NB) * lay.j_stride], P);
      Q = caxpy(tw_sin(w), s[(j + (R - m) * NB) * lay.j_stride], Q);
    }
    // -i Q forward, +i Q inverse
    const C e0 = cadd(v0, P), iq = mul_mi<INV>(Q);
    d[(base + r * NS) * lay.j_stride] = cadd(e0, iq);
    d[(base + (R - r) * NS) * lay.j_stride] = csub(e0, iq);
  }
}

// The stages `r[0..n)` of a run-time plan of length L over the pencils of a
// (partner b); returns the buffer holding the result.
template <bool INV, bool JFAST, class C>
__device__ __forceinline__ C* run_stages_rt(C* a, C* b, const PencilLayout& lay, const C* tw, int L, int n,
                                            const int* r) {
  int NS = 1;
  for (int st = 0; st < n; ++st) {
    const int R = r[st];
    __syncthreads();
    switch (R) {
      case 2: stockham_stage_rt<2, INV, JFAST>(a, b, lay, tw, L, NS); break;
      case 3: stockham_stage_rt<3, INV, JFAST>(a, b, lay, tw, L, NS); break;
      case 4: stockham_stage_rt<4, INV, JFAST>(a, b, lay, tw, L, NS); break;
      case 8: stockham_stage_rt<8, INV, JFAST>(a, b, lay, tw, L, NS); break;
      case 16: stockham_stage_rt<16, INV, JFAST>(a, b, lay, tw, L, NS); break;
      default: stockham_stage_odd<INV, JFAST>(a, b, lay, tw, L, R, NS); break;
    }
    C* t = a;
    a = b;
    b = t;
    NS *= R;
  }
  __syncthreads();
  return a;
}

// Prime length L by Rader's algorithm. With g a primitive root of L and
// M = L - 1: X_0 = sum_m v_m and, for q < M, X_{g^-q} = v_0 + sum_r v_{g^r}
// w^{g^(r-q)}, a cyclic convolution of a_r = v_{g^r} with b_s = w^{g^-s}
// (w = exp(-+ 2 pi i / L)). It is computed as IFFT_M(FFT_M(a) Bhat) with
// Bhat = FFT_M(b) / M precomputed for both directions. Tables at `tab`:
// length-M twiddles, Bhat forward, Bhat inverse, then (g^r, g^-r) as
// doubles. Each pencil keeps v_0 in slot 0 of both buffers and runs the
// inner transforms on slots 1..M; slot L (the pencil's padding) holds X_0.
template <bool INV, bool JFAST, class C>
__device__ __forceinline__ C* rader_pencils(C* a, C* b, const PencilLayout& lay, const C* tab, const FftPlan& p) {
  const int L = p.L, M = L - 1;
  const C* itw = tab;
  const C* bhat = tab + (INV ? 2 : 1) * M;
  const C* perm = tab + 3 * M;
  const int nq = (lay.np / lay.group) * lay.valid;
  const int js = lay.j_stride;
  __syncthreads();
  // gather a_r = v_{g^r} into slots 1..M of b; copy v_0
  for (int t = threadIdx.x; t < nq * L; t += blockDim.x) {
    const int q = pencil_of(JFAST ? t / L : t % nq, lay);
    const int e = JFAST ? t % L : t / nq;
    const C* s = a + q * lay.q_stride;
    C* d = b + q * lay.q_stride;
    d[e * js] = e == 0 ? s[0] : s[perm_first(perm[e - 1]) * js];
  }
  C* Cv = run_stages_rt<false, JFAST>(b + js, a + js, lay, itw, M, p.in_n, p.in_r) - js;
  // Ahat * Bhat; X_0 = v_0 + Ahat_0 into slot L
  for (int t = threadIdx.x; t < nq * M; t += blockDim.x) {
    const int q = pencil_of(JFAST ? t / M : t % nq, lay);
    const int k = JFAST ? t % M : t / nq;
    C* c = Cv + q * lay.q_stride;
    const C ah = c[(1 + k) * js];
    if (k == 0) c[L * js] = cadd(c[0], ah);
    c[(1 + k) * js] = cmul(ah, bhat[k]);
  }
  C* D = (Cv == a) ? b : a;
  C* E = run_stages_rt<true, JFAST>(Cv + js, D + js, lay, itw, M, p.in_n, p.in_r) - js;
  C* O = (E == a) ? b : a;
  // X_{g^-k} = v_0 + c_k, X_0 from slot L of Cv
  for (int t = threadIdx.x; t < nq * L; t += blockDim.x) {
    const int q = pencil_of(JFAST ? t / L : t % nq, lay);
    const int e = JFAST ? t % L : t / nq;
    const C* ee = E + q * lay.q_stride;
    C* o = O + q * lay.q_stride;
    if (e == 0) o[0] = Cv[q * lay.q_stride + L * js];
    else o[perm_second(perm[e - 1]) * js] = cadd(ee[0], ee[e * js]);
  }
  __syncthreads();
  return O;
}

// Transform all pencils of `a` with a run-time plan (see fft_pencils).
template <bool INV, bool JFAST, class C>
__device__ __noinline__ C* fft_pencils_rt(C* a, C* b, const PencilLayout lay, const C* tw, const FftPlan p) {
  if (p.rader) return rader_pencils<INV, JFAST>(a, b, lay, tw, p);
  return run_stages_rt<INV, JFAST>(a, b, lay, tw, p.L, p.n, p.r);
}

// twiddles of the y (AX = 1) or x (AX = 0) axis into shared memory: the
// compile-time table of L, or the run-time plan's table
template <int L, int AX, class C>
__device__ __forceinline__ void stage_axis_twiddles(C* dst, const C* __restrict__ tw, const Grid& g) {
  if constexpr (L > 0) {
    stage_fft_twiddles<L>(dst, tw, L);
  } else {
    const FftPlan& p = AX ? g.py : g.px;
    for (int i = threadIdx.x; i < p.tw_len; i += blockDim.x) dst[i] = tw[p.tw_off + i];
  }
}

// compile-time plan when L > 0, the run-time plan p otherwise
template <int L, bool INV, bool JFAST, class C>
__device__ __forceinline__ C* fft_pencils_any(C* a, C* b, const PencilLayout& lay, const C* tw, const FftPlan& p) {
  if constexpr (L > 0) return fft_pencils<L, INV, JFAST>(a, b, lay, tw);
  else return fft_pencils_rt<INV, JFAST>(a, b, lay, tw, p);
}

}  // namespace fh
