// Forward-mode automatic differentiation of second order in the nine entries
// of a 3x3 tensor, used to obtain the stress P = dW/dF (Eq. 2) and the tangent
// K = d2W/dF2 (Eq. 3) from a stored energy density W written once as a
// template over its scalar type (Section 3.1-3.2).
//
// A number T2<G, H> carries a value v, the gradient g[9] and the upper
// triangle h[45] of the Hessian with respect to the nine seeded inputs. The
// template arguments are compile-time masks of the entries that may be
// nonzero (bit i of G for g[i], bit k of H for h[k]). Arithmetic only touches
// entries inside the masks, so a product of two seeded entries costs a few
// multiplies instead of ~200: on hardware where FP64 issue is the scarce
// resource the sparsity is worth more than generality. The rules are the
// usual truncated Taylor rules:
//   (a b)_i  = a.v b_i + b.v a_i
//   (a b)_ij = a.v b_ij + b.v a_ij + a_i b_j + a_j b_i
//   f(a)_i   = f'(a.v) a_i,   f(a)_ij = f'(a.v) a_ij + f''(a.v) a_i a_j
#pragma once

#include <stdint.h>

#include <type_traits>

#include "fh_common.cuh"

namespace fh {
namespace ad {

template <int I>
struct IC {
  static constexpr int value = I;
};

template <int I, int N, class Fn>
__device__ __forceinline__ void static_for(Fn&& f) {
  if constexpr (I < N) {
    f(IC<I>{});
    static_for<I + 1, N>(f);
  }
}

__host__ __device__ constexpr int tri_row(int k) {
  int a = 0;
  while (k >= 9 - a) {
    k -= 9 - a;
    ++a;
  }
  return a;
}
__host__ __device__ constexpr int tri_col(int k) {
  int a = 0;
  while (k >= 9 - a) {
    k -= 9 - a;
    ++a;
  }
  return a + k;
}

// Hessian mask of the symmetric outer product of two gradient masks
__host__ __device__ constexpr uint64_t sym_outer(uint32_t a, uint32_t b) {
  uint64_t m = 0;
  for (int i = 0; i < 9; ++i)
    for (int j = i; j < 9; ++j)
      if ((((a >> i) & 1u) && ((b >> j) & 1u)) || (((a >> j) & 1u) && ((b >> i) & 1u)))
        m |= 1ull << tri(i, j);
  return m;
}

template <uint32_t G, uint64_t H>
struct T2 {
  static constexpr uint32_t gm = G;
  static constexpr uint64_t hm = H;
  double v;
  double g[9];
  double h[45];
};

template <class T>
struct is_t2 {
  static constexpr bool value = false;
};
template <uint32_t G, uint64_t H>
struct is_t2<T2<G, H>> {
  static constexpr bool value = true;
};

// ---- addition / subtraction ------------------------------------------------
template <int SB, uint32_t Ga, uint64_t Ha, uint32_t Gb, uint64_t Hb>
__device__ __forceinline__ T2<Ga | Gb, Ha | Hb> addsub(const T2<Ga, Ha>& a, const T2<Gb, Hb>& b) {
  T2<Ga | Gb, Ha | Hb> r;
  r.v = SB > 0 ? a.v + b.v : a.v - b.v;
  static_for<0, 9>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr bool ia = (Ga >> i) & 1u, ib = (Gb >> i) & 1u;
    if constexpr (ia && ib) r.g[i] = SB > 0 ? a.g[i] + b.g[i] : a.g[i] - b.g[i];
    else if constexpr (ia) r.g[i] = a.g[i];
    else if constexpr (ib) r.g[i] = SB > 0 ? b.g[i] : -b.g[i];
  });
  static_for<0, 45>([&](auto K) {
    constexpr int k = decltype(K)::value;
    constexpr bool ia = (Ha >> k) & 1ull, ib = (Hb >> k) & 1ull;
    if constexpr (ia && ib) r.h[k] = SB > 0 ? a.h[k] + b.h[k] : a.h[k] - b.h[k];
    else if constexpr (ia) r.h[k] = a.h[k];
    else if constexpr (ib) r.h[k] = SB > 0 ? b.h[k] : -b.h[k];
  });
  return r;
}

template <uint32_t Ga, uint64_t Ha, uint32_t Gb, uint64_t Hb>
__device__ __forceinline__ auto operator+(const T2<Ga, Ha>& a, const T2<Gb, Hb>& b) {
  return addsub<1>(a, b);
}
template <uint32_t Ga, uint64_t Ha, uint32_t Gb, uint64_t Hb>
__device__ __forceinline__ auto operator-(const T2<Ga, Ha>& a, const T2<Gb, Hb>& b) {
  return addsub<-1>(a, b);
}

template <uint32_t G, uint64_t H>
__device__ __forceinline__ T2<G, H> operator-(const T2<G, H>& a) {
  T2<G, H> r;
  r.v = -a.v;
  static_for<0, 9>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr ((G >> i) & 1u) r.g[i] = -a.g[i];
  });
  static_for<0, 45>([&](auto K) {
    constexpr int k = decltype(K)::value;
    if constexpr ((H >> k) & 1ull) r.h[k] = -a.h[k];
  });
  return r;
}

template <uint32_t G, uint64_t H>
__device__ __forceinline__ T2<G, H> operator+(const T2<G, H>& a, double c) {
  T2<G, H> r = a;
  r.v = a.v + c;
  return r;
}
template <uint32_t G, uint64_t H>
__device__ __forceinline__ T2<G, H> operator+(double c, const T2<G, H>& a) {
  return a + c;
}
template <uint32_t G, uint64_t H>
__device__ __forceinline__ T2<G, H> operator-(const T2<G, H>& a, double c) {
  return a + (-c);
}
template <uint32_t G, uint64_t H>
__device__ __forceinline__ T2<G, H> operator-(double c, const T2<G, H>& a) {
  return (-a) + c;
}

// ---- scaling -----------------------------------------------------------------
template <uint32_t G, uint64_t H>
__device__ __forceinline__ T2<G, H> operator*(const T2<G, H>& a, double c) {
  T2<G, H> r;
  r.v = a.v * c;
  static_for<0, 9>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr ((G >> i) & 1u) r.g[i] = a.g[i] * c;
  });
  static_for<0, 45>([&](auto K) {
    constexpr int k = decltype(K)::value;
    if constexpr ((H >> k) & 1ull) r.h[k] = a.h[k] * c;
  });
  return r;
}
template <uint32_t G, uint64_t H>
__device__ __forceinline__ T2<G, H> operator*(double c, const T2<G, H>& a) {
  return a * c;
}

// ---- product -------------------------------------------------------------------
template <uint32_t Ga, uint64_t Ha, uint32_t Gb, uint64_t Hb>
__device__ __forceinline__ auto operator*(const T2<Ga, Ha>& a, const T2<Gb, Hb>& b) {
  constexpr uint32_t G = Ga | Gb;
  constexpr uint64_t H = Ha | Hb | sym_outer(Ga, Gb);
  T2<G, H> r;
  r.v = a.v * b.v;
  static_for<0, 9>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr bool ia = (Ga >> i) & 1u, ib = (Gb >> i) & 1u;
    if constexpr (ia && ib) r.g[i] = fma(a.v, b.g[i], b.v * a.g[i]);
    else if constexpr (ia) r.g[i] = b.v * a.g[i];
    else if constexpr (ib) r.g[i] = a.v * b.g[i];
  });
  static_for<0, 45>([&](auto K) {
    constexpr int k = decltype(K)::value;
    constexpr int i = tri_row(k), j = tri_col(k);
    if constexpr ((H >> k) & 1ull) {
      // accumulate only the terms whose factors are structurally nonzero
      double acc = 0.0;
      bool have = false;
      if constexpr ((Hb >> k) & 1ull) {
        acc = a.v * b.h[k];
        have = true;
      }
      if constexpr ((Ha >> k) & 1ull) {
        acc = have ? fma(b.v, a.h[k], acc) : b.v * a.h[k];
        have = true;
      }
      if constexpr (i == j) {
        if constexpr (((Ga >> i) & 1u) && ((Gb >> i) & 1u)) {
          const double t = 2.0 * a.g[i];
          acc = have ? fma(t, b.g[i], acc) : t * b.g[i];
          have = true;
        }
      } else {
        if constexpr (((Ga >> i) & 1u) && ((Gb >> j) & 1u)) {
          acc = have ? fma(a.g[i], b.g[j], acc) : a.g[i] * b.g[j];
          have = true;
        }
        if constexpr (((Ga >> j) & 1u) && ((Gb >> i) & 1u)) {
          acc = have ? fma(a.g[j], b.g[i], acc) : a.g[j] * b.g[i];
          have = true;
        }
      }
      r.h[k] = acc;
    }
  });
  return r;
}

// ---- unary functions through f, f', f'' -------------------------------------------
template <uint32_t G, uint64_t H>
__device__ __forceinline__ auto unary(const T2<G, H>& a, double f0, double f1, double f2) {
  constexpr uint64_t HR = H | sym_outer(G, G);
  T2<G, HR> r;
  r.v = f0;
  static_for<0, 9>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr ((G >> i) & 1u) r.g[i] = f1 * a.g[i];
  });
  static_for<0, 45>([&](auto K) {
    constexpr int k = decltype(K)::value;
    constexpr int i = tri_row(k), j = tri_col(k);
    constexpr bool hh = (H >> k) & 1ull;
    constexpr bool gg = ((G >> i) & 1u) && ((G >> j) & 1u);
    if constexpr (hh && gg) r.h[k] = fma(f2 * a.g[i], a.g[j], f1 * a.h[k]);
    else if constexpr (hh) r.h[k] = f1 * a.h[k];
    else if constexpr (gg) r.h[k] = (f2 * a.g[i]) * a.g[j];
  });
  return r;
}

// natural logarithm: f' = 1/x, f'' = -1/x^2 (x <= 0 yields a non-finite value
// that the calling kernel reports as a non-physical state)
template <uint32_t G, uint64_t H>
__device__ __forceinline__ auto log(const T2<G, H>& a) {
  const double inv = 1.0 / a.v;
  return unary(a, ::log(a.v), inv, -inv * inv);
}
template <uint32_t G, uint64_t H>
__device__ __forceinline__ auto square(const T2<G, H>& a) {
  return unary(a, a.v * a.v, 2.0 * a.v, 2.0);
}
template <uint32_t G, uint64_t H>
__device__ __forceinline__ auto sqrt(const T2<G, H>& a) {
  const double r = ::sqrt(a.v);
  const double d1 = 0.5 / r;
  return unary(a, r, d1, -0.5 * d1 / a.v);
}
// every entry of a set to zero (a branch that contributes nothing)
template <uint32_t G, uint64_t H>
__device__ __forceinline__ void zero_out(T2<G, H>& a) {
  a.v = 0.0;
  static_for<0, 9>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr ((G >> i) & 1u) a.g[i] = 0.0;
  });
  static_for<0, 45>([&](auto Kk) {
    constexpr int k = decltype(Kk)::value;
    if constexpr ((H >> k) & 1ull) a.h[k] = 0.0;
  });
}
template <uint32_t G, uint64_t H>
__device__ __forceinline__ auto recip(const T2<G, H>& a) {
  const double inv = 1.0 / a.v;
  return unary(a, inv, -inv * inv, 2.0 * inv * inv * inv);
}
template <uint32_t Ga, uint64_t Ha, uint32_t Gb, uint64_t Hb>
__device__ __forceinline__ auto operator/(const T2<Ga, Ha>& a, const T2<Gb, Hb>& b) {
  return a * recip(b);
}

// plain-double overloads so an energy template also evaluates on doubles
__device__ __forceinline__ double log(double x) { return ::log(x); }
__device__ __forceinline__ double square(double x) { return x * x; }

// ---- seeding and extraction ---------------------------------------------------------
template <int I>
using Seed = T2<(1u << I), 0ull>;

template <int I>
__device__ __forceinline__ Seed<I> seed(double x) {
  Seed<I> s;
  s.v = x;
  s.g[I] = 1.0;
  return s;
}

// Evaluate W of Law at F; write P = dW/dF and packed K = d2W/dF2.
// Returns W. Entries outside the masks are structurally zero.
template <class Law>
__device__ __forceinline__ double energy_derivatives(const double F[9], double lam, double mu,
                                                     double P[9], double K[45]) {
  const auto w = Law::energy(seed<0>(F[0]), seed<1>(F[1]), seed<2>(F[2]), seed<3>(F[3]), seed<4>(F[4]),
                             seed<5>(F[5]), seed<6>(F[6]), seed<7>(F[7]), seed<8>(F[8]), lam, mu);
  using W = decltype(w);
  static_for<0, 9>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr ((W::gm >> i) & 1u) P[i] = w.g[i];
    else P[i] = 0.0;
  });
  static_for<0, 45>([&](auto Kk) {
    constexpr int k = decltype(Kk)::value;
    if constexpr ((W::hm >> k) & 1ull) K[k] = w.h[k];
    else K[k] = 0.0;
  });
  return w.v;
}

// Evaluate the stress function of a Law that returns the stress itself (laws
// whose stress is not the derivative of a stored energy, such as a return
// map); write P and the packed tangent K = dP/dF (the upper triangle of the
// Jacobian; the laws used here have symmetric Jacobians). Law::stress calls
// emit(IC<a>{}, sigma_a) once for every component a.
template <class Law, class State>
__device__ __forceinline__ void stress_derivatives(const double F[9], const State& st, double P[9], double K[45]) {
  Law::stress(seed<0>(F[0]), seed<1>(F[1]), seed<2>(F[2]), seed<3>(F[3]), seed<4>(F[4]), seed<5>(F[5]),
              seed<6>(F[6]), seed<7>(F[7]), seed<8>(F[8]), st, [&](auto A, const auto& sig) {
                constexpr int a = decltype(A)::value;
                using S = typename std::remove_cv<typename std::remove_reference<decltype(sig)>::type>::type;
                P[a] = sig.v;
                static_for<a, 9>([&](auto B) {
                  constexpr int b = decltype(B)::value;
                  if constexpr ((S::gm >> b) & 1u) K[tri(a, b)] = sig.g[b];
                  else K[tri(a, b)] = 0.0;
                });
              });
}

}  // namespace ad

// ---------------------------------------------------------------------------
// Stored energy densities, each written once as a template over the scalar
// type of the nine entries F00..F22 (row-major).
// ---------------------------------------------------------------------------
struct LinearElasticLaw {
  // small strain: the arguments are the displacement gradient H;
  // eps = sym(H), W = lambda/2 tr(eps)^2 + mu eps:eps
  template <class A0, class A1, class A2, class A3, class A4, class A5, class A6, class A7, class A8>
  __device__ static auto energy(const A0& H00, const A1& H01, const A2& H02, const A3& H10, const A4& H11,
                                const A5& H12, const A6& H20, const A7& H21, const A8& H22, double lam,
                                double mu) {
    using ad::square;
    const auto e01 = 0.5 * (H01 + H10);
    const auto e02 = 0.5 * (H02 + H20);
    const auto e12 = 0.5 * (H12 + H21);
    const auto tr = H00 + H11 + H22;
    const auto ee = square(H00) + square(H11) + square(H22) + 2.0 * (square(e01) + square(e02) + square(e12));
    return (0.5 * lam) * square(tr) + mu * ee;
  }
};

struct NeoHookeanLaw {
  // W = mu/2 (tr F^T F - 3) - mu ln J + lambda/2 (ln J)^2
  template <class A0, class A1, class A2, class A3, class A4, class A5, class A6, class A7, class A8>
  __device__ static auto energy(const A0& F00, const A1& F01, const A2& F02, const A3& F10, const A4& F11,
                                const A5& F12, const A6& F20, const A7& F21, const A8& F22, double lam,
                                double mu) {
    using ad::log;
    using ad::square;
    const auto I1 = square(F00) + square(F01) + square(F02) + square(F10) + square(F11) + square(F12) +
                    square(F20) + square(F21) + square(F22);
    const auto J = F00 * (F11 * F22 - F12 * F21) - F01 * (F10 * F22 - F12 * F20) + F02 * (F10 * F21 - F11 * F20);
    const auto lnJ = log(J);
    return (0.5 * mu) * (I1 - 3.0) - mu * lnJ + (0.5 * lam) * square(lnJ);
  }
};

struct SVKLaw {
  // W = lambda/2 tr(E)^2 + mu E:E with E = (F^T F - I)/2
  template <class A0, class A1, class A2, class A3, class A4, class A5, class A6, class A7, class A8>
  __device__ static auto energy(const A0& F00, const A1& F01, const A2& F02, const A3& F10, const A4& F11,
                                const A5& F12, const A6& F20, const A7& F21, const A8& F22, double lam,
                                double mu) {
    using ad::square;
    const auto E00 = 0.5 * (square(F00) + square(F10) + square(F20) - 1.0);
    const auto E11 = 0.5 * (square(F01) + square(F11) + square(F21) - 1.0);
    const auto E22 = 0.5 * (square(F02) + square(F12) + square(F22) - 1.0);
    const auto E01 = 0.5 * (F00 * F01 + F10 * F11 + F20 * F21);
    const auto E02 = 0.5 * (F00 * F02 + F10 * F12 + F20 * F22);
    const auto E12 = 0.5 * (F01 * F02 + F11 * F12 + F21 * F22);
    const auto trE = E00 + E11 + E22;
    const auto EE = square(E00) + square(E11) + square(E22) + 2.0 * (square(E01) + square(E02) + square(E12));
    return (0.5 * lam) * square(trE) + mu * EE;
  }
};

// ---------------------------------------------------------------------------
// Small-strain J2 plasticity with linear isotropic hardening (Section 4.1.2,
// Appendix B): elastic predictor from the plastic strain of the last
// converged increment, von Mises check, radial return. The branch is chosen
// on the value; both branches share one expression (the return factor is
// zeroed in the elastic branch), so AD differentiates the active one.
// ---------------------------------------------------------------------------
struct J2State {
  double ep[9];     // plastic strain of the last converged increment
  double p;         // cumulative plastic strain
  double lam, mu;   // Lame parameters
  double sy, h;     // yield stress and hardening modulus
};

struct J2Law {
  template <class A0, class A1, class A2, class A3, class A4, class A5, class A6, class A7, class A8, class Emit>
  __device__ static void stress(const A0& H00, const A1& H01, const A2& H02, const A3& H10, const A4& H11,
                                const A5& H12, const A6& H20, const A7& H21, const A8& H22, const J2State& st,
                                Emit&& emit) {
    using ad::IC;
    using ad::square;
    const double mu2 = 2.0 * st.mu;
    const auto e00 = H00 - st.ep[0];
    const auto e11 = H11 - st.ep[4];
    const auto e22 = H22 - st.ep[8];
    const auto e01 = 0.5 * (H01 + H10) - st.ep[1];
    const auto e02 = 0.5 * (H02 + H20) - st.ep[2];
    const auto e12 = 0.5 * (H12 + H21) - st.ep[5];
    const auto tr = e00 + e11 + e22;
    const auto third = tr * (1.0 / 3.0);
    const auto d00 = mu2 * (e00 - third);     // deviatoric trial stress
    const auto d11 = mu2 * (e11 - third);
    const auto d22 = mu2 * (e22 - third);
    const auto d01 = mu2 * e01;
    const auto d02 = mu2 * e02;
    const auto d12 = mu2 * e12;
    auto ss = square(d00) + square(d11) + square(d22) + 2.0 * (square(d01) + square(d02) + square(d12));
    const bool stress_free = !(ss.v > 0.0);  // a stress-free deviator is elastic
    ss.v += stress_free ? 1.0 : 0.0;         // keeps sqrt and the quotient below finite
    const auto q = ad::sqrt(1.5 * ss);
    const auto phi = q - (st.sy + st.h * st.p);
    auto kappa = (3.0 * st.mu / (3.0 * st.mu + st.h)) * (phi / q);  // 3 mu dp / q
    if (stress_free || !(phi.v > 0.0)) ad::zero_out(kappa);
    const auto vol = (st.lam + mu2 / 3.0) * tr;  // bulk part, unchanged by the return
    const auto s00 = vol + (d00 - kappa * d00);
    const auto s11 = vol + (d11 - kappa * d11);
    const auto s22 = vol + (d22 - kappa * d22);
    const auto s01 = d01 - kappa * d01;
    const auto s02 = d02 - kappa * d02;
    const auto s12 = d12 - kappa * d12;
    emit(IC<0>{}, s00);
    emit(IC<1>{}, s01);
    emit(IC<2>{}, s02);
    emit(IC<3>{}, s01);
    emit(IC<4>{}, s11);
    emit(IC<5>{}, s12);
    emit(IC<6>{}, s02);
    emit(IC<7>{}, s12);
    emit(IC<8>{}, s22);
  }
};

}  // namespace fh
