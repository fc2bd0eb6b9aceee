// Shared definitions of the CUDA library: complex helpers, index maps, error
// plumbing and the launch interface between the host driver and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fft_homog.h"

namespace fh {

constexpr int kThreads = 256;          // threads per CTA of every kernel
constexpr int kMaxN = 256;             // largest extent with a compile-time plan
constexpr int kMaxNAny = 512;          // largest x or y extent with a run-time plan

// transform lengths with a radix plan: 2^a and 3 * 2^a, up to 256
__host__ __device__ constexpr bool fft_length_ok(int L) {
  if (L < 1 || L > kMaxN) return false;
  if (L % 3 == 0) L /= 3;
  return (L & (L - 1)) == 0;
}

// offset of the twiddle table of length L: the tables of all supported lengths
// are stored back to back in increasing order
__host__ __device__ constexpr int twiddle_offset(int L) {
  int off = 0;
  for (int l = 1; l < L; ++l)
    if (fft_length_ok(l)) off += l;
  return off;
}
constexpr int kTwiddleTotal = twiddle_offset(kMaxN) + kMaxN;
// Every length has two tables: w_L^m as (cos, -sin) at twiddle_offset(L) + m,
// and the same roots in the tangent form of the twiddled FFT stages
// (fft_core.cuh) at kTwiddleTotal + twiddle_offset(L) + m. Run-time plans put
// their tables after both (from kTwiddleTables on).
constexpr int kTwiddleTables = 2 * kTwiddleTotal;

// ---------------------------------------------------------------------------
// complex helpers (double2 = re, im)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// a * w with w a unit twiddle: 2 DMUL + 2 DFMA
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 w) {
  return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
// a * conj(w)
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 w) {
  return make_double2(fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -a.x * w.y));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// symmetric 9x9 packing: slot of (a, b), a <= b, row by row
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int tri(int a, int b) { return 9 * a - a * (a - 1) / 2 + (b - a); }
__host__ __device__ constexpr int sym_slot(int a, int b) { return a <= b ? tri(a, b) : tri(b, a); }

// signed wave integer of index j on an n-point axis; the Nyquist index of an
// even axis maps to 0 (first spectral derivative convention)
__host__ __device__ __forceinline__ int wave_int(int j, int n) {
  if (2 * j == n) return 0;
  return (2 * j < n) ? j : j - n;
}

// the extents a grid may have: nx, ny any supported length, nz an even one
// whose half is supported too (the real-to-complex step transforms nz/2)
__host__ __device__ constexpr bool grid_extents_ok(int nx, int ny, int nz) {
  return fft_length_ok(nx) && fft_length_ok(ny) && nz >= 2 && nz % 2 == 0 && fft_length_ok(nz) &&
         fft_length_ok(nz / 2);
}

// the extents a solver context accepts: nx and ny any length 1 .. kMaxNAny
// (run-time plans for those without a compile-time one), nz as above or 1 (a
// cell one voxel thick: plane problems without a redundant second layer)
__host__ __device__ constexpr bool grid_extents_ok_any(int nx, int ny, int nz) {
  return nx >= 1 && nx <= kMaxNAny && ny >= 1 && ny <= kMaxNAny &&
         (nz == 1 || (nz >= 2 && nz % 2 == 0 && fft_length_ok(nz) && fft_length_ok(nz / 2)));
}

// Run-time FFT plan of an axis whose length has no compile-time plan (see
// fft_core.cuh): stage radices in order and the offset of the length's
// twiddle table.
struct FftPlan {
  int L;        // length (0 when the axis uses a compile-time plan)
  int n;        // number of stages (0 for a Rader plan)
  int tw_off;   // offset of the plan's tables in the context's twiddle table
  int tw_len;   // entries of those tables (L, or 4 (L - 1) for a Rader plan)
  int r[12];    // radix of each stage, in order
  int rader;    // 1: prime L by Rader's algorithm, a cyclic convolution of length L - 1
  int in_n;     // stages of the inner length-(L - 1) transforms
  int in_r[10]; // their radices
};

// ---------------------------------------------------------------------------
// Grid description passed by value to kernels
// ---------------------------------------------------------------------------
struct Grid {
  int nx, ny, nz, nzh;      // extents and half extent nz/2 + 1
  long long n;              // voxels
  long long nspec;          // complex entries per spectral component nx*ny*nzh
  double sx, sy, sz;        // wave-vector scale 1/L_a (2 pi cancels in Ghat)
  FftPlan px, py;           // run-time plans of x and y (L = 0: compile-time plan)
};

// Material tables passed by value (up to 256 phases live in a device buffer)
struct MatView {
  int kind;
  const uint8_t* phase;      // device
  const double* params;      // device [n_phase][2]
  const double* scale;       // device [N] modulus multiplier per voxel, or nullptr
  const double* plastic;     // device [n_phase][2] (yield stress, hardening modulus), J2 only
  const double* history;     // device [10][N] plastic strain and cumulative plastic strain, J2 only
};

__device__ __forceinline__ void voxel_lame(const MatView& m, long long v, double& lam, double& mu) {
  const int ph = m.phase[v];
  lam = m.params[2 * ph];
  mu = m.params[2 * ph + 1];
  if (m.scale) {
    const double s = m.scale[v];
    lam *= s;
    mu *= s;
  }
}

// ---------------------------------------------------------------------------
// device flags written by kernels, read by the host after a solve step
// ---------------------------------------------------------------------------
enum : int {
  kFlagNonPhysical = 1,
};

// ---------------------------------------------------------------------------
// deterministic reductions: fixed shuffle tree inside a warp, then warp 0
// adds the per-warp results in warp order
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Every thread of the CTA must call; the sum is valid in thread 0. `red`
// points to at least 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

}  // namespace fh
