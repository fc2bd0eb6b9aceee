// Learned warm start: forward, backward and Adam kernels of the factorized
// Fourier neural operator declared in include/fh_fno.h.
//
// Activations are stored channels-last, [sample][x][y][z][32 channels], so
// that a line of voxels along any axis is a run of 128-byte channel vectors:
// one warp handles one line with lane = channel, and every global access of
// the spectral kernels is a coalesced 128-byte row whatever the axis. The
// truncated real DFT along a line keeps 12 modes, so it is computed as a
// direct sum against precomputed twiddles (24 cosines/sines per position)
// rather than by an FFT (float32 on the CUDA cores). The channel
// contractions run on the tensor cores as bfloat16 MMAs (mma.sync m16n8k16)
// with float32 accumulation: the per-mode complex 32x32 mixing as a real
// 64x64 block per mode applied to the coefficients of the CTA's 8 lines at
// once, the pointwise 32x32 mixing and the 32 -> 128 -> 9 projection head on
// tiles of 16 voxels. The bfloat16 weights enter exactly; a float32 operand
// (activation, coefficient, effective head) enters as a pair of bfloat16
// terms hi + lo (about 16 significant bits), so each product takes two or
// three MMAs and the result stays close to float32 arithmetic. Every
// reduction over voxels (weight gradients, loss) runs in a fixed order
// through per-block partials, so a training step is deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/fh_fno.h"

extern "C" void fh_internal_set_error(const char* msg);
extern "C" void fh_internal_ctx_grid(const fh_ctx* ctx, int* nx, int* ny, int* nz);

namespace fh {
namespace fno {

constexpr int kC = 32;       // width
constexpr int kLayers = 4;
constexpr int kModes = 12;
constexpr int kJ = 2 * kModes;  // real coefficients per channel and line
constexpr int kHid = 128;
constexpr int kOut = 9;
constexpr int kHead = kOut * 9;  // per-voxel 9x9 response R_ij, applied to the load direction u
constexpr int kMinN = 2 * kModes;  // retained modes stay below the Nyquist index

constexpr long long kLift = kC + kC * 9 + kC;                       // 352
constexpr long long kWSize = 3LL * kModes * 2 * kC * kC;           // 73728
constexpr long long kWAxis = (long long)kModes * 2 * kC * kC;       // 24576
constexpr long long kLayer = kWSize + kC * kC + kC;                 // 74784
constexpr long long kOffA = 0, kOffB = kC, kOffB0 = kC + kC * 9;
__host__ __device__ constexpr long long off_W(int l) { return kLift + l * kLayer; }
__host__ __device__ constexpr long long off_M(int l) { return off_W(l) + kWSize; }
__host__ __device__ constexpr long long off_m(int l) { return off_M(l) + kC * kC; }
constexpr long long kOffP1 = kLift + kLayers * kLayer;
constexpr long long kOffp1 = kOffP1 + kHid * kC;
constexpr long long kOffP2 = kOffp1 + kHid;
constexpr long long kOffp2 = kOffP2 + kHead * kHid;
constexpr long long kNParam = kOffp2 + kHead;                       // 314161
// per-sample effective head: P2u[i][k] = sum_j P2[9i + j][k] u_j, p2u[i] = sum_j p2[9i + j] u_j
constexpr int kHeadEff = kOut * kHid + kOut;                        // 1161
// row of the projection weight-gradient partials: P1, p1, then the
// per-sample sums G[i][k] = sum gq_i t_k and Gp[i] = sum gq_i
constexpr int kProjRow = kHid * kC + kHid + kHeadEff;               // 5385
constexpr int kProjShared = kHid * kC + kHid;                       // 4224
constexpr int kPointLen = kC * kC + kC;                             // 1056
static_assert(kNParam == 314161, "parameter layout");

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kLinesPerChunk = 128;  // lines per block of the spectral weight gradient
constexpr long long kLiftChunk = 4096;  // voxels per block of the lifting gradient
constexpr double kPi = 3.14159265358979323846;

struct Geom {
  int nx, ny, nz;
  long long N;  // voxels per sample
};

// first voxel (global index over samples) and voxel stride of line li along axis ax
__device__ __forceinline__ void line_of(const Geom& g, int ax, long long li, long long& base, long long& stride) {
  if (ax == 0) {
    const long long per = (long long)g.ny * g.nz;
    const long long b = li / per, r = li - b * per;
    base = b * g.N + r;
    stride = per;
  } else if (ax == 1) {
    const long long per = (long long)g.nx * g.nz;
    const long long b = li / per, r = li - b * per;
    const long long x = r / g.nz, z = r - x * g.nz;
    base = b * g.N + x * g.ny * g.nz + z;
    stride = g.nz;
  } else {
    const long long per = (long long)g.nx * g.ny;
    const long long b = li / per, r = li - b * per;
    base = b * g.N + r * g.nz;
    stride = 1;
  }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}
__device__ __forceinline__ float bf(const __nv_bfloat16* p, long long i) { return __bfloat162float(p[i]); }

// ---------------------------------------------------------------------------
// tensor-core helpers. mma.sync m16n8k16, bf16 inputs, f32 accumulators; with
// g = lane / 4, t = lane % 4 a thread holds A[g][2t, 2t+1], A[g+8][2t, 2t+1],
// A[g][2t+8, 2t+9], A[g+8][2t+8, 2t+9] (four bf16 pairs), B[2t, 2t+1][g] and
// B[2t+8, 2t+9][g] (two pairs), and D[g][2t, 2t+1], D[g+8][2t, 2t+1].
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1) {
  mma_bf16(d, a.x, a.y, a.z, a.w, b0, b1);
}
__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }
// (x, y) -> hi = bf16(x, y) and lo = bf16(x - hi.x, y - hi.y)
__device__ __forceinline__ void split_bf2(float x, float y, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  const float2 hf = __bfloat1622float2(h);
  hi = bf2_bits(h);
  lo = bf2_bits(__floats2bfloat162_rn(x - hf.x, y - hf.y));
}

// Real 64x64 form of the complex mixing of mode k of layer l, axis ax:
// row r = (ri_o, o), column kap = (ri_c, c), each as 32 * ri + index, with
// [[Wr, -Wi], [Wi, Wr]] so that (Yr, Yi) = Wt (Xr, Xi) is Y = W X.
__device__ __forceinline__ float wtilde(const float* __restrict__ theta, int l, int ax, int k, int r, int kap) {
  const int ro = r >> 5, o = r & 31, rc = kap >> 5, c = kap & 31;
  const long long src = off_W(l) + ((long long)(ax * kModes + k) * 2) * kC * kC + (long long)o * kC + c;
  const float wr = theta[src], wi = theta[src + kC * kC];
  return ro == rc ? wr : (ro == 0 ? -wi : wi);
}

// A fragments of the mixing matrices in mma order, for the forward (Wt) and
// backward (Wt^T) passes: entry ((((l*3 + ax)*kModes + k)*4 + mt)*4 + ks)*32
// + lane is the uint4 that lane holds for row tile mt, k-step ks
constexpr long long kFragPerMode = 4 * 4 * 32;
constexpr long long kFrag = (long long)kLayers * 3 * kModes * kFragPerMode;

// ---------------------------------------------------------------------------
// parameters: bfloat16 copies, spectral weights also as (re, im) pairs in the
// two transposed orders the forward ([k][c][o]) and backward ([k][o][c])
// passes read with lane-contiguous addresses
// ---------------------------------------------------------------------------
__global__ void k_prepare(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wq, uint4* __restrict__ wfa,
                          uint4* __restrict__ wba) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < kNParam; i += stride)
    wq[i] = __float2bfloat16_rn(theta[i]);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < kFrag; e += stride) {
    const int lane = (int)(e & 31), g = lane >> 2, t = lane & 3;
    const int ks = (int)((e >> 5) & 3), mt = (int)((e >> 7) & 3);
    const long long lak = e >> 9;  // (l * 3 + ax) * kModes + k
    const int k = (int)(lak % kModes);
    const int ax = (int)((lak / kModes) % 3);
    const int l = (int)(lak / (3 * kModes));
    const int r0 = mt * 16 + g, r1 = r0 + 8, c0 = ks * 16 + 2 * t, c1 = c0 + 8;
    // forward: A[r][kap] = Wt[r][kap]; backward: A[kap][r] = Wt[r][kap]
    uint4 f, b;
    f.x = bf2_bits(__floats2bfloat162_rn(wtilde(theta, l, ax, k, r0, c0), wtilde(theta, l, ax, k, r0, c0 + 1)));
    f.y = bf2_bits(__floats2bfloat162_rn(wtilde(theta, l, ax, k, r1, c0), wtilde(theta, l, ax, k, r1, c0 + 1)));
    f.z = bf2_bits(__floats2bfloat162_rn(wtilde(theta, l, ax, k, r0, c1), wtilde(theta, l, ax, k, r0, c1 + 1)));
    f.w = bf2_bits(__floats2bfloat162_rn(wtilde(theta, l, ax, k, r1, c1), wtilde(theta, l, ax, k, r1, c1 + 1)));
    b.x = bf2_bits(__floats2bfloat162_rn(wtilde(theta, l, ax, k, c0, r0), wtilde(theta, l, ax, k, c0 + 1, r0)));
    b.y = bf2_bits(__floats2bfloat162_rn(wtilde(theta, l, ax, k, c0, r1), wtilde(theta, l, ax, k, c0 + 1, r1)));
    b.z = bf2_bits(__floats2bfloat162_rn(wtilde(theta, l, ax, k, c1, r0), wtilde(theta, l, ax, k, c1 + 1, r0)));
    b.w = bf2_bits(__floats2bfloat162_rn(wtilde(theta, l, ax, k, c1, r1), wtilde(theta, l, ax, k, c1 + 1, r1)));
    wfa[e] = f;
    wba[e] = b;
  }
}

// s = |Fbar - I|_F and u = (Fbar - I)/s per sample (u = 0 when s = 0)
__global__ void k_load_dir(const double* __restrict__ Fbar, int B, float* __restrict__ su) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double d[9], s2 = 0.0;
  for (int c = 0; c < 9; ++c) {
    d[c] = Fbar[9 * b + c] - ((c % 4 == 0) ? 1.0 : 0.0);
    s2 += d[c] * d[c];
  }
  const double s = sqrt(s2);
  su[10 * b] = (float)s;
  for (int c = 0; c < 9; ++c) su[10 * b + 1 + c] = s > 0.0 ? (float)(d[c] / s) : 0.0f;
}

// h0 = a phi + B u + b0
__global__ void k_lift(const uint8_t* const* __restrict__ phase, const float* __restrict__ su,
                       const __nv_bfloat16* __restrict__ wq, long long N, int B, float* __restrict__ h0) {
  const long long total = (long long)B * N * kC;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e & (kC - 1));
    const long long vox = e >> 5;
    const int b = (int)(vox / N);
    const long long v = vox - (long long)b * N;
    float bias = bf(wq, kOffB0 + c);
#pragma unroll
    for (int j = 0; j < 9; ++j) bias = fmaf(bf(wq, kOffB + c * 9 + j), su[10 * b + 1 + j], bias);
    const float phi = phase[b][v] != 0 ? 1.0f : 0.0f;
    h0[e] = fmaf(bf(wq, kOffA + c), phi, bias);
  }
}

// ---------------------------------------------------------------------------
// spectral convolution along one axis, forward: out (=/+=) S_ax(h)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// spectral convolution along one axis on the tensor cores. For a line h[x][c]
// (x < n positions, 32 channels) the truncated DFT X[j][c] = sum_x T[j][x]
// h[x][c] (j < 24: cosine and minus sine rows of the 12 modes) is an MMA with
// M = j (two 16-row tiles), N = c (four 8-column tiles), K = x; the inverse
// S[x][o] = sum_j I[x][j] Y[j][o] an MMA with M = x, N = o, K = j. The twiddle
// matrices T and I (and the transposes the backward pass needs) are split
// into bf16 hi + lo fragments once per CTA; the line values are split as
// they are loaded, and each product takes three MMAs (hi hi, hi lo, lo hi).
// ---------------------------------------------------------------------------
constexpr int kXStride = kJ * kC + 8;  // floats per line block (padding spreads the banks of the 8 lines)

__host__ __device__ constexpr int ksteps(int n) { return (n + 15) / 16; }
// fragments (hi and lo uint4 per lane) of a rows x cols matrix split into 16 x 16 tiles
__host__ __device__ constexpr int frag_count(int rows, int cols) { return ((rows + 15) / 16) * ksteps(cols) * 32; }
__host__ __device__ constexpr size_t spec_smem(int n, bool bwd) {
  // forward: T (24 x n) and I (n x 24); backward: T, I^T (24 x n) and T^T (n x 24); two line blocks per warp
  return (size_t)(bwd ? 2 * frag_count(kJ, n) + frag_count(n, kJ) : frag_count(kJ, n) + frag_count(n, kJ)) * 2 *
             sizeof(uint4) +
         2 * (size_t)kWarps * kXStride * sizeof(float);
}

// Build the hi/lo A fragments of the rows x cols matrix M(r, k) (zero outside)
// into Ah/Al: entry (mt * ksteps(cols) + ks) * 32 + lane.
template <class Fn>
__device__ __forceinline__ void build_frags(uint4* __restrict__ Ah, uint4* __restrict__ Al, int rows, int cols,
                                            Fn M) {
  const int nks = ksteps(cols);
  const int total = frag_count(rows, cols);
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int lane = e & 31, ks = (e >> 5) % nks, mt = (e >> 5) / nks, g = lane >> 2, t = lane & 3;
    const int r0 = mt * 16 + g, r1 = r0 + 8, k0 = ks * 16 + 2 * t, k1 = k0 + 8;
    auto at = [&](int r, int k) { return (r < rows && k < cols) ? M(r, k) : 0.0f; };
    uint4 h, l;
    split_bf2(at(r0, k0), at(r0, k0 + 1), h.x, l.x);
    split_bf2(at(r1, k0), at(r1, k0 + 1), h.y, l.y);
    split_bf2(at(r0, k1), at(r0, k1 + 1), h.z, l.z);
    split_bf2(at(r1, k1), at(r1, k1 + 1), h.w, l.w);
    Ah[e] = h;
    Al[e] = l;
  }
}

// d[mt][nt] += T[rows of tile mt][x] h[x][channels of tile nt] for one line of
// global memory (element x, channel c at src + x * step + c); two row tiles (24
// coefficient rows), four channel tiles, K = n positions
__device__ __forceinline__ void line_dft_tc(const float* __restrict__ src, long long step, int n,
                                            const uint4* __restrict__ Ah, const uint4* __restrict__ Al, int lane,
                                            float (&d)[2][4][4]) {
  const int g = lane >> 2, t = lane & 3, nks = ksteps(n);
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) d[mt][nt][0] = d[mt][nt][1] = d[mt][nt][2] = d[mt][nt][3] = 0.0f;
  for (int ks = 0; ks < nks; ++ks) {
    const int x0 = ks * 16 + 2 * t;
    const uint4 a0h = Ah[(0 * nks + ks) * 32 + lane], a0l = Al[(0 * nks + ks) * 32 + lane];
    const uint4 a1h = Ah[(1 * nks + ks) * 32 + lane], a1l = Al[(1 * nks + ks) * 32 + lane];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const float* col = src + nt * 8 + g;
      const float v0 = x0 < n ? col[x0 * step] : 0.0f, v1 = x0 + 1 < n ? col[(x0 + 1) * step] : 0.0f;
      const float v2 = x0 + 8 < n ? col[(x0 + 8) * step] : 0.0f, v3 = x0 + 9 < n ? col[(x0 + 9) * step] : 0.0f;
      uint32_t b0h, b0l, b1h, b1l;
      split_bf2(v0, v1, b0h, b0l);
      split_bf2(v2, v3, b1h, b1l);
      mma_bf16(d[0][nt], a0h, b0h, b1h);
      mma_bf16(d[0][nt], a0h, b0l, b1l);
      mma_bf16(d[0][nt], a0l, b0h, b1h);
      mma_bf16(d[1][nt], a1h, b0h, b1h);
      mma_bf16(d[1][nt], a1h, b0l, b1l);
      mma_bf16(d[1][nt], a1l, b0h, b1h);
    }
  }
}

// the D fragments of line_dft_tc as a [j][c] block (rows j < 24) in shared or global memory
__device__ __forceinline__ void store_coef(float* __restrict__ dst, int lane, const float (&d)[2][4][4]) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int j0 = mt * 16 + g, c = nt * 8 + 2 * t;
      if (j0 < kJ) *reinterpret_cast<float2*>(dst + j0 * kC + c) = make_float2(d[mt][nt][0], d[mt][nt][1]);
      if (j0 + 8 < kJ) *reinterpret_cast<float2*>(dst + (j0 + 8) * kC + c) = make_float2(d[mt][nt][2], d[mt][nt][3]);
    }
}

// dst[x][o] (+)= sum_j I[x][j] Y[j][o] for one line (x < n): Y a [j][o] block in
// shared memory, I as A fragments (row tiles of 16 positions, two k-steps of j)
template <bool ACCUM>
__device__ __forceinline__ void line_idft_tc(const float* __restrict__ Y, float* __restrict__ dst, long long step,
                                             int n, const uint4* __restrict__ Ah, const uint4* __restrict__ Al,
                                             int lane) {
  const int g = lane >> 2, t = lane & 3;
  uint32_t bh[2][4][2], bl[2][4][2];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int j0 = ks * 16 + 2 * t, o = nt * 8 + g;
      const float v0 = j0 < kJ ? Y[j0 * kC + o] : 0.0f, v1 = j0 + 1 < kJ ? Y[(j0 + 1) * kC + o] : 0.0f;
      const float v2 = j0 + 8 < kJ ? Y[(j0 + 8) * kC + o] : 0.0f, v3 = j0 + 9 < kJ ? Y[(j0 + 9) * kC + o] : 0.0f;
      split_bf2(v0, v1, bh[ks][nt][0], bl[ks][nt][0]);
      split_bf2(v2, v3, bh[ks][nt][1], bl[ks][nt][1]);
    }
  const int nmt = ksteps(n);
  for (int mt = 0; mt < nmt; ++mt) {
    const uint4 a0h = Ah[(mt * 2 + 0) * 32 + lane], a0l = Al[(mt * 2 + 0) * 32 + lane];
    const uint4 a1h = Ah[(mt * 2 + 1) * 32 + lane], a1l = Al[(mt * 2 + 1) * 32 + lane];
    const int x0 = mt * 16 + g, x1 = x0 + 8;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      mma_bf16(d, a0h, bh[0][nt][0], bh[0][nt][1]);
      mma_bf16(d, a0h, bl[0][nt][0], bl[0][nt][1]);
      mma_bf16(d, a0l, bh[0][nt][0], bh[0][nt][1]);
      mma_bf16(d, a1h, bh[1][nt][0], bh[1][nt][1]);
      mma_bf16(d, a1h, bl[1][nt][0], bl[1][nt][1]);
      mma_bf16(d, a1l, bh[1][nt][0], bh[1][nt][1]);
      const int o = nt * 8 + 2 * t;
      if (x0 < n) {
        float2* p = reinterpret_cast<float2*>(dst + x0 * step + o);
        float2 v = make_float2(d[0], d[1]);
        if (ACCUM) {
          const float2 u = *p;
          v.x += u.x;
          v.y += u.y;
        }
        *p = v;
      }
      if (x1 < n) {
        float2* p = reinterpret_cast<float2*>(dst + x1 * step + o);
        float2 v = make_float2(d[2], d[3]);
        if (ACCUM) {
          const float2 u = *p;
          v.x += u.x;
          v.y += u.y;
        }
        *p = v;
      }
    }
  }
}

// Complex mixing of the CTA's 8 lines on the tensor cores: for every mode k,
// Y_k = Wt_k X_k with Wt_k the real 64x64 block (rows (ri, o), columns
// (ri, c)) and X_k the 64 x 8 matrix of the 8 lines' coefficients of mode k
// (split hi + lo). Warp w takes row tile w % 4 of the modes k = w/4, w/4 + 2,
// ...; X and Y are [line][j][channel] blocks in shared memory (j = 2k + ri).
__device__ __forceinline__ void mix_modes_tc(const float* __restrict__ sX, float* __restrict__ sY,
                                             const uint4* __restrict__ WA, int warp, int lane) {
  const int mt = warp & 3, gi = lane >> 2, t = lane & 3;
  const float* Xl = sX + gi * kXStride;
  for (int k = warp >> 2; k < kModes; k += 2) {
    float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const uint4* wa = WA + (long long)((k * 4 + mt) * 4) * 32 + lane;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const uint4 af = __ldg(wa + ks * 32);
      const int kap0 = ks * 16 + 2 * t, kap1 = kap0 + 8;  // B rows kap, kap + 1 (same half of 32)
      const float2 x0 = *reinterpret_cast<const float2*>(Xl + (2 * k + (kap0 >> 5)) * kC + (kap0 & 31));
      const float2 x1 = *reinterpret_cast<const float2*>(Xl + (2 * k + (kap1 >> 5)) * kC + (kap1 & 31));
      uint32_t h0, l0, h1, l1;
      split_bf2(x0.x, x0.y, h0, l0);
      split_bf2(x1.x, x1.y, h1, l1);
      mma_bf16(d, af, h0, h1);
      mma_bf16(d, af, l0, l1);
    }
    // D rows r (output (ri, o)), columns = lines 2t, 2t + 1
    const int r0 = mt * 16 + gi, r1 = r0 + 8;
    float* y0 = sY + (2 * t) * kXStride;
    float* y1 = y0 + kXStride;
    y0[(2 * k + (r0 >> 5)) * kC + (r0 & 31)] = d[0];
    y1[(2 * k + (r0 >> 5)) * kC + (r0 & 31)] = d[1];
    y0[(2 * k + (r1 >> 5)) * kC + (r1 & 31)] = d[2];
    y1[(2 * k + (r1 >> 5)) * kC + (r1 & 31)] = d[3];
  }
}

// forward: out (=/+=) S_ax(h); each CTA takes 8 lines at a time, one per warp
template <bool ACCUM>
__global__ void __launch_bounds__(kThreads, 2) k_spec_fwd(const float* __restrict__ h, float* __restrict__ out,
                                                       const uint4* __restrict__ WA,
                                                       const float* __restrict__ tw, const float* __restrict__ itw,
                                                       Geom g, int ax, int n, long long n_lines) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int fT = frag_count(kJ, n), fI = frag_count(n, kJ);
  uint4* Th = reinterpret_cast<uint4*>(smem);
  uint4* Tl = Th + fT;
  uint4* Ih = Tl + fT;
  uint4* Il = Ih + fI;
  float* sX = reinterpret_cast<float*>(Il + fI);
  float* sY = sX + kWarps * kXStride;
  build_frags(Th, Tl, kJ, n, [&](int j, int x) { return tw[x * kJ + j]; });
  build_frags(Ih, Il, n, kJ, [&](int x, int j) { return itw[x * kJ + j]; });
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long l0 = (long long)blockIdx.x * kWarps; l0 < n_lines; l0 += (long long)gridDim.x * kWarps) {
    const long long li = l0 + warp;
    const bool valid = li < n_lines;
    long long base = 0, stride = 0;
    if (valid) line_of(g, ax, li, base, stride);
    const long long step = stride * kC;
    float d[2][4][4];
    if (valid) {
      line_dft_tc(h + base * kC, step, n, Th, Tl, lane, d);
    } else {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) d[mt][nt][0] = d[mt][nt][1] = d[mt][nt][2] = d[mt][nt][3] = 0.0f;
    }
    store_coef(sX + warp * kXStride, lane, d);
    __syncthreads();
    mix_modes_tc(sX, sY, WA, warp, lane);
    __syncthreads();
    if (valid) line_idft_tc<ACCUM>(sY + warp * kXStride, out + base * kC, step, n, Ih, Il, lane);
  }
}

// ---------------------------------------------------------------------------
// spectral convolution along one axis, backward: gh += S_ax^T(gz); stores the
// forward coefficients X of h and the coefficient gradient gY of every line
// for the weight gradient
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 2) k_spec_bwd(const float* __restrict__ h, const float* __restrict__ gz,
                                                       float* __restrict__ gh, float* __restrict__ xs,
                                                       float* __restrict__ gys, const uint4* __restrict__ WB,
                                                       const float* __restrict__ tw, const float* __restrict__ itw,
                                                       Geom g, int ax, int n, long long n_lines) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int fT = frag_count(kJ, n), fI = frag_count(n, kJ);
  uint4* Th = reinterpret_cast<uint4*>(smem);    // X = T h
  uint4* Tl = Th + fT;
  uint4* Uh = Tl + fT;                           // gY = I^T gz
  uint4* Ul = Uh + fT;
  uint4* Vh = Ul + fT;                           // gh += T^T gX
  uint4* Vl = Vh + fI;
  float* sG = reinterpret_cast<float*>(Vl + fI);  // coefficient gradients gY of the CTA's lines
  float* sGX = sG + kWarps * kXStride;           // gX = Wt^T gY
  build_frags(Th, Tl, kJ, n, [&](int j, int x) { return tw[x * kJ + j]; });
  build_frags(Uh, Ul, kJ, n, [&](int j, int x) { return itw[x * kJ + j]; });
  build_frags(Vh, Vl, n, kJ, [&](int x, int j) { return tw[x * kJ + j]; });
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long l0 = (long long)blockIdx.x * kWarps; l0 < n_lines; l0 += (long long)gridDim.x * kWarps) {
    const long long li = l0 + warp;
    const bool valid = li < n_lines;
    long long base = 0, stride = 0;
    if (valid) line_of(g, ax, li, base, stride);
    const long long step = stride * kC;
    float d[2][4][4];
    if (valid) {
      line_dft_tc(h + base * kC, step, n, Th, Tl, lane, d);
      store_coef(xs + li * (kJ * kC), lane, d);
      line_dft_tc(gz + base * kC, step, n, Uh, Ul, lane, d);
      store_coef(gys + li * (kJ * kC), lane, d);
    } else {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) d[mt][nt][0] = d[mt][nt][1] = d[mt][nt][2] = d[mt][nt][3] = 0.0f;
    }
    store_coef(sG + warp * kXStride, lane, d);
    __syncthreads();
    // gX = Wt^T gY on the tensor cores (same pattern as the forward mixing)
    mix_modes_tc(sG, sGX, WB, warp, lane);
    __syncthreads();
    if (valid) line_idft_tc<true>(sGX + warp * kXStride, gh + base * kC, step, n, Vh, Vl, lane);
  }
}

// spectral weight gradient of one axis: per block (chunk of 128 lines, mode k),
// gWr[o][c] = sum gYr[o] Xr[c] + gYi[o] Xi[c], gWi[o][c] = sum gYi[o] Xr[c] - gYr[o] Xi[c].
// On the tensor cores as the real product D[(ri, o)][(ri', c)] = sum_lines
// gY[(ri, o)] X[(ri', c)] (64 x 64, K = the chunk's lines, both operands split
// hi + lo), staged in shared memory, then combined per quadrant.
constexpr int kWgradSmem = 2 * kLinesPerChunk * 64 * (int)sizeof(float);
__global__ void __launch_bounds__(kThreads) k_wgrad(const float* __restrict__ xs, const float* __restrict__ gys,
                                                    long long n_lines, float* __restrict__ partial) {
  extern __shared__ __align__(16) float wsm[];
  float* sA = wsm;                          // [line][64] = gY of mode k, (ri, o)
  float* sB = wsm + kLinesPerChunk * 64;    // [line][64] = X of mode k, (ri, c)
  const int k = blockIdx.y;
  const long long l0 = (long long)blockIdx.x * kLinesPerChunk;
  const int nl = (int)(n_lines - l0 < kLinesPerChunk ? n_lines - l0 : kLinesPerChunk);
  for (int e = threadIdx.x; e < kLinesPerChunk * 64; e += blockDim.x) {
    const int l = e >> 6, q = e & 63;
    float a = 0.0f, b = 0.0f;
    if (l < nl) {
      const long long off = (l0 + l) * (kJ * kC) + (2 * k) * kC + q;  // rows 2k (re) and 2k + 1 (im) are contiguous
      a = gys[off];
      b = xs[off];
    }
    sA[e] = a;
    sB[e] = b;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gi = lane >> 2, t = lane & 3;
  const int mt = warp >> 1, nt0 = (warp & 1) * 4;
  float d[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) d[q][0] = d[q][1] = d[q][2] = d[q][3] = 0.0f;
  for (int ks = 0; ks < kLinesPerChunk / 16; ++ks) {
    const int v = ks * 16 + 2 * t, r0 = mt * 16 + gi, r1 = r0 + 8;
    uint32_t ah[4], al[4];
    split_bf2(sA[v * 64 + r0], sA[(v + 1) * 64 + r0], ah[0], al[0]);
    split_bf2(sA[v * 64 + r1], sA[(v + 1) * 64 + r1], ah[1], al[1]);
    split_bf2(sA[(v + 8) * 64 + r0], sA[(v + 9) * 64 + r0], ah[2], al[2]);
    split_bf2(sA[(v + 8) * 64 + r1], sA[(v + 9) * 64 + r1], ah[3], al[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = (nt0 + q) * 8 + gi;
      uint32_t b0h, b0l, b1h, b1l;
      split_bf2(sB[v * 64 + c], sB[(v + 1) * 64 + c], b0h, b0l);
      split_bf2(sB[(v + 8) * 64 + c], sB[(v + 9) * 64 + c], b1h, b1l);
      mma_bf16(d[q], ah[0], ah[1], ah[2], ah[3], b0h, b1h);
      mma_bf16(d[q], ah[0], ah[1], ah[2], ah[3], b0l, b1l);
      mma_bf16(d[q], al[0], al[1], al[2], al[3], b0h, b1h);
    }
  }
  __syncthreads();
  // the 64 x 64 product into shared memory (over sA), then the complex combination
  float* D = sA;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = mt * 16 + gi, c = (nt0 + q) * 8 + 2 * t;
    D[r * 64 + c] = d[q][0];
    D[r * 64 + c + 1] = d[q][1];
    D[(r + 8) * 64 + c] = d[q][2];
    D[(r + 8) * 64 + c + 1] = d[q][3];
  }
  __syncthreads();
  float* p = partial + ((long long)blockIdx.x * kModes + k) * 2 * kC * kC;
  for (int e = threadIdx.x; e < kC * kC; e += blockDim.x) {
    const int o = e >> 5, c = e & 31;
    // quadrants: (re, re) = D[o][c], (im, im) = D[32 + o][32 + c], (im, re) = D[32 + o][c], (re, im) = D[o][32 + c]
    p[e] = D[o * 64 + c] + D[(32 + o) * 64 + 32 + c];
    p[kC * kC + e] = D[(32 + o) * 64 + c] - D[o * 64 + 32 + c];
  }
}

// Deterministic two-stage sum over partial rows: block (x, g) adds rows
// g*group .. g*group+group-1 of partial[p * stride + i] in order into
// tmp[g][i]; k_reduce_final adds the groups in order. Both use doubles.
__global__ void k_reduce_groups(const float* __restrict__ partial, int n_part, int len, int stride, int group,
                                double* __restrict__ tmp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  const int p0 = blockIdx.y * group;
  const int p1 = p0 + group < n_part ? p0 + group : n_part;
  double s = 0.0;
#pragma unroll 8
  for (int p = p0; p < p1; ++p) s += (double)partial[(long long)p * stride + i];
  tmp[(long long)blockIdx.y * len + i] = s;
}

__global__ void k_reduce_final(const double* __restrict__ tmp, int n_groups, int len, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  double s = 0.0;
#pragma unroll 8
  for (int g = 0; g < n_groups; ++g) s += tmp[(long long)g * len + i];
  out[i] = (float)s;
}

// effective head of every sample from P2, p2 and the sample's load direction u
__global__ void k_head(const __nv_bfloat16* __restrict__ wq, const float* __restrict__ su, int B,
                       float* __restrict__ head) {
  const int total = B * kHeadEff;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int b = e / kHeadEff, r = e - b * kHeadEff;
    const float* u = su + 10 * b + 1;
    float acc = 0.0f;
    if (r < kOut * kHid) {
      const int i = r / kHid, k = r - i * kHid;
#pragma unroll
      for (int j = 0; j < 9; ++j) acc = fmaf(bf(wq, kOffP2 + (long long)(9 * i + j) * kHid + k), u[j], acc);
    } else {
      const int i = r - kOut * kHid;
#pragma unroll
      for (int j = 0; j < 9; ++j) acc = fmaf(bf(wq, kOffp2 + 9 * i + j), u[j], acc);
    }
    head[e] = acc;
  }
}

// head gradient from the per-sample sums: gP2[9i + j][k] = sum_b u_bj G_b[i][k], gp2[9i + j] = sum_b u_bj Gp_b[i]
__global__ void k_head_grad(const float* __restrict__ G, const float* __restrict__ su, int B,
                            float* __restrict__ grad) {
  const int total = kHead * kHid + kHead;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int src, j;
    if (e < kHead * kHid) {
      const int row = e / kHid, k = e - row * kHid;
      j = row % 9;
      src = (row / 9) * kHid + k;
    } else {
      const int row = e - kHead * kHid;
      j = row % 9;
      src = kOut * kHid + row / 9;
    }
    double acc = 0.0;
    for (int b = 0; b < B; ++b) acc += (double)su[10 * b + 1 + j] * (double)G[(long long)b * kHeadEff + src];
    grad[kOffP2 + e] = (float)acc;
  }
}

// ---------------------------------------------------------------------------
// pointwise part of a layer: z = acc + M h + m, h_next = gelu(z) (or z)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_point_fwd(const float* __restrict__ h, const float* __restrict__ acc,
                                                        const __nv_bfloat16* __restrict__ wq, int layer,
                                                        float* __restrict__ z, float* __restrict__ hn,
                                                        long long nvox, int act) {
  // tiles of 16 voxels per warp: D[vox][o] = sum_c h[vox][c] M[o][c] on the tensor cores
  // (A = h split hi + lo, B[c][o] = M[o][c] exact in bfloat16)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gi = lane >> 2, t = lane & 3;
  uint32_t bm[4][2][2];
  float mb[4][2];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int o = nt * 8 + gi;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const __nv_bfloat162* row = reinterpret_cast<const __nv_bfloat162*>(wq + off_M(layer) + o * kC + ks * 16 + 2 * t);
      bm[nt][ks][0] = bf2_bits(row[0]);
      bm[nt][ks][1] = bf2_bits(row[4]);
    }
    mb[nt][0] = bf(wq, off_m(layer) + nt * 8 + 2 * t);
    mb[nt][1] = bf(wq, off_m(layer) + nt * 8 + 2 * t + 1);
  }
  const long long tiles = (nvox + 15) / 16;
  for (long long tile = (long long)blockIdx.x * kWarps + warp; tile < tiles; tile += (long long)gridDim.x * kWarps) {
    const long long va = tile * 16 + gi, vb = va + 8;
    const bool oka = va < nvox, okb = vb < nvox;
    uint32_t ah[2][4], al[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const int c = ks * 16 + 2 * t;
      const float2 z2 = make_float2(0.0f, 0.0f);
      const float2 p0 = oka ? *reinterpret_cast<const float2*>(h + va * kC + c) : z2;
      const float2 p1 = okb ? *reinterpret_cast<const float2*>(h + vb * kC + c) : z2;
      const float2 p2 = oka ? *reinterpret_cast<const float2*>(h + va * kC + c + 8) : z2;
      const float2 p3 = okb ? *reinterpret_cast<const float2*>(h + vb * kC + c + 8) : z2;
      split_bf2(p0.x, p0.y, ah[ks][0], al[ks][0]);
      split_bf2(p1.x, p1.y, ah[ks][1], al[ks][1]);
      split_bf2(p2.x, p2.y, ah[ks][2], al[ks][2]);
      split_bf2(p3.x, p3.y, ah[ks][3], al[ks][3]);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        mma_bf16(d, ah[ks][0], ah[ks][1], ah[ks][2], ah[ks][3], bm[nt][ks][0], bm[nt][ks][1]);
        mma_bf16(d, al[ks][0], al[ks][1], al[ks][2], al[ks][3], bm[nt][ks][0], bm[nt][ks][1]);
      }
      const int o = nt * 8 + 2 * t;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const long long v = r ? vb : va;
        if (r ? !okb : !oka) continue;
        const long long e = v * kC + o;
        const float2 ac = *reinterpret_cast<const float2*>(acc + e);
        const float s0 = d[2 * r] + mb[nt][0] + ac.x, s1 = d[2 * r + 1] + mb[nt][1] + ac.y;
        if (z) *reinterpret_cast<float2*>(z + e) = make_float2(s0, s1);
        *reinterpret_cast<float2*>(hn + e) = act ? make_float2(gelu(s0), gelu(s1)) : make_float2(s0, s1);
      }
    }
  }
}

// pointwise part, backward, tiles of 16 voxels per warp on the tensor cores:
// gz = gn * gelu'(z) (or gn), gh = M^T gz (A = gz split, B[o][c] = M[o][c]
// exact), and the per-warp partial sums gM[o][c] = sum_vox gz[o] h[c] (A =
// gz^T, B = h, both split; K = the tile's voxels) and gm[o] = sum_vox gz[o]
__global__ void __launch_bounds__(kThreads) k_point_bwd(const float* __restrict__ gn, const float* __restrict__ z,
                                                        const float* __restrict__ h,
                                                        const __nv_bfloat16* __restrict__ wq, int layer,
                                                        float* __restrict__ gz, float* __restrict__ gh,
                                                        float* __restrict__ partial, long long nvox) {
  __shared__ __align__(16) float sg[kWarps][16 * kC];
  __shared__ __align__(16) float sh[kWarps][16 * kC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gi = lane >> 2, t = lane & 3;
  float* G = sg[warp];
  float* Hs = sh[warp];
  // B fragments of M for gh = gz M: B[k = o][n = c] = M[o][c]
  uint32_t bm[4][2][2];
  {
    const __nv_bfloat16* M = wq + off_M(layer);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const int c = nt * 8 + gi, o = ks * 16 + 2 * t;
        bm[nt][ks][0] = bf2_bits(__halves2bfloat162(M[o * kC + c], M[(o + 1) * kC + c]));
        bm[nt][ks][1] = bf2_bits(__halves2bfloat162(M[(o + 8) * kC + c], M[(o + 9) * kC + c]));
      }
  }
  float gM[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) gM[mt][nt][0] = gM[mt][nt][1] = gM[mt][nt][2] = gM[mt][nt][3] = 0.0f;
  float gm = 0.0f;
  const long long tiles = (nvox + 15) / 16;
  for (long long tile = (long long)blockIdx.x * kWarps + warp; tile < tiles; tile += (long long)gridDim.x * kWarps) {
    const long long v0 = tile * 16;
    // gz and h of the tile into shared memory (zero past the end), gz to global
    for (int i = 0; i < 16; ++i) {
      float gv = 0.0f, hv = 0.0f;
      if (v0 + i < nvox) {
        const long long e = (v0 + i) * kC + lane;
        gv = gn[e];
        if (z) gv *= gelu_d(z[e]);
        gz[e] = gv;
        hv = h[e];
      }
      G[i * kC + lane] = gv;
      Hs[i * kC + lane] = hv;
      gm += gv;
    }
    __syncwarp();
    // gh[vox][c] = sum_o gz[vox][o] M[o][c]
    uint32_t ah[2][4], al[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const int o = ks * 16 + 2 * t;
      split_bf2(G[gi * kC + o], G[gi * kC + o + 1], ah[ks][0], al[ks][0]);
      split_bf2(G[(gi + 8) * kC + o], G[(gi + 8) * kC + o + 1], ah[ks][1], al[ks][1]);
      split_bf2(G[gi * kC + o + 8], G[gi * kC + o + 9], ah[ks][2], al[ks][2]);
      split_bf2(G[(gi + 8) * kC + o + 8], G[(gi + 8) * kC + o + 9], ah[ks][3], al[ks][3]);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        mma_bf16(d, ah[ks][0], ah[ks][1], ah[ks][2], ah[ks][3], bm[nt][ks][0], bm[nt][ks][1]);
        mma_bf16(d, al[ks][0], al[ks][1], al[ks][2], al[ks][3], bm[nt][ks][0], bm[nt][ks][1]);
      }
      const int c = nt * 8 + 2 * t;
      if (v0 + gi < nvox) *reinterpret_cast<float2*>(gh + (v0 + gi) * kC + c) = make_float2(d[0], d[1]);
      if (v0 + gi + 8 < nvox) *reinterpret_cast<float2*>(gh + (v0 + gi + 8) * kC + c) = make_float2(d[2], d[3]);
    }
    // gM[o][c] += sum over the tile's voxels of gz[vox][o] h[vox][c] (K = 16 voxels)
    uint32_t gth[2][4], gtl[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int o0 = mt * 16 + gi, o1 = o0 + 8, v = 2 * t;
      split_bf2(G[v * kC + o0], G[(v + 1) * kC + o0], gth[mt][0], gtl[mt][0]);
      split_bf2(G[v * kC + o1], G[(v + 1) * kC + o1], gth[mt][1], gtl[mt][1]);
      split_bf2(G[(v + 8) * kC + o0], G[(v + 9) * kC + o0], gth[mt][2], gtl[mt][2]);
      split_bf2(G[(v + 8) * kC + o1], G[(v + 9) * kC + o1], gth[mt][3], gtl[mt][3]);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int c = nt * 8 + gi, v = 2 * t;
      uint32_t b0h, b0l, b1h, b1l;
      split_bf2(Hs[v * kC + c], Hs[(v + 1) * kC + c], b0h, b0l);
      split_bf2(Hs[(v + 8) * kC + c], Hs[(v + 9) * kC + c], b1h, b1l);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        mma_bf16(gM[mt][nt], gth[mt][0], gth[mt][1], gth[mt][2], gth[mt][3], b0h, b1h);
        mma_bf16(gM[mt][nt], gth[mt][0], gth[mt][1], gth[mt][2], gth[mt][3], b0l, b1l);
        mma_bf16(gM[mt][nt], gtl[mt][0], gtl[mt][1], gtl[mt][2], gtl[mt][3], b0h, b1h);
      }
    }
    __syncwarp();
  }
  float* p = partial + ((long long)blockIdx.x * kWarps + warp) * kPointLen;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int o = mt * 16 + gi, c = nt * 8 + 2 * t;
      p[o * kC + c] = gM[mt][nt][0];
      p[o * kC + c + 1] = gM[mt][nt][1];
      p[(o + 8) * kC + c] = gM[mt][nt][2];
      p[(o + 8) * kC + c + 1] = gM[mt][nt][3];
    }
  p[kC * kC + lane] = gm;
}

// ---------------------------------------------------------------------------
// projection: q = P2 gelu(P1 h4 + p1) + p2, written [9][N] per sample; with
// targets, the per-block partial sums of (q - target)^2
// ---------------------------------------------------------------------------
struct ProjSmem {
  float P1[kHid * kC];
  float p1[kHid];
  float P2[kOut * kHid];
  float p2[kOut];
};

__device__ __forceinline__ void load_proj(ProjSmem& s, const __nv_bfloat16* wq, const float* head) {
  for (int i = threadIdx.x; i < kHid * kC; i += blockDim.x) s.P1[i] = bf(wq, kOffP1 + i);
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) s.p1[i] = bf(wq, kOffp1 + i);
  for (int i = threadIdx.x; i < kOut * kHid; i += blockDim.x) s.P2[i] = head[i];
  for (int i = threadIdx.x; i < kOut; i += blockDim.x) s.p2[i] = head[kOut * kHid + i];
  __syncthreads();
}

__device__ __forceinline__ float hidden_pre(const ProjSmem& s, int j, const float hv[kC]) {
  float pre = s.p1[j];
  const float4* r = reinterpret_cast<const float4*>(&s.P1[j * kC]);
#pragma unroll
  for (int q = 0; q < kC / 4; ++q) {
    const float4 w = r[q];
    pre = fmaf(w.x, hv[4 * q], pre);
    pre = fmaf(w.y, hv[4 * q + 1], pre);
    pre = fmaf(w.z, hv[4 * q + 2], pre);
    pre = fmaf(w.w, hv[4 * q + 3], pre);
  }
  return pre;
}

__device__ __forceinline__ void load_h(const float* h4, long long vox, float hv[kC]) {
  const float4* r = reinterpret_cast<const float4*>(h4 + vox * kC);
#pragma unroll
  for (int q = 0; q < kC / 4; ++q) {
    const float4 v = r[q];
    hv[4 * q] = v.x;
    hv[4 * q + 1] = v.y;
    hv[4 * q + 2] = v.z;
    hv[4 * q + 3] = v.w;
  }
}

__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double red[kWarps];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kWarps; ++w) s += red[w];
  return s;
}

// Shared memory of the tensor-core projection: B fragments of P1 (hidden =
// h P1^T, exact bfloat16) and of the per-sample effective head P2u (q = t
// P2u^T, float32 as bfloat16 hi + lo), with the two bias vectors.
struct ProjFrag {
  uint2 P1[16 * 2 * 32];   // [n-tile of hidden units][k-step of channels][lane]
  uint2 P2h[2 * 8 * 32];   // [n-tile of outputs][k-step of hidden units][lane], hi terms
  uint2 P2l[2 * 8 * 32];   // lo terms
  float p1[kHid];
  float p2[16];
};

__device__ __forceinline__ void load_proj_frag(ProjFrag& s, const __nv_bfloat16* __restrict__ wq,
                                               const float* __restrict__ head) {
  for (int e = threadIdx.x; e < 16 * 2 * 32; e += blockDim.x) {
    const int lane = e & 31, ks = (e >> 5) & 1, nt = e >> 6, gi = lane >> 2, t = lane & 3;
    const __nv_bfloat162* row =
        reinterpret_cast<const __nv_bfloat162*>(wq + kOffP1 + (nt * 8 + gi) * kC + ks * 16 + 2 * t);
    s.P1[e] = make_uint2(bf2_bits(row[0]), bf2_bits(row[4]));
  }
  for (int e = threadIdx.x; e < 2 * 8 * 32; e += blockDim.x) {
    const int lane = e & 31, ks = (e >> 5) & 7, nt = e >> 8, gi = lane >> 2, t = lane & 3;
    const int i = nt * 8 + gi, j = ks * 16 + 2 * t;
    float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (i < kOut) {
      v[0] = head[i * kHid + j];
      v[1] = head[i * kHid + j + 1];
      v[2] = head[i * kHid + j + 8];
      v[3] = head[i * kHid + j + 9];
    }
    uint32_t h0, l0, h1, l1;
    split_bf2(v[0], v[1], h0, l0);
    split_bf2(v[2], v[3], h1, l1);
    s.P2h[e] = make_uint2(h0, h1);
    s.P2l[e] = make_uint2(l0, l1);
  }
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) s.p1[i] = bf(wq, kOffp1 + i);
  for (int i = threadIdx.x; i < 16; i += blockDim.x) s.p2[i] = i < kOut ? head[kOut * kHid + i] : 0.0f;
  __syncthreads();
}

// A fragments (hi, lo) of the 16 voxels va = tile*16 + g and vb = va + 8 of h4, both k-steps
__device__ __forceinline__ void load_h_frag(const float* __restrict__ h4, long long va, long long vb, bool oka,
                                            bool okb, int t, uint32_t (&ah)[2][4], uint32_t (&al)[2][4]) {
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    const int c = ks * 16 + 2 * t;
    const float2 z2 = make_float2(0.0f, 0.0f);
    const float2 p0 = oka ? *reinterpret_cast<const float2*>(h4 + va * kC + c) : z2;
    const float2 p1 = okb ? *reinterpret_cast<const float2*>(h4 + vb * kC + c) : z2;
    const float2 p2 = oka ? *reinterpret_cast<const float2*>(h4 + va * kC + c + 8) : z2;
    const float2 p3 = okb ? *reinterpret_cast<const float2*>(h4 + vb * kC + c + 8) : z2;
    split_bf2(p0.x, p0.y, ah[ks][0], al[ks][0]);
    split_bf2(p1.x, p1.y, ah[ks][1], al[ks][1]);
    split_bf2(p2.x, p2.y, ah[ks][2], al[ks][2]);
    split_bf2(p3.x, p3.y, ah[ks][3], al[ks][3]);
  }
}

// pre-activations of hidden units 16 kc .. 16 kc + 15 of the tile (two n-tiles of D = h P1^T + p1)
__device__ __forceinline__ void hidden_chunk(const ProjFrag& s, int kc, int lane, const uint32_t (&ah)[2][4],
                                             const uint32_t (&al)[2][4], float (&pre)[2][4]) {
  const int t = lane & 3;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int nt = 2 * kc + q;
    float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const uint2 b = s.P1[(nt * 2 + ks) * 32 + lane];
      mma_bf16(d, ah[ks][0], ah[ks][1], ah[ks][2], ah[ks][3], b.x, b.y);
      mma_bf16(d, al[ks][0], al[ks][1], al[ks][2], al[ks][3], b.x, b.y);
    }
    const float b0 = s.p1[nt * 8 + 2 * t], b1 = s.p1[nt * 8 + 2 * t + 1];
    pre[q][0] = d[0] + b0;
    pre[q][1] = d[1] + b1;
    pre[q][2] = d[2] + b0;
    pre[q][3] = d[3] + b1;
  }
}

// q[2][4] (D fragments of outputs 0..7 and 8..15 of the tile) = P2u gelu(P1 h + p1) + p2u
__device__ __forceinline__ void proj_q_tc(const ProjFrag& s, int lane, const uint32_t (&ah)[2][4],
                                          const uint32_t (&al)[2][4], float (&q)[2][4]) {
  const int t = lane & 3;
#pragma unroll
  for (int n2 = 0; n2 < 2; ++n2) {
    q[n2][0] = q[n2][2] = s.p2[n2 * 8 + 2 * t];
    q[n2][1] = q[n2][3] = s.p2[n2 * 8 + 2 * t + 1];
  }
  for (int kc = 0; kc < kHid / 16; ++kc) {
    float pre[2][4];
    hidden_chunk(s, kc, lane, ah, al, pre);
    // A fragment of t = gelu(pre) for k-step kc of the second product
    uint32_t th[4], tl[4];
    split_bf2(gelu(pre[0][0]), gelu(pre[0][1]), th[0], tl[0]);
    split_bf2(gelu(pre[0][2]), gelu(pre[0][3]), th[1], tl[1]);
    split_bf2(gelu(pre[1][0]), gelu(pre[1][1]), th[2], tl[2]);
    split_bf2(gelu(pre[1][2]), gelu(pre[1][3]), th[3], tl[3]);
#pragma unroll
    for (int n2 = 0; n2 < 2; ++n2) {
      const uint2 bh = s.P2h[(n2 * 8 + kc) * 32 + lane], bl = s.P2l[(n2 * 8 + kc) * 32 + lane];
      mma_bf16(q[n2], th[0], th[1], th[2], th[3], bh.x, bh.y);
      mma_bf16(q[n2], tl[0], tl[1], tl[2], tl[3], bh.x, bh.y);
      mma_bf16(q[n2], th[0], th[1], th[2], th[3], bl.x, bl.y);
    }
  }
}

// ---------------------------------------------------------------------------
// 5th-generation tensor-core (tcgen05) helpers: shared-memory operands in the
// canonical K-major layout without swizzle (core matrices of 8 rows x 16
// bytes; LBO = byte step between core matrices along K, SBO = between groups
// of 8 rows), fp32 accumulators in tensor memory (TMEM), one thread issuing
// the MMAs and an mbarrier signalled by tcgen05.commit. Every wait is bounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_smem_desc(const void* base, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((smem_u32(base) >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; base offset 0, relative LBO, no swizzle
  return d;
}
// kind::f16 instruction descriptor: bf16 A and B, both K-major, f32 accumulator, M x N
constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
// wait for the completion of phase `parity` of the mbarrier, for at most ~2^31 clock ticks; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1LL << 31)) return false;
  }
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 16 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
// byte offset of element (row r, k) in a K-major no-swizzle operand with rows of K elements (bf16)
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared memory of the tcgen05 projection: operand tiles (bf16, K-major) and the biases
constexpr int kT5 = 128;  // threads = voxels per tile = accumulator rows
struct ProjT5 {
  __nv_bfloat16 Ah[kT5 * kC], Al[kT5 * kC];     // h tile, hi and lo terms      (128 x 32)
  __nv_bfloat16 B1[kHid * kC];                  // P1 [hidden][channel]          (128 x 32)
  __nv_bfloat16 Th[kT5 * kHid], Tl[kT5 * kHid]; // gelu(hidden), hi and lo       (128 x 128)
  __nv_bfloat16 B2h[16 * kHid], B2l[16 * kHid]; // effective head [output][hidden] (16 x 128)
  float p1[kHid];
  float p2[16];
  uint64_t mbar;
  uint32_t tmem;
  double red[kT5 / 32];
};

// projection on the 5th-generation tensor cores: tiles of 128 voxels, one
// thread per voxel. hidden = h P1^T (M 128, N 128, K 32; h as hi + lo, P1 exact)
// accumulates in TMEM columns 0..127; t = gelu(hidden + p1) goes back to shared
// memory (hi + lo) as the A operand of q = t P2u^T (M 128, N 16, K 128; P2u as
// hi + lo, three products) in TMEM columns 128..143. q written [9][N] when qo
// is given, and the per-block partial sums of (q - target)^2. A wait that runs
// out sets *err and ends the kernel after releasing its TMEM.
__global__ void __launch_bounds__(kT5) k_proj_fwd(const float* __restrict__ h4, const __nv_bfloat16* __restrict__ wq,
                                                  const float* __restrict__ head, float* __restrict__ qo,
                                                  const float* __restrict__ target, long long N,
                                                  double* __restrict__ loss_part, int* __restrict__ err,
                                                  int skip_mma) {
  extern __shared__ __align__(128) unsigned char t5raw[];
  ProjT5& s = *reinterpret_cast<ProjT5*>(t5raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // constant operands: P1 (exact), P2u split, biases
  for (int e = tid; e < kHid * kC; e += kT5) {
    const int r = e / kC, k = e % kC;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(s.B1) + kmajor_off(r, k, kC)) =
        wq[kOffP1 + e];
  }
  for (int e = tid; e < 16 * kHid; e += kT5) {
    const int i = e / kHid, k = e % kHid;
    const float v = i < kOut ? head[i * kHid + k] : 0.0f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(s.B2h) + kmajor_off(i, k, kHid)) = hi;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(s.B2l) + kmajor_off(i, k, kHid)) = lo;
  }
  for (int i = tid; i < kHid; i += kT5) s.p1[i] = bf(wq, kOffp1 + i);
  if (tid < 16) s.p2[tid] = tid < kOut ? head[kOut * kHid + tid] : 0.0f;
  if (tid == 0) mbar_init(&s.mbar, 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s.tmem;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;  // this warp's TMEM lanes
  constexpr uint32_t id1 = umma_idesc_bf16(128, 128), id2 = umma_idesc_bf16(128, 16);
  uint32_t phase = 0;
  bool ok = true;
  double loss = 0.0;
  const long long tiles = (N + kT5 - 1) / kT5;
  for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
    const long long v = tile * kT5 + tid;
    const bool valid = v < N;
    // A operand of the first product: this thread's voxel row, split
#pragma unroll
    for (int q = 0; q < kC / 8; ++q) {
      float x[8];
      if (valid) {
        const float4 a = *reinterpret_cast<const float4*>(h4 + v * kC + 8 * q);
        const float4 b = *reinterpret_cast<const float4*>(h4 + v * kC + 8 * q + 4);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = 0.0f;
      }
      uint4 hi, lo;
      split_bf2(x[0], x[1], hi.x, lo.x);
      split_bf2(x[2], x[3], hi.y, lo.y);
      split_bf2(x[4], x[5], hi.z, lo.z);
      split_bf2(x[6], x[7], hi.w, lo.w);
      *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(s.Ah) + kmajor_off(tid, 8 * q, kC)) = hi;
      *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(s.Al) + kmajor_off(tid, 8 * q, kC)) = lo;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && !skip_mma) {
#pragma unroll
      for (int ks = 0; ks < kC / 16; ++ks) {
        const uint64_t b = umma_smem_desc(reinterpret_cast<unsigned char*>(s.B1) + ks * 256, 128, (kC / 8) * 128);
        umma_bf16(tmem, umma_smem_desc(reinterpret_cast<unsigned char*>(s.Ah) + ks * 256, 128, (kC / 8) * 128), b, id1,
                  ks > 0);
        umma_bf16(tmem, umma_smem_desc(reinterpret_cast<unsigned char*>(s.Al) + ks * 256, 128, (kC / 8) * 128), b, id1,
                  1);
      }
      umma_commit(&s.mbar);
    }
    ok = mbar_wait(&s.mbar, phase);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    tc_fence_after();
    // t = gelu(hidden + p1) into the A operand of the second product
#pragma unroll
    for (int c16 = 0; c16 < kHid / 16; ++c16) {
      float d[16];
      tmem_ld16(tmem + lane_base + (uint32_t)(c16 * 16), d);
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint4 hi, lo;
        const int k0 = c16 * 16 + half * 8;
        float t8[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) t8[e] = gelu(d[half * 8 + e] + s.p1[k0 + e]);
        split_bf2(t8[0], t8[1], hi.x, lo.x);
        split_bf2(t8[2], t8[3], hi.y, lo.y);
        split_bf2(t8[4], t8[5], hi.z, lo.z);
        split_bf2(t8[6], t8[7], hi.w, lo.w);
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(s.Th) + kmajor_off(tid, k0, kHid)) = hi;
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(s.Tl) + kmajor_off(tid, k0, kHid)) = lo;
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && !skip_mma) {
      constexpr uint32_t sbo = (kHid / 8) * 128;
      for (int ks = 0; ks < kHid / 16; ++ks) {
        const uint64_t th = umma_smem_desc(reinterpret_cast<unsigned char*>(s.Th) + ks * 256, 128, sbo);
        const uint64_t tl = umma_smem_desc(reinterpret_cast<unsigned char*>(s.Tl) + ks * 256, 128, sbo);
        const uint64_t bh = umma_smem_desc(reinterpret_cast<unsigned char*>(s.B2h) + ks * 256, 128, sbo);
        const uint64_t bl = umma_smem_desc(reinterpret_cast<unsigned char*>(s.B2l) + ks * 256, 128, sbo);
        umma_bf16(tmem + 128, th, bh, id2, ks > 0);
        umma_bf16(tmem + 128, tl, bh, id2, 1);
        umma_bf16(tmem + 128, th, bl, id2, 1);
      }
      umma_commit(&s.mbar);
    }
    ok = mbar_wait(&s.mbar, phase);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    tc_fence_after();
    float q[16];
    tmem_ld16(tmem + lane_base + 128u, q);
    if (valid) {
#pragma unroll
      for (int i = 0; i < kOut; ++i) {
        const float qi = q[i] + s.p2[i];
        if (qo) qo[i * N + v] = qi;
        if (target) {
          const double dd = (double)qi - (double)target[i * N + v];
          loss += dd * dd;
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // every thread has read TMEM and the operands may be rewritten
    tc_fence_after();
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  if (loss_part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) s.red[warp] = loss;
    __syncthreads();
    if (tid == 0) loss_part[blockIdx.x] = s.red[0] + s.red[1] + s.red[2] + s.red[3];
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

// B fragments of the backward products: gt = gq P2u (B[i][j] = P2u[i][j],
// float32 as hi + lo) and gh4 = gp P1 (B[j][c] = P1[j][c], exact)
struct ProjFragBwd {
  uint2 P2Th[8 * 2 * 32];  // [k-chunk of hidden units][n-tile][lane]
  uint2 P2Tl[8 * 2 * 32];
  uint2 P1T[8 * 4 * 32];   // [k-chunk of hidden units][n-tile of channels][lane]
};

__device__ __forceinline__ void load_proj_frag_bwd(ProjFragBwd& s, const __nv_bfloat16* __restrict__ wq,
                                                   const float* __restrict__ head) {
  for (int e = threadIdx.x; e < 8 * 2 * 32; e += blockDim.x) {
    const int lane = e & 31, nt = (e >> 5) & 1, kc = e >> 6, gi = lane >> 2, t = lane & 3;
    const int j = kc * 16 + nt * 8 + gi, i0 = 2 * t;
    const float v0 = i0 < kOut ? head[i0 * kHid + j] : 0.0f;
    const float v1 = i0 + 1 < kOut ? head[(i0 + 1) * kHid + j] : 0.0f;
    const float v2 = i0 + 8 < kOut ? head[(i0 + 8) * kHid + j] : 0.0f;
    const float v3 = i0 + 9 < kOut ? head[(i0 + 9) * kHid + j] : 0.0f;
    uint32_t h0, l0, h1, l1;
    split_bf2(v0, v1, h0, l0);
    split_bf2(v2, v3, h1, l1);
    s.P2Th[e] = make_uint2(h0, h1);
    s.P2Tl[e] = make_uint2(l0, l1);
  }
  for (int e = threadIdx.x; e < 8 * 4 * 32; e += blockDim.x) {
    const int lane = e & 31, nt = (e >> 5) & 3, kc = e >> 7, gi = lane >> 2, t = lane & 3;
    const int c = nt * 8 + gi, j = kc * 16 + 2 * t;
    const __nv_bfloat16* P1 = wq + kOffP1;
    const __nv_bfloat162 b0 = __halves2bfloat162(P1[j * kC + c], P1[(j + 1) * kC + c]);
    const __nv_bfloat162 b1 = __halves2bfloat162(P1[(j + 8) * kC + c], P1[(j + 9) * kC + c]);
    s.P1T[e] = make_uint2(bf2_bits(b0), bf2_bits(b1));
  }
  __syncthreads();
}

// projection backward on the tensor cores, tiles of 16 voxels per warp:
// gq = scale (q - target) (kept [vox][9]), gh4 = P1^T (gelu'(pre) . P2u^T gq),
// and the per-block partial sums of (q - target)^2
__global__ void __launch_bounds__(kThreads, 2) k_proj_bwd_a(const float* __restrict__ h4,
                                                         const __nv_bfloat16* __restrict__ wq,
                                                         const float* __restrict__ head,
                                                         const float* __restrict__ target, long long N, float scale,
                                                         float* __restrict__ gq_out, float* __restrict__ gh4,
                                                         double* __restrict__ loss_part) {
  __shared__ __align__(16) ProjFrag s;
  __shared__ __align__(16) ProjFragBwd sb;
  load_proj_frag(s, wq, head);
  load_proj_frag_bwd(sb, wq, head);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gi = lane >> 2, t = lane & 3;
  double loss = 0.0;
  const long long tiles = (N + 15) / 16;
  for (long long tile = (long long)blockIdx.x * kWarps + warp; tile < tiles; tile += (long long)gridDim.x * kWarps) {
    const long long va = tile * 16 + gi, vb = va + 8;
    const bool oka = va < N, okb = vb < N;
    uint32_t ah[2][4], al[2][4];
    load_h_frag(h4, va, vb, oka, okb, t, ah, al);
    float q[2][4];
    proj_q_tc(s, lane, ah, al, q);
    // q -> gq (zero outside the 9 outputs and the grid)
#pragma unroll
    for (int n2 = 0; n2 < 2; ++n2)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = n2 * 8 + 2 * t + (e & 1);
        const long long v = (e < 2) ? va : vb;
        float gv = 0.0f;
        if (i < kOut && (e < 2 ? oka : okb)) {
          const float d = q[n2][e] - target[i * N + v];
          loss += (double)d * (double)d;
          gv = scale * d;
          gq_out[v * kOut + i] = gv;
        }
        q[n2][e] = gv;
      }
    uint32_t gh_[4], gl_[4];
    split_bf2(q[0][0], q[0][1], gh_[0], gl_[0]);
    split_bf2(q[0][2], q[0][3], gh_[1], gl_[1]);
    split_bf2(q[1][0], q[1][1], gh_[2], gl_[2]);
    split_bf2(q[1][2], q[1][3], gh_[3], gl_[3]);
    float g4[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) g4[nt][0] = g4[nt][1] = g4[nt][2] = g4[nt][3] = 0.0f;
    for (int kc = 0; kc < kHid / 16; ++kc) {
      float pre[2][4];
      hidden_chunk(s, kc, lane, ah, al, pre);
      // gt = gq P2u over this chunk's 16 hidden units, then gp = gt gelu'(pre)
      float gp[2][4];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const uint2 bh = sb.P2Th[(kc * 2 + nt) * 32 + lane], bl = sb.P2Tl[(kc * 2 + nt) * 32 + lane];
        mma_bf16(d, gh_[0], gh_[1], gh_[2], gh_[3], bh.x, bh.y);
        mma_bf16(d, gl_[0], gl_[1], gl_[2], gl_[3], bh.x, bh.y);
        mma_bf16(d, gh_[0], gh_[1], gh_[2], gh_[3], bl.x, bl.y);
#pragma unroll
        for (int e = 0; e < 4; ++e) gp[nt][e] = d[e] * gelu_d(pre[nt][e]);
      }
      uint32_t ph[4], pl[4];
      split_bf2(gp[0][0], gp[0][1], ph[0], pl[0]);
      split_bf2(gp[0][2], gp[0][3], ph[1], pl[1]);
      split_bf2(gp[1][0], gp[1][1], ph[2], pl[2]);
      split_bf2(gp[1][2], gp[1][3], ph[3], pl[3]);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const uint2 b = sb.P1T[(kc * 4 + nt) * 32 + lane];
        mma_bf16(g4[nt], ph[0], ph[1], ph[2], ph[3], b.x, b.y);
        mma_bf16(g4[nt], pl[0], pl[1], pl[2], pl[3], b.x, b.y);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int c = nt * 8 + 2 * t;
      if (oka) *reinterpret_cast<float2*>(gh4 + va * kC + c) = make_float2(g4[nt][0], g4[nt][1]);
      if (okb) *reinterpret_cast<float2*>(gh4 + vb * kC + c) = make_float2(g4[nt][2], g4[nt][3]);
    }
  }
  const double tot = block_sum_d(loss);
  if (threadIdx.x == 0) loss_part[blockIdx.x] = tot;
}

// projection weight gradient of one sample on the tensor cores. Warp w owns
// the hidden units 16w .. 16w + 15; for every tile of 16 voxels of the CTA it
// recomputes pre = P1 h + p1 and gp = (P2u^T gq) gelu'(pre) for its units
// (as k_proj_bwd_a does) and accumulates gP1[j][c] += sum_vox gp[j] h[c] (A =
// gp^T, B = h), gp1[j] += sum gp, G[i][j] += sum_vox gq[i] gelu(pre)[j] (A =
// gq^T, B = t) and Gp[i] += sum gq[i], in a fixed order. Per-block rows of
// kProjRow entries (P1, p1, G, Gp).
struct ProjFragB2 {
  uint2 P2Th[8 * 2 * 32];
  uint2 P2Tl[8 * 2 * 32];
};
__global__ void __launch_bounds__(kThreads) k_proj_bwd_b(const float* __restrict__ h4, const float* __restrict__ gq,
                                                         const __nv_bfloat16* __restrict__ wq,
                                                         const float* __restrict__ head, long long nvox,
                                                         float* __restrict__ partial) {
  __shared__ __align__(16) ProjFrag s;
  __shared__ __align__(16) ProjFragB2 sb;
  __shared__ __align__(16) float sH[16 * kC];       // the tile's h
  __shared__ __align__(16) float sQ[16 * 16];       // the tile's gq (outputs 9..15 zero)
  __shared__ __align__(16) float sGP[kWarps][16 * 16];  // per warp: gp[vox][unit]
  __shared__ __align__(16) float sT[kWarps][16 * 16];   // per warp: gelu(pre)[vox][unit]
  load_proj_frag(s, wq, head);
  for (int e = threadIdx.x; e < 8 * 2 * 32; e += blockDim.x) {
    const int lane = e & 31, nt = (e >> 5) & 1, kc = e >> 6, gi = lane >> 2, t = lane & 3;
    const int j = kc * 16 + nt * 8 + gi, i0 = 2 * t;
    const float v0 = i0 < kOut ? head[i0 * kHid + j] : 0.0f;
    const float v1 = i0 + 1 < kOut ? head[(i0 + 1) * kHid + j] : 0.0f;
    const float v2 = i0 + 8 < kOut ? head[(i0 + 8) * kHid + j] : 0.0f;
    const float v3 = i0 + 9 < kOut ? head[(i0 + 9) * kHid + j] : 0.0f;
    uint32_t h0, l0, h1, l1;
    split_bf2(v0, v1, h0, l0);
    split_bf2(v2, v3, h1, l1);
    sb.P2Th[e] = make_uint2(h0, h1);
    sb.P2Tl[e] = make_uint2(l0, l1);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gi = lane >> 2, t = lane & 3;
  const int kc = warp;
  float* GP = sGP[warp];
  float* T = sT[warp];
  float a1[4][4], a2[2][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) a1[q][0] = a1[q][1] = a1[q][2] = a1[q][3] = 0.0f;
#pragma unroll
  for (int q = 0; q < 2; ++q) a2[q][0] = a2[q][1] = a2[q][2] = a2[q][3] = 0.0f;
  float ap1 = 0.0f, ap2 = 0.0f;
  const long long tiles = (nvox + 15) / 16;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long v0 = tile * 16;
    for (int e = threadIdx.x; e < 16 * kC; e += blockDim.x) sH[e] = v0 + e / kC < nvox ? h4[v0 * kC + e] : 0.0f;
    for (int e = threadIdx.x; e < 16 * 16; e += blockDim.x) {
      const int v = e >> 4, i = e & 15;
      sQ[e] = (i < kOut && v0 + v < nvox) ? gq[(v0 + v) * kOut + i] : 0.0f;
    }
    __syncthreads();
    // h fragments (rows = voxels g, g + 8), pre and t of this warp's 16 units
    uint32_t ah[2][4], al[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const int c = ks * 16 + 2 * t;
      split_bf2(sH[gi * kC + c], sH[gi * kC + c + 1], ah[ks][0], al[ks][0]);
      split_bf2(sH[(gi + 8) * kC + c], sH[(gi + 8) * kC + c + 1], ah[ks][1], al[ks][1]);
      split_bf2(sH[gi * kC + c + 8], sH[gi * kC + c + 9], ah[ks][2], al[ks][2]);
      split_bf2(sH[(gi + 8) * kC + c + 8], sH[(gi + 8) * kC + c + 9], ah[ks][3], al[ks][3]);
    }
    float pre[2][4];
    hidden_chunk(s, kc, lane, ah, al, pre);
    // gt = gq P2u over the units (A = gq [vox][i], K = 16 outputs)
    uint32_t qh[4], ql[4];
    split_bf2(sQ[gi * 16 + 2 * t], sQ[gi * 16 + 2 * t + 1], qh[0], ql[0]);
    split_bf2(sQ[(gi + 8) * 16 + 2 * t], sQ[(gi + 8) * 16 + 2 * t + 1], qh[1], ql[1]);
    split_bf2(sQ[gi * 16 + 2 * t + 8], sQ[gi * 16 + 2 * t + 9], qh[2], ql[2]);
    split_bf2(sQ[(gi + 8) * 16 + 2 * t + 8], sQ[(gi + 8) * 16 + 2 * t + 9], qh[3], ql[3]);
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      const uint2 bh = sb.P2Th[(kc * 2 + nt) * 32 + lane], bl = sb.P2Tl[(kc * 2 + nt) * 32 + lane];
      mma_bf16(d, qh[0], qh[1], qh[2], qh[3], bh.x, bh.y);
      mma_bf16(d, ql[0], ql[1], ql[2], ql[3], bh.x, bh.y);
      mma_bf16(d, qh[0], qh[1], qh[2], qh[3], bl.x, bl.y);
      // D rows vox g / g + 8, columns units nt*8 + 2t, + 1 (local to the warp's 16)
      const int u = nt * 8 + 2 * t;
      GP[gi * 16 + u] = d[0] * gelu_d(pre[nt][0]);
      GP[gi * 16 + u + 1] = d[1] * gelu_d(pre[nt][1]);
      GP[(gi + 8) * 16 + u] = d[2] * gelu_d(pre[nt][2]);
      GP[(gi + 8) * 16 + u + 1] = d[3] * gelu_d(pre[nt][3]);
      T[gi * 16 + u] = gelu(pre[nt][0]);
      T[gi * 16 + u + 1] = gelu(pre[nt][1]);
      T[(gi + 8) * 16 + u] = gelu(pre[nt][2]);
      T[(gi + 8) * 16 + u + 1] = gelu(pre[nt][3]);
    }
    __syncwarp();
    // gP1[unit][c] += sum_vox gp[vox][unit] h[vox][c]: A = gp^T (rows = units), B = h (K = voxels)
    uint32_t ph[4], pl[4];
    split_bf2(GP[(2 * t) * 16 + gi], GP[(2 * t + 1) * 16 + gi], ph[0], pl[0]);
    split_bf2(GP[(2 * t) * 16 + gi + 8], GP[(2 * t + 1) * 16 + gi + 8], ph[1], pl[1]);
    split_bf2(GP[(2 * t + 8) * 16 + gi], GP[(2 * t + 9) * 16 + gi], ph[2], pl[2]);
    split_bf2(GP[(2 * t + 8) * 16 + gi + 8], GP[(2 * t + 9) * 16 + gi + 8], ph[3], pl[3]);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int c = nt * 8 + gi;
      uint32_t b0h, b0l, b1h, b1l;
      split_bf2(sH[(2 * t) * kC + c], sH[(2 * t + 1) * kC + c], b0h, b0l);
      split_bf2(sH[(2 * t + 8) * kC + c], sH[(2 * t + 9) * kC + c], b1h, b1l);
      mma_bf16(a1[nt], ph[0], ph[1], ph[2], ph[3], b0h, b1h);
      mma_bf16(a1[nt], ph[0], ph[1], ph[2], ph[3], b0l, b1l);
      mma_bf16(a1[nt], pl[0], pl[1], pl[2], pl[3], b0h, b1h);
    }
    // G[i][unit] += sum_vox gq[vox][i] t[vox][unit]: A = gq^T (rows = outputs), B = t
    uint32_t gth[4], gtl[4];
    split_bf2(sQ[(2 * t) * 16 + gi], sQ[(2 * t + 1) * 16 + gi], gth[0], gtl[0]);
    split_bf2(sQ[(2 * t) * 16 + gi + 8], sQ[(2 * t + 1) * 16 + gi + 8], gth[1], gtl[1]);
    split_bf2(sQ[(2 * t + 8) * 16 + gi], sQ[(2 * t + 9) * 16 + gi], gth[2], gtl[2]);
    split_bf2(sQ[(2 * t + 8) * 16 + gi + 8], sQ[(2 * t + 9) * 16 + gi + 8], gth[3], gtl[3]);
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int u = nt * 8 + gi;
      uint32_t b0h, b0l, b1h, b1l;
      split_bf2(T[(2 * t) * 16 + u], T[(2 * t + 1) * 16 + u], b0h, b0l);
      split_bf2(T[(2 * t + 8) * 16 + u], T[(2 * t + 9) * 16 + u], b1h, b1l);
      mma_bf16(a2[nt], gth[0], gth[1], gth[2], gth[3], b0h, b1h);
      mma_bf16(a2[nt], gth[0], gth[1], gth[2], gth[3], b0l, b1l);
      mma_bf16(a2[nt], gtl[0], gtl[1], gtl[2], gtl[3], b0h, b1h);
    }
    // bias sums in voxel order: lane u < 16 takes unit u; lanes 0..8 of warp 0 take gq[i]
    if (lane < 16)
      for (int v = 0; v < 16; ++v) ap1 += GP[v * 16 + lane];
    if (warp == 0 && lane < kOut)
      for (int v = 0; v < 16; ++v) ap2 += sQ[v * 16 + lane];
    __syncthreads();
  }
  float* p = partial + (long long)blockIdx.x * kProjRow;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int j = kc * 16 + gi, c = nt * 8 + 2 * t;
    p[j * kC + c] = a1[nt][0];
    p[j * kC + c + 1] = a1[nt][1];
    p[(j + 8) * kC + c] = a1[nt][2];
    p[(j + 8) * kC + c + 1] = a1[nt][3];
  }
  if (lane < 16) p[kHid * kC + kc * 16 + lane] = ap1;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    const int i0 = gi, i1 = gi + 8, j = kc * 16 + nt * 8 + 2 * t;
    float* G = p + kHid * kC + kHid;
    if (i0 < kOut) {
      G[i0 * kHid + j] = a2[nt][0];
      G[i0 * kHid + j + 1] = a2[nt][1];
    }
    if (i1 < kOut) {
      G[i1 * kHid + j] = a2[nt][2];
      G[i1 * kHid + j + 1] = a2[nt][3];
    }
  }
  if (warp == 0 && lane < kOut) p[kHid * kC + kHid + kOut * kHid + lane] = ap2;
}

// lifting backward: per (sample, chunk) sums of gh0 and of gh0 phi per channel
__global__ void __launch_bounds__(kThreads) k_lift_bwd(const float* __restrict__ g0,
                                                       const uint8_t* const* __restrict__ phase, long long N,
                                                       long long chunk_vox, float* __restrict__ partial) {
  __shared__ float red[kWarps][2 * kC];
  const int b = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long v0 = (long long)blockIdx.x * chunk_vox;
  const long long v1 = v0 + chunk_vox < N ? v0 + chunk_vox : N;
  float s = 0.0f, sp = 0.0f;
  for (long long v = v0 + warp; v < v1; v += kWarps) {
    const float g = g0[((long long)b * N + v) * kC + lane];
    s += g;
    if (phase[b][v] != 0) sp += g;
  }
  red[warp][lane] = s;
  red[warp][kC + lane] = sp;
  __syncthreads();
  if (warp == 0) {
    float a = 0.0f, ap = 0.0f;
    for (int w = 0; w < kWarps; ++w) {
      a += red[w][lane];
      ap += red[w][kC + lane];
    }
    float* p = partial + ((long long)b * gridDim.x + blockIdx.x) * 2 * kC;
    p[lane] = a;
    p[kC + lane] = ap;
  }
}

__global__ void k_lift_finish(const float* __restrict__ partial, int B, int n_chunks, const float* __restrict__ su,
                              float* __restrict__ grad) {
  const int c = threadIdx.x;
  if (c >= kC) return;
  double ga = 0.0, gb0 = 0.0, gB[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < B; ++b) {
    double S = 0.0, Sp = 0.0;
    for (int k = 0; k < n_chunks; ++k) {
      S += partial[((long long)b * n_chunks + k) * 2 * kC + c];
      Sp += partial[((long long)b * n_chunks + k) * 2 * kC + kC + c];
    }
    ga += Sp;
    gb0 += S;
    for (int j = 0; j < 9; ++j) gB[j] += (double)su[10 * b + 1 + j] * S;
  }
  grad[kOffA + c] = (float)ga;
  grad[kOffB0 + c] = (float)gb0;
  for (int j = 0; j < 9; ++j) grad[kOffB + c * 9 + j] = (float)gB[j];
}

__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, int t, float lr, float b1, float b2, float eps, float wd) {
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * theta[i]);
  }
}

__global__ void k_make_target(const double* __restrict__ F, const double* __restrict__ Fbar, long long N,
                              float* __restrict__ target) {
  double s2 = 0.0;
  for (int c = 0; c < 9; ++c) {
    const double d = Fbar[c] - ((c % 4 == 0) ? 1.0 : 0.0);
    s2 += d * d;
  }
  const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < 9 * N;
       e += (long long)gridDim.x * blockDim.x)
    target[e] = (float)((F[e] - Fbar[e / N]) * inv);
}

// fluctuation s q of sample 0 as float64 [9][N]
__global__ void k_scale_q(const float* __restrict__ q, const float* __restrict__ su, long long N,
                          double* __restrict__ F) {
  const double s = su[0];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < 9 * N;
       e += (long long)gridDim.x * blockDim.x)
    F[e] = s * (double)q[e];
}

__global__ void k_add_fbar(const double* __restrict__ Fbar, long long N, double* __restrict__ F) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < 9 * N;
       e += (long long)gridDim.x * blockDim.x)
    F[e] += Fbar[e / N];
}

}  // namespace fno
}  // namespace fh

using namespace fh::fno;

struct fh_fno {
  int dev = 0;
  int nx = 0, ny = 0, nz = 0, max_batch = 0, train = 0, sms = 0;
  long long N = 0;
  cudaStream_t stream = nullptr;
  __nv_bfloat16* wq = nullptr;
  uint4* wfa = nullptr;  // mma fragments of the forward mixing matrices
  uint4* wba = nullptr;  // and of their transposes (backward)
  float* tw[3] = {nullptr, nullptr, nullptr};
  float* itw[3] = {nullptr, nullptr, nullptr};
  float* h[5] = {};
  float* z[3] = {};
  float* acc = nullptr;
  float* gz = nullptr;
  float* gn = nullptr;
  float* gh = nullptr;
  float* xs = nullptr;
  float* gys = nullptr;
  float* partial = nullptr;
  long long n_partial = 0;
  double* reduce_tmp = nullptr;
  long long n_reduce_tmp = 0;
  double* loss_part = nullptr;
  int n_loss_part = 0;
  double* fbar = nullptr;   // [max_batch][9]
  float* su = nullptr;      // [max_batch][10]: s, u
  float* head = nullptr;    // [max_batch][kHeadEff]: effective head of each sample
  float* gh_head = nullptr; // [max_batch][kHeadEff]: per-sample head-gradient sums
  const uint8_t** phase_tab = nullptr;
  float* qtmp = nullptr;    // [9][N] for the warm start
  int* err = nullptr;       // set by a kernel whose bounded wait ran out
  int test_skip_mma = 0;    // fh_fno_test_skip_mma
  std::vector<const uint8_t*> last_phase;
  int last_B = 0;
  bool params_set = false;
  std::vector<void*> allocs;
};

namespace {

int ffail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  fh_internal_set_error(buf);
  return code;
}

#define FN_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return ffail(FH_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct DevGuard {
  int old = -1;
  explicit DevGuard(int d) {
    cudaGetDevice(&old);
    if (old != d) cudaSetDevice(d);
  }
  ~DevGuard() {
    if (old >= 0) cudaSetDevice(old);
  }
};

template <class T>
cudaError_t nalloc(fh_fno* net, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e == cudaSuccess) {
    net->allocs.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

void free_all(fh_fno* net) {
  for (void* p : net->allocs) cudaFree(p);
  net->allocs.clear();
}

Geom geom(const fh_fno* net) { return Geom{net->nx, net->ny, net->nz, net->N}; }
int axis_len(const fh_fno* net, int ax) { return ax == 0 ? net->nx : (ax == 1 ? net->ny : net->nz); }

unsigned grid_for(long long work, int per_block, int cap) {
  long long b = (work + per_block - 1) / per_block;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

int spec_fwd(fh_fno* net, int B, int l, int ax, bool accum, const float* h, float* out) {
  const int n = axis_len(net, ax);
  const long long lines = (long long)B * (net->N / n);
  const unsigned grid = grid_for(lines, kWarps, 2 * net->sms);  // 2 resident CTAs per SM
  const uint4* W = net->wfa + (long long)(l * 3 + ax) * kModes * kFragPerMode;
  const size_t sm = spec_smem(n, false);
  if (accum)
    k_spec_fwd<true><<<grid, kThreads, sm, net->stream>>>(h, out, W, net->tw[ax], net->itw[ax], geom(net), ax, n, lines);
  else
    k_spec_fwd<false><<<grid, kThreads, sm, net->stream>>>(h, out, W, net->tw[ax], net->itw[ax], geom(net), ax, n, lines);
  FN_CUDA(cudaGetLastError());
  return FH_OK;
}

int group_size(int n_part) {
  int g = 1;
  while ((long long)g * g < n_part) ++g;
  return g;
}

int reduce_into(fh_fno* net, int n_part, int len, int stride, const float* partial, float* out) {
  const int group = group_size(n_part);
  const int n_groups = (n_part + group - 1) / group;
  if ((long long)n_groups * len > net->n_reduce_tmp) return ffail(FH_ERR_ARG, "reduction scratch too small");
  const unsigned bx = (unsigned)((len + kThreads - 1) / kThreads);
  k_reduce_groups<<<dim3(bx, (unsigned)n_groups), kThreads, 0, net->stream>>>(partial, n_part, len, stride, group,
                                                                             net->reduce_tmp);
  FN_CUDA(cudaGetLastError());
  k_reduce_final<<<bx, kThreads, 0, net->stream>>>(net->reduce_tmp, n_groups, len, out);
  FN_CUDA(cudaGetLastError());
  return FH_OK;
}

// FH_ERR_TIMEOUT (and the flag cleared) when a kernel's bounded wait ran out; call with the stream idle
int check_err(fh_fno* net) {
  int h = 0;
  FN_CUDA(cudaMemcpy(&h, net->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    FN_CUDA(cudaMemset(net->err, 0, sizeof(int)));
    return ffail(FH_ERR_TIMEOUT, "a tensor-core wait of the projection kernel ran out");
  }
  return FH_OK;
}

}  // namespace

extern "C" {

long long fh_fno_param_count(void) { return kNParam; }

int fh_fno_test_skip_mma(fh_fno* net, int skip) {
  fh_internal_set_error("");
  if (!net) return ffail(FH_ERR_ARG, "NULL argument");
  net->test_skip_mma = skip ? 1 : 0;
  return FH_OK;
}

int fh_fno_create(fh_fno** out, int nx, int ny, int nz, int max_batch, int train, void* cuda_stream) {
  fh_internal_set_error("");
  if (!out) return ffail(FH_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nx < kMinN || ny < kMinN || nz < kMinN)
    return ffail(FH_ERR_ARG, "every extent must be >= %d (got %d x %d x %d)", kMinN, nx, ny, nz);
  if (nx > 4096 || ny > 4096 || nz > 4096) return ffail(FH_ERR_ARG, "extent above 4096");
  if (max_batch < 1 || max_batch > 1024) return ffail(FH_ERR_ARG, "max_batch %d outside 1..1024", max_batch);
  fh_fno* net = new fh_fno();
  cudaGetDevice(&net->dev);
  net->nx = nx;
  net->ny = ny;
  net->nz = nz;
  net->N = (long long)nx * ny * nz;
  net->max_batch = max_batch;
  net->train = train ? 1 : 0;
  net->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaDeviceGetAttribute(&net->sms, cudaDevAttrMultiProcessorCount, net->dev);
  if (net->sms < 1) net->sms = 1;
  const long long act = (long long)max_batch * net->N * kC;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t count) {
    if (e == cudaSuccess) e = nalloc(net, p, count);
  };
  A(&net->wq, (size_t)kNParam);
  A(&net->wfa, (size_t)kFrag);
  A(&net->wba, (size_t)kFrag);
  for (int ax = 0; ax < 3; ++ax) {
    A(&net->tw[ax], (size_t)axis_len(net, ax) * kJ);
    A(&net->itw[ax], (size_t)axis_len(net, ax) * kJ);
  }
  A(&net->acc, (size_t)act);
  if (net->train) {
    for (int i = 0; i < 5; ++i) A(&net->h[i], (size_t)act);
    for (int i = 0; i < 3; ++i) A(&net->z[i], (size_t)act);
    A(&net->gz, (size_t)act);
    A(&net->gn, (size_t)act);
    A(&net->gh, (size_t)act);
    // per-line coefficients of the shortest axis bound every axis
    const int nmin = nx < ny ? (nx < nz ? nx : nz) : (ny < nz ? ny : nz);
    const long long coef = (long long)max_batch * (net->N / nmin) * kJ * kC;
    const long long gq = (long long)max_batch * net->N * kOut;
    A(&net->xs, (size_t)(coef > gq ? coef : gq));
    A(&net->gys, (size_t)coef);
    // partial sums: spectral weight gradient chunks, warps of the pointwise
    // backward, blocks of the projection backward, lifting chunks
    const long long lines_max = (long long)max_batch * (net->N / nmin);
    const long long n_chunks = (lines_max + kLinesPerChunk - 1) / kLinesPerChunk;
    long long np = n_chunks * kModes * 2 * kC * kC;
    np = np > (long long)4 * net->sms * kWarps * kPointLen ? np : (long long)4 * net->sms * kWarps * kPointLen;
    const long long proj = (long long)max_batch * 2 * net->sms * kProjRow;
    np = np > proj ? np : proj;
    const long long lift = (long long)max_batch * ((net->N + kLiftChunk - 1) / kLiftChunk) * 2 * kC;
    np = np > lift ? np : lift;
    net->n_partial = np;
    A(&net->partial, (size_t)np);
    // groups of the two-stage reduction: at most ceil(sqrt(rows)) + 1 of the longest row
    long long rows = n_chunks;
    rows = rows > (long long)4 * net->sms * kWarps ? rows : (long long)4 * net->sms * kWarps;
    rows = rows > (long long)max_batch * 2 * net->sms ? rows : (long long)max_batch * 2 * net->sms;
    long long gmax = 1;
    while (gmax * gmax < rows) ++gmax;
    net->n_reduce_tmp = (gmax + 1) * kWAxis;
    A(&net->reduce_tmp, (size_t)net->n_reduce_tmp);
  } else {
    A(&net->h[0], (size_t)act);
    A(&net->h[1], (size_t)act);
  }
  net->n_loss_part = 4 * net->sms;  // per sample
  A(&net->loss_part, (size_t)max_batch * net->n_loss_part);
  A(&net->fbar, (size_t)max_batch * 9);
  A(&net->su, (size_t)max_batch * 10);
  A(&net->head, (size_t)max_batch * kHeadEff);
  A(&net->gh_head, (size_t)max_batch * kHeadEff);
  A(&net->phase_tab, (size_t)max_batch);
  A(&net->qtmp, (size_t)9 * net->N);
  A(&net->err, (size_t)1);
  if (e == cudaSuccess) e = cudaMemset(net->err, 0, sizeof(int));
  if (e != cudaSuccess) {
    free_all(net);
    delete net;
    return ffail(FH_ERR_CUDA, "allocation failed: %s", cudaGetErrorString(e));
  }
  // twiddles: tw[x][2k] = cos(2 pi k x / n), tw[x][2k+1] = -sin(.);
  // itw = (c_k / n) tw with c_0 = 1 and c_k = 2 (the real inverse DFT)
  for (int ax = 0; ax < 3; ++ax) {
    const int n = axis_len(net, ax);
    std::vector<float> t((size_t)n * kJ), it((size_t)n * kJ);
    for (int x = 0; x < n; ++x)
      for (int k = 0; k < kModes; ++k) {
        const double ang = 2.0 * kPi * (double)(((long long)k * x) % n) / (double)n;
        const double ck = (k == 0 ? 1.0 : 2.0) / (double)n;
        t[(size_t)x * kJ + 2 * k] = (float)std::cos(ang);
        t[(size_t)x * kJ + 2 * k + 1] = (float)(-std::sin(ang));
        it[(size_t)x * kJ + 2 * k] = (float)(ck * std::cos(ang));
        it[(size_t)x * kJ + 2 * k + 1] = (float)(-ck * std::sin(ang));
      }
    e = cudaMemcpy(net->tw[ax], t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(net->itw[ax], it.data(), it.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
  }
  const int nmax = nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz);
  const size_t sm = spec_smem(nmax, false), smb = spec_smem(nmax, true);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgradSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_proj_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ProjT5));
  if (e != cudaSuccess) {
    free_all(net);
    delete net;
    return ffail(FH_ERR_CUDA, "set-up failed: %s", cudaGetErrorString(e));
  }
  *out = net;
  return FH_OK;
}

void fh_fno_destroy(fh_fno* net) {
  if (!net) return;
  DevGuard dg(net->dev);
  cudaStreamSynchronize(net->stream);
  free_all(net);
  delete net;
}

int fh_fno_set_params(fh_fno* net, const float* theta_dev) {
  fh_internal_set_error("");
  if (!net || !theta_dev) return ffail(FH_ERR_ARG, "NULL argument");
  DevGuard dg(net->dev);
  k_prepare<<<grid_for(kNParam, kThreads, 4 * net->sms), kThreads, 0, net->stream>>>(theta_dev, net->wq, net->wfa,
                                                                                     net->wba);
  FN_CUDA(cudaGetLastError());
  FN_CUDA(cudaStreamSynchronize(net->stream));
  net->params_set = true;
  return FH_OK;
}

int fh_fno_forward(fh_fno* net, int B, const unsigned char* const* phase_ptrs, const double* Fbar,
                   float* const* q_ptrs) {
  fh_internal_set_error("");
  if (!net || !phase_ptrs || !Fbar) return ffail(FH_ERR_ARG, "NULL argument");
  if (B < 1 || B > net->max_batch) return ffail(FH_ERR_ARG, "batch %d outside 1..%d", B, net->max_batch);
  if (!net->params_set) return ffail(FH_ERR_ARG, "parameters not set (fh_fno_set_params)");
  for (int b = 0; b < B; ++b) {
    if (!phase_ptrs[b]) return ffail(FH_ERR_ARG, "phase pointer %d is NULL", b);
    for (int c = 0; c < 9; ++c)
      if (!std::isfinite(Fbar[9 * b + c])) return ffail(FH_ERR_ARG, "non-finite Fbar of sample %d", b);
  }
  DevGuard dg(net->dev);
  cudaStream_t s = net->stream;
  net->last_phase.assign(phase_ptrs, phase_ptrs + B);
  FN_CUDA(cudaMemcpyAsync(net->phase_tab, phase_ptrs, B * sizeof(void*), cudaMemcpyHostToDevice, s));
  FN_CUDA(cudaMemcpyAsync(net->fbar, Fbar, (size_t)B * 9 * sizeof(double), cudaMemcpyHostToDevice, s));
  k_load_dir<<<(B + 63) / 64, 64, 0, s>>>(net->fbar, B, net->su);
  FN_CUDA(cudaGetLastError());
  k_head<<<grid_for((long long)B * kHeadEff, kThreads, 4 * net->sms), kThreads, 0, s>>>(net->wq, net->su, B,
                                                                                       net->head);
  FN_CUDA(cudaGetLastError());
  const long long nvox = (long long)B * net->N;
  auto H = [&](int l) { return net->train ? net->h[l] : net->h[l & 1]; };
  k_lift<<<grid_for(nvox * kC, kThreads, 8 * net->sms), kThreads, 0, s>>>(net->phase_tab, net->su, net->wq, net->N, B,
                                                                        H(0));
  FN_CUDA(cudaGetLastError());
  for (int l = 0; l < kLayers; ++l) {
    int rc;
    if ((rc = spec_fwd(net, B, l, 2, false, H(l), net->acc))) return rc;
    if ((rc = spec_fwd(net, B, l, 1, true, H(l), net->acc))) return rc;
    if ((rc = spec_fwd(net, B, l, 0, true, H(l), net->acc))) return rc;
    float* z = (net->train && l < kLayers - 1) ? net->z[l] : nullptr;
    k_point_fwd<<<grid_for((nvox + 15) / 16, kWarps, 4 * net->sms), kThreads, 0, s>>>(
        H(l), net->acc, net->wq, l, z, H(l + 1), nvox, l < kLayers - 1 ? 1 : 0);
    FN_CUDA(cudaGetLastError());
  }
  if (q_ptrs)
    for (int b = 0; b < B; ++b) {
      if (!q_ptrs[b]) continue;
      k_proj_fwd<<<grid_for(net->N, kT5, 2 * net->sms), kT5, sizeof(ProjT5), s>>>(
          H(kLayers) + (long long)b * net->N * kC, net->wq, net->head + (long long)b * kHeadEff, q_ptrs[b], nullptr,
          net->N, nullptr, net->err, net->test_skip_mma);
      FN_CUDA(cudaGetLastError());
    }
  FN_CUDA(cudaStreamSynchronize(s));
  int rc_err;
  if ((rc_err = check_err(net))) return rc_err;
  net->last_B = B;
  return FH_OK;
}

int fh_fno_loss_grad(fh_fno* net, const float* const* target_ptrs, double* loss_out, float* grad_dev) {
  fh_internal_set_error("");
  if (!net || !target_ptrs) return ffail(FH_ERR_ARG, "NULL argument");
  if (!net->train) return ffail(FH_ERR_ARG, "network created without training buffers");
  const int B = net->last_B;
  if (B < 1) return ffail(FH_ERR_ARG, "no forward pass to differentiate");
  for (int b = 0; b < B; ++b)
    if (!target_ptrs[b]) return ffail(FH_ERR_ARG, "target pointer %d is NULL", b);
  DevGuard dg(net->dev);
  cudaStream_t s = net->stream;
  const long long nvox = (long long)B * net->N;
  const double count = (double)nvox * kOut;
  const unsigned gl = (unsigned)net->n_loss_part;
  const long long N = net->N;
  if (!grad_dev) {
    for (int b = 0; b < B; ++b) {
      k_proj_fwd<<<gl, kT5, sizeof(ProjT5), s>>>(net->h[kLayers] + b * N * kC, net->wq,
                                                 net->head + (long long)b * kHeadEff, nullptr, target_ptrs[b], N,
                                                 net->loss_part + (long long)b * gl, net->err,
                                                 net->test_skip_mma);
      FN_CUDA(cudaGetLastError());
    }
  } else {
    int rc;
    // projection, sample by sample (each has its own effective head)
    const unsigned gp = (unsigned)(2 * net->sms);
    for (int b = 0; b < B; ++b) {
      const float* hb = net->h[kLayers] + b * N * kC;
      const float* headb = net->head + (long long)b * kHeadEff;
      k_proj_bwd_a<<<gl, kThreads, 0, s>>>(hb, net->wq, headb, target_ptrs[b], N, (float)(2.0 / count),
                                           net->xs + b * N * kOut, net->gn + b * N * kC,
                                           net->loss_part + (long long)b * gl);
      FN_CUDA(cudaGetLastError());
      k_proj_bwd_b<<<gp, kThreads, 0, s>>>(hb, net->xs + b * N * kOut, net->wq, headb, N,
                                           net->partial + (long long)b * gp * kProjRow);
      FN_CUDA(cudaGetLastError());
    }
    if ((rc = reduce_into(net, (int)(B * gp), kProjShared, kProjRow, net->partial, grad_dev + kOffP1))) return rc;
    for (int b = 0; b < B; ++b)
      if ((rc = reduce_into(net, (int)gp, kHeadEff, kProjRow, net->partial + (long long)b * gp * kProjRow + kProjShared,
                            net->gh_head + (long long)b * kHeadEff)))
        return rc;
    k_head_grad<<<grid_for(kHead * kHid + kHead, kThreads, 4 * net->sms), kThreads, 0, s>>>(net->gh_head, net->su, B,
                                                                                           grad_dev);
    FN_CUDA(cudaGetLastError());
    // layers, last to first
    for (int l = kLayers - 1; l >= 0; --l) {
      const unsigned gpw = grid_for((nvox + 15) / 16, kWarps, 4 * net->sms);
      k_point_bwd<<<gpw, kThreads, 0, s>>>(net->gn, l < kLayers - 1 ? net->z[l] : nullptr, net->h[l], net->wq, l,
                                           net->gz, net->gh, net->partial, nvox);
      FN_CUDA(cudaGetLastError());
      if ((rc = reduce_into(net, (int)(gpw * kWarps), kPointLen, kPointLen, net->partial, grad_dev + off_M(l))))
        return rc;
      for (int ax = 0; ax < 3; ++ax) {
        const int n = axis_len(net, ax);
        const long long lines = (long long)B * (net->N / n);
        const uint4* W = net->wba + (long long)(l * 3 + ax) * kModes * kFragPerMode;
        k_spec_bwd<<<grid_for(lines, kWarps, 2 * net->sms), kThreads, spec_smem(n, true), s>>>(
            net->h[l], net->gz, net->gh, net->xs, net->gys, W, net->tw[ax], net->itw[ax], geom(net), ax, n, lines);
        FN_CUDA(cudaGetLastError());
        const unsigned chunks = (unsigned)((lines + kLinesPerChunk - 1) / kLinesPerChunk);
        k_wgrad<<<dim3(chunks, kModes), kThreads, kWgradSmem, s>>>(net->xs, net->gys, lines, net->partial);
        FN_CUDA(cudaGetLastError());
        if ((rc = reduce_into(net, (int)chunks, (int)kWAxis, (int)kWAxis, net->partial, grad_dev + off_W(l) + ax * kWAxis)))
          return rc;
      }
      float* t = net->gn;
      net->gn = net->gh;
      net->gh = t;
    }
    // lifting: gn now holds the gradient with respect to h0
    const long long chunk_vox = kLiftChunk;
    const unsigned nch = (unsigned)((net->N + chunk_vox - 1) / chunk_vox);
    FN_CUDA(cudaMemcpyAsync(net->phase_tab, net->last_phase.data(), B * sizeof(void*), cudaMemcpyHostToDevice, s));
    k_lift_bwd<<<dim3(nch, B), kThreads, 0, s>>>(net->gn, net->phase_tab, net->N, chunk_vox, net->partial);
    FN_CUDA(cudaGetLastError());
    k_lift_finish<<<1, 32, 0, s>>>(net->partial, B, (int)nch, net->su, grad_dev);
    FN_CUDA(cudaGetLastError());
  }
  std::vector<double> lp((size_t)B * gl);
  FN_CUDA(cudaMemcpyAsync(lp.data(), net->loss_part, lp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  FN_CUDA(cudaStreamSynchronize(s));
  if (!grad_dev) {
    const int rc_err = check_err(net);
    if (rc_err) return rc_err;
  }
  double L = 0.0;
  for (double v : lp) L += v;
  if (loss_out) *loss_out = L / count;
  return FH_OK;
}

int fh_fno_adam(fh_fno* net, float* theta_dev, const float* grad_dev, float* m_dev, float* v_dev, int t, float lr,
                float beta1, float beta2, float eps, float wd) {
  fh_internal_set_error("");
  if (!net || !theta_dev || !grad_dev || !m_dev || !v_dev) return ffail(FH_ERR_ARG, "NULL argument");
  if (t < 1) return ffail(FH_ERR_ARG, "Adam step number must be >= 1");
  if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f && lr >= 0.0f && wd >= 0.0f))
    return ffail(FH_ERR_ARG, "invalid Adam hyper-parameters");
  DevGuard dg(net->dev);
  k_adam<<<grid_for(kNParam, kThreads, 4 * net->sms), kThreads, 0, net->stream>>>(theta_dev, grad_dev, m_dev, v_dev,
                                                                                 kNParam, t, lr, beta1, beta2, eps,
                                                                                 wd);
  FN_CUDA(cudaGetLastError());
  FN_CUDA(cudaStreamSynchronize(net->stream));
  return FH_OK;
}

int fh_fno_make_target(fh_fno* net, const double* F_dev, const double Fbar[9], float* target_dev) {
  fh_internal_set_error("");
  if (!net || !F_dev || !Fbar || !target_dev) return ffail(FH_ERR_ARG, "NULL argument");
  DevGuard dg(net->dev);
  FN_CUDA(cudaMemcpyAsync(net->fbar, Fbar, 9 * sizeof(double), cudaMemcpyHostToDevice, net->stream));
  k_make_target<<<grid_for(9 * net->N, kThreads, 4 * net->sms), kThreads, 0, net->stream>>>(F_dev, net->fbar, net->N,
                                                                                           target_dev);
  FN_CUDA(cudaGetLastError());
  FN_CUDA(cudaStreamSynchronize(net->stream));
  return FH_OK;
}

int fh_fno_warm_start(fh_fno* net, fh_ctx* ctx, const unsigned char* phase_dev, const double Fbar[9],
                      double* F_dev) {
  fh_internal_set_error("");
  if (!net || !ctx || !phase_dev || !Fbar || !F_dev) return ffail(FH_ERR_ARG, "NULL argument");
  int cx, cy, cz;
  fh_internal_ctx_grid(ctx, &cx, &cy, &cz);
  if (cx != net->nx || cy != net->ny || cz != net->nz)
    return ffail(FH_ERR_ARG, "context grid %dx%dx%d differs from the network grid %dx%dx%d", cx, cy, cz, net->nx,
                 net->ny, net->nz);
  const unsigned char* pp[1] = {phase_dev};
  float* qp[1] = {net->qtmp};
  int rc = fh_fno_forward(net, 1, pp, Fbar, qp);
  if (rc) return rc;
  {
    DevGuard dg(net->dev);
    k_scale_q<<<grid_for(9 * net->N, kThreads, 4 * net->sms), kThreads, 0, net->stream>>>(net->qtmp, net->su, net->N,
                                                                                         F_dev);
    FN_CUDA(cudaGetLastError());
    FN_CUDA(cudaStreamSynchronize(net->stream));
  }
  if ((rc = fh_project(ctx, F_dev, F_dev, 1.0, nullptr))) return rc;
  DevGuard dg(net->dev);
  FN_CUDA(cudaMemcpyAsync(net->fbar, Fbar, 9 * sizeof(double), cudaMemcpyHostToDevice, net->stream));
  k_add_fbar<<<grid_for(9 * net->N, kThreads, 4 * net->sms), kThreads, 0, net->stream>>>(net->fbar, net->N, F_dev);
  FN_CUDA(cudaGetLastError());
  FN_CUDA(cudaStreamSynchronize(net->stream));
  return FH_OK;
}

}  // extern "C"
