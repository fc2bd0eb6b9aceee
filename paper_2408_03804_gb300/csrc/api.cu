// C-ABI entry points and the host-side Newton-Krylov driver (Appendix A,
// Algorithm 1). The driver queues the kernels of kernels_pointwise.cu and
// kernels_fft.cu on the context's stream; the CG scalars stay on the device
// and the host reads them every `check_every` iterations, so a CG iteration
// costs no host round trip. Kernels queued after convergence see the device
// flag and return at once; the launch accounting books them apart (class
// "idle") so that per-kernel counts and times cover only launches that did
// work.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "df64.cuh"
#include "fh_kernels.h"

using namespace fh;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define FH_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return fail(FH_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)


struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

// device scalars of a context
struct DevScalars {
  CgScalars cg;
  double sums[16];
  int flags;
  int pad;
};

struct ProfPair {
  int cls;
  int tag;           // CG loop iteration of the launch, or -1 outside a CG loop
  cudaEvent_t a, b;  // null when events are off
};

// What a captured chunk of CG iterations depends on besides the context's own
// buffers: a replay is valid while these are unchanged (compared bytewise;
// zero-filled first so that padding compares equal)
struct CgGraphKey {
  Grid g;
  Tiling t;
  MatView mv;
  const double* F;
  double c_mv;
  int stored, first, check_every, n_iz, n_upd, df;
};

// One chunk of check_every CG iterations captured as a CUDA graph, with the
// class and iteration (0 .. check_every - 1) of each kernel it launches
struct CgGraph {
  CgGraphKey key;
  cudaGraphExec_t exec = nullptr;
  std::vector<ProfPair> nodes;
};

struct fh_ctx {
  int dev = 0;
  // launch accounting (fh_profile_enable / fh_profile_read)
  long long counts[FH_PROF_NCLASS] = {};
  double ms[FH_PROF_NCLASS] = {};
  bool prof = false;
  int cg_tag = -1;                  // CG loop iteration being queued (-1 outside CG loops)
  std::vector<cudaEvent_t> ev_pool;
  std::vector<ProfPair> pending;    // timed launches outside CG loops
  std::vector<ProfPair> tagged;     // launches of the current CG loop, booked once its products are known
  cudaStream_t stream = nullptr;
  Grid g{};
  Tiling tiling{};
  double2* S = nullptr;       // spectrum [9][nx][ny][nzh]
  double* x = nullptr;        // CG solution dF       [9][N]
  double* r = nullptr;        // CG residual          [9][N]
  double* p = nullptr;        // CG direction         [9][N]
  double* y = nullptr;        // G(K : p)             [9][N]
  double* P = nullptr;        // stress / jvp scratch [9][N]
  double* K = nullptr;        // packed tangent       [45][N]
  double* partials = nullptr;
  long long n_partials = 0;
  double* params = nullptr;   // [256][2] Lame pairs, then [256][2] J2 (yield stress, hardening)
  double2* tw = nullptr;      // twiddle tables
  dfc* tw_df = nullptr;       // the compile-time lengths' tables in double-float
  df64* K_df = nullptr;       // double-float copy of a packed tangent [45][N] (allocated on first use)
  DevScalars* sc = nullptr;
  // graph replay of the CG loop: chunk 0 starts a loop, chunk 1 continues it;
  // off after a failed capture (e.g. the legacy default stream)
  CgGraph cg_graph[2];
  bool graphs_ok = true;
  long long min_ctas = 0;     // CTAs per pass the default tiling aims for (two per SM)
  long long graph_replays = 0, graph_captures = 0;
};

namespace {

enum ProfClass : int {
  kPFwdZ = 0, kPFwdY, kPXGhat, kPInvY, kPInvZ, kPConst, kPJvp, kPCgScalar, kPCgUpdate, kPNewton, kPFill, kPReduce,
  kPContract, kPIdle
};
static_assert(kPIdle + 1 == FH_PROF_NCLASS, "profile classes");

cudaEvent_t ev_get(fh_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// book one launch under class cls: its count, and its device time if timed
void prof_book(fh_ctx* c, int cls, const ProfPair& q) {
  c->counts[cls]++;
  if (q.a) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) c->ms[cls] += ms;
    c->ev_pool.push_back(q.a);
    c->ev_pool.push_back(q.b);
  }
}

// accumulate the timed pairs; call only when the stream is idle
void prof_flush(fh_ctx* c) {
  for (const ProfPair& q : c->pending) prof_book(c, q.cls, q);
  c->pending.clear();
}

// Book the launches of a CG loop queued so far, once the stream is idle.
// `products` is the device's count of matrix-vector products that ran: the
// launches of loop iterations below it did work, the later ones found the
// done flag and returned at once, and go to the idle class.
void prof_commit_cg(fh_ctx* c, int products) {
  for (const ProfPair& q : c->tagged) prof_book(c, q.tag < products ? q.cls : (int)kPIdle, q);
  c->tagged.clear();
}

template <class Fn>
cudaError_t prof(fh_ctx* c, int cls, Fn&& fn) {
  ProfPair q{cls, c->cg_tag, nullptr, nullptr};
  cudaError_t e;
  if (c->prof) {
    q.a = ev_get(c);
    q.b = ev_get(c);
    cudaEventRecord(q.a, c->stream);
    e = fn();
    cudaEventRecord(q.b, c->stream);
  } else {
    e = fn();
  }
  if (q.tag >= 0) c->tagged.push_back(q);
  else if (q.a) c->pending.push_back(q);
  else c->counts[cls]++;
  return e;
}

Grid grid_with_lengths(const fh_ctx* ctx, const double* lengths) {
  Grid g = ctx->g;
  if (lengths) {
    g.sx = 1.0 / lengths[0];
    g.sy = 1.0 / lengths[1];
    g.sz = 1.0 / lengths[2];
  }
  return g;
}

bool lengths_ok(const double* L) { return !L || (L[0] > 0 && L[1] > 0 && L[2] > 0 && std::isfinite(L[0]) && std::isfinite(L[1]) && std::isfinite(L[2])); }

int check_material(const fh_material* m) {
  if (!m) return fail(FH_ERR_ARG, "material is NULL");
  if (m->kind < FH_LINEAR_ELASTIC || m->kind > FH_J2) return fail(FH_ERR_ARG, "unknown material kind %d", m->kind);
  if (m->n_phase < 1 || m->n_phase > 256) return fail(FH_ERR_ARG, "n_phase %d outside 1..256", m->n_phase);
  if (!m->phase || !m->params) return fail(FH_ERR_ARG, "phase or params is NULL");
  for (int i = 0; i < 2 * m->n_phase; ++i)
    if (!std::isfinite(m->params[i])) return fail(FH_ERR_ARG, "non-finite material parameter");
  if (m->kind == FH_J2) {
    if (!m->plastic || !m->history) return fail(FH_ERR_ARG, "J2 needs the plastic parameters and the history array");
    for (int i = 0; i < 2 * m->n_phase; ++i)
      if (!std::isfinite(m->plastic[i]) || m->plastic[i] < 0.0)
        return fail(FH_ERR_ARG, "J2 yield stress and hardening modulus must be finite and >= 0");
  }
  return FH_OK;
}

// upload the parameter table; rows >= n_phase hold NaN so that an
// out-of-range phase value surfaces as a non-physical state
int upload_material(fh_ctx* ctx, const fh_material* m, MatView* mv) {
  std::vector<double> tab(1024, std::nan(""));
  for (int i = 0; i < 2 * m->n_phase; ++i) tab[i] = m->params[i];
  if (m->kind == FH_J2)
    for (int i = 0; i < 2 * m->n_phase; ++i) tab[512 + i] = m->plastic[i];
  FH_CUDA(cudaMemcpyAsync(ctx->params, tab.data(), 1024 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  FH_CUDA(cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  mv->kind = m->kind;
  mv->phase = m->phase;
  mv->params = ctx->params;
  mv->scale = m->scale;
  mv->plastic = m->kind == FH_J2 ? ctx->params + 512 : nullptr;
  mv->history = m->kind == FH_J2 ? m->history : nullptr;
  return FH_OK;
}

// G applied to src (tau = src, K : src, or the CG direction), result to out
// (df: the transforms in double-float arithmetic, kernels_df64.cu)
// ctx->K_df = K in double-float (allocated on the first call: 360 bytes per voxel)
int tangent_to_df64(fh_ctx* ctx, const Grid& g, const double* K) {
  if (!ctx->K_df) FH_CUDA(cudaMalloc(&ctx->K_df, (size_t)45 * g.n * sizeof(df64)));
  FH_CUDA(prof(ctx, kPConst, [&] { return launch_tangent_to_df64(g, K, ctx->K_df, ctx->stream); }));
  return FH_OK;
}

// (df: the transforms in double-float arithmetic, kernels_df64.cu; a mode
// that reads K then reads the double-float copy ctx->K_df instead)
int run_projection(fh_ctx* ctx, const Grid& g, int zmode, const double* src, double* p, const double* K,
                   double scale, int izmode, double* out, const double* pdot, CgScalars* cg, double* x = nullptr,
                   bool df = false) {
  const Tiling& t = ctx->tiling;
  cudaStream_t s = ctx->stream;
  if (df) {
    const Tiling t = df_tiles(ctx->tiling);
    dfc* S = reinterpret_cast<dfc*>(ctx->S);
    const dfc* tw = ctx->tw_df;
    const df64* Kd = K ? ctx->K_df : nullptr;
    FH_CUDA(prof(ctx, kPFwdZ, [&] { return launch_fwd_z_df(g, t, zmode, src, p, x, Kd, cg, S, tw, s); }));
    FH_CUDA(prof(ctx, kPFwdY, [&] { return launch_fwd_y_df(g, t, S, tw, cg, s); }));
    FH_CUDA(prof(ctx, kPXGhat, [&] { return launch_x_ghat_df(g, t, S, tw, scale, cg, s); }));
    FH_CUDA(prof(ctx, kPInvY, [&] { return launch_inv_y_df(g, t, S, tw, cg, s); }));
    FH_CUDA(prof(ctx, kPInvZ, [&] { return launch_inv_z_df(g, t, izmode, S, out, pdot, ctx->partials, tw, cg, s); }));
    return FH_OK;
  }
  FH_CUDA(prof(ctx, kPFwdZ, [&] { return launch_fwd_z(g, t, zmode, src, p, x, K, cg, ctx->S, ctx->tw, s); }));
  FH_CUDA(prof(ctx, kPFwdY, [&] { return launch_fwd_y(g, t, ctx->S, ctx->tw, cg, s); }));
  FH_CUDA(prof(ctx, kPXGhat, [&] { return launch_x_ghat(g, t, ctx->S, ctx->tw, scale, cg, s); }));
  FH_CUDA(prof(ctx, kPInvY, [&] { return launch_inv_y(g, t, ctx->S, ctx->tw, cg, s); }));
  FH_CUDA(prof(ctx, kPInvZ, [&] { return launch_inv_z(g, t, izmode, ctx->S, out, pdot, ctx->partials, ctx->tw, cg, s); }));
  return FH_OK;
}

// Capture `queue` (the launches of one chunk of CG iterations, tagged
// 0 .. check_every - 1) into G. A stream that cannot be captured (the legacy
// default stream) turns graph replay off for the context, and a stream the
// caller is capturing gets plain launches; either way G.exec stays null and
// the chunk runs as plain launches.
template <class Queue>
int capture_cg_chunk(fh_ctx* ctx, CgGraph& G, const CgGraphKey& key, Queue&& queue) {
  cudaStream_t s = ctx->stream;
  if (G.exec) {
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
  }
  G.nodes.clear();
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    ctx->graphs_ok = false;
    return FH_OK;
  }
  if (st != cudaStreamCaptureStatusNone) return FH_OK;  // the caller is capturing: plain launches into its graph
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    ctx->graphs_ok = false;
    return FH_OK;
  }
  const int rc = queue();
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &graph);
  G.nodes.swap(ctx->tagged);
  ctx->tagged.clear();
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(FH_ERR_CUDA, "CG graph capture: %s", cudaGetErrorString(e));
  const cudaError_t ei = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    G.exec = nullptr;
    return fail(FH_ERR_CUDA, "CG graph instantiation: %s", cudaGetErrorString(ei));
  }
  G.key = key;
  ctx->graph_captures++;
  return FH_OK;
}

// Conjugate gradients on G(K : d) = b (Alg. 1 inner solve). On entry ctx->r
// holds b and ctx->partials the per-CTA sums of b . b from the inverse z pass
// that produced it; on return ctx->x holds d and *host_cg the final scalars.
int run_cg(fh_ctx* ctx, const Grid& g, const MatView& mv, const double* F_dev, bool stored, double cg_tol,
           const fh_options& opt, CgScalars* host_cg) {
  const int max_cg = opt.max_cg, check_every = opt.check_every;
  const bool plain = opt.launch_mode == FH_LAUNCH_PLAIN;
  const bool df = opt.matvec_arith == FH_ARITH_DF64;
  int rc;
  if (df && stored && (rc = tangent_to_df64(ctx, g, ctx->K))) return rc;
  cudaStream_t s = ctx->stream;
  CgScalars* cg = &ctx->sc->cg;
  // partial sums of the inverse z pass: the right-hand side's came from the FP64 tiles,
  // the CG products' from the tiles of their arithmetic
  const int n_iz_rhs = (int)z_pass_ctas(g, ctx->tiling);
  const int n_iz = (int)z_pass_ctas(g, df ? df_tiles(ctx->tiling) : ctx->tiling);
  const int n_upd = (int)cg_update_ctas(g);
  const double c_mv = 1.0 / (2.0 * (double)g.n);
  FH_CUDA(prof(ctx, kPCgScalar, [&] { return launch_cg_init(cg, ctx->partials, n_iz_rhs, cg_tol, max_cg, s); }));
  FH_CUDA(cudaMemsetAsync(ctx->x, 0, (size_t)9 * g.n * sizeof(double), s));
  int launched = 0;
  // every exit below clears the tag; launches of the loop are booked by prof_commit_cg
  struct TagReset {
    fh_ctx* c;
    ~TagReset() {
      c->cg_tag = -1;
      // launches still tagged here belong to an aborted loop: book them as idle
      if (!c->tagged.empty()) {
        cudaStreamSynchronize(c->stream);
        prof_commit_cg(c, 0);
      }
    }
  } tag_reset{ctx};
  // queue CG iterations base .. base + count - 1, tagged base-relative
  auto queue_iterations = [&](int base, int count, int tag0) -> int {
    for (int k = 0; k < count; ++k) {
      ctx->cg_tag = tag0 + k;
      const int zmode = base + k == 0 ? kZCgFirst : kZCg;
      int rc2;
      if (stored) {
        if ((rc2 = run_projection(ctx, g, zmode, ctx->r, ctx->p, ctx->K, c_mv, kIZDot, ctx->y, ctx->p, cg, ctx->x,
                                  df)))
          return rc2;
      } else {
        FH_CUDA(prof(ctx, kPJvp, [&] {
          return launch_jvp(g, mv, F_dev, ctx->r, ctx->p, ctx->x, ctx->P, zmode, cg, &ctx->sc->flags, s);
        }));
        if ((rc2 = run_projection(ctx, g, kZDirect, ctx->P, nullptr, nullptr, c_mv, kIZDot, ctx->y, ctx->p, cg,
                                  nullptr, df)))
          return rc2;
      }
      FH_CUDA(prof(ctx, kPCgScalar, [&] { return launch_cg_alpha(cg, ctx->partials, n_iz, s); }));
      FH_CUDA(prof(ctx, kPCgUpdate, [&] { return launch_cg_update(g, cg, ctx->r, ctx->y, ctx->partials, s); }));
      FH_CUDA(prof(ctx, kPCgScalar, [&] { return launch_cg_beta(cg, ctx->partials, n_upd, s); }));
    }
    return FH_OK;
  };
  while (true) {
    // Without per-launch timing, a chunk runs as a replay of a captured
    // graph (one launch instead of about 8 * check_every); the graph is
    // captured again only when what its kernels are given changes.
    bool replayed = false;
    if (!plain && !ctx->prof && ctx->graphs_ok) {
      CgGraphKey key;
      memset(&key, 0, sizeof key);
      key.g = g;
      key.t = ctx->tiling;
      key.mv = mv;
      key.F = stored ? nullptr : F_dev;  // only the jvp form reads F in the loop
      key.c_mv = c_mv;
      key.stored = stored;
      key.first = launched == 0;
      key.check_every = check_every;
      key.n_iz = n_iz;
      key.n_upd = n_upd;
      key.df = df;
      CgGraph& G = ctx->cg_graph[key.first ? 0 : 1];
      if (!G.exec || memcmp(&G.key, &key, sizeof key) != 0) {
        if ((rc = capture_cg_chunk(ctx, G, key, [&] { return queue_iterations(launched, check_every, 0); })))
          return rc;
      }
      if (G.exec) {
        FH_CUDA(cudaGraphLaunch(G.exec, s));
        ctx->graph_replays++;
        for (const ProfPair& q : G.nodes) ctx->tagged.push_back(ProfPair{q.cls, launched + q.tag, nullptr, nullptr});
        launched += check_every;
        replayed = true;
      }
    }
    if (!replayed) {
      if ((rc = queue_iterations(launched, check_every, launched))) return rc;
      launched += check_every;
    }
    ctx->cg_tag = -1;
    FH_CUDA(cudaMemcpyAsync(host_cg, cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    FH_CUDA(cudaStreamSynchronize(s));
    prof_flush(ctx);
    prof_commit_cg(ctx, host_cg->done ? host_cg->products : launched);
    if (host_cg->done) {
      FH_CUDA(prof(ctx, kPCgUpdate, [&] { return launch_cg_finalize(g, cg, ctx->x, ctx->p, s); }));
      return FH_OK;
    }
    if (launched > max_cg + 2 * check_every) return fail(FH_ERR_CUDA, "CG loop did not report completion");
  }
}

int read_flags(fh_ctx* ctx, int* flags) {
  FH_CUDA(cudaMemcpyAsync(flags, &ctx->sc->flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FH_CUDA(cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  return FH_OK;
}

int reduce9(fh_ctx* ctx, int n_parts, double out[9]) {
  FH_CUDA(prof(ctx, kPReduce, [&] { return launch_sum_partials(ctx->partials, n_parts, 9, ctx->sc->sums, ctx->stream); }));
  FH_CUDA(cudaMemcpyAsync(out, ctx->sc->sums, 9 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FH_CUDA(cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  return FH_OK;
}

}  // namespace

extern "C" {

void fh_default_options(fh_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->newton_tol = 1e-8;
  o->cg_tol = 0.0;
  o->max_newton = 50;
  o->max_cg = 5000;
  o->init = FH_INIT_REFERENCE;
  o->tangent_mode = FH_TANGENT_STORED;
  o->check_every = 16;
  o->launch_mode = FH_LAUNCH_GRAPH;
  o->matvec_arith = FH_ARITH_FP64;
  o->lengths[0] = o->lengths[1] = o->lengths[2] = 1.0;
}

const char* fh_last_error_string(void) { return g_err; }

// error text of entry points defined in other translation units (not exported)
void fh_internal_set_error(const char* msg) {
  snprintf(g_err, sizeof(g_err), "%s", msg ? msg : "");
}

// grid of a context, for entry points of other translation units (not exported)
void fh_internal_ctx_grid(const fh_ctx* ctx, int* nx, int* ny, int* nz) {
  *nx = ctx->g.nx;
  *ny = ctx->g.ny;
  *nz = ctx->g.nz;
}

int fh_create(fh_ctx** out, int nx, int ny, int nz, void* cuda_stream) {
  g_err[0] = 0;
  if (!out) return fail(FH_ERR_ARG, "out is NULL");
  if (!grid_extents_ok_any(nx, ny, nz))
    return fail(FH_ERR_ARG,
                "grid %dx%dx%d: nx and ny must be 1..%d, nz 1 or even with nz and nz/2 of the form 2^a or 3*2^a up to 256",
                nx, ny, nz, kMaxNAny);
  fh_ctx* c = new fh_ctx();
  FH_CUDA(cudaGetDevice(&c->dev));
  c->stream = (cudaStream_t)cuda_stream;
  Grid& g = c->g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.nzh = nz / 2 + 1;
  g.n = (long long)nx * ny * nz;
  g.nspec = (long long)nx * ny * g.nzh;
  g.sx = g.sy = g.sz = 1.0;
  // lengths without a compile-time plan get a run-time plan and their own
  // twiddle table after the tables of the compile-time lengths
  int tw_len = kTwiddleTables;
  g.px = make_fft_plan(nx, tw_len);
  tw_len += g.px.tw_len;
  g.py = make_fft_plan(ny, tw_len);
  tw_len += g.py.tw_len;
  // default tiles, smaller on small grids so that every pass keeps two CTAs per SM busy
  int sms = 0;
  FH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  c->min_ctas = 2LL * sms;
  c->tiling = choose_tiling(g, c->min_ctas);
  const size_t f9 = (size_t)9 * g.n * sizeof(double);
  long long np = 9LL * constitutive_ctas(g);
  np = std::max(np, (long long)nx * ny);  // z passes with one line per CTA (any autotuned tiling)
  np = std::max(np, cg_update_ctas(g));
  np = std::max(np, newton_update_ctas(g));
  c->n_partials = np;
  auto cleanup = [&](int code) {
    fh_destroy(c);
    return code;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&c->S, (size_t)9 * g.nspec * sizeof(double2))) ||
      (e = cudaMalloc(&c->x, f9)) || (e = cudaMalloc(&c->r, f9)) || (e = cudaMalloc(&c->p, f9)) ||
      (e = cudaMalloc(&c->y, f9)) || (e = cudaMalloc(&c->P, f9)) ||
      (e = cudaMalloc(&c->K, (size_t)45 * g.n * sizeof(double))) ||
      (e = cudaMalloc(&c->partials, (size_t)np * sizeof(double))) ||
      (e = cudaMalloc(&c->params, 1024 * sizeof(double))) ||
      (e = cudaMalloc(&c->tw, tw_len * sizeof(double2))) || (e = cudaMalloc(&c->tw_df, tw_len * sizeof(dfc))) ||
      (e = cudaMalloc(&c->sc, sizeof(DevScalars)))) {
    fail(FH_ERR_CUDA, "fh_create: allocation failed: %s", cudaGetErrorString(e));
    return cleanup(FH_ERR_CUDA);
  }
  std::vector<double2> tw(tw_len);
  fill_twiddle_table(tw.data());
  if (g.px.L) fill_plan_tables(tw.data() + g.px.tw_off, g.px);
  if (g.py.L) fill_plan_tables(tw.data() + g.py.tw_off, g.py);
  std::vector<dfc> tw_df(tw_len);
  twiddles_to_df64(tw.data(), tw_df.data(), tw_len);
  if ((e = cudaMemcpy(c->tw, tw.data(), tw_len * sizeof(double2), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(c->tw_df, tw_df.data(), tw_len * sizeof(dfc), cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(c->sc, 0, sizeof(DevScalars))) || (e = setup_fft_kernels(g, c->tiling))) {
    fail(FH_ERR_CUDA, "fh_create: setup failed: %s", cudaGetErrorString(e));
    return cleanup(FH_ERR_CUDA);
  }
  *out = c;
  return FH_OK;
}

void fh_destroy(fh_ctx* c) {
  if (!c) return;
  DeviceGuard dg(c->dev);
  if (c->stream) cudaStreamSynchronize(c->stream);
  prof_flush(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (CgGraph& G : c->cg_graph)
    if (G.exec) cudaGraphExecDestroy(G.exec);
  cudaFree(c->S);
  cudaFree(c->x);
  cudaFree(c->r);
  cudaFree(c->p);
  cudaFree(c->y);
  cudaFree(c->P);
  cudaFree(c->K);
  cudaFree(c->partials);
  cudaFree(c->params);
  cudaFree(c->tw);
  cudaFree(c->tw_df);
  cudaFree(c->K_df);
  cudaFree(c->sc);
  delete c;
}

int fh_constitutive(fh_ctx* ctx, const fh_material* mat, const double* F_dev, double* P_dev, double* K_dev,
                    double Pbar_out[9]) {
  g_err[0] = 0;
  if (!ctx || !F_dev) return fail(FH_ERR_ARG, "context or F is NULL");
  int rc = check_material(mat);
  if (rc) return rc;
  DeviceGuard dg(ctx->dev);
  MatView mv;
  if ((rc = upload_material(ctx, mat, &mv))) return rc;
  FH_CUDA(cudaMemsetAsync(&ctx->sc->flags, 0, sizeof(int), ctx->stream));
  FH_CUDA(prof(ctx, kPConst, [&] { return launch_constitutive(ctx->g, mv, F_dev, P_dev, K_dev, ctx->partials, &ctx->sc->flags, ctx->stream); }));
  if (Pbar_out) {
    double s[9];
    if ((rc = reduce9(ctx, (int)constitutive_ctas(ctx->g), s))) return rc;
    for (int c = 0; c < 9; ++c) Pbar_out[c] = s[c] / (double)ctx->g.n;
  }
  int flags = 0;
  if ((rc = read_flags(ctx, &flags))) return rc;
  if (flags & kFlagNonPhysical) return fail(FH_ERR_NONPHYSICAL, "det F <= 0 or non-finite value in some voxel");
  return FH_OK;
}

int fh_project(fh_ctx* ctx, const double* A_dev, double* out_dev, double scale, const double lengths[3]) {
  g_err[0] = 0;
  if (!ctx || !A_dev || !out_dev) return fail(FH_ERR_ARG, "NULL argument");
  if (!lengths_ok(lengths)) return fail(FH_ERR_ARG, "box lengths must be positive");
  DeviceGuard dg(ctx->dev);
  const Grid g = grid_with_lengths(ctx, lengths);
  const double c = scale / (2.0 * (double)g.n);
  int rc = run_projection(ctx, g, kZDirect, A_dev, nullptr, nullptr, c, kIZOut, out_dev, nullptr, nullptr);
  if (rc) return rc;
  FH_CUDA(cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  return FH_OK;
}

int fh_matvec(fh_ctx* ctx, const fh_material* mat, const double* F_dev, const double* K_dev, const double* p_dev,
              double* y_dev, const double lengths[3], int arith) {
  g_err[0] = 0;
  if (!ctx || !p_dev || !y_dev) return fail(FH_ERR_ARG, "NULL argument");
  if (p_dev == y_dev) return fail(FH_ERR_ARG, "y must not alias p");
  if (!lengths_ok(lengths)) return fail(FH_ERR_ARG, "box lengths must be positive");
  if (arith != FH_ARITH_FP64 && arith != FH_ARITH_DF64) return fail(FH_ERR_ARG, "invalid arith");
  const bool df = arith == FH_ARITH_DF64;
  DeviceGuard dg(ctx->dev);
  const Grid g = grid_with_lengths(ctx, lengths);
  const double c = 1.0 / (2.0 * (double)g.n);
  int rc;
  if (K_dev) {
    if (df && (rc = tangent_to_df64(ctx, g, K_dev))) return rc;
    rc = run_projection(ctx, g, kZKApply, p_dev, nullptr, K_dev, c, kIZOut, y_dev, nullptr, nullptr, nullptr, df);
    if (rc) return rc;
  } else {
    if (!F_dev) return fail(FH_ERR_ARG, "jvp form needs F");
    if ((rc = check_material(mat))) return rc;
    MatView mv;
    if ((rc = upload_material(ctx, mat, &mv))) return rc;
    FH_CUDA(cudaMemsetAsync(&ctx->sc->flags, 0, sizeof(int), ctx->stream));
    FH_CUDA(prof(ctx, kPJvp, [&] { return launch_jvp(g, mv, F_dev, p_dev, nullptr, nullptr, ctx->P, kZKApply, nullptr, &ctx->sc->flags, ctx->stream); }));
    rc = run_projection(ctx, g, kZDirect, ctx->P, nullptr, nullptr, c, kIZOut, y_dev, nullptr, nullptr, nullptr, df);
    if (rc) return rc;
    int flags = 0;
    if ((rc = read_flags(ctx, &flags))) return rc;
    if (flags & kFlagNonPhysical) return fail(FH_ERR_NONPHYSICAL, "det F <= 0 or non-finite value in some voxel");
  }
  FH_CUDA(cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  return FH_OK;
}

int fft_homog_solve(fh_ctx* ctx, const fh_material* mat, const double Fbar[9], int n_increments,
                    const fh_options* opt_in, double* F_dev, double Pbar_out[9], fh_stats* stats) {
  g_err[0] = 0;
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctx || !F_dev || !Fbar) return fail(FH_ERR_ARG, "NULL argument");
  int rc = check_material(mat);
  if (rc) return rc;
  fh_options opt;
  if (opt_in) opt = *opt_in;
  else fh_default_options(&opt);
  if (n_increments < 1) return fail(FH_ERR_ARG, "n_increments must be >= 1");
  if (!(opt.newton_tol > 0.0) || opt.max_newton < 1 || opt.max_cg < 0 || opt.check_every < 1 ||
      (opt.launch_mode != FH_LAUNCH_GRAPH && opt.launch_mode != FH_LAUNCH_PLAIN) ||
      (opt.matvec_arith != FH_ARITH_FP64 && opt.matvec_arith != FH_ARITH_DF64))
    return fail(FH_ERR_ARG, "invalid options");
  if (opt.init != FH_INIT_REFERENCE && opt.init != FH_INIT_GIVEN) return fail(FH_ERR_ARG, "invalid init");
  if (opt.tangent_mode != FH_TANGENT_STORED && opt.tangent_mode != FH_TANGENT_JVP)
    return fail(FH_ERR_ARG, "invalid tangent_mode");
  if (!lengths_ok(opt.lengths)) return fail(FH_ERR_ARG, "box lengths must be positive");
  for (int c = 0; c < 9; ++c)
    if (!std::isfinite(Fbar[c])) return fail(FH_ERR_ARG, "non-finite Fbar");
  const double cg_tol = opt.cg_tol > 0.0 ? opt.cg_tol : 1e-2 * opt.newton_tol;
  DeviceGuard dg(ctx->dev);
  cudaStream_t s = ctx->stream;
  const Grid g = grid_with_lengths(ctx, opt.lengths);
  const double N = (double)g.n;
  MatView mv;
  if ((rc = upload_material(ctx, mat, &mv))) return rc;
  FH_CUDA(cudaMemsetAsync(&ctx->sc->flags, 0, sizeof(int), s));
  const bool stored = opt.tangent_mode == FH_TANGENT_STORED;
  const long long replays0 = ctx->graph_replays, captures0 = ctx->graph_captures;

  // start tensor and load step (a1)
  double start[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (opt.init == FH_INIT_REFERENCE) {
    if (mat->kind != FH_LINEAR_ELASTIC && mat->kind != FH_J2) start[0] = start[4] = start[8] = 1.0;
    FH_CUDA(prof(ctx, kPFill, [&] { return launch_fill(g, F_dev, start, 0, s); }));
  } else {
    FH_CUDA(prof(ctx, kPFill, [&] { return launch_field_sums(g, F_dev, ctx->partials, s); }));
    if ((rc = reduce9(ctx, (int)constitutive_ctas(g), start))) return rc;
    for (int c = 0; c < 9; ++c) start[c] /= N;
  }
  double dFbar[9];
  for (int c = 0; c < 9; ++c) dFbar[c] = (Fbar[c] - start[c]) / n_increments;

  const int n_nu = (int)newton_update_ctas(g);
  const double c_rhs = -1.0 / (2.0 * N);
  int n_newton = 0, n_cg = 0, status = FH_OK;

  for (int inc = 1; inc <= n_increments && status == FH_OK; ++inc) {
    double Fn[9], nrm = 0.0;
    for (int c = 0; c < 9; ++c) {
      Fn[c] = start[c] + inc * dFbar[c];
      nrm += Fn[c] * Fn[c];
    }
    const double denom = (nrm > 0.0 ? std::sqrt(nrm) : 1.0) * std::sqrt(N);
    FH_CUDA(prof(ctx, kPFill, [&] { return launch_fill(g, F_dev, dFbar, 1, s); }));
    bool inc_converged = false;
    for (int it = 0; it < opt.max_newton; ++it) {
      // stress and tangent by AD (a2)
      FH_CUDA(prof(ctx, kPConst, [&] { return launch_constitutive(g, mv, F_dev, ctx->P, stored ? ctx->K : nullptr, ctx->partials,
                                  &ctx->sc->flags, s); }));
      int flags = 0;
      if ((rc = read_flags(ctx, &flags))) return rc;
      if (flags & kFlagNonPhysical) {
        status = fail(FH_ERR_NONPHYSICAL, "det F <= 0 or non-finite value (increment %d, Newton iteration %d)", inc,
                      it);
        break;
      }
      // right-hand side b = -G(P) (a3), r = b
      if ((rc = run_projection(ctx, g, kZDirect, ctx->P, nullptr, nullptr, c_rhs, kIZRhs, ctx->r, nullptr,
                               nullptr)))
        return rc;
      // CG on G(K : dF) = b (a4, a5); scalars stay on the device
      CgScalars host_cg{};
      if ((rc = run_cg(ctx, g, mv, F_dev, stored, cg_tol, opt, &host_cg))) return rc;
      // Newton update and convergence test (a6)
      FH_CUDA(prof(ctx, kPNewton, [&] { return launch_newton_update(g, F_dev, ctx->x, ctx->partials, s); }));
      FH_CUDA(prof(ctx, kPReduce, [&] { return launch_sum_partials(ctx->partials, n_nu, 1, ctx->sc->sums, s); }));
      double dd = 0.0;
      FH_CUDA(cudaMemcpyAsync(&dd, ctx->sc->sums, sizeof(double), cudaMemcpyDeviceToHost, s));
      FH_CUDA(cudaStreamSynchronize(s));
      prof_flush(ctx);
      const double e = std::sqrt(dd) / denom;
      if (stats && stats->newton_residuals && n_newton < stats->capacity) stats->newton_residuals[n_newton] = e;
      if (stats && stats->cg_iterations && n_newton < stats->capacity) stats->cg_iterations[n_newton] = host_cg.it;
      ++n_newton;
      n_cg += host_cg.it;
      if (host_cg.done != 1) {
        status = fail(FH_ERR_NOT_CONVERGED, "CG %s after %d products (increment %d, Newton iteration %d)",
                      host_cg.done == 2 ? "hit max_cg" : "broke down", host_cg.it, inc, it);
        break;
      }
      if (!std::isfinite(e)) {
        status = fail(FH_ERR_NONPHYSICAL, "non-finite Newton update");
        break;
      }
      if (e < opt.newton_tol) {
        inc_converged = true;
        break;
      }
    }
    if (inc_converged && mat->kind == FH_J2) {
      // plastic strain and cumulative plastic strain of the converged increment
      FH_CUDA(prof(ctx, kPConst, [&] { return launch_j2_update(g, mv, F_dev, mat->history, s); }));
    }
    if (status == FH_OK && !inc_converged)
      status = fail(FH_ERR_NOT_CONVERGED, "Newton hit max_newton=%d in increment %d", opt.max_newton, inc);
  }

  // homogenized stress of the final state (a7, Eq. 4)
  if (Pbar_out) {
    FH_CUDA(prof(ctx, kPConst, [&] { return launch_constitutive(g, mv, F_dev, nullptr, nullptr, ctx->partials, &ctx->sc->flags, s); }));
    double sums[9];
    if ((rc = reduce9(ctx, (int)constitutive_ctas(g), sums))) return rc;
    for (int c = 0; c < 9; ++c) Pbar_out[c] = sums[c] / N;
  }
  FH_CUDA(cudaStreamSynchronize(s));
  prof_flush(ctx);
  if (stats) {
    stats->n_newton = n_newton;
    stats->n_cg = n_cg;
    stats->n_recorded = stats->capacity < n_newton ? stats->capacity : n_newton;
    stats->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    stats->cg_graph_replays = (int)(ctx->graph_replays - replays0);
    stats->cg_graph_captures = (int)(ctx->graph_captures - captures0);
  }
  return status;
}

namespace {

int options_or_default(const fh_ctx* ctx, const fh_options* in, fh_options* o) {
  if (in) *o = *in;
  else fh_default_options(o);
  if (!(o->newton_tol > 0.0) || o->max_cg < 0 || o->check_every < 1 ||
      (o->launch_mode != FH_LAUNCH_GRAPH && o->launch_mode != FH_LAUNCH_PLAIN) ||
      (o->matvec_arith != FH_ARITH_FP64 && o->matvec_arith != FH_ARITH_DF64))
    return fail(FH_ERR_ARG, "invalid options");
  if (!lengths_ok(o->lengths)) return fail(FH_ERR_ARG, "box lengths must be positive");
  return FH_OK;
}

// unit response E_cd + d: b = -G(K : E_cd) into r, then CG; d in ctx->x
int unit_response(fh_ctx* ctx, const Grid& g, const MatView& mv, int cd, double cg_tol, const fh_options& opt,
                  CgScalars* host_cg) {
  double e[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  e[cd] = 1.0;
  FH_CUDA(prof(ctx, kPFill, [&] { return launch_fill(g, ctx->y, e, 0, ctx->stream); }));
  int rc = run_projection(ctx, g, kZKApply, ctx->y, nullptr, ctx->K, -1.0 / (2.0 * (double)g.n), kIZRhs, ctx->r,
                          nullptr, nullptr);
  if (rc) return rc;
  if ((rc = run_cg(ctx, g, mv, nullptr, true, cg_tol, opt, host_cg))) return rc;
  if (host_cg->done != 1)
    return fail(FH_ERR_NOT_CONVERGED, "tangent CG %s after %d products (column %d)",
                host_cg->done == 2 ? "hit max_cg" : "broke down", host_cg->it, cd);
  return FH_OK;
}

}  // namespace

int fft_homog_tangent(fh_ctx* ctx, const fh_material* mat, const double* F_dev, const fh_options* opt_in,
                      double Cbar_out[81]) {
  g_err[0] = 0;
  if (!ctx || !F_dev || !Cbar_out) return fail(FH_ERR_ARG, "NULL argument");
  int rc = check_material(mat);
  if (rc) return rc;
  if (mat->kind == FH_J2)
    return fail(FH_ERR_UNSUPPORTED, "the homogenized tangent is implemented for hyperelastic laws");
  fh_options opt;
  if ((rc = options_or_default(ctx, opt_in, &opt))) return rc;
  const double cg_tol = opt.cg_tol > 0.0 ? opt.cg_tol : 1e-2 * opt.newton_tol;
  DeviceGuard dg(ctx->dev);
  cudaStream_t s = ctx->stream;
  const Grid g = grid_with_lengths(ctx, opt.lengths);
  MatView mv;
  if ((rc = upload_material(ctx, mat, &mv))) return rc;
  FH_CUDA(cudaMemsetAsync(&ctx->sc->flags, 0, sizeof(int), s));
  FH_CUDA(prof(ctx, kPConst, [&] {
    return launch_constitutive(g, mv, F_dev, nullptr, ctx->K, ctx->partials, &ctx->sc->flags, s);
  }));
  int flags = 0;
  if ((rc = read_flags(ctx, &flags))) return rc;
  if (flags & kFlagNonPhysical) return fail(FH_ERR_NONPHYSICAL, "det F <= 0 or non-finite value in some voxel");
  const int n_k = (int)kapply_sums_ctas(g);
  for (int cd = 0; cd < 9; ++cd) {
    CgScalars host_cg{};
    if ((rc = unit_response(ctx, g, mv, cd, cg_tol, opt, &host_cg))) return rc;
    FH_CUDA(prof(ctx, kPContract, [&] { return launch_kapply_sums(g, ctx->K, ctx->x, cd, ctx->partials, s); }));
    double col[9];
    if ((rc = reduce9(ctx, n_k, col))) return rc;
    for (int ab = 0; ab < 9; ++ab) Cbar_out[9 * ab + cd] = col[ab] / (double)g.n;
  }
  return FH_OK;
}

int fft_homog_sensitivity(fh_ctx* ctx, const fh_material* mat, const fh_options* opt_in, int i, int j, int k, int l,
                          const double* dscale_dev, double* out_dev) {
  g_err[0] = 0;
  if (!ctx || !dscale_dev || !out_dev) return fail(FH_ERR_ARG, "NULL argument");
  int rc = check_material(mat);
  if (rc) return rc;
  if (mat->kind != FH_LINEAR_ELASTIC)
    return fail(FH_ERR_UNSUPPORTED, "sensitivities are implemented for small-strain linear elasticity only");
  if (i < 0 || i > 2 || j < 0 || j > 2 || k < 0 || k > 2 || l < 0 || l > 2)
    return fail(FH_ERR_ARG, "tensor indices must be 0, 1 or 2");
  fh_options opt;
  if ((rc = options_or_default(ctx, opt_in, &opt))) return rc;
  const double cg_tol = opt.cg_tol > 0.0 ? opt.cg_tol : 1e-2 * opt.newton_tol;
  DeviceGuard dg(ctx->dev);
  cudaStream_t s = ctx->stream;
  const Grid g = grid_with_lengths(ctx, opt.lengths);
  MatView mv;
  if ((rc = upload_material(ctx, mat, &mv))) return rc;
  FH_CUDA(cudaMemsetAsync(&ctx->sc->flags, 0, sizeof(int), s));
  // the linear tangent does not depend on the state: evaluate it at H = 0
  FH_CUDA(cudaMemsetAsync(ctx->p, 0, (size_t)9 * g.n * sizeof(double), s));
  FH_CUDA(prof(ctx, kPConst, [&] {
    return launch_constitutive(g, mv, ctx->p, nullptr, ctx->K, ctx->partials, &ctx->sc->flags, s);
  }));
  int flags = 0;
  if ((rc = read_flags(ctx, &flags))) return rc;
  if (flags & kFlagNonPhysical) return fail(FH_ERR_NONPHYSICAL, "non-finite modulus in some voxel");
  const int ab = 3 * i + j, cd = 3 * k + l;
  CgScalars host_cg{};
  if ((rc = unit_response(ctx, g, mv, ab, cg_tol, opt, &host_cg))) return rc;
  const double* xa = ctx->x;
  if (cd != ab) {
    FH_CUDA(cudaMemcpyAsync(ctx->P, ctx->x, (size_t)9 * g.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    xa = ctx->P;
    if ((rc = unit_response(ctx, g, mv, cd, cg_tol, opt, &host_cg))) return rc;
  }
  MatView base = mv;
  base.scale = nullptr;
  FH_CUDA(prof(ctx, kPContract, [&] {
    return launch_sensitivity(g, base, xa, ab, ctx->x, cd, dscale_dev, out_dev, s);
  }));
  FH_CUDA(cudaStreamSynchronize(s));
  prof_flush(ctx);
  return FH_OK;
}

int fft_homog_stress_sensitivity(fh_ctx* ctx, const fh_material* mat, const double* F_dev, const fh_options* opt_in,
                                 int i, int j, const double* dscale_dev, double* out_dev) {
  g_err[0] = 0;
  if (!ctx || !F_dev || !dscale_dev || !out_dev) return fail(FH_ERR_ARG, "NULL argument");
  int rc = check_material(mat);
  if (rc) return rc;
  if (mat->kind == FH_J2)
    return fail(FH_ERR_UNSUPPORTED, "stress sensitivities are implemented for hyperelastic and linear elastic laws");
  if (i < 0 || i > 2 || j < 0 || j > 2) return fail(FH_ERR_ARG, "tensor indices must be 0, 1 or 2");
  fh_options opt;
  if ((rc = options_or_default(ctx, opt_in, &opt))) return rc;
  const double cg_tol = opt.cg_tol > 0.0 ? opt.cg_tol : 1e-2 * opt.newton_tol;
  DeviceGuard dg(ctx->dev);
  cudaStream_t s = ctx->stream;
  const Grid g = grid_with_lengths(ctx, opt.lengths);
  MatView mv;
  if ((rc = upload_material(ctx, mat, &mv))) return rc;
  FH_CUDA(cudaMemsetAsync(&ctx->sc->flags, 0, sizeof(int), s));
  // tangent of the converged state with the scaled moduli, then the unit response d_ab
  FH_CUDA(prof(ctx, kPConst, [&] {
    return launch_constitutive(g, mv, F_dev, nullptr, ctx->K, ctx->partials, &ctx->sc->flags, s);
  }));
  int flags = 0;
  if ((rc = read_flags(ctx, &flags))) return rc;
  if (flags & kFlagNonPhysical) return fail(FH_ERR_NONPHYSICAL, "det F <= 0 or non-finite value in some voxel");
  const int ab = 3 * i + j;
  CgScalars host_cg{};
  if ((rc = unit_response(ctx, g, mv, ab, cg_tol, opt, &host_cg))) return rc;
  FH_CUDA(prof(ctx, kPContract, [&] {
    return launch_stress_sensitivity(g, mv, F_dev, ctx->x, ab, dscale_dev, out_dev, s);
  }));
  FH_CUDA(cudaStreamSynchronize(s));
  prof_flush(ctx);
  return FH_OK;
}

namespace {

// z lines per CTA must divide nx*ny; shared memory of a z pass must fit a CTA
bool tiling_fits(const Grid& g, const Tiling& t) {
  const long long lines = (long long)g.nx * g.ny;
  if (t.lines_z < 1 || lines % t.lines_z) return false;
  if (t.bk_y < 1 || t.bk_y > g.nzh || t.bk_x < 1 || t.bk_x > g.nzh) return false;
  const size_t limit = 227 * 1024;
  const size_t zs = ((size_t)9 * t.lines_z * g.nz + g.nz) * sizeof(double2);
  const int twy = g.py.L ? g.py.tw_len : g.ny, twx = g.px.L ? g.px.tw_len : g.nx;
  const size_t ys = ((size_t)2 * 3 * t.bk_y * (g.ny + 1) + twy) * sizeof(double2);
  const size_t xs = ((size_t)2 * 6 * t.bk_x * (g.nx + 1) + twx) * sizeof(double2);
  return zs <= limit && ys <= limit && xs <= limit;
}

}  // namespace

int fh_autotune(fh_ctx* ctx, int reps, double* best_ms, int chosen[3]) {
  g_err[0] = 0;
  if (!ctx) return fail(FH_ERR_ARG, "context is NULL");
  if (reps < 1) reps = 3;
  DeviceGuard dg(ctx->dev);
  cudaStream_t s = ctx->stream;
  const Grid& g = ctx->g;
  const Tiling base = choose_tiling(g, ctx->min_ctas);
  std::vector<Tiling> cand;
  for (int fz : {1, 2, 4}) {
    for (int fy : {1, 2}) {
      for (int fx : {1, 2}) {
        Tiling t = base;
        t.lines_z = std::max(1, base.lines_z * fz / 2);
        while ((long long)g.nx * g.ny % t.lines_z) --t.lines_z;
        t.bk_y = std::min(g.nzh, std::max(1, base.bk_y * fy));
        t.bk_x = std::min(g.nzh, std::max(1, base.bk_x * fx));
        if (!tiling_fits(g, t)) continue;
        bool dup = false;
        for (const Tiling& u : cand) dup |= (u.lines_z == t.lines_z && u.bk_y == t.bk_y && u.bk_x == t.bk_x);
        if (!dup) cand.push_back(t);
      }
    }
  }
  cudaEvent_t e0, e1;
  FH_CUDA(cudaEventCreate(&e0));
  FH_CUDA(cudaEventCreate(&e1));
  FH_CUDA(cudaMemsetAsync(ctx->y, 0, (size_t)9 * g.n * sizeof(double), s));
  const Tiling keep = ctx->tiling;
  float best = 1e30f;
  Tiling best_t = keep;
  for (const Tiling& t : cand) {
    ctx->tiling = t;
    cudaError_t e = setup_fft_kernels(g, t);
    if (e != cudaSuccess) continue;
    int rc = run_projection(ctx, g, kZDirect, ctx->y, nullptr, nullptr, 1.0, kIZOut, ctx->p, nullptr, nullptr);
    if (rc) continue;
    FH_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r)
      if ((rc = run_projection(ctx, g, kZDirect, ctx->y, nullptr, nullptr, 1.0, kIZOut, ctx->p, nullptr, nullptr)))
        break;
    FH_CUDA(cudaEventRecord(e1, s));
    FH_CUDA(cudaEventSynchronize(e1));
    if (rc) continue;
    float ms = 0.f;
    FH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    ms /= reps;
    if (ms < best) {
      best = ms;
      best_t = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  prof_flush(ctx);
  ctx->tiling = best_t;
  FH_CUDA(setup_fft_kernels(g, best_t));
  if (best_ms) *best_ms = best;
  if (chosen) {
    chosen[0] = best_t.lines_z;
    chosen[1] = best_t.bk_y;
    chosen[2] = best_t.bk_x;
  }
  return FH_OK;
}

int fh_profile_enable(fh_ctx* ctx, int enable) {
  g_err[0] = 0;
  if (!ctx) return fail(FH_ERR_ARG, "context is NULL");
  DeviceGuard dg(ctx->dev);
  FH_CUDA(cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  for (int i = 0; i < FH_PROF_NCLASS; ++i) {
    ctx->counts[i] = 0;
    ctx->ms[i] = 0.0;
  }
  ctx->prof = enable != 0;
  return FH_OK;
}

int fh_twiddle_tables(double* out, int capacity) {
  g_err[0] = 0;
  if (!out || capacity < kTwiddleTables) return kTwiddleTables;
  std::vector<double2> t(kTwiddleTables);
  fill_twiddle_table(t.data());
  for (int i = 0; i < kTwiddleTables; ++i) {
    out[2 * i] = t[i].x;
    out[2 * i + 1] = t[i].y;
  }
  return kTwiddleTables;
}

int fh_profile_read(fh_ctx* ctx, long long counts[FH_PROF_NCLASS], double ms[FH_PROF_NCLASS]) {
  g_err[0] = 0;
  if (!ctx) return fail(FH_ERR_ARG, "context is NULL");
  DeviceGuard dg(ctx->dev);
  FH_CUDA(cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  for (int i = 0; i < FH_PROF_NCLASS; ++i) {
    if (counts) counts[i] = ctx->counts[i];
    if (ms) ms[i] = ctx->ms[i];
  }
  return FH_OK;
}

}  // extern "C"
