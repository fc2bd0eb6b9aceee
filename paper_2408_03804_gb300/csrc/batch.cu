// Batched solve of many independent cells of uneven grids (the paper's
// uncertainty-quantification setting of Section 4.4.1, Monte-Carlo style):
// every cell runs Algorithm 1 with its own Newton and CG state, but each pass
// is one launch per group of equal grids (blockIdx.y = cell), and a cell whose
// CG or Newton loop has finished is masked out of the launches by its device
// flag. The CG iterations of all groups are captured once as a CUDA graph and
// replayed, so the host issues one graph launch per `check_every` iterations
// of the whole batch.
#include <chrono>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "fh_kernels.h"

using namespace fh;

extern "C" void fh_internal_set_error(const char* msg);

namespace {

int bfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  fh_internal_set_error(buf);
  return code;
}

#define FB_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return bfail(FH_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct Group {
  Grid g{};
  Tiling t{};
  std::vector<int> cells;       // indices into the batch's cells
  CellState* states = nullptr;  // device [n]
  CellView* views_rhs = nullptr;  // device [n]: P -> r, masked by the Newton flag
  CellView* views_cg = nullptr;   // device [n]: r -> y, masked by the CG flag
  int n_iz = 0, n_pw = 0;
};

}  // namespace

struct fh_batch {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;         // created here because the caller passed the legacy stream
  std::vector<fh_cell> cells;
  std::vector<Group> groups;
  std::vector<void*> allocs;       // every device allocation of the batch
  CgScalars* cg = nullptr;         // device [n_cells]
  double* sums = nullptr;          // device [n_cells][16]
  int* newton_done = nullptr;      // device [n_cells]
  int* flags = nullptr;            // device [n_cells]
  double* params = nullptr;        // device [256][2]
  double2* tw = nullptr;
  cudaGraphExec_t chunk = nullptr;  // check_every CG iterations of every group
  int chunk_len = 0;
};

namespace {

template <class T>
int dalloc(fh_batch* b, T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return bfail(FH_ERR_CUDA, "fh_batch_create: allocation of %zu bytes failed: %s", bytes,
                                     cudaGetErrorString(e));
  b->allocs.push_back(q);
  *p = (T*)q;
  return FH_OK;
}

// one CG iteration (after the first) for every group
int launch_cg_iteration(fh_batch* b, bool first) {
  cudaStream_t s = b->stream;
  for (Group& G : b->groups) {
    const int n = (int)G.cells.size();
    const double c_mv = 1.0 / (2.0 * (double)G.g.n);
    FB_CUDA(launch_fwd_z_batch(G.g, G.t, first ? kZCgFirst : kZCg, G.views_cg, n, b->tw, s));
    FB_CUDA(launch_fwd_y_batch(G.g, G.t, G.views_cg, n, b->tw, s));
    FB_CUDA(launch_x_ghat_batch(G.g, G.t, G.views_cg, n, b->tw, c_mv, s));
    FB_CUDA(launch_inv_y_batch(G.g, G.t, G.views_cg, n, b->tw, s));
    FB_CUDA(launch_inv_z_batch(G.g, G.t, kIZDot, G.views_cg, n, b->tw, s));
    FB_CUDA(launch_cg_alpha_batch(G.states, n, G.n_iz, s));
    FB_CUDA(launch_cg_update_batch(G.g, G.states, n, s));
    FB_CUDA(launch_cg_beta_batch(G.states, n, G.n_pw, s));
  }
  return FH_OK;
}

int capture_chunk(fh_batch* b, int len) {
  if (b->chunk && b->chunk_len == len) return FH_OK;
  if (b->chunk) {
    cudaGraphExecDestroy(b->chunk);
    b->chunk = nullptr;
  }
  cudaGraph_t graph = nullptr;
  FB_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int rc = FH_OK;
  for (int k = 0; k < len && rc == FH_OK; ++k) rc = launch_cg_iteration(b, false);
  cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return bfail(FH_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->chunk, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(FH_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  b->chunk_len = len;
  return FH_OK;
}

}  // namespace

extern "C" {

int fh_batch_create(fh_batch** out, const fh_cell* cells, int n_cells, void* cuda_stream) {
  fh_internal_set_error("");
  if (!out || !cells || n_cells < 1) return bfail(FH_ERR_ARG, "fh_batch_create: no cells");
  for (int i = 0; i < n_cells; ++i) {
    const fh_cell& c = cells[i];
    if (!grid_extents_ok(c.nx, c.ny, c.nz))
      return bfail(FH_ERR_ARG, "fh_batch_create: cell %d grid %dx%dx%d unsupported (extents 2^a or 3*2^a up to 256, "
                   "nz even with nz/2 of that form)", i, c.nx, c.ny, c.nz);
    if (!c.phase || !c.F) return bfail(FH_ERR_ARG, "fh_batch_create: cell %d has a NULL phase or F", i);
  }
  fh_batch* b = new fh_batch();
  auto cleanup = [&](int code) {
    fh_batch_destroy(b);
    return code;
  };
  if (cudaGetDevice(&b->dev) != cudaSuccess) return cleanup(bfail(FH_ERR_CUDA, "cudaGetDevice failed"));
  b->stream = (cudaStream_t)cuda_stream;
  if (!b->stream) {
    // graphs cannot be captured on the legacy stream: use a blocking stream of
    // our own, which orders itself with the legacy stream
    if (cudaStreamCreate(&b->stream) != cudaSuccess) return cleanup(bfail(FH_ERR_CUDA, "cudaStreamCreate failed"));
    b->own_stream = true;
  }
  b->cells.assign(cells, cells + n_cells);
  int rc;
  if ((rc = dalloc(b, &b->cg, sizeof(CgScalars) * n_cells)) || (rc = dalloc(b, &b->sums, 16 * sizeof(double) * n_cells)) ||
      (rc = dalloc(b, &b->newton_done, sizeof(int) * n_cells)) || (rc = dalloc(b, &b->flags, sizeof(int) * n_cells)) ||
      (rc = dalloc(b, &b->params, 512 * sizeof(double))) || (rc = dalloc(b, &b->tw, kTwiddleTotal * sizeof(double2))))
    return cleanup(rc);
  std::vector<double2> tw(kTwiddleTotal);
  fill_twiddle_table(tw.data());
  if (cudaMemcpy(b->tw, tw.data(), kTwiddleTotal * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess)
    return cleanup(bfail(FH_ERR_CUDA, "twiddle upload failed"));
  // group the cells by grid shape
  std::map<long long, int> key_to_group;
  for (int i = 0; i < n_cells; ++i) {
    const long long key = ((long long)cells[i].nx << 40) | ((long long)cells[i].ny << 20) | cells[i].nz;
    auto it = key_to_group.find(key);
    if (it == key_to_group.end()) {
      Group G;
      G.g.nx = cells[i].nx;
      G.g.ny = cells[i].ny;
      G.g.nz = cells[i].nz;
      G.g.nzh = G.g.nz / 2 + 1;
      G.g.n = (long long)G.g.nx * G.g.ny * G.g.nz;
      G.g.nspec = (long long)G.g.nx * G.g.ny * G.g.nzh;
      G.g.sx = G.g.sy = G.g.sz = 1.0;
      G.t = choose_tiling(G.g);
      G.n_iz = (int)z_pass_ctas(G.g, G.t);
      G.n_pw = (int)cg_update_ctas(G.g);
      key_to_group[key] = (int)b->groups.size();
      b->groups.push_back(G);
      it = key_to_group.find(key);
    }
    b->groups[it->second].cells.push_back(i);
  }
  for (Group& G : b->groups) {
    const int n = (int)G.cells.size();
    const size_t f9 = (size_t)9 * G.g.n * sizeof(double);
    long long np = 9LL * constitutive_ctas(G.g);
    if (np < G.n_iz) np = G.n_iz;
    std::vector<CellState> st(n);
    std::vector<CellView> vr(n), vc(n);
    for (int j = 0; j < n; ++j) {
      const int i = G.cells[j];
      CellState& c = st[j];
      if ((rc = dalloc(b, &c.x, f9)) || (rc = dalloc(b, &c.r, f9)) || (rc = dalloc(b, &c.p, f9)) ||
          (rc = dalloc(b, &c.y, f9)) || (rc = dalloc(b, &c.P, f9)) ||
          (rc = dalloc(b, &c.K, (size_t)45 * G.g.n * sizeof(double))) ||
          (rc = dalloc(b, &c.S, (size_t)9 * G.g.nspec * sizeof(double2))) ||
          (rc = dalloc(b, &c.partials, (size_t)np * sizeof(double))))
        return cleanup(rc);
      c.F = cells[i].F;
      c.sums = b->sums + 16 * i;
      c.cg = b->cg + i;
      c.phase = cells[i].phase;
      c.scale = cells[i].scale;
      c.newton_done = b->newton_done + i;
      c.flags = b->flags + i;
      vr[j] = CellView{c.newton_done, c.P, c.p, c.x, c.K, c.cg, c.S, c.r, c.partials};
      vc[j] = CellView{&c.cg->done, c.r, c.p, c.x, c.K, c.cg, c.S, c.y, c.partials};
    }
    if ((rc = dalloc(b, &G.states, sizeof(CellState) * n)) || (rc = dalloc(b, &G.views_rhs, sizeof(CellView) * n)) ||
        (rc = dalloc(b, &G.views_cg, sizeof(CellView) * n)))
      return cleanup(rc);
    if (cudaMemcpy(G.states, st.data(), sizeof(CellState) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.views_rhs, vr.data(), sizeof(CellView) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.views_cg, vc.data(), sizeof(CellView) * n, cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup(bfail(FH_ERR_CUDA, "fh_batch_create: descriptor upload failed"));
    if (setup_fft_kernels(G.g, G.t) != cudaSuccess) return cleanup(bfail(FH_ERR_CUDA, "kernel set-up failed"));
  }
  *out = b;
  return FH_OK;
}

void fh_batch_destroy(fh_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->chunk) cudaGraphExecDestroy(b->chunk);
  for (void* p : b->allocs) cudaFree(p);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

int fft_homog_solve_batched(fh_batch* b, int kind, int n_phase, const double* params, const double Fbar[9],
                            int n_increments, const fh_options* opt_in, double* Pbar_out, int* status_out,
                            int* newton_out, int* cg_out) {
  fh_internal_set_error("");
  const auto t0 = std::chrono::steady_clock::now();
  (void)t0;
  if (!b || !params || !Fbar) return bfail(FH_ERR_ARG, "fft_homog_solve_batched: NULL argument");
  if (kind < FH_LINEAR_ELASTIC || kind > FH_SVK)
    return bfail(kind == FH_J2 ? FH_ERR_UNSUPPORTED : FH_ERR_ARG, "material kind %d not available in batched solves",
                 kind);
  if (n_phase < 1 || n_phase > 256) return bfail(FH_ERR_ARG, "n_phase %d outside 1..256", n_phase);
  if (n_increments < 1) return bfail(FH_ERR_ARG, "n_increments must be >= 1");
  fh_options opt;
  if (opt_in) opt = *opt_in;
  else fh_default_options(&opt);
  if (!(opt.newton_tol > 0.0) || opt.max_newton < 1 || opt.max_cg < 0 || opt.check_every < 1)
    return bfail(FH_ERR_ARG, "invalid options");
  if (opt.init != FH_INIT_REFERENCE) return bfail(FH_ERR_UNSUPPORTED, "batched solves start from the reference state");
  if (opt.tangent_mode != FH_TANGENT_STORED) return bfail(FH_ERR_UNSUPPORTED, "batched solves store the tangent");
  if (opt.lengths[0] != 1.0 || opt.lengths[1] != 1.0 || opt.lengths[2] != 1.0)
    return bfail(FH_ERR_UNSUPPORTED, "batched solves use unit boxes");
  const double cg_tol = opt.cg_tol > 0.0 ? opt.cg_tol : 1e-2 * opt.newton_tol;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->dev) cudaSetDevice(b->dev);
  cudaStream_t s = b->stream;
  const int nc = (int)b->cells.size();
  {
    std::vector<double> tab(512, std::nan(""));
    for (int i = 0; i < 2 * n_phase; ++i) tab[i] = params[i];
    FB_CUDA(cudaMemcpyAsync(b->params, tab.data(), 512 * sizeof(double), cudaMemcpyHostToDevice, s));
    FB_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int> status(nc, FH_OK), newton(nc, 0), cgs(nc, 0), done(nc, 0);
  std::vector<CgScalars> hcg(nc);
  std::vector<double> hs(16 * (size_t)nc);
  FB_CUDA(cudaMemsetAsync(b->flags, 0, sizeof(int) * nc, s));
  FB_CUDA(cudaMemsetAsync(b->newton_done, 0, sizeof(int) * nc, s));

  double start[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (kind != FH_LINEAR_ELASTIC) start[0] = start[4] = start[8] = 1.0;
  double dFbar[9], nrm = 0.0;
  for (int c = 0; c < 9; ++c) dFbar[c] = (Fbar[c] - start[c]) / n_increments;
  for (Group& G : b->groups) FB_CUDA(launch_fill_batch(G.g, G.states, (int)G.cells.size(), 0, start, 0, s));
  int rc = capture_chunk(b, opt.check_every);
  if (rc) return rc;

  for (int inc = 1; inc <= n_increments; ++inc) {
    nrm = 0.0;
    for (int c = 0; c < 9; ++c) {
      const double v = start[c] + inc * dFbar[c];
      nrm += v * v;
    }
    for (Group& G : b->groups) FB_CUDA(launch_fill_batch(G.g, G.states, (int)G.cells.size(), 0, dFbar, 1, s));
    for (int i = 0; i < nc; ++i) done[i] = status[i] != FH_OK;
    FB_CUDA(cudaMemcpyAsync(b->newton_done, done.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    for (int it = 0; it < opt.max_newton; ++it) {
      // stress and tangent (a2), right-hand side (a3)
      for (Group& G : b->groups) {
        const int n = (int)G.cells.size();
        FB_CUDA(launch_constitutive_batch(G.g, kind, b->params, G.states, n, 1, s));
        FB_CUDA(launch_fwd_z_batch(G.g, G.t, kZDirect, G.views_rhs, n, b->tw, s));
        FB_CUDA(launch_fwd_y_batch(G.g, G.t, G.views_rhs, n, b->tw, s));
        FB_CUDA(launch_x_ghat_batch(G.g, G.t, G.views_rhs, n, b->tw, -1.0 / (2.0 * (double)G.g.n), s));
        FB_CUDA(launch_inv_y_batch(G.g, G.t, G.views_rhs, n, b->tw, s));
        FB_CUDA(launch_inv_z_batch(G.g, G.t, kIZRhs, G.views_rhs, n, b->tw, s));
        FB_CUDA(launch_cg_init_batch(G.states, n, G.n_iz, cg_tol, opt.max_cg, s));
        const double zero[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        FB_CUDA(launch_fill_batch(G.g, G.states, n, 1, zero, 0, s));
      }
      // CG (a4, a5): the first iteration by hand, then graph chunks
      if ((rc = launch_cg_iteration(b, true))) return rc;
      int launched = 1;
      while (true) {
        FB_CUDA(cudaGraphLaunch(b->chunk, s));
        launched += b->chunk_len;
        FB_CUDA(cudaMemcpyAsync(hcg.data(), b->cg, sizeof(CgScalars) * nc, cudaMemcpyDeviceToHost, s));
        FB_CUDA(cudaStreamSynchronize(s));
        bool all = true;
        for (int i = 0; i < nc; ++i) all = all && hcg[i].done != 0;
        if (all) break;
        if (launched > opt.max_cg + 2 * opt.check_every) return bfail(FH_ERR_CUDA, "batched CG did not finish");
      }
      for (Group& G : b->groups) {
        const int n = (int)G.cells.size();
        FB_CUDA(launch_cg_finalize_batch(G.g, G.states, n, s));
        FB_CUDA(launch_newton_update_batch(G.g, G.states, n, s));
        FB_CUDA(launch_sum_partials_batch(G.states, n, G.n_pw, 1, s));
      }
      std::vector<int> flags(nc);
      FB_CUDA(cudaMemcpyAsync(hs.data(), b->sums, sizeof(double) * 16 * nc, cudaMemcpyDeviceToHost, s));
      FB_CUDA(cudaMemcpyAsync(flags.data(), b->flags, sizeof(int) * nc, cudaMemcpyDeviceToHost, s));
      FB_CUDA(cudaStreamSynchronize(s));
      bool all_done = true;
      for (Group& G : b->groups) {
        const double denom = (nrm > 0.0 ? std::sqrt(nrm) : 1.0) * std::sqrt((double)G.g.n);
        for (int i : G.cells) {
          if (done[i]) continue;
          newton[i] += 1;
          cgs[i] += hcg[i].it;
          const double e = std::sqrt(hs[16 * i]) / denom;
          if (flags[i]) {
            status[i] = FH_ERR_NONPHYSICAL;
            done[i] = 1;
          } else if (hcg[i].done != 1) {
            status[i] = FH_ERR_NOT_CONVERGED;
            done[i] = 1;
          } else if (e < opt.newton_tol) {
            done[i] = 1;
          }
          all_done = all_done && done[i];
        }
      }
      FB_CUDA(cudaMemcpyAsync(b->newton_done, done.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
      if (all_done) break;
      if (it == opt.max_newton - 1)
        for (int i = 0; i < nc; ++i)
          if (!done[i]) status[i] = FH_ERR_NOT_CONVERGED;
    }
  }
  // homogenized stress of every cell (a7)
  std::vector<int> zeros(nc, 0);
  FB_CUDA(cudaMemcpyAsync(b->newton_done, zeros.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
  for (Group& G : b->groups) {
    const int n = (int)G.cells.size();
    FB_CUDA(launch_constitutive_batch(G.g, kind, b->params, G.states, n, 0, s));
    FB_CUDA(launch_sum_partials_batch(G.states, n, (int)constitutive_ctas(G.g), 9, s));
  }
  FB_CUDA(cudaMemcpyAsync(hs.data(), b->sums, sizeof(double) * 16 * nc, cudaMemcpyDeviceToHost, s));
  FB_CUDA(cudaStreamSynchronize(s));
  int worst = FH_OK;
  for (Group& G : b->groups)
    for (int i : G.cells) {
      if (Pbar_out)
        for (int c = 0; c < 9; ++c) Pbar_out[9 * i + c] = hs[16 * i + c] / (double)G.g.n;
      if (status_out) status_out[i] = status[i];
      if (newton_out) newton_out[i] = newton[i];
      if (cg_out) cg_out[i] = cgs[i];
      if (status[i] != FH_OK && worst == FH_OK) worst = status[i];
    }
  if (prev >= 0 && prev != b->dev) cudaSetDevice(prev);
  if (worst != FH_OK) return bfail(worst, "fft_homog_solve_batched: some cells did not converge (see status_out)");
  return FH_OK;
}

}  // extern "C"
