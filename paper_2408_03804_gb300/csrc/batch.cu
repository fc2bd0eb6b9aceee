// Batched solve of many independent cells of uneven grids (the paper's
// uncertainty-quantification setting of Section 4.4.1, Monte-Carlo style):
// every cell runs Algorithm 1 with its own Newton and CG state, but each pass
// is one launch per group of equal grids (blockIdx.y = cell), and a cell that
// takes no part in a launch is masked out of it by a device flag.
//
// The Newton loop runs on the device, one state machine per cell (stage:
// load increment, right-hand side, CG, done): one captured CUDA graph holds,
// for every group, the end of a Newton iteration for the cells whose CG has
// stopped (x += alpha p, F += x, ||x||, the convergence test of Algorithm 1
// and the next stage), the load increment, the stress/tangent evaluation and
// right-hand side for the cells starting a Newton iteration, and then
// `check_every` CG iterations. The host replays the graph and reads the cells'
// stages after each replay, so no cell waits for another at a Newton step:
// a cell whose CG has converged goes on with its own next Newton iteration at
// the next replay.
#include <chrono>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "df64.cuh"
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
  std::vector<int> cells;         // indices into the batch's cells
  int* cell_ids = nullptr;        // device [n]: the same indices
  CellState* states = nullptr;    // device [n]: every cell takes part
  CellState* states_end = nullptr;  // device [n]: masked but for cells ending a Newton iteration
  CellState* states_inc = nullptr;  // device [n]: masked but for cells starting a load increment
  CellState* states_rhs = nullptr;  // device [n]: masked but for cells starting a Newton iteration
  CellView* views_rhs = nullptr;  // device [n]: P -> r, masked like states_rhs
  CellView* views_cg = nullptr;   // device [n]: r -> y, masked by the CG done flag
  int n_iz = 0, n_pw = 0;
};

// per-cell Newton state on the device
struct CellCtl {
  int stage;          // kStage*
  int inc;            // current load increment (1-based)
  int newton_it;      // Newton iterations in this increment
  int newton_total;
  int cg_total;
  int status;         // FH_OK, FH_ERR_NOT_CONVERGED or FH_ERR_NONPHYSICAL once done
  int mask_end, mask_inc, mask_rhs;  // 0: the cell takes part in that phase of the current replay
  int zero;           // always 0 (mask of the every-cell descriptors)
};
enum : int { kStageInc = 0, kStageRhs = 1, kStageCg = 2, kStageDone = 3 };

// solve parameters baked into the captured graph
struct SolveParams {
  double start[9], dfbar[9];
  double newton_tol, cg_tol;
  int n_inc, max_newton, max_cg, check_every, kind;
  int df;  // CG products with double-float transforms (FH_ARITH_DF64)
  bool operator==(const SolveParams& o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};

// phase masks; phase 0: cells whose CG has stopped end their Newton iteration;
// 1: cells at a new increment apply it (and go on to the right-hand side);
// 2: cells at the right-hand side compute it (and go on to CG)
__global__ void k_batch_masks(CellCtl* __restrict__ ctl, const CgScalars* __restrict__ cg,
                              const int* __restrict__ ids, int n, int phase) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  CellCtl& c = ctl[ids[j]];
  if (phase == 0) {
    c.mask_end = !(c.stage == kStageCg && cg[ids[j]].done != 0);
  } else if (phase == 1) {
    c.mask_inc = c.stage != kStageInc;
    if (c.stage == kStageInc) c.stage = kStageRhs;
  } else {
    c.mask_rhs = c.stage != kStageRhs;
    if (c.stage == kStageRhs) c.stage = kStageCg;
  }
}

// the end of a Newton iteration (Algorithm 1): with ||dF||^2 in sums[0],
// e = ||dF|| / (||Fbar_n|| sqrt(N)); converged increments move on to the next
// one or finish, failures (iteration caps, CG breakdown, det F <= 0) finish
// with their status, the rest start another Newton iteration
__global__ void k_batch_decide(CellCtl* __restrict__ ctl, const CgScalars* __restrict__ cg,
                               const double* __restrict__ sums, const int* __restrict__ flags,
                               const int* __restrict__ ids, int n, SolveParams sp, double sqrt_n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int i = ids[j];
  CellCtl& c = ctl[i];
  if (c.mask_end) return;
  const CgScalars& s = cg[i];
  c.newton_it += 1;
  c.newton_total += 1;
  c.cg_total += s.it;
  double nrm = 0.0;
  for (int k = 0; k < 9; ++k) {
    const double v = sp.start[k] + c.inc * sp.dfbar[k];
    nrm += v * v;
  }
  const double e = sqrt(sums[16 * i]) / ((nrm > 0.0 ? sqrt(nrm) : 1.0) * sqrt_n);
  if (flags[i] & kFlagNonPhysical) {
    c.status = FH_ERR_NONPHYSICAL;
    c.stage = kStageDone;
  } else if (s.done != 1) {
    c.status = FH_ERR_NOT_CONVERGED;
    c.stage = kStageDone;
  } else if (!isfinite(e)) {
    c.status = FH_ERR_NONPHYSICAL;
    c.stage = kStageDone;
  } else if (e < sp.newton_tol) {
    if (c.inc >= sp.n_inc) {
      c.stage = kStageDone;
    } else {
      c.inc += 1;
      c.newton_it = 0;
      c.stage = kStageInc;
    }
  } else if (c.newton_it >= sp.max_newton) {
    c.status = FH_ERR_NOT_CONVERGED;
    c.stage = kStageDone;
  } else {
    c.stage = kStageRhs;
  }
}

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
  CellCtl* ctl = nullptr;          // device [n_cells]
  int* flags = nullptr;            // device [n_cells]
  double* params = nullptr;        // device [256][2]
  double2* tw = nullptr;
  dfc* tw_df = nullptr;            // the same tables in double-float
  cudaGraphExec_t chunk = nullptr;  // one Newton tick and check_every CG iterations of every group
  SolveParams chunk_params;         // the parameters chunk was captured with (valid while chunk != nullptr)
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

// One replay of the solve for every group: the Newton tick (end of
// iteration, increment, right-hand side, CG start) for the cells concerned,
// then check_every CG iterations. With alpha = beta = 0 after CG start and
// x = 0, the first iteration's p = r + beta p is the CG start p = r (p holds
// finite values: zero at the solve start, then the last direction).
int launch_replay(fh_batch* b, const SolveParams& sp) {
  cudaStream_t s = b->stream;
  for (Group& G : b->groups) {
    const int n = (int)G.cells.size();
    const unsigned nb = (unsigned)((n + 127) / 128);
    const double zero9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    // end of a Newton iteration: x += alpha p, F += x, ||x||^2, decide
    k_batch_masks<<<nb, 128, 0, s>>>(b->ctl, b->cg, G.cell_ids, n, 0);
    FB_CUDA(cudaGetLastError());
    FB_CUDA(launch_cg_finalize_batch(G.g, G.states_end, n, s));
    FB_CUDA(launch_newton_update_batch(G.g, G.states_end, n, s));
    FB_CUDA(launch_sum_partials_batch(G.states_end, n, G.n_pw, 1, s));
    k_batch_decide<<<nb, 128, 0, s>>>(b->ctl, b->cg, b->sums, b->flags, G.cell_ids, n, sp,
                                       std::sqrt((double)G.g.n));
    FB_CUDA(cudaGetLastError());
    // load increment: F += dFbar
    k_batch_masks<<<nb, 128, 0, s>>>(b->ctl, b->cg, G.cell_ids, n, 1);
    FB_CUDA(cudaGetLastError());
    FB_CUDA(launch_fill_batch(G.g, G.states_inc, n, 0, sp.dfbar, 1, s));
    // stress and tangent (a2), right-hand side b = -G(P) (a3), CG start
    k_batch_masks<<<nb, 128, 0, s>>>(b->ctl, b->cg, G.cell_ids, n, 2);
    FB_CUDA(cudaGetLastError());
    FB_CUDA(launch_constitutive_batch(G.g, sp.kind, b->params, G.states_rhs, n, 1, s));
    FB_CUDA(launch_fwd_z_batch(G.g, G.t, kZDirect, G.views_rhs, n, b->tw, s));
    FB_CUDA(launch_fwd_y_batch(G.g, G.t, G.views_rhs, n, b->tw, s));
    FB_CUDA(launch_x_ghat_batch(G.g, G.t, G.views_rhs, n, b->tw, -1.0 / (2.0 * (double)G.g.n), s));
    FB_CUDA(launch_inv_y_batch(G.g, G.t, G.views_rhs, n, b->tw, s));
    FB_CUDA(launch_inv_z_batch(G.g, G.t, kIZRhs, G.views_rhs, n, b->tw, s));
    // the fresh tangents in double-float, in place, for the double-float CG products
    if (sp.df) FB_CUDA(launch_tangent_to_df64_batch(G.g, G.states_rhs, n, s));
    FB_CUDA(launch_cg_init_batch(G.states_rhs, n, G.n_iz, sp.cg_tol, sp.max_cg, s));
    FB_CUDA(launch_fill_batch(G.g, G.states_rhs, n, 1, zero9, 0, s));
  }
  for (int k = 0; k < sp.check_every; ++k) {
    for (Group& G : b->groups) {
      const int n = (int)G.cells.size();
      const double c_mv = 1.0 / (2.0 * (double)G.g.n);
      if (sp.df) {
        const Tiling td = df_tiles(G.t);
        FB_CUDA(launch_fwd_z_batch_df(G.g, td, kZCg, G.views_cg, n, b->tw_df, s));
        FB_CUDA(launch_fwd_y_batch_df(G.g, td, G.views_cg, n, b->tw_df, s));
        FB_CUDA(launch_x_ghat_batch_df(G.g, td, G.views_cg, n, b->tw_df, c_mv, s));
        FB_CUDA(launch_inv_y_batch_df(G.g, td, G.views_cg, n, b->tw_df, s));
        FB_CUDA(launch_inv_z_batch_df(G.g, td, G.views_cg, n, b->tw_df, s));
      } else {
        FB_CUDA(launch_fwd_z_batch(G.g, G.t, kZCg, G.views_cg, n, b->tw, s));
        FB_CUDA(launch_fwd_y_batch(G.g, G.t, G.views_cg, n, b->tw, s));
        FB_CUDA(launch_x_ghat_batch(G.g, G.t, G.views_cg, n, b->tw, c_mv, s));
        FB_CUDA(launch_inv_y_batch(G.g, G.t, G.views_cg, n, b->tw, s));
        FB_CUDA(launch_inv_z_batch(G.g, G.t, kIZDot, G.views_cg, n, b->tw, s));
      }
      FB_CUDA(launch_cg_alpha_batch(G.states, n, sp.df ? (int)z_pass_ctas(G.g, df_tiles(G.t)) : G.n_iz, s));
      FB_CUDA(launch_cg_update_batch(G.g, G.states, n, s));
      FB_CUDA(launch_cg_beta_batch(G.states, n, G.n_pw, s));
    }
  }
  return FH_OK;
}

int capture_replay(fh_batch* b, const SolveParams& sp) {
  if (b->chunk && b->chunk_params == sp) return FH_OK;
  if (b->chunk) {
    cudaGraphExecDestroy(b->chunk);
    b->chunk = nullptr;
  }
  cudaGraph_t graph = nullptr;
  FB_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  const int rc = launch_replay(b, sp);
  cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return bfail(FH_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->chunk, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(FH_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  b->chunk_params = sp;
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
      (rc = dalloc(b, &b->ctl, sizeof(CellCtl) * n_cells)) || (rc = dalloc(b, &b->flags, sizeof(int) * n_cells)) ||
      (rc = dalloc(b, &b->params, 512 * sizeof(double))) || (rc = dalloc(b, &b->tw, kTwiddleTables * sizeof(double2))) ||
      (rc = dalloc(b, &b->tw_df, kTwiddleTables * sizeof(dfc))))
    return cleanup(rc);
  std::vector<double2> tw(kTwiddleTables);
  fill_twiddle_table(tw.data());
  std::vector<dfc> tw_df(kTwiddleTables);
  twiddles_to_df64(tw.data(), tw_df.data(), kTwiddleTables);
  if (cudaMemcpy(b->tw, tw.data(), kTwiddleTables * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->tw_df, tw_df.data(), kTwiddleTables * sizeof(dfc), cudaMemcpyHostToDevice) != cudaSuccess)
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
    std::vector<CellState> st(n), st_end(n), st_inc(n), st_rhs(n);
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
      c.flags = b->flags + i;
      c.newton_done = &b->ctl[i].zero;
      st_end[j] = c;
      st_end[j].newton_done = &b->ctl[i].mask_end;
      st_inc[j] = c;
      st_inc[j].newton_done = &b->ctl[i].mask_inc;
      st_rhs[j] = c;
      st_rhs[j].newton_done = &b->ctl[i].mask_rhs;
      vr[j] = CellView{&b->ctl[i].mask_rhs, c.P, c.p, c.x, c.K, c.cg, c.S, c.r, c.partials};
      vc[j] = CellView{&c.cg->done, c.r, c.p, c.x, c.K, c.cg, c.S, c.y, c.partials};
    }
    if ((rc = dalloc(b, &G.states, sizeof(CellState) * n)) || (rc = dalloc(b, &G.states_end, sizeof(CellState) * n)) ||
        (rc = dalloc(b, &G.states_inc, sizeof(CellState) * n)) ||
        (rc = dalloc(b, &G.states_rhs, sizeof(CellState) * n)) || (rc = dalloc(b, &G.views_rhs, sizeof(CellView) * n)) ||
        (rc = dalloc(b, &G.views_cg, sizeof(CellView) * n)) || (rc = dalloc(b, &G.cell_ids, sizeof(int) * n)))
      return cleanup(rc);
    if (cudaMemcpy(G.states, st.data(), sizeof(CellState) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.states_end, st_end.data(), sizeof(CellState) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.states_inc, st_inc.data(), sizeof(CellState) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.states_rhs, st_rhs.data(), sizeof(CellState) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.views_rhs, vr.data(), sizeof(CellView) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.views_cg, vc.data(), sizeof(CellView) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.cell_ids, G.cells.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess)
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
  if (!(opt.newton_tol > 0.0) || opt.max_newton < 1 || opt.max_cg < 0 || opt.check_every < 1 ||
      (opt.matvec_arith != FH_ARITH_FP64 && opt.matvec_arith != FH_ARITH_DF64))
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
  SolveParams sp;
  std::memset(&sp, 0, sizeof(sp));  // the graph is keyed on the bytes of sp, padding included
  if (kind != FH_LINEAR_ELASTIC) sp.start[0] = sp.start[4] = sp.start[8] = 1.0;
  for (int c = 0; c < 9; ++c) sp.dfbar[c] = (Fbar[c] - sp.start[c]) / n_increments;
  sp.newton_tol = opt.newton_tol;
  sp.cg_tol = cg_tol;
  sp.n_inc = n_increments;
  sp.max_newton = opt.max_newton;
  sp.max_cg = opt.max_cg;
  sp.check_every = opt.check_every;
  sp.kind = kind;
  sp.df = opt.matvec_arith == FH_ARITH_DF64;  // every batched grid has compile-time plans and an even nz
  // every cell at its first load increment, CG idle (done = 1), flags clear
  {
    std::vector<CellCtl> c0(nc);
    for (CellCtl& c : c0) c = CellCtl{kStageInc, 1, 0, 0, 0, FH_OK, 1, 1, 1, 0};
    std::vector<CgScalars> g0(nc);
    for (CgScalars& g : g0) {
      std::memset(&g, 0, sizeof(g));
      g.done = 1;
    }
    FB_CUDA(cudaMemcpyAsync(b->ctl, c0.data(), sizeof(CellCtl) * nc, cudaMemcpyHostToDevice, s));
    FB_CUDA(cudaMemcpyAsync(b->cg, g0.data(), sizeof(CgScalars) * nc, cudaMemcpyHostToDevice, s));
    FB_CUDA(cudaMemsetAsync(b->flags, 0, sizeof(int) * nc, s));
    const double zero9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (Group& G : b->groups) {
      const int n = (int)G.cells.size();
      FB_CUDA(launch_fill_batch(G.g, G.states, n, 0, sp.start, 0, s));
      FB_CUDA(launch_fill_batch(G.g, G.states, n, 1, zero9, 0, s));
      FB_CUDA(launch_fill_batch(G.g, G.states, n, 2, zero9, 0, s));
    }
    FB_CUDA(cudaStreamSynchronize(s));
  }
  int rc = capture_replay(b, sp);
  if (rc) return rc;
  // replays until every cell is done; each replay moves every active cell by at least one CG iteration
  const long long max_replays =
      (long long)n_increments * opt.max_newton * ((opt.max_cg + opt.check_every) / opt.check_every + 2) + 4;
  std::vector<CellCtl> hc(nc);
  bool all_done = false;
  for (long long r = 0; r < max_replays && !all_done; ++r) {
    FB_CUDA(cudaGraphLaunch(b->chunk, s));
    FB_CUDA(cudaMemcpyAsync(hc.data(), b->ctl, sizeof(CellCtl) * nc, cudaMemcpyDeviceToHost, s));
    FB_CUDA(cudaStreamSynchronize(s));
    all_done = true;
    for (int i = 0; i < nc; ++i) all_done = all_done && hc[i].stage == kStageDone;
  }
  if (!all_done) return bfail(FH_ERR_CUDA, "batched solve did not finish within its iteration caps");
  std::vector<int> status(nc), newton(nc), cgs(nc);
  for (int i = 0; i < nc; ++i) {
    status[i] = hc[i].status;
    newton[i] = hc[i].newton_total;
    cgs[i] = hc[i].cg_total;
  }
  // homogenized stress of every cell (a7)
  std::vector<double> hs(16 * (size_t)nc);
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
