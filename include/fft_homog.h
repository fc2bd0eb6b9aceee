/*
 * fft_homog.h -- C-ABI of the GB300 Fourier-Galerkin homogenization library.
 *
 * The library solves the periodic cell problem of Pundir & Kammer,
 * "Simplifying FFT-based methods for solid mechanics with automatic
 * differentiation": a representative volume element under a prescribed
 * macroscopic deformation gradient Fbar (Section 3), equilibrium in Fourier
 * form  IFFT{ Ghat(xi) : FFT{P} } = 0  (Eq. 1), stress P = dW/dF (Eq. 2) and
 * tangent K = dP/dF (Eq. 3) by forward-mode automatic differentiation of the
 * stored energy W, a Newton-Krylov solve (Appendix A, Algorithm 1) and the
 * homogenized stress Pbar = volume mean of P (Eq. 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid        nx x ny x nz voxels, N = nx*ny*nz. nx and ny are any length
 *             1..512 (2^a and 3*2^a up to 256 use compile-time radix-16/8/4/2/3
 *             plans; other lengths, e.g. the paper's odd grids 199 or 299,
 *             run-time plans: prime lengths from 37 up by Rader's algorithm,
 *             other prime factors above 3 as direct DFT stages); nz is 1 (a
 *             plane problem: every field is z-invariant and xi_z = 0), or
 *             even with nz and nz/2 of the form 2^a or 3*2^a up to 256.
 *             fh_project_static and batched solves take only the
 *             compile-time lengths on every axis and an even nz. Box side
 *             lengths default to 1 (see fh_options.lengths).
 * Fields      device float64 arrays in structure-of-arrays order
 *             [9][nx][ny][nz] (z fastest); component c = 3*i + j holds the
 *             tensor entry T_ij (row-major 3x3; F_ij = dx_i/dX_j).
 * Tangents    device float64 arrays [45][nx][ny][nz]: the upper triangle of
 *             the symmetric 9x9 matrix K[a][b] = dP_a/dF_b (a, b component
 *             indices), row by row: slot s(a,b) = 9a - a(a-1)/2 + (b - a) for
 *             a <= b. Hyperelastic tangents have this major symmetry.
 * Phase map   device uint8 array [nx][ny][nz]; value p selects row p of the
 *             host parameter table params[n_phase][2] = (lambda, mu).
 * Ownership   the caller owns every pointer it passes; the context owns only
 *             its own scratch (spectrum, CG vectors, tangent, partial sums),
 *             allocated by fh_create and released by fh_destroy.
 * Streams     all device work of a context runs on the stream given to
 *             fh_create; every call has finished on that stream when it
 *             returns.
 * Errors      every int-returning call returns FH_OK (0) or one of the codes
 *             below; fh_last_error_string() describes the last failure of the
 *             calling thread. No C++ exception crosses this interface.
 * Precision   all arithmetic of the solver is IEEE float64.
 */
#ifndef FFT_HOMOG_H
#define FFT_HOMOG_H

#if defined(__GNUC__)
#define FH_API __attribute__((visibility("default")))
#else
#define FH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define FH_OK 0
#define FH_ERR_ARG 1            /* invalid argument (size, pointer, option) */
#define FH_ERR_CUDA 2           /* a CUDA runtime call failed */
#define FH_ERR_NOT_CONVERGED 3  /* Newton or CG hit its iteration cap; outputs hold the last iterate */
#define FH_ERR_NONPHYSICAL 4    /* det F <= 0 or a non-finite value in a voxel */
#define FH_ERR_TIMEOUT 5        /* reserved: a bounded device-side wait ran out */
#define FH_ERR_UNSUPPORTED 6    /* valid request this build does not implement */

/* ---- material laws (energy densities differentiated in the kernels) ----
 * FH_LINEAR_ELASTIC  small strain; the unknown is the displacement gradient
 *                    H, eps = sym(H), W = lambda/2 tr(eps)^2 + mu eps:eps
 *                    (Section 3.2; the paper omits the 1/2 on lambda).
 * FH_NEO_HOOKEAN     W = mu/2 (tr F^T F - 3) - mu ln J + lambda/2 (ln J)^2.
 * FH_SVK             St. Venant-Kirchhoff, W = lambda/2 tr(E)^2 + mu E:E with
 *                    E = (F^T F - I)/2 (Eq. 6).
 * FH_J2              small-strain J2 plasticity with linear isotropic hardening
 *                    (Section 4.1.2, Appendix B): elastic predictor from the
 *                    plastic strain of the last converged increment, von Mises
 *                    yield check, radial return; the stress is the return map
 *                    itself (no energy) and K its AD derivative. Needs
 *                    fh_material.plastic and .history. */
#define FH_LINEAR_ELASTIC 0
#define FH_NEO_HOOKEAN 1
#define FH_SVK 2
#define FH_J2 3

/* ---- how the CG matrix-vector product gets K : dF (Section 3.2) ----
 * FH_TANGENT_STORED  K is evaluated by AD once per Newton step and stored
 *                    (45 doubles per voxel; Listing 2's explicit tangent).
 * FH_TANGENT_JVP     K : dF is re-derived from F by AD inside every product
 *                    (Listing 3's push-forward); nothing is stored. */
#define FH_TANGENT_STORED 0
#define FH_TANGENT_JVP 1

/* ---- start state of a solve ----
 * FH_INIT_REFERENCE  F starts at I (finite strain) or 0 (small strain).
 * FH_INIT_GIVEN      F_dev holds the start field; its voxel mean is taken as
 *                    the macroscopic tensor it is in equilibrium with. */
#define FH_INIT_REFERENCE 0
#define FH_INIT_GIVEN 1

/* ---- how the kernels of a CG loop are launched (fh_options.launch_mode) ---- */
#define FH_LAUNCH_GRAPH 0
#define FH_LAUNCH_PLAIN 1

/* ---- arithmetic of the transforms in the CG matrix-vector product ----
 * FH_ARITH_FP64  IEEE FP64 throughout (the default; the method as stated).
 * FH_ARITH_DF64  an option, not the default: the five projection passes of
 *                every CG product transform in double-float arithmetic
 *                (each real number an unevaluated sum of two FP32 values,
 *                about 48 significant bits, on the FP32 pipe, which issues
 *                about 75 times faster than FP64 on GB300), and K : p is
 *                formed in double-float from a double-float copy of the
 *                packed tangent. The CG vector updates and dot products,
 *                the Newton right-hand side, residuals and stress stay
 *                FP64. Every grid. */
#define FH_ARITH_FP64 0
#define FH_ARITH_DF64 1

typedef struct fh_ctx fh_ctx;

typedef struct fh_material {
  int kind;                     /* FH_LINEAR_ELASTIC, FH_NEO_HOOKEAN, FH_SVK or FH_J2 */
  int n_phase;                  /* rows of params, 1..256 */
  const unsigned char* phase;   /* device uint8[N], every value < n_phase */
  const double* params;         /* host double[n_phase][2] = (lambda, mu) */
  const double* scale;          /* device double[N] multiplying both Lame parameters of each voxel
                                   (a modulus field such as E = rho^p at fixed Poisson ratio), or NULL */
  const double* plastic;        /* FH_J2: host double[n_phase][2] = (yield stress, hardening modulus) */
  double* history;              /* FH_J2: device double[10][N], the plastic strain (9 components,
                                   symmetric) and the cumulative plastic strain; zero for a virgin
                                   material; fft_homog_solve updates it after each converged
                                   increment, the other entry points only read it */
} fh_material;

typedef struct fh_options {
  double newton_tol;    /* stop when ||dF||_2 / (||Fbar_n||_F sqrt(N)) < newton_tol (Alg. 1) */
  double cg_tol;        /* CG stops when ||r|| <= cg_tol ||b||; <= 0 selects 1e-2 * newton_tol */
  int max_newton;       /* Newton iterations per load increment */
  int max_cg;           /* CG matrix-vector products per Newton iteration */
  int init;             /* FH_INIT_REFERENCE or FH_INIT_GIVEN */
  int tangent_mode;     /* FH_TANGENT_STORED or FH_TANGENT_JVP */
  int check_every;      /* CG iterations queued between host convergence reads (>= 1) */
  int launch_mode;      /* FH_LAUNCH_GRAPH: each chunk of check_every CG iterations is the replay
                           of a CUDA graph captured on the context's stream (captured again when
                           the material, the field pointer or the grid scale changes; plain
                           launches on the legacy default stream, on a stream the caller is
                           capturing and while fh_profile_enable timing is on); FH_LAUNCH_PLAIN:
                           every kernel launched from the host. Results are identical. */
  double lengths[3];    /* box side lengths L_x, L_y, L_z (> 0) */
  int matvec_arith;     /* FH_ARITH_FP64 or FH_ARITH_DF64 */
  int reserved;         /* 0 */
} fh_options;

typedef struct fh_stats {
  int n_newton;               /* Newton iterations over all increments */
  int n_cg;                   /* CG matrix-vector products over all increments */
  int capacity;               /* length of the two caller-owned arrays below (may be 0) */
  int n_recorded;             /* entries written to them (min(n_newton, capacity)) */
  double* newton_residuals;   /* host array: e after each Newton iteration, or NULL */
  int* cg_iterations;         /* host array: CG products of each Newton iteration, or NULL */
  double time_ms;             /* wall time of the call */
  int cg_graph_replays;       /* chunks of CG iterations run as replays of a captured graph */
  int cg_graph_captures;      /* graph captures the call needed (0 when the context's graphs were current) */
} fh_stats;

/* Fill *o with the defaults: newton_tol 1e-8, cg_tol 0 (= 1e-2 newton_tol),
 * max_newton 50, max_cg 5000, FH_INIT_REFERENCE, FH_TANGENT_STORED,
 * check_every 16, FH_LAUNCH_GRAPH, lengths (1, 1, 1), FH_ARITH_FP64. */
FH_API void fh_default_options(fh_options* o);

/* Create a context for an nx x ny x nz grid whose work runs on cuda_stream
 * (a cudaStream_t; NULL = the legacy default stream) of the current device.
 * Allocates the context's device scratch: about 650 bytes per voxel.
 * Returns FH_ERR_ARG for unsupported extents, FH_ERR_CUDA if allocation
 * fails; *out is set only on success. */
FH_API int fh_create(fh_ctx** out, int nx, int ny, int nz, void* cuda_stream);

/* Release a context and its scratch; NULL is accepted. */
FH_API void fh_destroy(fh_ctx* ctx);

/* Description of the last error on the calling thread ("" if none). */
FH_API const char* fh_last_error_string(void);

/* Stress and tangent of every voxel (Eqs. 2-3, Section 3.1-3.2), from the
 * energy of mat->kind by forward-mode dual numbers of second order; for
 * FH_J2, the return-mapped stress from mat->history and its first-order AD
 * derivative (Section 4.1.2). The history is only read.
 *   F_dev      in   [9][N] deformation gradient (H for small strain)
 *   P_dev      out  [9][N] stress dW/dF, or NULL
 *   K_dev      out  [45][N] packed tangent d2W/dF2, or NULL
 *   Pbar_out   out  host double[9], volume mean of P (Eq. 4), or NULL
 * Returns FH_ERR_NONPHYSICAL if any voxel has det F <= 0 or a non-finite
 * result (outputs are still written). */
FH_API int fh_constitutive(fh_ctx* ctx, const fh_material* mat, const double* F_dev,
                    double* P_dev, double* K_dev, double Pbar_out[9]);

/* out = scale * G(A): the compatibility projection of Eq. 1,
 * IFFT{ Ghat(xi) : FFT{A} } with Ghat(xi)[Ahat] = (Ahat xi) (x) xi / |xi|^2
 * and Ghat(0) = 0. On an even axis the Nyquist index has xi = 0.
 *   A_dev    in   [9][N]     out_dev  out  [9][N] (may equal A_dev)
 * lengths: box side lengths (NULL = unit box). */
FH_API int fh_project(fh_ctx* ctx, const double* A_dev, double* out_dev, double scale,
               const double lengths[3]);

/* y = G(K : p), the CG matrix-vector product of the linearised Eq. 1.
 * With K_dev != NULL the stored packed tangent [45][N] is applied; with
 * K_dev == NULL, K : p is re-derived from F_dev and mat by AD (jvp form).
 *   p_dev in [9][N], y_dev out [9][N] (must not alias p_dev).
 * arith: FH_ARITH_FP64, or FH_ARITH_DF64 for the transforms in double-float. */
FH_API int fh_matvec(fh_ctx* ctx, const fh_material* mat, const double* F_dev,
              const double* K_dev, const double* p_dev, double* y_dev,
              const double lengths[3], int arith);

/* Solve the cell under the macroscopic tensor Fbar (Appendix A, Algorithm 1;
 * Listing 5's solve_microscale). The load goes from the start tensor to Fbar
 * in n_increments equal additive steps; each step runs Newton iterations
 *   P, K = AD(W)(F);  b = -G(P);  CG on G(K : dF) = b from dF = 0;  F += dF
 * until ||dF||/(||Fbar_n|| sqrt(N)) < newton_tol.
 *   F_dev      in/out [9][N]: start field if opt->init == FH_INIT_GIVEN;
 *              the converged field on return (H for small strain)
 *   Fbar       host double[9] macroscopic target
 *   Pbar_out   host double[9] homogenized stress (Eq. 4), or NULL
 *   stats      optional convergence record, or NULL
 *   opt        NULL = defaults
 * FH_J2: every Newton iteration of an increment starts its return map from
 * mat->history, which is advanced in place once the increment has converged
 * (a failed increment leaves it at the last converged one); a second call
 * with opt->init = FH_INIT_GIVEN continues the loading path.
 * Returns FH_ERR_NOT_CONVERGED when an iteration cap is hit (F_dev and
 * Pbar_out then hold the last iterate), FH_ERR_NONPHYSICAL on det F <= 0. */
FH_API int fft_homog_solve(fh_ctx* ctx, const fh_material* mat, const double Fbar[9],
                    int n_increments, const fh_options* opt, double* F_dev,
                    double Pbar_out[9], fh_stats* stats);

/* Homogenized tangent Cbar = dPbar/dFbar at a converged state (Section 3.3,
 * Eq. 4; the forward derivative of Listing 5's solve_microscale). For each of
 * the nine unit macroscopic entries E_cd one conjugate-gradient solve gives
 * the fluctuation d with G(K : (E_cd + d)) = 0, and column cd of Cbar is
 * mean(K : (E_cd + d)), with K evaluated by AD at F_dev.
 *   F_dev      in   [9][N] converged field (H for small strain)
 *   opt        CG tolerance (cg_tol, or 1e-2 newton_tol), max_cg, lengths; NULL = defaults
 *   Cbar_out   out  host double[81], Cbar[9*ab + cd] = dPbar_ab / dFbar_cd
 * Returns FH_ERR_NOT_CONVERGED if a CG solve hits max_cg, FH_ERR_UNSUPPORTED
 * for FH_J2. */
FH_API int fft_homog_tangent(fh_ctx* ctx, const fh_material* mat, const double* F_dev,
                             const fh_options* opt, double Cbar_out[81]);

/* Sensitivity of one homogenized modulus to a voxel density field
 * (Section 4.4.2's topology-optimisation gradient), for small-strain linear
 * elasticity with per-voxel moduli s(rho_v) * C0(phase_v) (mat->scale holds
 * s). Because the cell problem is self-adjoint, no adjoint solve is needed:
 *   dCbar_ab,cd / d rho_v = (1/N) (E_ab + d_ab)_v : C0_v : (E_cd + d_cd)_v * ds/drho_v
 * with d_ab, d_cd the unit responses of fft_homog_tangent (one CG solve, two
 * when ab != cd). ab = 3*i + j, cd = 3*k + l.
 *   dscale_dev  in   device double[N], ds/drho per voxel
 *   out_dev     out  device double[N], the sensitivity per voxel
 * Returns FH_ERR_UNSUPPORTED for finite-strain laws and FH_J2. */
FH_API int fft_homog_sensitivity(fh_ctx* ctx, const fh_material* mat, const fh_options* opt, int i, int j,
                                 int k, int l, const double* dscale_dev, double* out_dev);

/* Sensitivity of one homogenized stress entry to a voxel density field at a
 * converged state, for laws whose voxel moduli are s(rho_v) times those of the
 * voxel's phase (mat->scale holds s): P = s(rho) P0(F) (Section 4.4's
 * gradients for finite strain; the linear law too). Differentiating the
 * equilibrium of Eq. 1 and using the major symmetry of K, the adjoint solve is
 * the unit response d_ab of fft_homog_tangent (one CG solve):
 *   dPbar_ab / d rho_v = (1/N) (E_ab + d_ab)_v : P0(F_v) * ds/drho_v,
 * with ab = 3*i + j and P0 by AD with the unscaled moduli.
 *   F_dev       in   [9][N] converged field (H for small strain)
 *   opt         CG tolerance (cg_tol, or 1e-2 newton_tol), max_cg, lengths; NULL = defaults
 *   dscale_dev  in   device double[N], ds/drho per voxel
 *   out_dev     out  device double[N], the sensitivity per voxel
 * Returns FH_ERR_UNSUPPORTED for FH_J2, FH_ERR_NOT_CONVERGED if the CG solve
 * hits max_cg. */
FH_API int fft_homog_stress_sensitivity(fh_ctx* ctx, const fh_material* mat, const double* F_dev,
                                        const fh_options* opt, int i, int j, const double* dscale_dev,
                                        double* out_dev);

/* Pick the tile shapes of the five projection passes for this context's grid
 * by timing them: z lines per CTA in the z passes, kz columns per CTA in the
 * y and x passes (a handful of candidates around the default, all within the
 * per-CTA shared-memory limit), `reps` projections each. The fastest is kept
 * for every later call on the context. Optional outputs: best_ms (time of
 * one projection) and chosen[3] = (z lines, y columns, x columns). */
FH_API int fh_autotune(fh_ctx* ctx, int reps, double* best_ms, int chosen[3]);

/* ---- batched solves of many cells (Section 4.4.1's many-sample setting) ----
 * A batch binds cells of possibly different grids; each keeps its own Newton
 * and CG state (its own convergence, decided on the device), while every pass
 * of the solve is one launch per group of equal grids. One captured CUDA
 * graph (the Newton step bookkeeping of every cell, then check_every CG
 * iterations of every group) is replayed until every cell has finished, so a
 * cell never waits for another cell's CG at a Newton step. */
typedef struct fh_batch fh_batch;

typedef struct fh_cell {
  int nx, ny, nz;               /* grid, as for fh_create */
  const unsigned char* phase;   /* device uint8[N] */
  const double* scale;          /* device double[N] modulus multiplier, or NULL */
  double* F;                    /* device [9][N]: the cell's converged field on return */
} fh_cell;

/* Create a batch over n_cells cells whose device arrays the caller owns and
 * keeps alive until fh_batch_destroy. Allocates each cell's scratch (about
 * 700 bytes per voxel). cuda_stream NULL: the batch uses a stream of its own
 * (CUDA graphs cannot be captured on the legacy stream). */
FH_API int fh_batch_create(fh_batch** out, const fh_cell* cells, int n_cells, void* cuda_stream);
FH_API void fh_batch_destroy(fh_batch* batch);

/* Solve every cell of the batch under the same material law (kind, n_phase,
 * host params[n_phase][2]), macroscopic tensor and options, as
 * fft_homog_solve does for one cell (Algorithm 1), from the reference state,
 * with the tangent stored and unit boxes. Per-cell outputs (host arrays of
 * n_cells entries, each may be NULL): Pbar_out[9 * i + c], status_out[i]
 * (FH_OK, FH_ERR_NOT_CONVERGED or FH_ERR_NONPHYSICAL), newton_out[i] and
 * cg_out[i] (iteration totals). Returns FH_OK when every cell converged,
 * else the first failing cell's status; FH_ERR_UNSUPPORTED for FH_J2 (no
 * per-cell history). opt->matvec_arith = FH_ARITH_DF64 runs every cell's CG
 * products with double-float transforms (each cell's tangent buffer then
 * holds its double-float copy during CG). */
FH_API int fft_homog_solve_batched(fh_batch* batch, int kind, int n_phase, const double* params,
                                   const double Fbar[9], int n_increments, const fh_options* opt,
                                   double* Pbar_out, int* status_out, int* newton_out, int* cg_out);

/* ---- launch accounting and per-kernel device time ----
 * Kernel classes, in slot order: 0 forward z pass (stress/tangent apply +
 * real-to-complex), 1 forward y pass, 2 x pass with Ghat, 3 inverse y pass,
 * 4 inverse z pass (complex-to-real + dot), 5 constitutive AD, 6 jvp tangent
 * apply, 7 CG scalar kernels, 8 CG vector update, 9 Newton update,
 * 10 fills and field sums, 11 partial-sum reductions, 12 tangent/sensitivity
 * contractions, 13 idle: CG-loop launches queued after the loop had
 * converged (the host reads the done flag only every check_every
 * iterations), which found the flag set and returned without work. Classes
 * 0-12 therefore count and time only launches that did work. */
#define FH_PROF_NCLASS 14

/* Reset the context's launch counters and, with enable != 0, bracket every
 * later launch with a pair of CUDA events on the context's stream (adds one
 * event record before and after each kernel). */
FH_API int fh_profile_enable(fh_ctx* ctx, int enable);

/* Launches per class since the last fh_profile_enable, and the summed device
 * time in milliseconds of those launched while events were enabled (0 when
 * disabled). Waits for the context's stream. Either array may be NULL. */
FH_API int fh_profile_read(fh_ctx* ctx, long long counts[FH_PROF_NCLASS], double ms[FH_PROF_NCLASS]);

/* FP64 issue rate of the current device, measured (the roofline of the
 * FP64-bound CG matrix-vector product; no counterpart in the paper). Runs
 * ctas_per_sm (1..8) CTAs of 256 threads per SM, each thread `iters`
 * (1..2^34) rounds of `chains` (4, 8 or 16) independent FMA chains, on
 * cuda_stream (NULL = legacy stream), after one untimed launch of iters/16
 * rounds. Outputs: *ms_out the CUDA-event time of the timed launch,
 * *lane_ops_out its FP64 FMA lane operations (threads x chains x iters; 2 flops
 * each). Returns when done. */
FH_API int fh_probe_fp64(int ctas_per_sm, int chains, long long iters, void* cuda_stream, double* ms_out,
                         double* lane_ops_out);

/* The twiddle tables of the compile-time FFT plans (the transforms of Eq. 1),
 * for checking on the host (no counterpart in the paper; touches no device).
 * out receives 2 * count doubles: count complex entries, count = 2 * T where
 * T = 892 is the total length of the tables of all lengths L in {1, 2, 3, 4, 6,
 * 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256}, stored back to back in that
 * order. Entry o(L) + m (o(L) the sum of the shorter lengths) is w_L^m =
 * exp(-2 pi i m / L) as (cos, -sin); entry T + o(L) + m the same root in the
 * tangent form (rho, tau) of the FP64 stages: with qr = floor((8 m + L) / (2 L))
 * (the nearest quarter turn), w_L^m = (-i)^qr rho (1 + i tau), |tau| <= 1.
 * Returns count (and writes nothing) when out is NULL or capacity (in complex
 * entries) is below count; otherwise writes the tables and returns count. */
FH_API int fh_twiddle_tables(double* out, int capacity);

/* The double-float conversions of FH_ARITH_DF64, for checking (no
 * counterpart in the paper): for each of the n device doubles in_dev, hi_dev
 * and lo_dev (device floats, NULL to skip) get the split the double-float
 * kernels make of it (hi: the significand cut after 23 bits; lo: the rest
 * truncated to 24 significant bits; |x - hi - lo| < max(2^-47 |x|, 2^-125);
 * 0 below the smallest normal float), and out_dev (device doubles) hi + lo joined back
 * with one FP64 addition. n >= 0; out_dev may equal in_dev. Runs on
 * cuda_stream and returns when done. */
FH_API int fh_df64_roundtrip(const double* in_dev, float* hi_dev, float* lo_dev, double* out_dev, long long n,
                             void* cuda_stream);

/* ---- projection without device allocation ----
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory, such as a plug-in inside an application that
 * owns the GPU's memory, or a loop that must not allocate once it runs. It
 * computes exactly what fh_project computes (out = scale * G(A)), with the
 * same kernels, but needs no fh_ctx: its scratch is a static device array of
 * 9 * 32768 complex doubles (4.5 MiB) plus the twiddle tables (1784 complex
 * doubles, about 28 KiB), which every GPU that loads this library holds until
 * the process exits.
 *   A_dev, out_dev  device [9][nx][ny][nz] fields (out may equal A)
 *   nx, ny, nz      extents as for fh_create, nx*ny*nz <= 32768;
 *                   larger grids return FH_ERR_ARG (use fh_project)
 *   lengths         box side lengths, or NULL for the unit box
 *   cuda_stream     stream to run on (NULL = legacy default stream)
 * Every call resolves the static arrays' device addresses on the current
 * device and reads back one twiddle entry on cuda_stream; the first call on a
 * device (and the first after its context was recreated, e.g. by
 * cudaDeviceReset) also writes the twiddle tables, so make that first call
 * before any stream capture. Every call on a device shares the one
 * array and leaves its contents behind; no value carries over from one call
 * to the next (each call overwrites all scratch it reads), but calls whose
 * work overlaps on the GPU (for example on two streams) race on the array and
 * must be serialised by the caller. Returns when the work has finished. */
FH_API int fh_project_static(const double* A_dev, double* out_dev, int nx, int ny, int nz, double scale,
                             const double lengths[3], void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FFT_HOMOG_H */
