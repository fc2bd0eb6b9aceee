/*
 * fh_fno.h -- C-ABI of the learned warm start: a factorized Fourier neural
 * operator trained on solutions of the cell problem and used to start the
 * Newton-Krylov solve of fft_homog.h from a predicted fluctuation field.
 *
 * The paper solves every cell from the macroscopic tensor itself (Algorithm 1
 * with the fluctuation started at zero) and has no learned component; this
 * interface adds one around that solver without changing it. The solver
 * still refines the start field to the requested tolerance, so the network
 * can only change the number of iterations, never the answer.
 *
 * Network (all sizes fixed at build time)
 * ---------------------------------------
 *   s = |Fbar - I|_F, u = (Fbar - I)/s (u = 0 when s = 0)
 *   h0(x)  = a phi(x) + B u + b0                   width 32, phi = (phase != 0)
 *   z_l    = sum_{d = x, y, z} S_{l,d}(h_l) + M_l h_l + m_l,   l = 0..3
 *   h_l+1  = gelu(z_l) (l < 3),  h_4 = z_3         gelu(z) = z Phi(z), exact erf form
 *   R(x)   = P2 gelu(P1 h_4 + p1) + p2             hidden 128, 81 outputs R_ij
 *   q_i(x) = sum_j R_ij(x) u_j                     (a response per load direction)
 *   predicted fluctuation F - Fbar = s q(x)
 * S_{l,d} acts along axis d alone: the real DFT of each channel along d,
 * the 12 lowest modes k = 0..11 multiplied by a complex 32x32 matrix
 * W_{l,d}[k] (output channel o, input channel c), higher modes dropped, and
 * the real inverse DFT (1/n, the imaginary part of the k = 0 term dropped).
 * Every axis of the grid must have at least 24 voxels.
 *
 * Parameter vector (float32, n = fh_fno_param_count() = 314161), in order:
 *   a[32], B[32][9], b0[32];
 *   for l = 0..3: W_l[3 axes x,y,z][12 modes][2 re,im][32 o][32 c], M_l[32 o][32 c], m_l[32];
 *   P1[128][32], p1[128], P2[81][128] (row 9i + j), p2[81].
 * The forward and backward passes use a bfloat16 copy of every parameter
 * (made by fh_fno_set_params); activations and gradients are stored as
 * float32. The channel contractions (truncated DFTs, spectral mixing,
 * pointwise mixing, projection head, weight gradients) run on the tensor
 * cores as bfloat16 MMAs with float32 accumulation, float32 operands split
 * into a bfloat16 pair hi + lo (about 16 significant bits).
 *
 * Layouts: phase maps are device uint8 [nx][ny][nz] (z fastest); q, targets
 * and gradients are float32, q and targets [9][nx][ny][nz] per sample.
 * Ownership: the caller owns every pointer passed; an fh_fno owns its
 * activation and gradient scratch. All work runs on the stream given to
 * fh_fno_create and has finished when a call returns. Errors: FH_OK or an
 * FH_ERR_* code of fft_homog.h with fh_last_error_string().
 */
#ifndef FH_FNO_H
#define FH_FNO_H

#include "fft_homog.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fh_fno fh_fno;

/* Number of float32 entries of the parameter vector (314161). */
FH_API long long fh_fno_param_count(void);

/* Network scratch for batches of up to max_batch cells of nx x ny x nz voxels
 * (each >= 24). train != 0 also allocates what fh_fno_loss_grad needs (about
 * 14 float32 fields of 32 channels per voxel and sample, versus 3 for
 * inference). cuda_stream NULL = legacy default stream. */
FH_API int fh_fno_create(fh_fno** out, int nx, int ny, int nz, int max_batch, int train, void* cuda_stream);
FH_API void fh_fno_destroy(fh_fno* net);

/* Load the parameters: theta_dev device float32[n]; the bfloat16 copies used
 * by every later pass are made from it (theta_dev is not kept). */
FH_API int fh_fno_set_params(fh_fno* net, const float* theta_dev);

/* Forward pass for a batch of B <= max_batch cells.
 *   phase_ptrs  host array of B device pointers to uint8 phase maps
 *   Fbar        host double[B][9] macroscopic tensors
 *   q_ptrs      host array of B device pointers to float32 [9][N] outputs
 *               (the normalised prediction q), or NULL
 * In training mode the activations are kept for fh_fno_loss_grad, which also
 * reads the phase maps again: they must stay valid until then. */
FH_API int fh_fno_forward(fh_fno* net, int B, const unsigned char* const* phase_ptrs, const double* Fbar,
                          float* const* q_ptrs);

/* Loss of the last forward pass against normalised targets and its gradient
 * with respect to the parameter vector (training mode only):
 *   loss = mean over samples, components and voxels of (q - target)^2
 *   target_ptrs  host array of B device pointers to float32 [9][N]
 *   loss_out     host double, or NULL
 *   grad_dev     device float32[n] (overwritten), or NULL for the loss alone
 * Reductions run in a fixed order: the result is deterministic. */
FH_API int fh_fno_loss_grad(fh_fno* net, const float* const* target_ptrs, double* loss_out, float* grad_dev);

/* One Adam step (Kingma and Ba) on float32 device vectors of length n, step
 * number t >= 1 (bias correction 1 - beta^t), with decoupled weight decay wd:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
 *   theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps) + lr wd theta */
FH_API int fh_fno_adam(fh_fno* net, float* theta_dev, const float* grad_dev, float* m_dev, float* v_dev, int t,
                       float lr, float beta1, float beta2, float eps, float wd);

/* Normalised training target of one solved cell: target = (F - Fbar)/s.
 *   F_dev device float64 [9][N] (a converged field), Fbar host double[9],
 *   target_dev device float32 [9][N]. Fbar = I gives a zero target. */
FH_API int fh_fno_make_target(fh_fno* net, const double* F_dev, const double Fbar[9], float* target_dev);

/* Warm start for fft_homog_solve with opt->init = FH_INIT_GIVEN:
 *   F_dev = Fbar + G(s q)
 * with q the network's prediction for the cell (phase_dev, Fbar) and G the
 * compatibility projection of ctx (fh_project), so that the start field is
 * compatible and its voxel mean is exactly Fbar. ctx must have the grid of
 * net. F_dev device float64 [9][N]. */
FH_API int fh_fno_warm_start(fh_fno* net, fh_ctx* ctx, const unsigned char* phase_dev, const double Fbar[9],
                             double* F_dev);

/* Failure-detection test hook (no counterpart in the paper). The projection
 * head runs on the tcgen05 tensor cores and waits on an mbarrier for its MMAs,
 * a wait bounded at about 2^31 clock ticks (about a second), after which the
 * kernel records the failure, releases its tensor memory and returns, and the
 * calling entry point reports FH_ERR_TIMEOUT. With skip != 0 the kernel issues
 * no MMA and never signals the mbarrier, so that wait runs out: a test can
 * check the reported status, with no MMA in flight and the GPU context still
 * usable. skip = 0 restores normal operation. */
FH_API int fh_fno_test_skip_mma(fh_fno* net, int skip);

#ifdef __cplusplus
}
#endif

#endif /* FH_FNO_H */
