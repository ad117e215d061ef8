/*
 * flatlayer_diff.h -- derivatives of the flat-layer reconstruction (Algorithm 2
 * of arXiv 1911.10487, Sec. 4) at a fixed Tikhonov parameter per frequency.
 *
 * The differentiated map.  With alpha_omega = exp(log_alpha[omega]) fixed (no
 * discrepancy search), for every frequency omega and wavenumber nu
 *   b = W~_nu (2D FFT of the data planes, Sec. 2),
 *   V~_nu = A_nu^H (A_nu A_nu^H + alpha_omega I)^-1 b  (eq. 8, the Tikhonov normal
 *           solution of Sec. 4 comment b; V~ = 0 on modes with |nu| = k0),
 *   U~_nu = U~0_nu + omega^2 T_nu V~_nu (eq. 9),  V = F^-1[V~],  u = F^-1[U~],
 *   xi = Re(sum_omega conj(u) V) / sum_omega |u|^2, 0 where that sum is below
 *        eps_u^2 n_omega (step 3; the mask is held fixed when differentiating),
 *   Phi_omega = sum_nu ||A_nu V~_nu - b||^2   (the discrepancy of Sec. 4, summed
 *        over all N^2 modes; an excluded mode contributes ||b||^2).
 * The library computes xi, c = (c0^-2 - xi)^(-1/2) and Phi, and the derivatives
 *   VJP: (xi-bar, Phi-bar) -> (W-bar, log_alpha-bar)
 *   JVP: (W-dot, log_alpha-dot) -> (xi-dot, Phi-dot)
 * For complex W the gradient is dL/dRe W + i dL/dIm W (so dL = Re sum conj(W-bar) dW),
 * the convention of PyTorch's complex autograd.
 *
 * Precision.  FS_FP64: everything in FP64.  FS_MIXED: W, xi, c, the FFTs and the
 * pointwise step 3 in FP32 (complex64 / float32 arrays); the per-mode normal
 * matrices, their Cholesky factors and the solves stay in FP64.
 *
 * Memory.  A plan owns the per-mode normal matrices A_nu A_nu^H (they depend on
 * the geometry and frequencies only; 16 n_omega N^2 M1 (M1+1)/2 bytes).  Every
 * other buffer is caller-owned device memory: a tape (written by the forward,
 * read by VJP and JVP) and a scratch buffer, both 256-byte aligned, of the sizes
 * the *_bytes functions return.  A tape stays valid until the next forward into
 * it.  All calls enqueue on the context's stream, allocate nothing, do not
 * synchronise (so they can be captured in a CUDA graph) and are deterministic.
 * Shapes as in flatlayer.h: W [n_omega][M1][N][N], xi and c [M][N][N].
 */
#ifndef FLATLAYER_DIFF_H
#define FLATLAYER_DIFF_H

#include <stddef.h>

#include "flatlayer.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fs_diff_plan fs_diff_plan;

/* Plan for one geometry, precision and frequency list (omega: host, n_omega
   entries).  Allocates the normal matrices and enqueues their computation.
   FS_EINVAL / FS_EUNSUPPORTED as fs_reconstruct; FS_ENOMEM if the allocation
   fails.  The plan keeps `ctx` (not owned) and must be destroyed before it. */
fs_status fs_diff_plan_create(fs_ctx* ctx, const fs_geometry* geom, fs_precision prec, const double* omega,
                              int n_omega, double c0, double eps_u, fs_diff_plan** plan);
void fs_diff_plan_destroy(fs_diff_plan* plan);

/* Sizes of the caller-owned buffers.  The scratch for fs_reconstruct_jvp with
   n_dir directions holds min(n_dir, 16) of them (larger n_dir run in chunks of
   16); n_dir = 1 suffices for the forward and the VJP. */
size_t fs_diff_tape_bytes(const fs_diff_plan* plan);
size_t fs_diff_scratch_bytes(const fs_diff_plan* plan, int n_dir);

/* Forward: xi [M][N][N] (device, real), c (device or NULL), phi [n_omega]
   (device FP64 or NULL) from W (device, complex) and log_alpha [n_omega]
   (device, FP64).  Records the tape. */
fs_status fs_reconstruct_diff(fs_diff_plan* plan, void* tape, void* scratch, const void* W,
                              const double* log_alpha, void* xi, void* c, double* phi);

/* VJP of the last forward recorded in `tape`: grad_xi [M][N][N] (device, real,
   or NULL for zero), grad_phi [n_omega] (device FP64 or NULL) ->
   grad_W [n_omega][M1][N][N] (device complex, or NULL to skip) and
   grad_log_alpha [n_omega] (device FP64, or NULL to skip). */
fs_status fs_reconstruct_vjp(fs_diff_plan* plan, const void* tape, void* scratch, const void* grad_xi,
                             const double* grad_phi, void* grad_W, double* grad_log_alpha);

/* JVP of the last forward recorded in `tape` for n_dir >= 1 directions:
   dW [n_dir][n_omega][M1][N][N] (device complex), dlog_alpha [n_dir][n_omega]
   (device FP64, or NULL for zero) -> dxi [n_dir][M][N][N] (device real) and
   dphi [n_dir][n_omega] (device FP64 or NULL). */
fs_status fs_reconstruct_jvp(fs_diff_plan* plan, const void* tape, void* scratch, int n_dir, const void* dW,
                             const double* dlog_alpha, void* dxi, double* dphi);

#ifdef __cplusplus
}
#endif

#endif /* FLATLAYER_DIFF_H */
