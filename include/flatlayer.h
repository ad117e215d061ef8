/*
 * flatlayer.h -- C ABI of the GB300 (sm_103a) implementation of the flat-layer
 * inverse multi-frequency scalar acoustics algorithm of Bakushinsky & Leonov
 * (arXiv 1911.10487): Algorithm 2 of Sec. 4, with the discretisation of Sec. 5.
 *
 * Problem (Sec. 1-2).  The Helmholtz equation  Lap u + k0^2 u = f + omega^2 xi u
 * (eq. 1), k0 = omega/c0, xi = c0^-2 - c^-2, with Green function
 * G(rho) = -exp(i k0 rho)/(4 pi rho).  The coefficient xi is supported in the
 * flat layer X = R^2 x [z1, z2]; the scattered field W = u - u0 is measured on
 * M1 planes of the layer Y above it, at one or more frequencies (eq. 2-3).
 * The incident field is the plane wave u0 = exp(-i k0 z).
 *
 * Discretisation.  The horizontal directions are periodic with period L on an
 * N x N grid (nodes x0 + i L/N); the horizontal Fourier transform of Sec. 2 is
 * the 2D DFT.  X is cut into M cells of height h_z = (z2 - z1)/M with planes at
 * the midpoints z'_l = z1 + (l + 1/2) h_z (midpoint quadrature, Sec. 5.2).  Y
 * planes are given explicitly and must all lie above z2.
 *
 * Method (Algorithm 2).  For every frequency omega and wavenumber nu = 2 pi m/L:
 *   1. b = W~_nu (2D FFT of the data planes); A_nu[k, l] = omega^2 h_z K_nu(z_k - z'_l)
 *      with K_nu(dz) = -i exp(i k_z |dz|)/(2 k_z), k_z = sqrt(k0^2 - |nu|^2),
 *      Im k_z >= 0 (eq. 8);  V~_nu = (A^H A + alpha I)^-1 A^H b (Tikhonov, Sec. 5.2),
 *      alpha chosen per mode by the discrepancy principle ||A V~ - b|| = delta_nu,
 *      delta_nu = tau max(delta, delta_floor) ||W_omega||_2;  ||b|| <= delta_nu gives
 *      V~ = 0; alpha is never below alpha_rel tr(A A^H).  Modes with |nu| = k0
 *      exactly (k_z = 0) are excluded (V~ = 0).
 *   2. U~ = U~0 + omega^2 T_nu V~, T_nu[l, l'] = h_z K_nu(z'_l - z'_l') (eq. 9);
 *      V = F^-1[V~], u = F^-1[U~].
 *   3. xi = Re(sum_omega conj(u) V) / sum_omega |u|^2 (least squares over the
 *      frequencies; V/u for one frequency); c = (c0^-2 - xi)^(-1/2).
 *
 * Conventions of every entry point.
 *   - Pointers documented as "device" must be device memory of the context's
 *     device; "host" pointers are ordinary host memory.  The library never frees
 *     caller memory.  It owns only the context's workspace.
 *   - Complex arrays are interleaved (re, im); real arrays are contiguous.  Array
 *     shapes are listed outermost first; x (the last index) is fastest.
 *   - Calls are asynchronous on the context's stream unless stated otherwise and
 *     return FS_OK once all work is enqueued.  Results are deterministic.
 *   - Errors are returned as fs_status; fs_last_error() gives a message.  Invalid
 *     arguments are detected on the host before any work is enqueued.
 */
#ifndef FLATLAYER_H
#define FLATLAYER_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FS_OK = 0,
  FS_EINVAL = 1,      /* invalid argument (shape, range, null pointer)           */
  FS_ENOMEM = 2,      /* device or pinned allocation failed                      */
  FS_ECUDA = 3,       /* a CUDA call failed; see fs_last_error                   */
  FS_EUNSUPPORTED = 4, /* size outside the compiled limits (see below)           */
  FS_ENOCONV = 5,      /* fs_forward: the fixed point did not converge            */
  FS_ENONFINITE = 6,   /* fs_sync_status: the last reconstruction met a non-finite
                          value (NaN or Inf in W, or in a recovered xi)            */
  FS_ETIMEOUT = 7      /* fs_sync_status: a device-side wait of the last
                          reconstruction gave up after its poll limit               */
} fs_status;

typedef enum {
  FS_FP64 = 0, /* every step in FP64: W complex128 in, xi/c float64 out               */
  FS_MIXED = 1 /* FFTs, kernel assembly, normal matrix and its reduction in FP32;
                  the dense solve's alpha root-find and its refinement against a
                  two-float residual (FP64 factorisation when alpha/tr(A A^H) <
                  fp64_switch); the rank-one form in two-float arithmetic;
                  W complex64 in, xi/c float32 out                                  */
} fs_precision;

/* Smallest noise level max(delta, delta_floor) the FS_MIXED reconstruction accepts
   when alpha comes from the discrepancy principle: the FP32 transform of W rounds
   each mode to about 1e-7 of ||W||, and the test ||b|| <= delta_nu needs delta_nu well
   above that.  Below it (the paper's noise levels 0 and 1e-7 of Sec. 5 with a small
   delta_floor) fs_reconstruct returns FS_EUNSUPPORTED: FS_FP64 is the path for such
   data.  Given alpha (alpha_mode 1) and the truncated SVD (whose route transforms W
   in FP64) are not limited. */
#define FS_MIXED_MIN_NOISE 1e-6

/* Limits of this build: N in {8,12,16,24,32,48,64,96,128,192,256}; 1 <= M <= 128;
   1 <= M1 <= 128; 1 <= n_omega <= 64.  The dense per-mode solve (solve_form 0, the
   default; the sampled kernel; the derivatives of flatlayer_diff.h) holds A_nu in
   shared memory and takes M <= 64, M1 <= 32; the rank-one form serves the rest. */

typedef struct {
  int n;            /* N: horizontal grid points per axis                           */
  int m;            /* M: X planes                                                  */
  int m1;           /* M1: data (Y) planes                                          */
  double period;    /* L > 0: horizontal period                                     */
  double z1, z2;    /* X slab [z1, z2], z2 > z1                                     */
  const double* zy; /* host, M1 heights of the data planes, each > z2               */
} fs_geometry;

typedef struct fs_kernel_plan fs_kernel_plan;

typedef struct {
  double tau;          /* discrepancy factor: delta_nu = tau max(delta, delta_floor) ||W|| (default 2) */
  double delta_floor;  /* lower bound of the relative noise level (default 1e-5)          */
  double alpha_rel;    /* alpha >= alpha_rel tr(A A^H) (default 1e-6)                     */
  double eps_u;        /* xi := 0 where sum |u|^2 < eps_u^2 n_omega (default 1e-8)        */
  int alpha_mode;      /* 0: per-mode discrepancy principle; 1: alpha_given per frequency,
                          every non-grazing mode solved (default 0)                       */
  const double* alpha_given; /* host, n_omega values, read when alpha_mode == 1           */
  int max_iter;        /* root-find iteration cap (default 100)                           */
  int refine_iters;    /* FS_MIXED: cap on FP64 refinement sweeps (default 8)             */
  double fp64_switch;  /* FS_MIXED: FP64 factorisation below alpha/tr = this (default 1e-4) */
  int stage_timing;    /* 1: record CUDA events between the kernels of fs_reconstruct; the
                          durations appear in fs_report.ms_stage (default 0)              */
  int solve_blocks_per_sm; /* 1, 2 or 3: resident blocks per SM of the per-mode solve (grid =
                          this x SM count); a tuning knob (default 2)                      */
  int solve_form;      /* 0: dense -- the normal matrix A A^H formed and reduced per mode
                          (default); 1: rank-one closed form.  Every data plane lies above
                          X, so K_nu(z_k - z'_l) factors and A_nu = E P^T has rank one
                          exactly: the Tikhonov solution is conj(P) (E^H b)/(tr + alpha) and
                          the discrepancy root is explicit, O(M1 + M) per mode.  FS_MIXED:
                          the factors E, P rounded to FP32, every sum, the root, V~ and
                          eq. (9) in two-float arithmetic on the FP32 pipe.  The two forms
                          agree to rounding.                                              */
  int regularizer;     /* 0: Tikhonov (default); 1: truncated SVD (Sec. 5: the paper's best
                          regularising algorithm), truncation rank by the discrepancy
                          principle -- rank one on these kernels, i.e. the pseudo-inverse on
                          every active mode.  Requires solve_form 1 and alpha_mode 0
                          (FS_EUNSUPPORTED / FS_EINVAL otherwise); alpha output 0.        */
  const fs_kernel_plan* kernel_plan; /* NULL (default): the Weyl closed form of K_nu.  Else
                          the sampled-G kernel of Sec. 5 tabulated by fs_kernel_plan_create,
                          which must have been made for the same geometry, precision,
                          frequencies and c0 on the context's device (FS_EINVAL otherwise).
                          A_nu is then numerically full rank and only the dense form solves
                          it (solve_form 1 gives FS_EUNSUPPORTED); eq. (9) is applied as the
                          Toeplitz matrix T_nu; no mode is excluded as grazing.  Only
                          fs_reconstruct and fs_reconstruct_host accept it.             */
  int classify_single_pass; /* 0 (default): the norms of the modes, the discrepancy test and the
                          active list in three kernels.  1: in one cooperative launch whose
                          blocks meet at two bounded device-side barriers (a wait that runs
                          out is reported by fs_sync_status as FS_ETIMEOUT); taken when the
                          device holds the grid co-resident, else the three-kernel form.
                          Fewer launches (batches); on one 128^2 problem the three kernels,
                          overlapped by programmatic dependent launch, are faster (measured).
                          Results are identical up to the rounding of the sum ||W||^2 (its
                          terms are grouped differently).                                  */
  int fft_tile;        /* tile shape of the transform passes, a tuning knob: 0 (default)
                          shared-memory tiles of 2048 elements, 16 (FP32) / 8 (FP64) columns
                          per column tile, radix cap 16; 1: tiles of 1024 elements, 8 / 4
                          columns, radix cap 8 (twice the blocks, half the shared memory
                          each).  Applies to the two-pass transforms.  Results agree to
                          rounding.                                                      */
  int forward_single_pass; /* FS_MIXED, N <= 128: 1 (default): the forward 2D transform of W in one pass,
                          a cluster of CTAs per data plane exchanging rows and columns
                          through distributed shared memory; 0: two passes (rows, then
                          columns) through global memory.  FS_FP64 always takes the two
                          passes.  The results agree to rounding.                       */
  int inverse_single_pass; /* FS_MIXED, N <= 128 except 96: 1: the inverse transform along y,
                          along x and the recovery of xi and c in one pass, a cluster of
                          CTAs per X plane (the transformed active columns go to the CTAs
                          that own their rows through distributed shared memory); 0
                          (default, measured faster on one 128^2 problem): two passes (the
                          column pass writes the transformed active columns to global
                          memory, the row pass reads them).  FS_FP64 always takes the two
                          passes.  The results agree to rounding.                       */
  int fp64_sums;        /* FS_MIXED: the least-squares sums of Sec. 5.2 (step 3 of Algorithm 2)
                          over the frequencies: 0 (default) in FP32, redone in FP64 for the
                          rows where they overflow; 1: in FP64 from the start.  FS_FP64
                          always sums in FP64.                                          */
  const void* incident;  /* NULL (default): the incident field is the plane wave exp(-i k0 z).
                          Else device, [n_omega][M][N][N] complex in the working precision:
                          the incident field u0 on the X planes (for instance the point
                          sources of fs_incident_point_sources, Sec. 5); Algorithm 2 step 2
                          then takes u = u0 + F^-1[omega^2 T_nu V~].  fs_reconstruct,
                          fs_reconstruct_host and fs_reconstruct_static accept it.      */
} fs_options;

typedef struct {
  long long n_modes;         /* wavenumbers examined (n_omega N^2)                   */
  long long n_active;        /* modes solved                                         */
  long long n_zeroed;        /* modes with ||b|| <= delta_nu (V~ = 0)                */
  long long n_grazing;       /* modes with |nu| = k0 (excluded)                      */
  long long n_alpha_floor;   /* active modes where alpha = alpha_rel tr(A A^H)       */
  long long n_root_capped;   /* root-finds stopped by max_iter                        */
  long long n_u_guard;       /* voxels where sum |u|^2 < eps_u^2 n_omega (xi := 0)   */
  long long n_nan_c;         /* voxels where xi >= c0^-2 (c := NaN)                  */
  long long n_fp64_fallback; /* FS_MIXED: modes refactorised in FP64                  */
  long long n_refine_iters;  /* FS_MIXED: refinement sweeps performed                 */
  long long n_columns;       /* columns nu1 holding a nonzero mode, summed over omega:
                                the inverse transform along y runs on these only       */
  long long n_nonfinite;     /* modes whose ||W~_nu||^2 is not finite (W holds a NaN or
                                Inf) plus voxels whose recovered xi is not finite plus
                                modes whose solution leaves the range of the working
                                precision; when nonzero the outputs are unspecified     */
  long long n_timeouts;      /* device-side waits that ran out (the single-pass
                                classification); when nonzero the outputs are unspecified */
  float ms_stage[6];         /* with stage_timing: device milliseconds of the kernels
                                [0] forward FFT along x, [1] forward FFT along y + mode
                                norms, [2] mode classification, [3] per-mode solve,
                                [4] inverse FFT along y (gather), [5] inverse FFT along x
                                + xi/c; zeros otherwise                                  */
} fs_report;

typedef struct fs_ctx fs_ctx;

/* Library version string (static storage). */
const char* fs_version(void);

/* Fill *opts with the defaults listed in fs_options.  Returns FS_EINVAL on NULL. */
fs_status fs_default_options(fs_options* opts);

/* Create a context on CUDA device `device`, enqueueing on `stream` (a
   cudaStream_t; NULL = the legacy default stream).  The context owns a workspace
   that grows on demand and is released by fs_destroy.  *ctx receives the handle.
   A growth reallocates the workspace: CUDA graphs captured earlier around calls on
   this context refer to the old one and must be captured again after any call that
   needed more (a larger problem, fs_forward_born, fs_forward); fs_reserve sizes it up
   front, fs_workspace_generation tells whether it has moved, and a growth during a
   capture is refused (FS_EUNSUPPORTED). */
fs_status fs_create(fs_ctx** ctx, int device, void* stream);

/* Release the context and its workspace (synchronises its stream).  NULL is a no-op. */
void fs_destroy(fs_ctx* ctx);

/* Grow the context's workspace now (synchronously) to what fs_reconstruct needs for
   this geometry, frequency count and precision, and make the twiddle tables of N, so
   that later calls up to that size allocate nothing and can be captured into CUDA
   graphs.  A call that would have to
   grow the workspace while the context's stream is being captured returns
   FS_EUNSUPPORTED instead (nothing is enqueued).  Errors: FS_EINVAL, FS_EUNSUPPORTED,
   FS_ENOMEM, FS_ECUDA. */
fs_status fs_reserve(fs_ctx* ctx, const fs_geometry* geom, int n_omega, fs_precision prec);

/* How many times the context's workspace has been reallocated (0 for NULL).  A graph
   captured when this count was g refers to freed memory once it has changed: compare
   before replaying. */
unsigned long long fs_workspace_generation(const fs_ctx* ctx);

/* Message describing the last error of this context (never NULL). */
const char* fs_last_error(const fs_ctx* ctx);

/* Bytes of device workspace fs_reconstruct needs for this geometry. */
fs_status fs_workspace_size(const fs_geometry* geom, int n_omega, fs_precision prec, size_t* bytes);

/* Algorithm 2 (Sec. 4 steps 1-3) on one problem.
     W         device, [n_omega][M1][N][N] complex (complex128 for FS_FP64,
               complex64 for FS_MIXED): scattered field on the data planes.
     omega     host, n_omega angular frequencies (> 0).
     delta     relative noise level of W (>= 0).
     c0        background sound speed (> 0).
     opts      NULL for defaults.
     xi        device, [M][N][N] real (float64 / float32): reconstructed xi.
     c         device, [M][N][N] real, or NULL: sound speed (NaN where xi >= c0^-2).
     alpha_out device, [n_omega][N][N] float64, or NULL: chosen alpha of each active
               mode (other entries are left untouched).
   The workspace grows (synchronously) when a larger problem arrives; otherwise the
   call only enqueues work.  Counters of the call are read with fs_get_report.
   Every buffer must be aligned to its element (W and the incident field to the complex
   element, xi and c to the real one, alpha_out to 8 bytes): FS_EINVAL otherwise. */
fs_status fs_reconstruct(fs_ctx* ctx, const fs_geometry* geom, fs_precision prec, const void* W,
                         const double* omega, int n_omega, double delta, double c0,
                         const fs_options* opts, void* xi, void* c, double* alpha_out);

/* Same as fs_reconstruct with HOST buffers W, xi, c (c may be NULL), synchronising
   the stream before returning.  Page-locked buffers mapped into the device's address
   space at the same address (cudaHostAlloc / torch pin_memory under unified
   addressing), aligned to their elements: the kernels read W and write xi and c there
   directly over the host link (on a Grace-Blackwell node the coherent NVLink-C2C), no
   staging copy; a repeated call replays a graph captured after the first.  Other host
   buffers: W is copied to a device staging buffer, xi (and c) copied back. */
fs_status fs_reconstruct_host(fs_ctx* ctx, const fs_geometry* geom, fs_precision prec, const void* W_host,
                              const double* omega, int n_omega, double delta, double c0,
                              const fs_options* opts, void* xi_host, void* c_host);

/* One entry of a batch: a complete problem (arguments as for fs_reconstruct). */
typedef struct {
  fs_geometry geom;
  const void* W;        /* device, [n_omega][M1][N][N] complex                */
  const double* omega;  /* host, n_omega                                      */
  int n_omega;
  double delta, c0;
  void* xi;             /* device, [M][N][N] real                             */
  void* c;              /* device, [M][N][N] real, or NULL                    */
} fs_problem;

/* Many independent problems of uneven size in one call (the paper reconstructs one
   problem at a time; batching is a throughput device).  Each problem is solved
   exactly as by fs_reconstruct; the problems are dealt, largest first, over
   n_streams (1..64) streams forked from the context's stream and joined back to
   it, so independent problems run concurrently.  The workspace is the sum of the
   problems' workspaces.  Fork and join use events only, so the call can be
   captured into a CUDA graph once the workspace has been sized by an earlier call.
   Counters of fs_get_report are summed over the batch; stage timing is off.
   Errors: FS_EINVAL (names the first bad problem), FS_EUNSUPPORTED, FS_ENOMEM. */
fs_status fs_reconstruct_batch(fs_ctx* ctx, const fs_problem* probs, int n_probs, fs_precision prec,
                               const fs_options* opts, int n_streams);

/* Forward data generator in the single-scattering (Born) form: Algorithm 1 of
   Sec. 3 with zero iterations, i.e. U~ = U~0 in eq. (7):
     W = F^-1[ omega^2 sum_l h_z K_nu(z_k - z'_l) F[xi u0](z'_l) ]  on the data planes,
   with k0 = omega/c0 and grazing modes excluded as above.
     xi        device, [M][N][N] real (float64 for FS_FP64, float32 for FS_MIXED).
     incident  device, [n_omega][M][N][N] complex (complex128 / complex64): u0 on the X
               planes; or NULL for the plane wave u0 = exp(-i k0 z).
     W         device, [n_omega][M1][N][N] complex (complex128 / complex64), written.
   Uses the context workspace; asynchronous. */
fs_status fs_forward_born(fs_ctx* ctx, const fs_geometry* geom, fs_precision prec, const void* xi,
                          const void* incident, const double* omega, int n_omega, double c0, void* W);

/* The incident field of point sources on the X planes (Sec. 5: sources f = sum_s a_s
   delta(x - x_s), u0 = sum_s a_s G(|x - x_s|)), in the horizontally periodic model of
   this library: for every frequency and mode
     U~0_nu(z'_l) = (N^2/L^2) sum_s a_s K_nu(z'_l - z_s) exp(-i nu . (r_s - x0)),
   K_nu the Weyl form (grazing modes zero), x0 = -L/2 the first grid node on both
   horizontal axes (nodes x0 + i L/N), then u0 = F^-1[U~0] on each X plane.
     sources  host, [n_sources][4] doubles (x, y, z, a): position and real amplitude;
              every source lies above X (z > z2).
     u0       device, [n_omega][M][N][N] complex (complex128 / complex64), written.
   Synchronises the context's stream.  Errors: FS_EINVAL, FS_EUNSUPPORTED, FS_ECUDA. */
fs_status fs_incident_point_sources(fs_ctx* ctx, const fs_geometry* geom, fs_precision prec, const double* sources,
                                    int n_sources, const double* omega, int n_omega, double c0, void* u0);

/* Solver of the full-scattering forward problem u = u0 + omega^2 T(xi u) on X (first
   line of eq. 2) for fs_forward. */
typedef enum {
  FS_FIXED_POINT = 0,       /* Algorithm 1 of Sec. 3 (the fixed point of eq. 6)          */
  FS_GMRES = 1,             /* restarted GMRES on u - omega^2 T(xi u) = u0                */
  FS_FIXED_POINT_GMRES = 2  /* Algorithm 1, and GMRES for a frequency where it fails      */
} fs_forward_method;

/* Forward data generator with full scattering.  FS_FIXED_POINT iterates Algorithm 1,
     U~_{n+1} = U~0 + omega^2 T_nu F_r[xi F^-1 U~_n],  T_nu[l, l'] = h_z K_nu(z'_l - z'_l'),
   from U~_1 = U~0 (the plane wave u0 = exp(-i k0 z)), to the first n with
   ||U~_{n+1} - U~_n|| <= rtol ||U~0|| (Frobenius norms over the M planes of one
   frequency; the stopping rule of Sec. 5.1 with rtol = 1e-13).  FS_GMRES solves the
   same equation in X by restarted GMRES (30 vectors per cycle, from u = 0) to
   ||u0 - u + omega^2 T(xi u)|| <= rtol ||u0||, the residual computed afresh at each
   restart.  Either way the data of eq. (7) follow from the converged field.  Each
   frequency is solved on its own.
     xi        device, [M][N][N] real (float64 for FS_FP64, float32 for FS_MIXED).
     incident  device, [n_omega][M][N][N] complex: the incident field u0 on X (for
               instance fs_incident_point_sources), whose U~0 = F_r[u0] starts
               Algorithm 1 and enters each step; or NULL for the plane wave.  The
               stopping rule then takes ||U~0|| of that field.
     omega     host, n_omega values > 0.
     max_iter  >= 0: iterations of Algorithm 1, or operator applications of GMRES (each
               method of FS_FIXED_POINT_GMRES gets max_iter); FS_FIXED_POINT with 0
               gives the single-scattering data of fs_forward_born.
     rtol      > 0; FP32 rounding bounds it below near 1e-6 in FS_MIXED.
     W         device, [n_omega][M1][N][N] complex, written.
     u         device, [n_omega][M][N][N] complex (the total field on X), written; or NULL.
     iterations host, n_omega ints, or NULL: iterations of Algorithm 1 plus Arnoldi
               steps of GMRES (each one operator application; the residual computed at
               each restart is one more, not counted).
   Returns FS_ENOCONV, with W and u of the remaining frequencies unwritten, when a
   frequency has not converged within max_iter or its iterate grows past 1e30 times the
   incident field (Algorithm 1 with a scatterer too strong for the fixed point:
   omega^2 ||T xi|| >= 1).  Uses the context workspace; synchronises the context's
   stream at each stopping test and GMRES inner product, so it cannot be captured in a
   graph. */
fs_status fs_forward(fs_ctx* ctx, const fs_geometry* geom, fs_precision prec, const void* xi,
                     const void* incident, const double* omega, int n_omega, double c0, fs_forward_method method,
                     int max_iter, double rtol, void* W, void* u, int* iterations);

/* Sampled-G kernel (Sec. 5: the discrete analogue of G~ computed from the values of G
   by the FFT), the alternative to the Weyl closed form.  For every frequency and mode
     K~_nu(dz) = h^2 sum_{i,j} G(sqrt(x_i^2 + y_j^2 + dz^2)) exp(-i nu . (x_i, y_j)),
   over the offsets x_i = i h (i < N/2), (i - N) h (otherwise) of one period of the
   grid (the horizontal convolution with G cut to one period, periodised), h = L/N;
   at rho = 0 the sample is the integral of G over the grid cell (taken over the ball
   of equal volume) divided by h_z.  The plan tabulates, per frequency and mode, the
   M1 x M entries of A_nu = omega^2 h_z K~_nu(z_k - z'_l) and the M values
   omega^2 h_z K~_nu(j h_z) of eq. (9), and tr(A_nu A_nu^H): (M1 M + M) N^2 n_omega x 16
   bytes of device memory, built synchronously on the current device (the batched
   FFTs of G sampled at every offset) and owned by the plan.  ctx is used for its
   argument checks and messages.  Errors: FS_EINVAL, FS_EUNSUPPORTED, FS_ENOMEM,
   FS_ECUDA. */
fs_status fs_kernel_plan_create(fs_ctx* ctx, const fs_geometry* geom, fs_precision prec, const double* omega,
                                int n_omega, double c0, fs_kernel_plan** plan);
/* Release the plan's tables (synchronises the device).  NULL is a no-op. */
void fs_kernel_plan_destroy(fs_kernel_plan* plan);
/* Device bytes held by the plan (0 for NULL). */
size_t fs_kernel_plan_bytes(const fs_kernel_plan* plan);

/* Size of the device array that holds every intermediate of fs_reconstruct_static. */
#define FS_STATIC_SCRATCH_BYTES (32u << 20)

/* fs_reconstruct without any device allocation.  The paper has no counterpart:
   this entry point exists for callers that cannot call cudaMalloc -- a host
   framework that hands out all device memory from its own pool, or a real-time
   or embedded caller that must not grow its memory or synchronise the device
   once it is running (a cudaMalloc may do both).  It takes no context and
   allocates nothing: the caller passes W, xi and c (same layouts, precisions and
   results as fs_reconstruct; no alpha_out, no report), and every intermediate
   lives in one device array of FS_STATIC_SCRATCH_BYTES (32 MiB) that every GPU
   which loads the library holds until the process exits.  `stream` is a
   cudaStream_t (NULL = the legacy default stream); the call is asynchronous on it.
   A problem whose intermediates do not fit returns FS_EUNSUPPORTED before any
   work is enqueued: for one frequency, 128 x 128 x 32 with 32 data planes fits in
   FS_MIXED, 128 x 128 x 64 does not, and 64 x 64 x 64 with 32 planes fits in FS_FP64.
   The first call on a device looks up the device address of that array
   (cudaGetSymbolAddress) and keeps it.  Under CUDA's lazy module loading that
   lookup may itself load the library's device code onto the device, which
   allocates device memory and can synchronise: make the first call on each
   device during start-up, before any stream capture and before the phase in
   which the caller may not allocate.  Every call uses the same array: calls whose work overlaps on the GPU
   (different streams, or different host threads without ordering) race and
   corrupt each other's results, so serialise them.  Other errors as for
   fs_reconstruct (FS_EINVAL, FS_EUNSUPPORTED, FS_ECUDA), without a message. */
fs_status fs_reconstruct_static(const fs_geometry* geom, fs_precision prec, const void* W, const double* omega,
                                int n_omega, double delta, double c0, const fs_options* opts, void* xi, void* c,
                                void* stream);

/* Synchronise the context's stream and return the counters of the last
   fs_reconstruct call. */
fs_status fs_get_report(fs_ctx* ctx, fs_report* report);

/* Device-side status of the last fs_reconstruct (or fs_reconstruct_batch) call on
   this context.  The calls return once their work is enqueued, so what the
   kernels find is reported here: synchronises the context's stream, then returns
   FS_ECUDA if the stream reports an error, FS_ETIMEOUT if a device-side wait ran
   out (fs_report.n_timeouts > 0), FS_ENONFINITE if the call met a non-finite value
   (fs_report.n_nonfinite > 0: a NaN or Inf in W makes delta_nu undefined, so no mode
   is solved and xi, c are unspecified; or a solution beyond the range of the working
   precision), and FS_OK otherwise.  The message of fs_last_error says what was found. */
fs_status fs_sync_status(fs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* FLATLAYER_H */
