// Internal interface between the C-ABI layer (api.cu) and the kernel
// translation units.  Not installed; the public interface is include/flatlayer.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/flatlayer.h"
#include "common.cuh"

namespace fl {

constexpr int MAX_M1 = 128;     // data planes per problem
constexpr int MAX_M = 128;      // X planes per problem
// the dense per-mode solve and the derivative kernels hold A_nu (M1 x M) and its
// factorisations in shared memory: their limits
constexpr int DENSE_M1 = 32;
constexpr int DENSE_M = 64;
constexpr int MAX_OMEGA = 64;   // frequencies per problem
constexpr int MAX_N = 256;      // horizontal points per axis

// Device counters (index into Work::ctr); summed over the call.
enum Ctr {
  C_MODES = 0, C_ACTIVE, C_ZEROED, C_GRAZING, C_ALPHA_FLOOR, C_ROOT_CAPPED,
  C_U_GUARD, C_NAN_C, C_FP64_FALLBACK, C_NONFINITE, C_REFINE_ITERS, C_COLUMNS, C_TIMEOUT, C_COUNT
};

// Scalars of one problem, passed by value to every kernel.
struct Problem {
  int n, m, m1, n_omega;
  int alpha_mode;     // 0: per-mode discrepancy, 1: given alpha per frequency
  int max_iter;       // root-find iteration cap
  int refine_iters;   // mixed precision: FP64 residual refinement sweeps
  int solve_bps;      // resident blocks per SM of the solve
  int solve_form;     // 0: dense per-mode solve; 1: rank-one closed form
  int regularizer;    // 0: Tikhonov; 1: truncated SVD (rank-one form only)
  double period, z1, hz, c0;
  double delta, tau, delta_floor, alpha_rel, eps_u;
  double fp64_switch; // mixed precision: FP64 factor when alpha/tr(Gram) is below this
  double zy[MAX_M1];
  double zy_min;  // the lowest data plane
  double omega[MAX_OMEGA];
  double alpha_given[MAX_OMEGA];
  // grazing modes |nu| = k0: integer window [graz_lo, graz_hi] of m1^2 + m2^2, the
  // integers within a relative 1e-9 of (k0 L / 2 pi)^2 (empty when lo > hi)
  int graz_lo[MAX_OMEGA], graz_hi[MAX_OMEGA];
  // derived on the host (derive_constants), so that the kernels spend no FP64
  // division on them: k0 = omega/c0, g0 = omega^2 h_z / 2, kn = 2 pi / L
  double k0[MAX_OMEGA], g0[MAX_OMEGA];
  double kn;
  double inv_c02, u_guard;  // c0^-2 and the |u|^2 guard eps_u^2 n_omega of the recovery
  double u_guard_raw;       // the same guard on the sums of the unscaled transforms: u_guard N^4
  double inv_n2, dscale;    // 1/N^2 and tau max(delta, delta_floor): delta_nu = dscale ||W||
  int sampled;  // 1: the sampled-G kernel of a kernel plan (Work::ktab) replaces the Weyl form
  int incident; // 1: the incident field on X is given (Work::u0) instead of the plane wave
  int classify_single;  // 1: single-pass classification (one cooperative launch)
  int fft_tile;         // tile shape of the transform passes (0 large, 1 small)
  int forward_single;   // 1: the mixed path's forward 2D transform in one pass (clusters)
  int inverse_single;   // 1: the mixed path's inverse transform and recovery in one pass
  int sums64;           // 1: the mixed path's least-squares sums of step 3 in FP64 from the start
  // two-float (hi, lo) copies of the constants the mixed rank-one solve needs, so that
  // its per-mode set-up runs on the FP32 pipe: k0, k0^2, g0 per frequency, kn^2, h_z,
  // z1, alpha_rel, zy[k] - zy_min and zy_min - z_top (z_top = z1 + (M - 1/2) h_z)
  float2 k0_f[MAX_OMEGA], k0sq_f[MAX_OMEGA], g0_f[MAX_OMEGA];
  float2 knsq_f, hz_f, z1_f, alpha_rel_f, d0_f;
  float2 zyd_f[MAX_M1];
};

inline bool classify_fused_ok(const Problem& P) { return P.classify_single != 0; }

inline float2 two_float(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

// Element alignment of the caller's buffers (the kernels load and store whole complex
// and real elements): W (and a given incident field) to its complex element, xi and c
// to the real one.  NULL passes.
inline bool elems_aligned(bool fp64, const void* W, const void* xi, const void* c, const void* u0 = nullptr) {
  const uintptr_t cx = fp64 ? 16 : 8, re = cx / 2;
  return ((uintptr_t)W % cx) == 0 && ((uintptr_t)u0 % cx) == 0 && ((uintptr_t)xi % re) == 0 &&
         ((uintptr_t)c % re) == 0;
}

inline void derive_constants(Problem& P) {
  P.kn = 2.0 * M_PI / P.period;
  P.inv_c02 = 1.0 / (P.c0 * P.c0);
  P.u_guard = P.eps_u * P.eps_u * P.n_omega;
  P.u_guard_raw = P.u_guard * ((double)P.n * P.n) * ((double)P.n * P.n);
  P.inv_n2 = 1.0 / ((double)P.n * (double)P.n);
  P.dscale = P.tau * fmax(P.delta, P.delta_floor);
  for (int j = 0; j < P.n_omega; ++j) {
    const double om2 = P.omega[j] * P.omega[j];
    P.k0[j] = P.omega[j] / P.c0;
    P.g0[j] = 0.5 * om2 * P.hz;
    P.k0_f[j] = two_float(P.k0[j]);
    P.k0sq_f[j] = two_float(P.k0[j] * P.k0[j]);
    P.g0_f[j] = two_float(P.g0[j]);
  }
  P.knsq_f = two_float(P.kn * P.kn);
  P.hz_f = two_float(P.hz);
  P.z1_f = two_float(P.z1);
  P.alpha_rel_f = two_float(P.alpha_rel);
  P.d0_f = two_float(P.zy_min - (P.z1 + (P.m - 0.5) * P.hz));
  for (int k = 0; k < P.m1; ++k) P.zyd_f[k] = two_float(P.zy[k] - P.zy_min);
}

// Workspace views (device pointers).  R = bulk real type (double / float).
template <typename R> struct Work {
  cx<R>* wt;        // [n_omega][M1][N][N] W~ (mode space)                      (aliases t2)
  cx<R>* t2;        // [n_omega][2][M][N][N] y-inverse-transformed V~, U~ (compact columns)
  cx<R>* prof;      // [n_omega][N*N][2][M] solved profiles V~, U~ of active modes
  double* norms;    // [n_omega][N*N] ||b_nu||^2
  double* partial;  // [n_omega][n_partial] block sums of norms (fixed order)
  int n_partial;
  int* slot;        // [n_omega][N*N] slot of an active mode or -1
  int* act;         // [n_omega][N*N] active mode list (mode index, ascending)
  unsigned* flagbits;  // [n_omega][classify_blocks][32] active-mode bitmask (classification)
  int* blkcnt;      // [n_omega][classify_blocks] active modes per classification block
  int* blkgz;       // [n_omega][classify_blocks] grazing modes per classification block
  unsigned* colblk; // [n_omega][classify_blocks][8] columns holding an active mode, per block
  int* cols;        // [n_omega][N] columns nu1 holding a nonzero mode
  int* ncol;        // [n_omega]
  int* count;       // [n_omega] active modes
  double* dnu;      // [n_omega] delta_nu
  unsigned* bar;    // [n_omega] barrier counters of the single-pass classification
  unsigned long long* ctr;  // [C_COUNT]
  const cx<R>* tw;  // [N] twiddles exp(-2 pi i j/N)
  double* alpha_out;  // [n_omega][N*N] or null
  // FP32 data transformed in FP64 (the truncated-SVD route of the mixed precision,
  // whose pseudo-inverse passes the rounding of W~ through undamped): when set, the
  // forward transform reads the complex64 W, writes W~ here in complex128 (over the
  // start of the t12 region, sized for it by layout) with the FP64
  // twiddles tw64, and the solve reads b from here.  Null otherwise.
  double2* wt64;
  const double2* tw64;
  // sampled-G kernel (Problem::sampled): per frequency and mode the D = M1 M + M
  // values [A_nu row-major (k, l) | omega^2 h_z K~_nu(j h_z), j < M] at
  // ktab + ((omega N^2) + nu) D -- double2 in FP64; in the mixed precision float4
  // two-float pairs (hi.re, lo.re, hi.im, lo.im), the A part scaled by 1/sqrt(tr) --
  // and tr(A_nu A_nu^H) at ktr[omega N^2 + nu].  Null otherwise.
  const void* ktab;
  const double* ktr;
  // the incident field u0 on the X planes, [n_omega][M][N][N] (Problem::incident): the
  // solve then writes U~ - U~0 and the recovery adds u0 pointwise.  Null otherwise.
  const cx<R>* u0;
};

// blocks of 1024 consecutive modes in the classification of an N x N grid
inline int classify_blocks(int n) { return (n * n + 1023) / 1024; }

// Workspace of one problem: byte offsets (multiples of 256) of every Work array
// from the base of the workspace, and its total size.  The context entry points
// and the allocation-free entry point carve their workspace from this one layout.
struct Layout {
  size_t t12, prof, norms, partial, slot, act, flagbits, blkcnt, blkgz, colblk, cols, ncol, count, dnu, bar, total;
  int n_partial;
};
// (the W~ part of the t12 region is sized for complex128 in both precisions, so
// that the mixed truncated-SVD route can hold W~ in FP64: Work::wt64)
Layout layout(int n, int m, int m1, int n_omega, bool fp64);
// the Work views of a workspace laid out by `L` at `base`; counters, twiddles and the
// alpha output live elsewhere and are passed in
template <typename R>
Work<R> carve_work(void* base, const Layout& L, unsigned long long* ctr, const cx<R>* tw, double* alpha_out);

// The kernels of Algorithm 2 for one problem, enqueued on `s`: forward transform,
// classification, per-mode solve, inverse transform and recovery.  With `ev` (7
// events) the boundaries of the stages are recorded.  On failure *stage names the
// stage whose launch failed.
template <typename R>
cudaError_t launch_pipeline(const Problem& P, const Work<R>& w, const void* W, void* xi, void* c, cudaStream_t s,
                            cudaEvent_t* ev, const char** stage);

// The mixed-precision truncated SVD transforms its (complex64) data in FP64: the
// pseudo-inverse damps nothing, so FP32 rounding of W~ would reach V~ amplified by
// the inverse of each mode's singular value.
inline bool wide_route(const Problem& P, bool fp64) { return !fp64 && P.regularizer == 1; }

// Argument checks shared by the entry points (the rules of include/flatlayer.h).
// ctx may be null: the status is returned without a message.  dense_solve: the call
// runs the per-mode solve, whose dense form (o null or o->solve_form 0) is limited to
// DENSE_M x DENSE_M1; the forward generators pass false.
fs_status validate_args(fs_ctx* ctx, const fs_geometry* g, fs_precision prec, int n_omega, const double* omega,
                        double delta, double c0, const fs_options* o, bool dense_solve = true);
// The by-value problem description of validated arguments.
Problem make_problem(const fs_geometry* g, int n_omega, const double* omega, double delta, double c0,
                     const fs_options& o);

// kernel plans (kernel_plan.cu): whether a plan was made for these arguments, and
// its tables
bool kernel_plan_matches(const fs_kernel_plan* p, const fs_geometry* g, fs_precision prec, const double* omega,
                         int n_omega, double c0);
void kernel_plan_tables(const fs_kernel_plan* p, const void** tab, const double** tr);
int kernel_plan_device(const fs_kernel_plan* p);

// Launch facts kept per device, since one process may drive several GPUs:
//   sm_count()    SM count of the current device (looked up once per device)
//   opt_in_smem() cudaFuncSetAttribute(MaxDynamicSharedMemorySize) for `kernel`
//                 (and, max_shared, the largest shared-memory carveout of the unified
//                 L1/shared array, so that as many CTAs as the registers allow stay
//                 resident), done once per device; `flag` is the call site's own record
constexpr int MAX_DEVICES = 64;
int sm_count();
struct SmemOptIn {
  std::atomic<unsigned long long> done{0};  // bit d: set on device d
};
cudaError_t opt_in_smem(SmemOptIn& flag, const void* kernel, size_t bytes, bool max_shared = false);

// Launchers (return the launch error).
// `mid` (may be null) is recorded on `s` between the two kernels of the stage
// norms: also the per-mode norms and their block sums (k_mode_norms); without them the
// column pass zeroes the barrier counters of the single-pass classification instead
template <typename R>
cudaError_t launch_fft2_forward(const cx<R>* W, const Problem& P, const Work<R>& w, cudaStream_t s,
                                cudaEvent_t mid = nullptr, bool norms = true);
template <typename R>
cudaError_t launch_mode_norms(const Problem& P, const Work<R>& w, cudaStream_t s);
// classification from the norms: two kernels (flags, scatter)
template <typename R>
cudaError_t launch_classify(const Problem& P, const Work<R>& w, cudaStream_t s);
// classification in one cooperative launch that computes the norms itself (forward
// transform run with norms = false); returns an error without enqueueing anything
// when the device cannot hold the grid co-resident (the caller then falls back)
template <typename R>
cudaError_t launch_classify_fused(const Problem& P, const Work<R>& w, cudaStream_t s);
cudaError_t launch_solve_fp64(const Problem& P, const Work<double>& w, cudaStream_t s);
cudaError_t launch_solve_mixed(const Problem& P, const Work<float>& w, cudaStream_t s);
// rank-one closed form of the per-mode problem (Problem::solve_form == 1), either precision
template <typename R>
cudaError_t launch_solve_rank1(const Problem& P, const Work<R>& w, cudaStream_t s);
template <typename R>
cudaError_t launch_recover(const Problem& P, const Work<R>& w, R* xi, R* c, cudaStream_t s,
                           cudaEvent_t mid = nullptr);
template <typename R>
cudaError_t launch_twiddles(cx<R>* tw, int n, cudaStream_t s);
// dense 2D FFT of `planes` N x N planes: forward (unnormalised) in -> out, or
// inverse (with 1/N^2) transforming `in` in place along y, then in -> out along x
template <typename R>
cudaError_t launch_fft2_dense(cx<R>* in, cx<R>* out, int n, long long planes, bool inverse, const cx<R>* tw,
                              cudaStream_t s);
// the sampled-G kernel tables of one frequency (kernel_plan.cu): G sampled on the grid
// offsets, its 2D FFT, packed mode-major with omega^2 h_z applied and the traces;
// gs and ft are scratch of D N^2 complex128 each, tw64 the FP64 twiddles of N
cudaError_t launch_kernel_tables(const Problem& P, int om, double2* gs, double2* ft, const double2* tw64, bool mixed,
                                 void* tab, double* tr, cudaStream_t s);
inline int kernel_table_width(const Problem& P) { return P.m1 * P.m + P.m; }

// forward data generator (single scattering): W = F^-1[ A_nu F[omega^2 xi u0] ], u0 the
// plane wave or, when given, the incident field u0 [n_omega][M][N][N] on X
template <typename R>
cudaError_t launch_forward_born(const Problem& P, const R* xi, const cx<R>* u0, cx<R>* src, cx<R>* W,
                                const cx<R>* tw, cudaStream_t s);
// the field of point sources on the X planes in the periodic model (Sec. 5): for every
// frequency and mode U~0_nu(z'_l) = (N^2/L^2) sum_s a_s K_nu(z'_l - z_s) e^{-i nu.(r_s - x0)}
// (grazing modes zero), then its inverse 2D FFT; spec [n_src][4] = (x, y, z, a), device;
// u0 [n_omega][M][N][N]; tw the twiddles of N
template <typename R>
cudaError_t launch_point_sources(const Problem& P, const double* spec, int n_src, cx<R>* u0, const cx<R>* tw,
                                 cudaStream_t s);
// Full-scattering field per frequency -- method 0: Algorithm 1 (fixed point of eq. 6);
// 1: restarted GMRES on u - omega^2 T(xi u) = u0; 2: Algorithm 1, GMRES where it does
// not converge -- then the data of eq. (7).  iters and converged (host arrays of
// n_omega, may be null) report each frequency.  ws holds forward_bytes(P) bytes.
// Synchronises the stream at each stopping test and inner product.
template <typename R>
size_t forward_bytes(const Problem& P);
// incident: u0 [n_omega][M][N][N] on X, or null for the plane wave
template <typename R>
cudaError_t forward_solve(const Problem& P, const R* xi, const cx<R>* incident, cx<R>* W, cx<R>* u_out, void* ws,
                          int method, double rtol, int max_iter, const cx<R>* tw, cudaStream_t s, int* iters,
                          int* converged);

bool fft_size_supported(int n);

}  // namespace fl
