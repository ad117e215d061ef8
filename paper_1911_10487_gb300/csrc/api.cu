// C ABI of the flat-layer reconstruction (declared in include/flatlayer.h):
// argument validation, context/workspace management and the launch sequence of
// Algorithm 2 (Sec. 4):
//   fft2_forward (W -> W~, ||W~_nu||^2) -> classify (delta_nu, active modes)
//   -> solve (eq. 8 Tikhonov + discrepancy, eq. 9) -> recover (F^-1, step 3).
#include <stdarg.h>
#include <stdio.h>
#include <new>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cmath>

#include <atomic>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/flatlayer.h"
#include "../../include/flatlayer_diff.h"
#include "diff.cuh"
#include "pipeline.cuh"

using namespace fl;

namespace {

constexpr int N_SIZES = 11;
const int kSizes[N_SIZES] = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256};

int size_index(int n) {
  for (int i = 0; i < N_SIZES; ++i)
    if (kSizes[i] == n) return i;
  return -1;
}

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

struct fs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  unsigned long long ws_generation = 0;  // reallocations of ws so far
  void* tw[2][N_SIZES] = {};  // [fp64?][size]
  unsigned long long* ctr = nullptr;
  unsigned long long* ctr_host = nullptr;
  // staging for fs_reconstruct_host
  void* stage = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t ev[7] = {};
  bool timed = false;
  // batches: side streams forked from `stream` and joined back with events
  static constexpr int MAX_SIDE = 64;
  cudaStream_t side[MAX_SIDE] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[MAX_SIDE] = {};
  // fs_reconstruct_host: the last call captured as a CUDA graph, replayed while the
  // call repeats (same problem, options and buffers; pinned host memory)
  std::vector<unsigned char> host_key;
  cudaGraphExec_t host_exec = nullptr;
  char err[512] = {0};
};

namespace {

fs_status fail(fs_ctx* ctx, fs_status st, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

// page-locked (or registered) host memory: copies from it can be captured in a graph
bool pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// page-locked host memory that the current device reaches at the same address (mapped
// under unified addressing): kernels may read and write it directly
bool mapped_here(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

template <typename T> void key_put(std::vector<unsigned char>& k, const T& v) {
  const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
  k.insert(k.end(), b, b + sizeof(T));
}

fs_status cuda_fail(fs_ctx* ctx, cudaError_t e, const char* where) {
  if (ctx) snprintf(ctx->err, sizeof(ctx->err), "%s: %s", where, cudaGetErrorString(e));
  return FS_ECUDA;
}

}  // namespace

namespace fl {

Layout layout(int n, int m, int m1, int n_omega, bool fp64) {
  const size_t cxs = fp64 ? 16 : 8;
  const size_t N2 = (size_t)n * n;
  // W~ in complex128 in both precisions (the mixed truncated-SVD route), then the
  // y-inverse output in the working precision over it
  const size_t a = 16 * (size_t)n_omega * m1 * N2, b = cxs * (size_t)n_omega * 2 * m * N2;
  Layout L;
  size_t off = 0;
  L.t12 = off; off = align_up(off + (a > b ? a : b));  // W~, later the y-inverse pass output
  L.prof = off; off = align_up(off + cxs * (size_t)n_omega * N2 * 2 * m);
  L.norms = off; off = align_up(off + 8 * (size_t)n_omega * N2);
  L.n_partial = (int)((N2 + 63) / 64);  // blocks of the norms kernel (64 modes each)
  L.partial = off; off = align_up(off + 8 * (size_t)n_omega * L.n_partial);
  L.slot = off; off = align_up(off + 4 * (size_t)n_omega * N2);
  L.act = off; off = align_up(off + 4 * (size_t)n_omega * N2);
  const size_t cb = (size_t)n_omega * classify_blocks(n);
  L.flagbits = off; off = align_up(off + 4 * cb * 32);
  L.blkcnt = off; off = align_up(off + 4 * cb);
  L.blkgz = off; off = align_up(off + 4 * cb);
  L.colblk = off; off = align_up(off + 4 * cb * 8);
  L.cols = off; off = align_up(off + 4 * (size_t)n_omega * n);
  L.ncol = off; off = align_up(off + 4 * (size_t)n_omega);
  L.count = off; off = align_up(off + 4 * (size_t)n_omega);
  L.dnu = off; off = align_up(off + 8 * (size_t)n_omega);
  L.bar = off; off = align_up(off + 4 * (size_t)n_omega);
  L.total = off;
  return L;
}

fs_status validate_args(fs_ctx* ctx, const fs_geometry* g, fs_precision prec, int n_omega, const double* omega,
                        double delta, double c0, const fs_options* o, bool dense_solve) {
  if (!g) return fail(ctx, FS_EINVAL, "geometry is NULL");
  if (prec != FS_FP64 && prec != FS_MIXED) return fail(ctx, FS_EINVAL, "unknown precision");
  if (g->n <= 0 || g->m <= 0 || g->m1 <= 0) return fail(ctx, FS_EINVAL, "grid sizes must be positive");
  if (!fft_size_supported(g->n))
    return fail(ctx, FS_EUNSUPPORTED, "N=%d not supported (8,12,16,24,32,48,64,96,128,192,256)",
                g->n);
  if (g->m > MAX_M) return fail(ctx, FS_EUNSUPPORTED, "M=%d exceeds %d", g->m, MAX_M);
  if (g->m1 > MAX_M1) return fail(ctx, FS_EUNSUPPORTED, "M1=%d exceeds %d", g->m1, MAX_M1);
  // the dense per-mode solve (solve_form 0, the default) holds A_nu in shared memory
  const bool dense = dense_solve && (!o || o->solve_form == 0);
  if (dense && (g->m > DENSE_M || g->m1 > DENSE_M1))
    return fail(ctx, FS_EUNSUPPORTED,
                "the dense form solves M <= %d, M1 <= %d (got M=%d, M1=%d); larger layers take the rank-one form "
                "(solve_form 1)",
                DENSE_M, DENSE_M1, g->m, g->m1);
  if (n_omega <= 0) return fail(ctx, FS_EINVAL, "n_omega must be positive");
  if (n_omega > MAX_OMEGA) return fail(ctx, FS_EUNSUPPORTED, "n_omega=%d exceeds 64", n_omega);
  if (!omega) return fail(ctx, FS_EINVAL, "omega is NULL");
  for (int j = 0; j < n_omega; ++j)
    if (!(omega[j] > 0.0)) return fail(ctx, FS_EINVAL, "omega[%d] must be > 0", j);
  if (!(g->period > 0.0)) return fail(ctx, FS_EINVAL, "period must be > 0");
  if (!(g->z2 > g->z1)) return fail(ctx, FS_EINVAL, "need z2 > z1");
  if (!g->zy) return fail(ctx, FS_EINVAL, "zy is NULL");
  for (int k = 0; k < g->m1; ++k)
    if (!(g->zy[k] > g->z2)) return fail(ctx, FS_EINVAL, "data plane %d is not above X", k);
  if (!(delta >= 0.0)) return fail(ctx, FS_EINVAL, "delta must be >= 0");
  if (!(c0 > 0.0)) return fail(ctx, FS_EINVAL, "c0 must be > 0");
  if (o) {
    if (!(o->tau > 0.0) || !(o->delta_floor >= 0.0) || !(o->alpha_rel > 0.0) || !(o->eps_u >= 0.0))
      return fail(ctx, FS_EINVAL, "options out of range (tau>0, delta_floor>=0, alpha_rel>0, eps_u>=0)");
    if (o->alpha_mode != 0 && o->alpha_mode != 1) return fail(ctx, FS_EINVAL, "alpha_mode must be 0 or 1");
    if (o->alpha_mode == 1) {
      if (!o->alpha_given) return fail(ctx, FS_EINVAL, "alpha_given is NULL");
      for (int j = 0; j < n_omega; ++j)
        if (!(o->alpha_given[j] > 0.0)) return fail(ctx, FS_EINVAL, "alpha_given[%d] must be > 0", j);
    }
    if (o->max_iter < 1 || o->refine_iters < 1) return fail(ctx, FS_EINVAL, "max_iter >= 1, refine_iters >= 1");
    if (o->solve_blocks_per_sm < 1 || o->solve_blocks_per_sm > 3)
      return fail(ctx, FS_EINVAL, "solve_blocks_per_sm must be 1, 2 or 3");
    if (o->solve_form != 0 && o->solve_form != 1) return fail(ctx, FS_EINVAL, "solve_form must be 0 or 1");
    if (o->classify_single_pass != 0 && o->classify_single_pass != 1)
      return fail(ctx, FS_EINVAL, "classify_single_pass must be 0 or 1");
    if (o->fft_tile != 0 && o->fft_tile != 1) return fail(ctx, FS_EINVAL, "fft_tile must be 0 or 1");
    if ((o->forward_single_pass != 0 && o->forward_single_pass != 1) ||
        (o->inverse_single_pass != 0 && o->inverse_single_pass != 1) || (o->fp64_sums != 0 && o->fp64_sums != 1))
      return fail(ctx, FS_EINVAL, "forward_single_pass, inverse_single_pass and fp64_sums must be 0 or 1");
    if (o->regularizer != 0 && o->regularizer != 1) return fail(ctx, FS_EINVAL, "regularizer must be 0 or 1");
    if (o->regularizer == 1 && o->solve_form != 1)
      return fail(ctx, FS_EUNSUPPORTED, "the truncated SVD is implemented in the rank-one form (solve_form 1)");
    if (o->regularizer == 1 && o->alpha_mode != 0)
      return fail(ctx, FS_EINVAL, "the truncated SVD takes no alpha (alpha_mode must be 0)");
    if (dense_solve && prec == FS_MIXED && o->alpha_mode == 0 && o->regularizer == 0 &&
        !(delta >= FS_MIXED_MIN_NOISE || o->delta_floor >= FS_MIXED_MIN_NOISE))
      return fail(ctx, FS_EUNSUPPORTED,
                  "the mixed path transforms W in FP32: its discrepancy test resolves noise levels down to %g "
                  "(delta=%g, delta_floor=%g); take FS_FP64",
                  FS_MIXED_MIN_NOISE, delta, o->delta_floor);
    if (o->kernel_plan) {
      if (!kernel_plan_matches(o->kernel_plan, g, prec, omega, n_omega, c0))
        return fail(ctx, FS_EINVAL, "the kernel plan was made for another geometry, precision, frequency list or c0");
      if (o->solve_form != 0)
        return fail(ctx, FS_EUNSUPPORTED, "the sampled-G kernel is solved by the dense form only (solve_form 0)");
    }
  }
  return FS_OK;
}

Problem make_problem(const fs_geometry* g, int n_omega, const double* omega, double delta, double c0,
                     const fs_options& o) {
  Problem P;
  memset(&P, 0, sizeof(P));
  P.n = g->n; P.m = g->m; P.m1 = g->m1; P.n_omega = n_omega;
  P.alpha_mode = o.alpha_mode; P.max_iter = o.max_iter; P.refine_iters = o.refine_iters;
  P.period = g->period; P.z1 = g->z1; P.hz = (g->z2 - g->z1) / g->m; P.c0 = c0;
  P.delta = delta; P.tau = o.tau; P.delta_floor = o.delta_floor; P.alpha_rel = o.alpha_rel; P.eps_u = o.eps_u;
  P.fp64_switch = o.fp64_switch;
  P.solve_bps = o.solve_blocks_per_sm;
  P.solve_form = o.solve_form;
  P.regularizer = o.regularizer;
  P.sampled = o.kernel_plan ? 1 : 0;
  P.incident = o.incident ? 1 : 0;
  P.classify_single = o.classify_single_pass;
  P.fft_tile = o.fft_tile;
  P.forward_single = o.forward_single_pass;
  P.inverse_single = o.inverse_single_pass;
  P.sums64 = o.fp64_sums;
  for (int k = 0; k < g->m1; ++k) P.zy[k] = g->zy[k];
  P.zy_min = g->zy[0];
  for (int k = 1; k < g->m1; ++k) P.zy_min = fmin(P.zy_min, g->zy[k]);
  for (int j = 0; j < n_omega; ++j) {
    P.omega[j] = omega[j];
    P.alpha_given[j] = (o.alpha_mode == 1) ? o.alpha_given[j] : 0.0;
    // |m|^2 = (k0 L / 2 pi)^2 within a relative 1e-9 (k_z = 0: excluded modes); the
    // sampled kernel is finite there and excludes nothing (an empty window)
    const double sL = omega[j] / c0 * g->period / (2.0 * M_PI);
    const double s2 = sL * sL;
    const double lo = ceil(s2 - 1e-9 * s2), hi = floor(s2 + 1e-9 * s2);
    P.graz_lo[j] = lo > 1e9 ? 1000000001 : (int)lo;  // |m|^2 <= 2 (N/2)^2 never reaches 1e9
    P.graz_hi[j] = hi > 1e9 ? 1000000000 : (int)hi;
    if (P.sampled) {
      P.graz_lo[j] = 1;
      P.graz_hi[j] = 0;
    }
  }
  derive_constants(P);
  return P;
}

template <typename R>
Work<R> carve_work(void* base, const Layout& L, unsigned long long* ctr, const cx<R>* tw, double* alpha_out) {
  char* b = (char*)base;
  Work<R> w;
  w.wt = (cx<R>*)(b + L.t12);
  w.t2 = (cx<R>*)(b + L.t12);
  w.prof = (cx<R>*)(b + L.prof);
  w.norms = (double*)(b + L.norms);
  w.partial = (double*)(b + L.partial);
  w.n_partial = L.n_partial;
  w.slot = (int*)(b + L.slot);
  w.act = (int*)(b + L.act);
  w.flagbits = (unsigned*)(b + L.flagbits);
  w.blkcnt = (int*)(b + L.blkcnt);
  w.blkgz = (int*)(b + L.blkgz);
  w.colblk = (unsigned*)(b + L.colblk);
  w.cols = (int*)(b + L.cols);
  w.ncol = (int*)(b + L.ncol);
  w.count = (int*)(b + L.count);
  w.dnu = (double*)(b + L.dnu);
  w.bar = (unsigned*)(b + L.bar);
  w.ctr = ctr;
  w.tw = tw;
  w.alpha_out = alpha_out;
  w.wt64 = nullptr;
  w.tw64 = nullptr;
  w.ktab = nullptr;
  w.ktr = nullptr;
  w.u0 = nullptr;
  return w;
}

template Work<double> carve_work<double>(void*, const Layout&, unsigned long long*, const double2*, double*);
template Work<float> carve_work<float>(void*, const Layout&, unsigned long long*, const float2*, double*);

template <typename R>
cudaError_t launch_pipeline(const Problem& P, const Work<R>& w, const void* W, void* xi, void* c, cudaStream_t s,
                            cudaEvent_t* ev, const char** stage) {
  cudaError_t e;
  // the single-pass classification computes the norms itself; the mixed truncated-SVD
  // route (W~ in FP64) keeps the separate norms kernel
  const bool fused = w.wt64 == nullptr && classify_fused_ok(P);
  if (ev) cudaEventRecord(ev[0], s);
  *stage = "fft2_forward";
  if ((e = launch_fft2_forward<R>((const cx<R>*)W, P, w, s, ev ? ev[1] : nullptr, !fused)) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[2], s);
  *stage = "classify";
  if (fused) {
    e = launch_classify_fused<R>(P, w, s);
    if (e != cudaSuccess) {  // not co-resident on this device: norms, then the two-kernel classification
      cudaGetLastError();
      if ((e = launch_mode_norms<R>(P, w, s)) != cudaSuccess) return e;
      e = launch_classify<R>(P, w, s);
    }
  } else {
    e = launch_classify<R>(P, w, s);
  }
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[3], s);
  *stage = "solve";
  if (P.solve_form == 1) e = launch_solve_rank1<R>(P, w, s);
  else if (sizeof(R) == 8) e = launch_solve_fp64(P, *(const Work<double>*)&w, s);
  else e = launch_solve_mixed(P, *(const Work<float>*)&w, s);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[4], s);
  *stage = "recover";
  if ((e = launch_recover<R>(P, w, (R*)xi, (R*)c, s, ev ? ev[5] : nullptr)) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[6], s);
  return cudaSuccess;
}
template cudaError_t launch_pipeline<double>(const Problem&, const Work<double>&, const void*, void*, void*,
                                             cudaStream_t, cudaEvent_t*, const char**);
template cudaError_t launch_pipeline<float>(const Problem&, const Work<float>&, const void*, void*, void*,
                                            cudaStream_t, cudaEvent_t*, const char**);

int sm_count() {
  static std::atomic<int> cache[MAX_DEVICES];
  int dev = 0;
  cudaGetDevice(&dev);
  int v = (dev >= 0 && dev < MAX_DEVICES) ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (v <= 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 152;
    }
    if (dev >= 0 && dev < MAX_DEVICES) cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

cudaError_t opt_in_smem(SmemOptIn& flag, const void* kernel, size_t bytes, bool max_shared) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < MAX_DEVICES) ? 1ull << dev : 0ull;
  if (bit && (flag.done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && max_shared)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess && bit) flag.done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

}  // namespace fl

namespace {

fs_status ensure_workspace(fs_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return FS_OK;
  // a growth frees the workspace a graph being captured (or captured before) refers
  // to: refused during a capture, counted otherwise (fs_workspace_generation)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return fail(ctx, FS_EUNSUPPORTED,
                "the workspace must grow to %lld bytes during a stream capture: size it first (fs_reserve, or "
                "an uncaptured call on the largest problem)",
                (long long)bytes);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  e = cudaMalloc(&ctx->ws, bytes);
  if (e != cudaSuccess) {
    ctx->ws = nullptr;
    return fail(ctx, FS_ENOMEM, "workspace allocation of %lld bytes failed", (long long)bytes);
  }
  ctx->ws_bytes = bytes;
  ++ctx->ws_generation;
  return FS_OK;
}

template <typename R>
fs_status ensure_twiddles(fs_ctx* ctx, int n, const cx<R>** out) {
  const int fp = sizeof(R) == 8 ? 1 : 0;
  const int si = size_index(n);
  if (!ctx->tw[fp][si]) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      return fail(ctx, FS_EUNSUPPORTED,
                  "the twiddle table of N=%d must be made during a stream capture: make it first (fs_reserve, or "
                  "an uncaptured call of that size)", n);
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(cx<R>) * n) != cudaSuccess) return fail(ctx, FS_ENOMEM, "twiddle table");
    cudaError_t e = launch_twiddles<R>((cx<R>*)p, n, ctx->stream);
    // complete before any transform: those read the table before their programmatic
    // dependency wait
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { cudaFree(p); return cuda_fail(ctx, e, "twiddles"); }
    ctx->tw[fp][si] = p;
  }
  *out = (const cx<R>*)ctx->tw[fp][si];
  return FS_OK;
}

// Enqueue the pipeline of one problem on `s` with workspace `base` (counters are
// not reset here).  Twiddles for P.n must exist.
template <typename R>
fs_status run_on(fs_ctx* ctx, const Problem& P, const Layout& L, void* base, cudaStream_t s, const void* W,
                 void* xi, void* c, double* alpha_out, cudaEvent_t* ev, const fs_kernel_plan* kp = nullptr,
                 const void* u0 = nullptr) {
  const cx<R>* tw = (const cx<R>*)ctx->tw[sizeof(R) == 8 ? 1 : 0][size_index(P.n)];
  Work<R> w = carve_work<R>(base, L, ctx->ctr, tw, alpha_out);
  if (wide_route(P, sizeof(R) == 8)) {
    w.wt64 = (double2*)((char*)base + L.t12);
    w.tw64 = (const double2*)ctx->tw[1][size_index(P.n)];
  }
  if (kp) kernel_plan_tables(kp, &w.ktab, &w.ktr);
  if (P.incident) w.u0 = (const cx<R>*)u0;
  const char* stage = "";
  const cudaError_t e = launch_pipeline<R>(P, w, W, xi, c, s, ev, &stage);
  return e == cudaSuccess ? FS_OK : cuda_fail(ctx, e, stage);
}

template <typename R>
fs_status run(fs_ctx* ctx, const Problem& P, const Layout& L, const void* W, void* xi, void* c,
              double* alpha_out, bool timed, const fs_kernel_plan* kp, const void* u0) {
  const cx<R>* tw = nullptr;
  fs_status st = ensure_twiddles<R>(ctx, P.n, &tw);
  if (st != FS_OK) return st;
  if (wide_route(P, sizeof(R) == 8)) {
    const double2* tw64 = nullptr;
    if ((st = ensure_twiddles<double>(ctx, P.n, &tw64)) != FS_OK) return st;
  }
  cudaError_t e = cudaMemsetAsync(ctx->ctr, 0, sizeof(unsigned long long) * C_COUNT, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync");
  ctx->timed = timed;
  return run_on<R>(ctx, P, L, ctx->ws, ctx->stream, W, xi, c, alpha_out, timed ? ctx->ev : nullptr, kp, u0);
}

}  // namespace

extern "C" {

const char* fs_version(void) { return "flatlayer-gb300 0.1 (sm_103a)"; }

fs_status fs_default_options(fs_options* o) {
  if (!o) return FS_EINVAL;
  o->tau = 2.0;
  o->delta_floor = 1e-5;
  o->alpha_rel = 1e-6;
  o->eps_u = 1e-8;
  o->alpha_mode = 0;
  o->alpha_given = nullptr;
  o->max_iter = 100;
  o->refine_iters = 8;
  o->fp64_switch = 1e-4;
  o->stage_timing = 0;
  o->solve_blocks_per_sm = 2;
  o->solve_form = 0;
  o->regularizer = 0;
  o->kernel_plan = nullptr;
  o->incident = nullptr;
  o->classify_single_pass = 0;
  o->fft_tile = 0;
  o->forward_single_pass = 1;
  o->inverse_single_pass = 0;
  o->fp64_sums = 0;
  return FS_OK;
}

fs_status fs_create(fs_ctx** out, int device, void* stream) {
  if (!out) return FS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FS_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return FS_ECUDA;
  fs_ctx* ctx = new (std::nothrow) fs_ctx();
  if (!ctx) return FS_ENOMEM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  if (cudaMalloc(&ctx->ctr, sizeof(unsigned long long) * C_COUNT) != cudaSuccess) {
    delete ctx;
    return FS_ENOMEM;
  }
  if (cudaMallocHost(&ctx->ctr_host, sizeof(unsigned long long) * C_COUNT) != cudaSuccess) {
    cudaFree(ctx->ctr);
    delete ctx;
    return FS_ENOMEM;
  }
  memset(ctx->ctr_host, 0, sizeof(unsigned long long) * C_COUNT);
  for (auto& e : ctx->ev) cudaEventCreate(&e);
  cudaMemsetAsync(ctx->ctr, 0, sizeof(unsigned long long) * C_COUNT, ctx->stream);
  *out = ctx;
  return FS_OK;
}

void fs_destroy(fs_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->host_exec) cudaGraphExecDestroy(ctx->host_exec);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->stage) cudaFree(ctx->stage);
  for (auto& a : ctx->tw)
    for (void* p : a)
      if (p) cudaFree(p);
  if (ctx->ctr) cudaFree(ctx->ctr);
  if (ctx->ctr_host) cudaFreeHost(ctx->ctr_host);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (int k = 0; k < fs_ctx::MAX_SIDE; ++k) {
    if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
    if (ctx->join_ev[k]) cudaEventDestroy(ctx->join_ev[k]);
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  delete ctx;
}

const char* fs_last_error(const fs_ctx* ctx) { return ctx ? ctx->err : "null context"; }

fs_status fs_workspace_size(const fs_geometry* g, int n_omega, fs_precision prec, size_t* bytes) {
  if (!g || !bytes || n_omega <= 0 || g->n <= 0 || g->m <= 0 || g->m1 <= 0) return FS_EINVAL;
  *bytes = layout(g->n, g->m, g->m1, n_omega, prec == FS_FP64).total;
  return FS_OK;
}

extern "C" fs_status fs_reserve(fs_ctx* ctx, const fs_geometry* g, int n_omega, fs_precision prec) {
  if (!ctx) return FS_EINVAL;
  if (!g || g->n <= 0 || g->m <= 0 || g->m1 <= 0 || n_omega <= 0 || (prec != FS_FP64 && prec != FS_MIXED))
    return fail(ctx, FS_EINVAL, "fs_reserve: geometry, n_omega or precision out of range");
  if (!fft_size_supported(g->n) || g->m > MAX_M || g->m1 > MAX_M1 || n_omega > MAX_OMEGA)
    return fail(ctx, FS_EUNSUPPORTED, "fs_reserve: N=%d, M=%d, M1=%d, n_omega=%d beyond this build's limits", g->n,
                g->m, g->m1, n_omega);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  fs_status st = ensure_workspace(ctx, layout(g->n, g->m, g->m1, n_omega, prec == FS_FP64).total);
  // the twiddle tables of N in both real types (FP64 also serves the mixed truncated-SVD route)
  const double2* t64;
  const float2* t32;
  if (st == FS_OK) st = ensure_twiddles<double>(ctx, g->n, &t64);
  if (st == FS_OK) st = ensure_twiddles<float>(ctx, g->n, &t32);
  if (st == FS_OK && (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "sync");
  return st;
}

extern "C" unsigned long long fs_workspace_generation(const fs_ctx* ctx) { return ctx ? ctx->ws_generation : 0; }

fs_status fs_reconstruct(fs_ctx* ctx, const fs_geometry* g, fs_precision prec, const void* W, const double* omega,
                         int n_omega, double delta, double c0, const fs_options* opts, void* xi, void* c,
                         double* alpha_out) {
  if (!ctx) return FS_EINVAL;
  fs_status st = validate_args(ctx, g, prec, n_omega, omega, delta, c0, opts);
  if (st != FS_OK) return st;
  if (!W || !xi) return fail(ctx, FS_EINVAL, "W and xi must be device pointers");
  fs_options o;
  fs_default_options(&o);
  if (opts) o = *opts;
  if (!elems_aligned(prec == FS_FP64, W, xi, c, o.incident) || ((uintptr_t)alpha_out % 8) != 0)
    return fail(ctx, FS_EINVAL, "W, xi, c, alpha_out and the incident field must be aligned to their elements");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  const bool fp64 = prec == FS_FP64;
  const Layout L = layout(g->n, g->m, g->m1, n_omega, fp64);
  if ((st = ensure_workspace(ctx, L.total)) != FS_OK) return st;
  const Problem P = make_problem(g, n_omega, omega, delta, c0, o);
  const bool timed = o.stage_timing != 0;
  if (o.kernel_plan && kernel_plan_device(o.kernel_plan) != ctx->device)
    return fail(ctx, FS_EINVAL, "the kernel plan lives on another device");
  return fp64 ? run<double>(ctx, P, L, W, xi, c, alpha_out, timed, o.kernel_plan, o.incident)
              : run<float>(ctx, P, L, W, xi, c, alpha_out, timed, o.kernel_plan, o.incident);
}

fs_status fs_reconstruct_host(fs_ctx* ctx, const fs_geometry* g, fs_precision prec, const void* W_host,
                              const double* omega, int n_omega, double delta, double c0, const fs_options* opts,
                              void* xi_host, void* c_host) {
  if (!ctx) return FS_EINVAL;
  fs_status st = validate_args(ctx, g, prec, n_omega, omega, delta, c0, opts);
  if (st != FS_OK) return st;
  if (!W_host || !xi_host) return fail(ctx, FS_EINVAL, "W_host and xi_host must be non-NULL");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  const size_t cxs = prec == FS_FP64 ? 16 : 8, rs = cxs / 2;
  const size_t N2 = (size_t)g->n * g->n;
  const size_t wbytes = cxs * (size_t)n_omega * g->m1 * N2;
  const size_t obytes = rs * (size_t)g->m * N2;
  fs_options o;
  fs_default_options(&o);
  if (opts) o = *opts;
  const bool graphable = o.stage_timing == 0 && pinned(W_host) && pinned(xi_host) && (!c_host || pinned(c_host));
  // mapped, aligned page-locked buffers: the kernels read W and write xi and c in host
  // memory themselves (no staging buffers, no copies)
  const bool direct = graphable && mapped_here(W_host) && mapped_here(xi_host) && (!c_host || mapped_here(c_host)) &&
                      elems_aligned(prec == FS_FP64, W_host, xi_host, c_host);
  const size_t need = direct ? 0 : align_up(wbytes) + 2 * align_up(obytes);
  if (need > ctx->stage_bytes) {
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "sync");
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    if (cudaMalloc(&ctx->stage, need) != cudaSuccess) return fail(ctx, FS_ENOMEM, "staging buffers");
    ctx->stage_bytes = need;
  }
  char* dW = (char*)ctx->stage;
  char* dxi = dW + align_up(wbytes);
  char* dc = dxi + align_up(obytes);
  // A repeated call (same key: every argument that shapes the work, the host and
  // device buffers) replays the graph captured after its first run: one launch
  // instead of the copies and eight kernel launches.  Only with page-locked host
  // buffers (copies from pageable memory cannot be captured) and without stage timing.
  std::vector<unsigned char> key;
  if (graphable) {
    // values only (no struct padding, no pointers to argument arrays)
    const int ints[16] = {g->n, g->m, g->m1, n_omega, (int)prec, o.alpha_mode, o.max_iter, o.refine_iters,
                          o.solve_blocks_per_sm, o.solve_form, o.regularizer, o.classify_single_pass, o.fft_tile,
                          o.forward_single_pass, o.inverse_single_pass, o.fp64_sums};
    const double dbl[10] = {g->period, g->z1, g->z2, delta, c0, o.tau, o.delta_floor, o.alpha_rel, o.eps_u,
                            o.fp64_switch};
    key_put(key, ints);
    key_put(key, dbl);
    key.insert(key.end(), (const unsigned char*)g->zy, (const unsigned char*)(g->zy + g->m1));
    key.insert(key.end(), (const unsigned char*)omega, (const unsigned char*)(omega + n_omega));
    if (o.alpha_mode == 1)
      key.insert(key.end(), (const unsigned char*)o.alpha_given, (const unsigned char*)(o.alpha_given + n_omega));
    const void* ptrs[8] = {W_host, xi_host, c_host, ctx->stage, ctx->ws, ctx->stream, o.kernel_plan, o.incident};
    key_put(key, ptrs);
    if (ctx->host_exec && key == ctx->host_key) {
      if ((e = cudaGraphLaunch(ctx->host_exec, ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
      if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "sync");
      return FS_OK;
    }
  }
  auto enqueue = [&]() -> fs_status {
    if (direct) return fs_reconstruct(ctx, g, prec, W_host, omega, n_omega, delta, c0, opts, xi_host, c_host, nullptr);
    cudaError_t e2;
    if ((e2 = cudaMemcpyAsync(dW, W_host, wbytes, cudaMemcpyHostToDevice, ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e2, "H2D W");
    fs_status s2 = fs_reconstruct(ctx, g, prec, dW, omega, n_omega, delta, c0, opts, dxi, c_host ? dc : nullptr, nullptr);
    if (s2 != FS_OK) return s2;
    if ((e2 = cudaMemcpyAsync(xi_host, dxi, obytes, cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e2, "D2H xi");
    if (c_host && (e2 = cudaMemcpyAsync(c_host, dc, obytes, cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e2, "D2H c");
    return FS_OK;
  };
  if ((st = enqueue()) != FS_OK) return st;
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "sync");
  if (graphable) {
    // the run above sized the workspace and twiddles, so the capture allocates
    // nothing; the key is taken again in case the workspace moved
    const void* ptrs[8] = {W_host, xi_host, c_host, ctx->stage, ctx->ws, ctx->stream, o.kernel_plan, o.incident};
    key.resize(key.size() - sizeof(ptrs));
    key_put(key, ptrs);
    if (ctx->host_exec) {
      cudaGraphExecDestroy(ctx->host_exec);
      ctx->host_exec = nullptr;
      ctx->host_key.clear();
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const fs_status cap = enqueue();
      const cudaError_t end = cudaStreamEndCapture(ctx->stream, &graph);
      if (cap == FS_OK && end == cudaSuccess && graph &&
          cudaGraphInstantiate(&ctx->host_exec, graph, 0) == cudaSuccess) {
        ctx->host_key = key;
      } else {
        ctx->host_exec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();  // a failed capture leaves the uncaptured path in use
  }
  return FS_OK;
}

fs_status fs_reconstruct_batch(fs_ctx* ctx, const fs_problem* probs, int n_probs, fs_precision prec,
                               const fs_options* opts, int n_streams) {
  if (!ctx) return FS_EINVAL;
  if (!probs || n_probs <= 0) return fail(ctx, FS_EINVAL, "empty batch");
  if (n_streams < 1 || n_streams > fs_ctx::MAX_SIDE)
    return fail(ctx, FS_EINVAL, "n_streams must be in [1, %d]", fs_ctx::MAX_SIDE);
  fs_options o;
  fs_default_options(&o);
  if (opts) o = *opts;
  if (o.kernel_plan) return fail(ctx, FS_EUNSUPPORTED, "batches take the Weyl kernel only (kernel_plan must be NULL)");
  if (o.incident) return fail(ctx, FS_EUNSUPPORTED, "batches take the plane incident wave only (incident must be NULL)");
  const bool fp64 = prec == FS_FP64;
  size_t total = 0;
  for (int i = 0; i < n_probs; ++i) {
    const fs_problem& q = probs[i];
    fs_status st = validate_args(ctx, &q.geom, prec, q.n_omega, q.omega, q.delta, q.c0, opts);
    if (st != FS_OK) {
      char m[256];
      snprintf(m, sizeof(m), "%s", ctx->err);
      return fail(ctx, st, "problem %d: %s", i, m);
    }
    if (!q.W || !q.xi) return fail(ctx, FS_EINVAL, "problem %d: W and xi must be device pointers", i);
    if (!elems_aligned(prec == FS_FP64, q.W, q.xi, q.c))
      return fail(ctx, FS_EINVAL, "problem %d: W, xi and c must be aligned to their elements", i);
    total += align_up(layout(q.geom.n, q.geom.m, q.geom.m1, q.n_omega, fp64).total);
  }
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  fs_status st = ensure_workspace(ctx, total);
  if (st != FS_OK) return st;
  for (int i = 0; i < n_probs; ++i) {
    const double2* t64;
    const float2* t32;
    if (fp64 || o.regularizer == 1) st = ensure_twiddles<double>(ctx, probs[i].geom.n, &t64);
    if (st == FS_OK && !fp64) st = ensure_twiddles<float>(ctx, probs[i].geom.n, &t32);
    if (st != FS_OK) return st;
  }
  if (!ctx->fork_ev) {
    if (cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) != cudaSuccess) return FS_ECUDA;
    for (int k = 0; k < fs_ctx::MAX_SIDE; ++k)
      if (cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ctx->join_ev[k], cudaEventDisableTiming) != cudaSuccess)
        return fail(ctx, FS_ECUDA, "side streams");
  }
  if ((e = cudaMemsetAsync(ctx->ctr, 0, sizeof(unsigned long long) * C_COUNT, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "cudaMemsetAsync");
  ctx->timed = false;
  // largest problems first, dealt round-robin over the side streams
  int* order = new (std::nothrow) int[n_probs];
  size_t* off = new (std::nothrow) size_t[n_probs];
  if (!order || !off) { delete[] order; delete[] off; return FS_ENOMEM; }
  size_t acc = 0;
  for (int i = 0; i < n_probs; ++i) {
    order[i] = i;
    off[i] = acc;
    acc += align_up(layout(probs[i].geom.n, probs[i].geom.m, probs[i].geom.m1, probs[i].n_omega, fp64).total);
  }
  auto work = [&](int i) {
    const fs_problem& q = probs[i];
    return (double)q.n_omega * q.geom.n * q.geom.n * (q.geom.m + q.geom.m1);
  };
  for (int i = 1; i < n_probs; ++i)  // insertion sort, stable, by decreasing work
    for (int j = i; j > 0 && work(order[j]) > work(order[j - 1]); --j) {
      const int t = order[j]; order[j] = order[j - 1]; order[j - 1] = t;
    }
  const int S = n_streams < n_probs ? n_streams : n_probs;
  cudaEventRecord(ctx->fork_ev, ctx->stream);
  for (int k = 0; k < S; ++k) cudaStreamWaitEvent(ctx->side[k], ctx->fork_ev, 0);
  for (int r = 0; r < n_probs && st == FS_OK; ++r) {
    const int i = order[r];
    const fs_problem& q = probs[i];
    const Layout L = layout(q.geom.n, q.geom.m, q.geom.m1, q.n_omega, fp64);
    const Problem P = make_problem(&q.geom, q.n_omega, q.omega, q.delta, q.c0, o);
    char* base = (char*)ctx->ws + off[i];
    cudaStream_t s = ctx->side[r % S];
    st = fp64 ? run_on<double>(ctx, P, L, base, s, q.W, q.xi, q.c, nullptr, nullptr)
              : run_on<float>(ctx, P, L, base, s, q.W, q.xi, q.c, nullptr, nullptr);
  }
  for (int k = 0; k < S; ++k) {
    cudaEventRecord(ctx->join_ev[k], ctx->side[k]);
    cudaStreamWaitEvent(ctx->stream, ctx->join_ev[k], 0);
  }
  delete[] order;
  delete[] off;
  return st;
}

fs_status fs_forward_born(fs_ctx* ctx, const fs_geometry* g, fs_precision prec, const void* xi,
                          const void* incident, const double* omega, int n_omega, double c0, void* W) {
  if (!ctx) return FS_EINVAL;
  fs_status st = validate_args(ctx, g, prec, n_omega, omega, 0.0, c0, nullptr, false);
  if (st != FS_OK) return st;
  if (!xi || !W) return fail(ctx, FS_EINVAL, "xi and W must be device pointers");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  const bool fp64 = prec == FS_FP64;
  const size_t need = (fp64 ? 16 : 8) * (size_t)n_omega * g->m * g->n * g->n;
  if ((st = ensure_workspace(ctx, need)) != FS_OK) return st;
  fs_options o;
  fs_default_options(&o);
  const Problem P = make_problem(g, n_omega, omega, 0.0, c0, o);
  if (fp64) {
    const double2* tw = nullptr;
    if ((st = ensure_twiddles<double>(ctx, g->n, &tw)) != FS_OK) return st;
    e = launch_forward_born<double>(P, (const double*)xi, (const double2*)incident, (double2*)ctx->ws, (double2*)W, tw,
                                    ctx->stream);
  } else {
    const float2* tw = nullptr;
    if ((st = ensure_twiddles<float>(ctx, g->n, &tw)) != FS_OK) return st;
    e = launch_forward_born<float>(P, (const float*)xi, (const float2*)incident, (float2*)ctx->ws, (float2*)W, tw,
                                   ctx->stream);
  }
  return e == cudaSuccess ? FS_OK : cuda_fail(ctx, e, "forward_born");
}

fs_status fs_forward(fs_ctx* ctx, const fs_geometry* g, fs_precision prec, const void* xi, const void* incident,
                     const double* omega, int n_omega, double c0, fs_forward_method method, int max_iter, double rtol,
                     void* W, void* u, int* iterations) {
  if (!ctx) return FS_EINVAL;
  fs_status st = validate_args(ctx, g, prec, n_omega, omega, 0.0, c0, nullptr, false);
  if (st != FS_OK) return st;
  if (!xi || !W) return fail(ctx, FS_EINVAL, "xi and W must be device pointers");
  if (max_iter < 0) return fail(ctx, FS_EINVAL, "max_iter must be >= 0");
  if (method < FS_FIXED_POINT || method > FS_FIXED_POINT_GMRES) return fail(ctx, FS_EINVAL, "unknown forward method");
  if (!(rtol > 0.0)) return fail(ctx, FS_EINVAL, "rtol must be > 0");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  fs_options o;
  fs_default_options(&o);
  const Problem P = make_problem(g, n_omega, omega, 0.0, c0, o);
  const bool fp64 = prec == FS_FP64;
  const size_t need = fp64 ? forward_bytes<double>(P) : forward_bytes<float>(P);
  if ((st = ensure_workspace(ctx, need)) != FS_OK) return st;
  std::vector<int> it(n_omega, 0), conv(n_omega, 0);
  if (fp64) {
    const double2* tw = nullptr;
    if ((st = ensure_twiddles<double>(ctx, g->n, &tw)) != FS_OK) return st;
    e = forward_solve<double>(P, (const double*)xi, (const double2*)incident, (double2*)W, (double2*)u, ctx->ws,
                              (int)method, rtol, max_iter, tw, ctx->stream, it.data(), conv.data());
  } else {
    const float2* tw = nullptr;
    if ((st = ensure_twiddles<float>(ctx, g->n, &tw)) != FS_OK) return st;
    e = forward_solve<float>(P, (const float*)xi, (const float2*)incident, (float2*)W, (float2*)u, ctx->ws,
                             (int)method, rtol, max_iter, tw, ctx->stream, it.data(), conv.data());
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "forward");
  if (iterations)
    for (int j = 0; j < n_omega; ++j) iterations[j] = it[j];
  for (int j = 0; j < n_omega; ++j)
    if (!conv[j])
      return fail(ctx, FS_ENOCONV, "the forward solve did not converge for omega[%d] after %d iterations", j, it[j]);
  return FS_OK;
}

fs_status fs_incident_point_sources(fs_ctx* ctx, const fs_geometry* g, fs_precision prec, const double* sources,
                                    int n_sources, const double* omega, int n_omega, double c0, void* u0) {
  if (!ctx) return FS_EINVAL;
  fs_status st = validate_args(ctx, g, prec, n_omega, omega, 0.0, c0, nullptr, false);
  if (st != FS_OK) return st;
  if (!u0) return fail(ctx, FS_EINVAL, "u0 must be a device pointer");
  if (n_sources < 1 || !sources) return fail(ctx, FS_EINVAL, "at least one source is needed");
  std::vector<double> spec(4 * (size_t)n_sources);
  for (int j = 0; j < n_sources; ++j) {
    for (int c = 0; c < 4; ++c) spec[4 * j + c] = sources[4 * j + c];
    if (!std::isfinite(spec[4 * j]) || !std::isfinite(spec[4 * j + 1]) || !std::isfinite(spec[4 * j + 3]))
      return fail(ctx, FS_EINVAL, "source %d is not finite", j);
    if (!(spec[4 * j + 2] > g->z2)) return fail(ctx, FS_EINVAL, "source %d is not above X", j);
  }
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  const size_t need = align_up(32 * (size_t)n_sources);
  if ((st = ensure_workspace(ctx, need)) != FS_OK) return st;
  if ((e = cudaMemcpyAsync(ctx->ws, spec.data(), 32 * (size_t)n_sources, cudaMemcpyHostToDevice, ctx->stream)) !=
      cudaSuccess)
    return cuda_fail(ctx, e, "source copy");
  fs_options o;
  fs_default_options(&o);
  const Problem P = make_problem(g, n_omega, omega, 0.0, c0, o);
  if (prec == FS_FP64) {
    const double2* tw = nullptr;
    if ((st = ensure_twiddles<double>(ctx, g->n, &tw)) != FS_OK) return st;
    e = launch_point_sources<double>(P, (const double*)ctx->ws, n_sources, (double2*)u0, tw, ctx->stream);
  } else {
    const float2* tw = nullptr;
    if ((st = ensure_twiddles<float>(ctx, g->n, &tw)) != FS_OK) return st;
    e = launch_point_sources<float>(P, (const double*)ctx->ws, n_sources, (float2*)u0, tw, ctx->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // the host copy of spec must outlive it
  return e == cudaSuccess ? FS_OK : cuda_fail(ctx, e, "point sources");
}

fs_status fs_get_report(fs_ctx* ctx, fs_report* r) {
  if (!ctx || !r) return FS_EINVAL;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->ctr_host, ctx->ctr, sizeof(unsigned long long) * C_COUNT, cudaMemcpyDeviceToHost,
                        ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fs_get_report");
  const unsigned long long* h = ctx->ctr_host;
  r->n_modes = (long long)h[C_MODES];
  r->n_active = (long long)h[C_ACTIVE];
  r->n_zeroed = (long long)h[C_ZEROED];
  r->n_grazing = (long long)h[C_GRAZING];
  r->n_alpha_floor = (long long)h[C_ALPHA_FLOOR];
  r->n_root_capped = (long long)h[C_ROOT_CAPPED];
  r->n_u_guard = (long long)h[C_U_GUARD];
  r->n_nan_c = (long long)h[C_NAN_C];
  r->n_fp64_fallback = (long long)h[C_FP64_FALLBACK];
  r->n_refine_iters = (long long)h[C_REFINE_ITERS];
  r->n_columns = (long long)h[C_COLUMNS];
  r->n_nonfinite = (long long)h[C_NONFINITE];
  r->n_timeouts = (long long)h[C_TIMEOUT];
  for (int i = 0; i < 6; ++i) {
    float ms = 0.f;
    if (ctx->timed && cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]) != cudaSuccess) ms = 0.f;
    r->ms_stage[i] = ms;
  }
  return FS_OK;
}

fs_status fs_sync_status(fs_ctx* ctx) {
  if (!ctx) return FS_EINVAL;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->ctr_host, ctx->ctr, sizeof(unsigned long long) * C_COUNT, cudaMemcpyDeviceToHost,
                        ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fs_sync_status");
  const unsigned long long to = ctx->ctr_host[C_TIMEOUT];
  if (to) return fail(ctx, FS_ETIMEOUT, "%llu device-side waits ran out (results unspecified)", to);
  const unsigned long long nf = ctx->ctr_host[C_NONFINITE];
  if (nf) return fail(ctx, FS_ENONFINITE, "%llu non-finite values (modes of W~ or voxels of xi)", nf);
  return FS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// derivatives at fixed alpha (include/flatlayer_diff.h)
// ---------------------------------------------------------------------------
struct fs_diff_plan {
  fs_ctx* ctx = nullptr;
  Problem P;
  bool fp64 = true;
  int gb = 1;              // blocks per frequency of the per-mode kernels
  size_t P1 = 0;           // packed lower-triangle entries per mode
  void* buf = nullptr;     // normal matrices, then the twiddle table
  double2* gram = nullptr;
  void* tw = nullptr;
};

namespace {

struct TapeLayout {
  size_t L, y, Vx, ux, xi, la, total;
};
struct ScratchLayout {
  size_t min, mout, xsp, partial, total;
  int nd;
};

TapeLayout tape_layout(const fs_diff_plan* p) {
  const Problem& P = p->P;
  const size_t cxs = p->fp64 ? 16 : 8, rs = cxs / 2;
  const size_t N2 = (size_t)P.n * P.n, F = P.n_omega;
  TapeLayout T;
  size_t off = 0;
  T.L = off; off = align_up(off + 16 * F * N2 * p->P1);
  T.y = off; off = align_up(off + 16 * F * N2 * P.m1);
  T.Vx = off; off = align_up(off + cxs * F * P.m * N2);
  T.ux = off; off = align_up(off + cxs * F * P.m * N2);
  T.xi = off; off = align_up(off + rs * P.m * N2);
  T.la = off; off = align_up(off + 8 * F);
  T.total = off;
  return T;
}

ScratchLayout scratch_layout(const fs_diff_plan* p, int n_dir) {
  const Problem& P = p->P;
  const size_t cxs = p->fp64 ? 16 : 8;
  const size_t N2 = (size_t)P.n * P.n, F = P.n_omega;
  ScratchLayout S;
  S.nd = n_dir < 1 ? 1 : (n_dir > JVP_CHUNK ? JVP_CHUNK : n_dir);
  const size_t nd = S.nd;
  size_t off = 0;
  S.min = off; off = align_up(off + cxs * nd * F * P.m1 * N2);
  S.mout = off; off = align_up(off + cxs * 2 * nd * F * P.m * N2);
  S.xsp = off; off = align_up(off + cxs * 2 * nd * F * P.m * N2);
  S.partial = off; off = align_up(off + 8 * nd * F * (size_t)p->gb);
  S.total = off;
  return S;
}

bool aligned256(const void* p) { return ((uintptr_t)p & 255) == 0; }

template <typename R>
fs_status diff_forward(fs_diff_plan* p, char* tape, char* scr, const void* W, const double* log_alpha, void* xi,
                       void* c, double* phi) {
  fs_ctx* ctx = p->ctx;
  const Problem& P = p->P;
  const TapeLayout T = tape_layout(p);
  const ScratchLayout S = scratch_layout(p, 1);
  const long long F = P.n_omega, N2 = (long long)P.n * P.n;
  cudaStream_t s = ctx->stream;
  const cx<R>* tw = (const cx<R>*)p->tw;
  cx<R>* wt = (cx<R>*)(scr + S.min);
  cx<R>* vt = (cx<R>*)(scr + S.mout);
  cx<R>* ut = vt + F * P.m * N2;
  double* part = (double*)(scr + S.partial);
  double* la = (double*)(tape + T.la);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(la, log_alpha, 8 * F, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "log_alpha copy");
  if ((e = launch_fft2_dense<R>((cx<R>*)W, wt, P.n, F * P.m1, false, tw, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "fft2 W");
  if ((e = launch_diff_forward<R>(P, p->gb, p->gram, wt, la, (double2*)(tape + T.L), (double2*)(tape + T.y), vt, ut,
                                  part, ctx->ctr, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "diff forward");
  // V~ and U~ are adjacent, as are V and u in the tape: one inverse transform
  if ((e = launch_fft2_dense<R>(vt, (cx<R>*)(tape + T.Vx), P.n, 2 * F * P.m, true, tw, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "ifft2 V, u");
  if ((e = launch_diff_combine<R>(P, (const cx<R>*)(tape + T.Vx), (const cx<R>*)(tape + T.ux), (R*)xi, (R*)c,
                                  (R*)(tape + T.xi), s)) != cudaSuccess)
    return cuda_fail(ctx, e, "combine");
  if (phi && (e = launch_reduce_rows(part, (int)F, p->gb, phi, s)) != cudaSuccess) return cuda_fail(ctx, e, "phi");
  return FS_OK;
}

template <typename R>
fs_status diff_vjp(fs_diff_plan* p, const char* tape, char* scr, const void* gxi, const double* gphi, void* gW,
                   double* gla) {
  fs_ctx* ctx = p->ctx;
  const Problem& P = p->P;
  const TapeLayout T = tape_layout(p);
  const ScratchLayout S = scratch_layout(p, 1);
  const long long F = P.n_omega, N2 = (long long)P.n * P.n;
  cudaStream_t s = ctx->stream;
  const cx<R>* tw = (const cx<R>*)p->tw;
  cx<R>* wbt = (cx<R>*)(scr + S.min);
  cx<R>* vbt = (cx<R>*)(scr + S.mout);
  cx<R>* ubt = vbt + F * P.m * N2;
  cx<R>* Vb = (cx<R>*)(scr + S.xsp);
  cx<R>* ub = Vb + F * P.m * N2;
  double* part = (double*)(scr + S.partial);
  const double* la = (const double*)(tape + T.la);
  cudaError_t e;
  if (gxi) {
    if ((e = launch_diff_vjp_point<R>(P, (const R*)gxi, (const cx<R>*)(tape + T.Vx), (const cx<R>*)(tape + T.ux),
                                      (const R*)(tape + T.xi), Vb, ub, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "vjp pointwise");
    if ((e = launch_fft2_dense<R>(Vb, vbt, P.n, 2 * F * P.m, false, tw, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "fft2 V-bar, u-bar");
  }
  if ((e = launch_diff_vjp<R>(P, p->gb, (const double2*)(tape + T.L), (const double2*)(tape + T.y),
                              gxi ? vbt : nullptr, gxi ? ubt : nullptr, la, gphi, gW ? wbt : nullptr, part, s)) !=
      cudaSuccess)
    return cuda_fail(ctx, e, "diff vjp");
  if (gW && (e = launch_fft2_dense<R>(wbt, (cx<R>*)gW, P.n, F * P.m1, true, tw, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "ifft2 W-bar");
  if (gla && (e = launch_reduce_rows(part, (int)F, p->gb, gla, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "log_alpha-bar");
  return FS_OK;
}

template <typename R>
fs_status diff_jvp(fs_diff_plan* p, const char* tape, char* scr, int n_dir, const void* dW, const double* dla,
                   void* dxi, double* dphi) {
  fs_ctx* ctx = p->ctx;
  const Problem& P = p->P;
  const TapeLayout T = tape_layout(p);
  const ScratchLayout S = scratch_layout(p, n_dir);
  const long long F = P.n_omega, N2 = (long long)P.n * P.n, MN2 = (long long)P.m * N2;
  cudaStream_t s = ctx->stream;
  const cx<R>* tw = (const cx<R>*)p->tw;
  const double* la = (const double*)(tape + T.la);
  double* part = (double*)(scr + S.partial);
  cudaError_t e;
  for (int d0 = 0; d0 < n_dir; d0 += S.nd) {
    const int nd = n_dir - d0 < S.nd ? n_dir - d0 : S.nd;
    const cx<R>* dWc = (const cx<R>*)dW + (long long)d0 * F * P.m1 * N2;
    cx<R>* dwt = (cx<R>*)(scr + S.min);
    cx<R>* dvt = (cx<R>*)(scr + S.mout);
    cx<R>* dut = dvt + (long long)nd * F * MN2;
    cx<R>* dVx = (cx<R>*)(scr + S.xsp);
    cx<R>* dux = dVx + (long long)nd * F * MN2;
    if ((e = launch_fft2_dense<R>((cx<R>*)dWc, dwt, P.n, (long long)nd * F * P.m1, false, tw, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "fft2 dW");
    if ((e = launch_diff_jvp<R>(P, p->gb, nd, (const double2*)(tape + T.L), (const double2*)(tape + T.y), dwt, la,
                                dla ? dla + (long long)d0 * F : nullptr, dvt, dut, part, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "diff jvp");
    if ((e = launch_fft2_dense<R>(dvt, dVx, P.n, 2LL * nd * F * P.m, true, tw, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "ifft2 dV, du");
    if ((e = launch_diff_jvp_point<R>(P, nd, (const cx<R>*)(tape + T.Vx), (const cx<R>*)(tape + T.ux),
                                      (const R*)(tape + T.xi), dVx, dux, (R*)dxi + (long long)d0 * MN2, s)) !=
        cudaSuccess)
      return cuda_fail(ctx, e, "jvp pointwise");
    if (dphi && (e = launch_reduce_rows(part, nd * (int)F, p->gb, dphi + (long long)d0 * F, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "phi-dot");
  }
  return FS_OK;
}

}  // namespace

extern "C" {

fs_status fs_diff_plan_create(fs_ctx* ctx, const fs_geometry* g, fs_precision prec, const double* omega,
                              int n_omega, double c0, double eps_u, fs_diff_plan** out) {
  if (!ctx || !out) return FS_EINVAL;
  *out = nullptr;
  fs_status st = validate_args(ctx, g, prec, n_omega, omega, 0.0, c0, nullptr);
  if (st != FS_OK) return st;
  if (!(eps_u >= 0.0)) return fail(ctx, FS_EINVAL, "eps_u must be >= 0");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  fs_diff_plan* p = new (std::nothrow) fs_diff_plan();
  if (!p) return fail(ctx, FS_ENOMEM, "plan");
  fs_options o;
  fs_default_options(&o);
  o.eps_u = eps_u;
  p->ctx = ctx;
  p->P = make_problem(g, n_omega, omega, 0.0, c0, o);
  p->fp64 = prec == FS_FP64;
  p->gb = diff_blocks_per_omega(g->n, n_omega);
  p->P1 = (size_t)g->m1 * (g->m1 + 1) / 2;
  const size_t gbytes = align_up(16 * (size_t)n_omega * g->n * g->n * p->P1);
  const size_t twb = (p->fp64 ? 16 : 8) * (size_t)g->n;
  if (cudaMalloc(&p->buf, gbytes + twb) != cudaSuccess) {
    delete p;
    return fail(ctx, FS_ENOMEM, "normal matrices (%lld bytes)", (long long)(gbytes + twb));
  }
  p->gram = (double2*)p->buf;
  p->tw = (char*)p->buf + gbytes;
  e = p->fp64 ? launch_twiddles<double>((double2*)p->tw, g->n, ctx->stream)
              : launch_twiddles<float>((float2*)p->tw, g->n, ctx->stream);
  if (e == cudaSuccess) e = launch_diff_gram(p->P, p->gram, ctx->stream);
  if (e != cudaSuccess) {
    cudaFree(p->buf);
    delete p;
    return cuda_fail(ctx, e, "plan kernels");
  }
  *out = p;
  return FS_OK;
}

void fs_diff_plan_destroy(fs_diff_plan* p) {
  if (!p) return;
  cudaSetDevice(p->ctx->device);
  cudaStreamSynchronize(p->ctx->stream);
  cudaFree(p->buf);
  delete p;
}

size_t fs_diff_tape_bytes(const fs_diff_plan* p) { return p ? tape_layout(p).total : 0; }

size_t fs_diff_scratch_bytes(const fs_diff_plan* p, int n_dir) { return p ? scratch_layout(p, n_dir).total : 0; }

fs_status fs_reconstruct_diff(fs_diff_plan* p, void* tape, void* scratch, const void* W, const double* log_alpha,
                              void* xi, void* c, double* phi) {
  if (!p) return FS_EINVAL;
  if (!tape || !scratch || !W || !log_alpha || !xi)
    return fail(p->ctx, FS_EINVAL, "tape, scratch, W, log_alpha and xi must be device pointers");
  if (!aligned256(tape) || !aligned256(scratch)) return fail(p->ctx, FS_EINVAL, "tape and scratch must be 256-byte aligned");
  cudaError_t e = cudaSetDevice(p->ctx->device);
  if (e != cudaSuccess) return cuda_fail(p->ctx, e, "cudaSetDevice");
  return p->fp64 ? diff_forward<double>(p, (char*)tape, (char*)scratch, W, log_alpha, xi, c, phi)
                 : diff_forward<float>(p, (char*)tape, (char*)scratch, W, log_alpha, xi, c, phi);
}

fs_status fs_reconstruct_vjp(fs_diff_plan* p, const void* tape, void* scratch, const void* grad_xi,
                             const double* grad_phi, void* grad_W, double* grad_log_alpha) {
  if (!p) return FS_EINVAL;
  if (!tape || !scratch) return fail(p->ctx, FS_EINVAL, "tape and scratch must be device pointers");
  if (!aligned256(tape) || !aligned256(scratch)) return fail(p->ctx, FS_EINVAL, "tape and scratch must be 256-byte aligned");
  cudaError_t e = cudaSetDevice(p->ctx->device);
  if (e != cudaSuccess) return cuda_fail(p->ctx, e, "cudaSetDevice");
  return p->fp64 ? diff_vjp<double>(p, (const char*)tape, (char*)scratch, grad_xi, grad_phi, grad_W, grad_log_alpha)
                 : diff_vjp<float>(p, (const char*)tape, (char*)scratch, grad_xi, grad_phi, grad_W, grad_log_alpha);
}

fs_status fs_reconstruct_jvp(fs_diff_plan* p, const void* tape, void* scratch, int n_dir, const void* dW,
                             const double* dlog_alpha, void* dxi, double* dphi) {
  if (!p) return FS_EINVAL;
  if (n_dir < 1) return fail(p->ctx, FS_EINVAL, "n_dir must be >= 1");
  if (!tape || !scratch || !dW || !dxi) return fail(p->ctx, FS_EINVAL, "tape, scratch, dW and dxi must be device pointers");
  if (!aligned256(tape) || !aligned256(scratch)) return fail(p->ctx, FS_EINVAL, "tape and scratch must be 256-byte aligned");
  cudaError_t e = cudaSetDevice(p->ctx->device);
  if (e != cudaSuccess) return cuda_fail(p->ctx, e, "cudaSetDevice");
  return p->fp64 ? diff_jvp<double>(p, (const char*)tape, (char*)scratch, n_dir, dW, dlog_alpha, dxi, dphi)
                 : diff_jvp<float>(p, (const char*)tape, (char*)scratch, n_dir, dW, dlog_alpha, dxi, dphi);
}

}  // extern "C"
