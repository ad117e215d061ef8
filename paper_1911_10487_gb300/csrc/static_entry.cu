// fs_reconstruct_static: the reconstruction of fs_reconstruct for callers that
// cannot allocate device memory -- code running where cudaMalloc is unavailable
// or forbidden (a host framework that owns all device memory through its own
// pool, an embedded caller that must not grow its footprint after start-up, or a
// caller that may not synchronise the device, which a first cudaMalloc can do).
// The caller passes inputs and outputs; every intermediate array lives in one
// file-scope device array of fixed size, so this entry point allocates nothing.
#include <math.h>
#include <mutex>
#include <string.h>

#include <cuda_runtime.h>

#include "../../include/flatlayer.h"
#include "pipeline.cuh"

using namespace fl;

namespace {

constexpr size_t STATIC_SCRATCH_BYTES = size_t(32) << 20;  // FS_STATIC_SCRATCH_BYTES in the header
constexpr int MAX_DEVICES = 64;

// Scratch shared by every call on a device: intermediates, counters, twiddles.
// Host code must not pass this symbol to a kernel (on the host it names a
// stand-in, not device memory); it uses the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

std::mutex g_setup_mutex;
void* g_scratch_addr[MAX_DEVICES] = {};

size_t up(size_t v) { return (v + 255) & ~size_t(255); }

// device address of the scratch array on the current device (looked up once)
fs_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= MAX_DEVICES) return FS_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return FS_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return FS_OK;
}

template <typename R>
fs_status run_static(const Problem& P, unsigned char* base, const void* W, void* xi, void* c, cudaStream_t s) {
  const size_t cxs = sizeof(cx<R>);
  const size_t N2 = (size_t)P.n * P.n;
  const size_t F = (size_t)P.n_omega;
  const size_t a = F * P.m1 * N2, b = F * 2 * P.m * N2;
  const int n_partial = (int)((N2 + 255) / 256);
  Work<R> w;
  size_t off = 0;
  w.wt = (cx<R>*)(base + off);
  w.t2 = w.wt;
  off = up(off + cxs * (a > b ? a : b));
  w.prof = (cx<R>*)(base + off); off = up(off + cxs * F * N2 * 2 * P.m);
  w.norms = (double*)(base + off); off = up(off + 8 * F * N2);
  w.partial = (double*)(base + off); off = up(off + 8 * F * n_partial);
  w.n_partial = n_partial;
  w.slot = (int*)(base + off); off = up(off + 4 * F * N2);
  w.act = (int*)(base + off); off = up(off + 4 * F * N2);
  const size_t cb = F * classify_blocks(P.n);
  w.flagbits = (unsigned*)(base + off); off = up(off + 4 * cb * 32);
  w.blkcnt = (int*)(base + off); off = up(off + 4 * cb);
  w.blkgz = (int*)(base + off); off = up(off + 4 * cb);
  w.colblk = (unsigned*)(base + off); off = up(off + 4 * cb * 8);
  w.cols = (int*)(base + off); off = up(off + 4 * F * P.n);
  w.ncol = (int*)(base + off); off = up(off + 4 * F);
  w.count = (int*)(base + off); off = up(off + 4 * F);
  w.dnu = (double*)(base + off); off = up(off + 8 * F);
  w.ctr = (unsigned long long*)(base + off); off = up(off + sizeof(unsigned long long) * C_COUNT);
  cx<R>* tw = (cx<R>*)(base + off); off = up(off + cxs * P.n);
  if (off > STATIC_SCRATCH_BYTES) return FS_EUNSUPPORTED;
  w.tw = tw;
  w.alpha_out = nullptr;
  // the scratch keeps the previous call's contents: the counters start at zero,
  // the twiddles are rewritten for this N and precision
  if (cudaMemsetAsync(w.ctr, 0, sizeof(unsigned long long) * C_COUNT, s) != cudaSuccess) return FS_ECUDA;
  if (launch_twiddles<R>(tw, P.n, s) != cudaSuccess) return FS_ECUDA;
  if (launch_fft2_forward<R>((const cx<R>*)W, P, w, s) != cudaSuccess) return FS_ECUDA;
  if (launch_classify<R>(P, w, s) != cudaSuccess) return FS_ECUDA;
  cudaError_t e = P.solve_form == 1 ? launch_solve_rank1<R>(P, w, s)
                  : sizeof(R) == 8   ? launch_solve_fp64(P, *(const Work<double>*)&w, s)
                                     : launch_solve_mixed(P, *(const Work<float>*)&w, s);
  if (e != cudaSuccess) return FS_ECUDA;
  if (launch_recover<R>(P, w, (R*)xi, (R*)c, s) != cudaSuccess) return FS_ECUDA;
  return FS_OK;
}

}  // namespace

extern "C" fs_status fs_reconstruct_static(const fs_geometry* g, fs_precision prec, const void* W,
                                           const double* omega, int n_omega, double delta, double c0,
                                           const fs_options* opts, void* xi, void* c, void* stream) {
  if (!g || !W || !xi || !omega || !g->zy) return FS_EINVAL;
  if (prec != FS_FP64 && prec != FS_MIXED) return FS_EINVAL;
  if (g->n <= 0 || g->m <= 0 || g->m1 <= 0 || n_omega <= 0) return FS_EINVAL;
  if (!fft_size_supported(g->n) || g->m > MAX_M || g->m1 > MAX_M1 || n_omega > MAX_OMEGA) return FS_EUNSUPPORTED;
  if (!(g->period > 0.0) || !(g->z2 > g->z1) || !(delta >= 0.0) || !(c0 > 0.0)) return FS_EINVAL;
  for (int k = 0; k < g->m1; ++k)
    if (!(g->zy[k] > g->z2)) return FS_EINVAL;
  for (int j = 0; j < n_omega; ++j)
    if (!(omega[j] > 0.0)) return FS_EINVAL;
  fs_options o;
  fs_default_options(&o);
  if (opts) o = *opts;
  if (!(o.tau > 0.0) || !(o.delta_floor >= 0.0) || !(o.alpha_rel > 0.0) || !(o.eps_u >= 0.0) ||
      o.max_iter < 1 || o.refine_iters < 1 || (o.alpha_mode != 0 && o.alpha_mode != 1))
    return FS_EINVAL;
  if (o.solve_form != 0 && o.solve_form != 1) return FS_EINVAL;
  if (o.regularizer != 0 && o.regularizer != 1) return FS_EINVAL;
  if (o.regularizer == 1 && o.solve_form != 1) return FS_EUNSUPPORTED;
  if (o.regularizer == 1 && o.alpha_mode != 0) return FS_EINVAL;
  if (o.alpha_mode == 1) {
    if (!o.alpha_given) return FS_EINVAL;
    for (int j = 0; j < n_omega; ++j)
      if (!(o.alpha_given[j] > 0.0)) return FS_EINVAL;
  }
  Problem P;
  memset(&P, 0, sizeof(P));
  P.n = g->n; P.m = g->m; P.m1 = g->m1; P.n_omega = n_omega;
  P.alpha_mode = o.alpha_mode; P.max_iter = o.max_iter; P.refine_iters = o.refine_iters;
  P.period = g->period; P.z1 = g->z1; P.hz = (g->z2 - g->z1) / g->m; P.c0 = c0;
  P.delta = delta; P.tau = o.tau; P.delta_floor = o.delta_floor; P.alpha_rel = o.alpha_rel; P.eps_u = o.eps_u;
  P.fp64_switch = o.fp64_switch;
  P.solve_bps = (o.solve_blocks_per_sm >= 1 && o.solve_blocks_per_sm <= 3) ? o.solve_blocks_per_sm : 2;
  P.solve_form = o.solve_form;
  P.regularizer = o.regularizer;
  for (int k = 0; k < g->m1; ++k) P.zy[k] = g->zy[k];
  for (int j = 0; j < n_omega; ++j) {
    P.omega[j] = omega[j];
    P.alpha_given[j] = o.alpha_mode == 1 ? o.alpha_given[j] : 0.0;
    const double sL = omega[j] / c0 * g->period / (2.0 * M_PI);
    const double s2 = sL * sL;
    const double lo = ceil(s2 - 1e-9 * s2), hi = floor(s2 + 1e-9 * s2);
    P.graz_lo[j] = lo > 1e9 ? 1000000001 : (int)lo;
    P.graz_hi[j] = hi > 1e9 ? 1000000000 : (int)hi;
  }
  derive_constants(P);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FS_ECUDA;
  unsigned char* base = nullptr;
  fs_status st = scratch_address(dev, &base);
  if (st != FS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  return prec == FS_FP64 ? run_static<double>(P, base, W, xi, c, s) : run_static<float>(P, base, W, xi, c, s);
}
