// fs_reconstruct_static: the reconstruction of fs_reconstruct for callers that
// cannot allocate device memory -- code running where cudaMalloc is unavailable
// or forbidden (a host framework that owns all device memory through its own
// pool, an embedded caller that must not grow its footprint after start-up, or a
// caller that may not synchronise the device, which a first cudaMalloc can do).
// The caller passes inputs and outputs; every intermediate array lives in one
// file-scope device array of fixed size, so this entry point allocates nothing.
// Argument checks, the problem set-up, the workspace layout and the launch
// sequence are those of fs_reconstruct (api.cu); only the memory differs.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/flatlayer.h"
#include "pipeline.cuh"

using namespace fl;

namespace {

constexpr size_t STATIC_SCRATCH_BYTES = size_t(32) << 20;  // FS_STATIC_SCRATCH_BYTES in the header
static_assert(STATIC_SCRATCH_BYTES == (size_t)FS_STATIC_SCRATCH_BYTES, "scratch size of the header");

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
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FS_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return FS_OK;
}

// bytes of scratch a problem needs: the fs_reconstruct workspace, then the counters,
// the twiddle table and the FP64 twiddles of the mixed truncated-SVD route
size_t static_bytes(const Layout& L, int n, bool fp64, size_t* ctr_off, size_t* tw_off, size_t* tw64_off) {
  *ctr_off = L.total;
  *tw_off = up(*ctr_off + sizeof(unsigned long long) * C_COUNT);
  *tw64_off = up(*tw_off + (fp64 ? 16 : 8) * (size_t)n);
  return up(*tw64_off + 16 * (size_t)n);
}

template <typename R>
fs_status run_static(const Problem& P, const Layout& L, unsigned char* base, const void* W, void* xi, void* c,
                     cudaStream_t s) {
  size_t ctr_off, tw_off, tw64_off;
  static_bytes(L, P.n, sizeof(R) == 8, &ctr_off, &tw_off, &tw64_off);
  unsigned long long* ctr = (unsigned long long*)(base + ctr_off);
  cx<R>* tw = (cx<R>*)(base + tw_off);
  Work<R> w = carve_work<R>(base, L, ctr, tw, nullptr);
  // the scratch keeps the previous call's contents: the counters start at zero,
  // the twiddles are rewritten for this N and precision
  if (cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * C_COUNT, s) != cudaSuccess) return FS_ECUDA;
  if (launch_twiddles<R>(tw, P.n, s) != cudaSuccess) return FS_ECUDA;
  if (wide_route(P, sizeof(R) == 8)) {
    double2* tw64 = (double2*)(base + tw64_off);
    if (launch_twiddles<double>(tw64, P.n, s) != cudaSuccess) return FS_ECUDA;
    w.wt64 = (double2*)(base + L.t12);
    w.tw64 = tw64;
  }
  const char* stage = "";
  return launch_pipeline<R>(P, w, W, xi, c, s, nullptr, &stage) == cudaSuccess ? FS_OK : FS_ECUDA;
}

}  // namespace

extern "C" fs_status fs_reconstruct_static(const fs_geometry* g, fs_precision prec, const void* W,
                                           const double* omega, int n_omega, double delta, double c0,
                                           const fs_options* opts, void* xi, void* c, void* stream) {
  fs_status st = validate_args(nullptr, g, prec, n_omega, omega, delta, c0, opts);
  if (st != FS_OK) return st;
  if (opts && opts->kernel_plan) return FS_EUNSUPPORTED;  // the sampled kernel needs its plan's memory
  if (!W || !xi) return FS_EINVAL;
  if (!elems_aligned(prec == FS_FP64, W, xi, c, opts ? opts->incident : nullptr)) return FS_EINVAL;
  const bool fp64 = prec == FS_FP64;
  const Layout L = layout(g->n, g->m, g->m1, n_omega, fp64);
  size_t ctr_off, tw_off, tw64_off;
  if (static_bytes(L, g->n, fp64, &ctr_off, &tw_off, &tw64_off) > STATIC_SCRATCH_BYTES) return FS_EUNSUPPORTED;
  fs_options o;
  fs_default_options(&o);
  if (opts) o = *opts;
  const Problem P = make_problem(g, n_omega, omega, delta, c0, o);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FS_ECUDA;
  unsigned char* base = nullptr;
  if ((st = scratch_address(dev, &base)) != FS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  return fp64 ? run_static<double>(P, L, base, W, xi, c, s) : run_static<float>(P, L, base, W, xi, c, s);
}
