// Sampled-G kernel of Sec. 5 ("discrete analogues of G~ ... calculated from the
// known values of G using the FFT"): the alternative to the Weyl closed form.
//
// For every frequency, mode nu and vertical offset dz the horizontal transform is
// the 2D DFT of G sampled on the offsets of one period of the grid,
//     K~_nu(dz) = h^2 sum_{i,j} G(sqrt(x_i^2 + y_j^2 + dz^2)) exp(-i nu . (x_i, y_j)),
// x_i = i h (i < N/2), (i - N) h (i >= N/2): the horizontal convolution with G cut to
// one period and periodised.  Where rho = 0 (dz = 0, offset 0) the sample is the
// integral of G over the cell, taken over the ball of the same volume, divided by
// h_z, so that h_z K~ holds that integral.
//
// The offsets a reconstruction needs: dz = z_k - z'_l for the M1 x M entries of A_nu
// (eq. 8) and dz = j h_z, j < M, for the Toeplitz T_nu of eq. (9).  The tables are
// built once per geometry, precision and frequency list (fs_kernel_plan_create), one
// frequency at a time: the samples of D = M1 M + M offsets (FP64), their batched 2D
// FFT (the library's own FFT kernels), and a transpose into mode-major rows of D
// values with omega^2 h_z applied, plus tr(A_nu A_nu^H) per mode.  The mixed precision
// stores each value as a two-float pair (FP32 high and low parts), A scaled by
// 1/sqrt(tr) as its per-mode solve uses it, so that the solve reads A without FP64
// conversions.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/flatlayer.h"
#include "pipeline.cuh"

using namespace fl;

namespace {

// Integral of G = -exp(i k0 rho)/(4 pi rho) over the ball of radius a:
// (1 - (1 - i x) e^{i x}) / k0^2 with x = k0 a; for x <= 1 the difference cancels and
// the power series a^2 sum_{n>=2} (n - 1) i^n x^(n-2) / n! is summed instead.
__device__ double2 ball_integral(double k0, double a) {
  const double x = k0 * a;
  if (x > 1.0) {
    double s, c;
    sincos(x, &s, &c);
    // (1 - i x) e^{i x} = (c + x s) + i (s - x c)
    const double re = 1.0 - (c + x * s), im = -(s - x * c);
    const double ik2 = 1.0 / (k0 * k0);
    return make_double2(re * ik2, im * ik2);
  }
  // sum_{n>=2} (n-1) i^n x^(n-2) / n!: i^n cycles -1, -i, 1, i for n = 2, 3, 4, 5
  double re = 0.0, im = 0.0, xp = 1.0, fact = 2.0;
  for (int n = 2; n < 40; ++n) {
    const double t = (n - 1) * xp / fact;
    switch (n & 3) {
      case 2: re -= t; break;
      case 3: im -= t; break;
      case 0: re += t; break;
      default: im += t; break;
    }
    xp *= x;
    fact *= n + 1;
  }
  return make_double2(a * a * re, a * a * im);
}

// samples h^2 G(rho) of one frequency: [D][N][N] (y, x), offset d < M1 M is the data
// entry (k, l) = (d / M, d % M), d = M1 M + j the interior offset j h_z
__global__ void k_sample_green(Problem P, int om, double2* __restrict__ gs, long long total) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int N = P.n, M = P.m, M1 = P.m1;
  const long long N2 = (long long)N * N;
  const int d = (int)(t / N2);
  const int r = (int)(t - (long long)d * N2);
  const int iy = r / N, ix = r - iy * N;
  const double h = P.period / N;
  const double x = (ix < N / 2 ? ix : ix - N) * h, y = (iy < N / 2 ? iy : iy - N) * h;
  double dz;
  if (d < M1 * M) {
    const int k = d / M, l = d - k * M;
    dz = P.zy[k] - (P.z1 + (l + 0.5) * P.hz);
  } else {
    dz = (d - M1 * M) * P.hz;
  }
  const double k0 = P.k0[om];
  const double r2 = x * x + y * y + dz * dz;
  double2 v;
  if (r2 == 0.0) {
    const double a = cbrt(3.0 * h * h * P.hz / (4.0 * M_PI));
    const double2 b = ball_integral(k0, a);
    v = make_double2(b.x / P.hz, b.y / P.hz);
  } else {
    const double rho = sqrt(r2);
    double s, c;
    sincos(k0 * rho, &s, &c);
    const double f = -h * h / (4.0 * M_PI * rho);
    v = make_double2(f * c, f * s);
  }
  gs[t] = v;
}

// ft[d][nu] (the transforms) -> rows of D values per mode, times omega^2 h_z, and the
// traces tr[nu] = sum_{d < M1 M} |A_d|^2.  Block: 32 modes x all d, in two passes: the
// traces (fixed-order sums), then the transpose through 32 x 32 tiles.  The mixed
// precision stores the entries of A scaled by 1/sqrt(tr) (|A_kl| / sqrt(tr) <= 1,
// where FP32 cannot hold the unscaled entries of strongly evanescent modes) and the
// Toeplitz row of eq. (9) unscaled, each value as two floats (high part, remainder).
constexpr int PT = 32, PR = 8;  // tile width, rows of threads
template <bool MIXED>
__global__ void __launch_bounds__(PT * PR)
k_pack_tables(const double2* __restrict__ ft, int D, int n_a, long long N2, double scale, void* __restrict__ tab,
              double* __restrict__ tr) {
  __shared__ double2 tile[PT][PT + 1];
  __shared__ double red[PR][PT];
  __shared__ double sc[PT];  // 1/sqrt(tr) of the block's modes (mixed)
  const int tx = threadIdx.x % PT, ty = threadIdx.x / PT;
  const long long nu0 = (long long)blockIdx.x * PT;
  {
    double a = 0.0;
    const long long nu = nu0 + tx;
    if (nu < N2)
      for (int d = ty; d < n_a; d += PR) {
        const double2 v = ft[(long long)d * N2 + nu];
        a += v.x * v.x + v.y * v.y;
      }
    red[ty][tx] = a;
    __syncthreads();
    if (ty == 0) {
      double t = 0.0;
      for (int r = 0; r < PR; ++r) t += red[r][tx];
      t *= scale * scale;
      if (nu < N2) tr[nu] = t;
      sc[tx] = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
    }
    __syncthreads();
  }
  for (int d0 = 0; d0 < D; d0 += PT) {
#pragma unroll
    for (int r = 0; r < PT / PR; ++r) {  // read along nu (coalesced)
      const int d = d0 + ty + r * PR;
      const long long nu = nu0 + tx;
      tile[ty + r * PR][tx] = (d < D && nu < N2) ? ft[(long long)d * N2 + nu] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PT / PR; ++r) {  // write along d (coalesced)
      const int mi = ty + r * PR;
      const long long nu = nu0 + mi;
      const int d = d0 + tx;
      if (nu < N2 && d < D) {
        const double2 t = tile[tx][mi];
        if (MIXED) {
          const double f = d < n_a ? scale * sc[mi] : scale;
          const double vr = f * t.x, vi = f * t.y;
          const float hr = (float)vr, hi = (float)vi;
          reinterpret_cast<float4*>(tab)[nu * D + d] =
              make_float4(hr, (float)(vr - (double)hr), hi, (float)(vi - (double)hi));
        } else {
          reinterpret_cast<double2*>(tab)[nu * D + d] = make_double2(scale * t.x, scale * t.y);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

namespace fl {

cudaError_t launch_kernel_tables(const Problem& P, int om, double2* gs, double2* ft, const double2* tw64, bool mixed,
                                 void* tab, double* tr, cudaStream_t s) {
  const int D = kernel_table_width(P);
  const long long N2 = (long long)P.n * P.n;
  const long long total = (long long)D * N2;
  k_sample_green<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(P, om, gs, total);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = launch_fft2_dense<double>(gs, ft, P.n, D, false, tw64, s)) != cudaSuccess) return e;
  const double scale = P.omega[om] * P.omega[om] * P.hz;
  const unsigned grid = (unsigned)((N2 + PT - 1) / PT);
  if (mixed) k_pack_tables<true><<<grid, PT * PR, 0, s>>>(ft, D, P.m1 * P.m, N2, scale, tab, tr);
  else k_pack_tables<false><<<grid, PT * PR, 0, s>>>(ft, D, P.m1 * P.m, N2, scale, tab, tr);
  return cudaGetLastError();
}

}  // namespace fl

struct fs_kernel_plan {
  int device = 0;
  fs_precision prec = FS_FP64;
  int n = 0, m = 0, m1 = 0, n_omega = 0;
  double period = 0, z1 = 0, z2 = 0, c0 = 0;
  std::vector<double> zy, omega;
  void* tab = nullptr;   // [n_omega][N^2][D] double2 (FP64) or float4 two-float (mixed)
  double* tr = nullptr;  // [n_omega][N^2]
  size_t bytes = 0;
};

namespace fl {

bool kernel_plan_matches(const fs_kernel_plan* p, const fs_geometry* g, fs_precision prec, const double* omega,
                         int n_omega, double c0) {
  if (!p || p->prec != prec || p->n != g->n || p->m != g->m || p->m1 != g->m1 || p->n_omega != n_omega) return false;
  if (p->period != g->period || p->z1 != g->z1 || p->z2 != g->z2 || p->c0 != c0) return false;
  for (int k = 0; k < g->m1; ++k)
    if (p->zy[k] != g->zy[k]) return false;
  for (int j = 0; j < n_omega; ++j)
    if (p->omega[j] != omega[j]) return false;
  return true;
}

void kernel_plan_tables(const fs_kernel_plan* p, const void** tab, const double** tr) {
  *tab = p->tab;
  *tr = p->tr;
}

int kernel_plan_device(const fs_kernel_plan* p) { return p->device; }

}  // namespace fl

extern "C" {

fs_status fs_kernel_plan_create(fs_ctx* ctx, const fs_geometry* g, fs_precision prec, const double* omega,
                                int n_omega, double c0, fs_kernel_plan** out) {
  if (!ctx || !out) return FS_EINVAL;
  *out = nullptr;
  fs_status st = validate_args(ctx, g, prec, n_omega, omega, 0.0, c0, nullptr);
  if (st != FS_OK) return st;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FS_ECUDA;
  fs_options o;
  fs_default_options(&o);
  Problem P = make_problem(g, n_omega, omega, 0.0, c0, o);
  const int D = kernel_table_width(P);
  const size_t N2 = (size_t)g->n * g->n;
  const size_t per = (size_t)D * N2 * 16;
  fs_kernel_plan* p = new (std::nothrow) fs_kernel_plan();
  if (!p) return FS_ENOMEM;
  p->device = dev;
  p->prec = prec;
  p->n = g->n; p->m = g->m; p->m1 = g->m1; p->n_omega = n_omega;
  p->period = g->period; p->z1 = g->z1; p->z2 = g->z2; p->c0 = c0;
  p->zy.assign(g->zy, g->zy + g->m1);
  p->omega.assign(omega, omega + n_omega);
  p->bytes = per * n_omega + 8 * N2 * n_omega;
  void *gs = nullptr, *ft = nullptr, *tw = nullptr;
  cudaError_t e = cudaMalloc(&p->tab, per * n_omega);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->tr, 8 * N2 * n_omega);
  if (e == cudaSuccess) e = cudaMalloc(&gs, per);
  if (e == cudaSuccess) e = cudaMalloc(&ft, per);
  if (e == cudaSuccess) e = cudaMalloc(&tw, 16 * (size_t)g->n);
  cudaStream_t s = nullptr;  // the legacy stream: the plan is built synchronously
  if (e == cudaSuccess) e = launch_twiddles<double>((double2*)tw, g->n, s);
  for (int j = 0; j < n_omega && e == cudaSuccess; ++j)
    e = launch_kernel_tables(P, j, (double2*)gs, (double2*)ft, (const double2*)tw, prec == FS_MIXED,
                             (char*)p->tab + per * j, p->tr + N2 * j, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (gs) cudaFree(gs);
  if (ft) cudaFree(ft);
  if (tw) cudaFree(tw);
  if (e != cudaSuccess) {
    if (p->tab) cudaFree(p->tab);
    if (p->tr) cudaFree(p->tr);
    delete p;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FS_ENOMEM : FS_ECUDA;
  }
  *out = p;
  return FS_OK;
}

void fs_kernel_plan_destroy(fs_kernel_plan* p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  cudaFree(p->tab);
  cudaFree(p->tr);
  cudaSetDevice(cur);
  delete p;
}

size_t fs_kernel_plan_bytes(const fs_kernel_plan* p) { return p ? p->bytes : 0; }

}  // extern "C"
