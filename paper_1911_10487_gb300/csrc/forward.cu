// Forward data generator on the device.
//
// Single scattering (Born): Algorithm 1 (Sec. 3) stopped before its first
// iteration, so U~ = U~0 and eq. (7) gives
//   V~ = F_r[xi F^-1 U~0] = F_r[xi u0],   W~_k = omega^2 sum_l h_z K_nu(z_k - z'_l) V~_l,
//   W = F^-1[W~]  on the data planes.
// Full scattering: Algorithm 1 itself, the fixed point of eq. (6),
//   U~_{n+1} = U~0 + omega^2 T_nu F_r[xi F^-1 U~_n],  T_nu[l, l'] = h_z K_nu(z'_l - z'_l'),
// stopped when ||U~_{n+1} - U~_n|| <= rtol ||U~0|| (Sec. 5.1), then eq. (7) with the
// converged field.  T_nu is applied as in eq. (9) of the inverse: with q = e^{i k_z h_z},
// h_z K_nu(z'_l - z'_l') = gamma q^|l - l'| / omega^2, a forward and a backward first-order
// recurrence over the planes, one thread per mode.
// The incident field is the plane wave u0 = exp(-i k0 z).  As in the solve, every
// data plane lies above X, so exp(i k_z (z_k - z'_l)) = exp(i k_z (z_k - z'_top)) *
// exp(i k_z (z'_top - z'_l)) and the sum over l is shared by all k.  Grazing modes
// (|nu| = k0) carry K = 0.
#include <math.h>

#include <vector>

#include "pipeline.cuh"

namespace fl {

namespace {

template <typename R>
__global__ void k_source(Problem P, const R* __restrict__ xi, cx<R>* __restrict__ src) {
  const long long N2 = (long long)P.n * P.n;
  const long long per = (long long)P.m * N2;
  const long long total = per * P.n_omega;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int om = (int)(e / per);
    const long long r = e - om * per;
    const int l = (int)(r / N2);
    const double k0 = P.omega[om] / P.c0;
    double s, c;
    sincos(-k0 * (P.z1 + (l + 0.5) * P.hz), &s, &c);
    const double x = (double)xi[r];  // V = xi u0; omega^2 sits in the kernel factor
    src[e] = from_d<R>(make_double2(x * c, x * s));
  }
}

__device__ __forceinline__ double2 exp_ikz(double2 kz, double d) {
  const double mag = exp(-kz.y * d);
  double s, c;
  sincos(kz.x * d, &s, &c);
  return make_double2(mag * c, mag * s);
}

template <typename R>
__global__ void k_apply_data(Problem P, const cx<R>* __restrict__ vt, cx<R>* __restrict__ wt) {
  const int N = P.n;
  const long long N2 = (long long)N * N;
  const long long total = N2 * P.n_omega;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int om = (int)(e / N2);
    const int nu = (int)(e - om * N2);
    const int i2 = nu / N, i1 = nu - i2 * N;
    const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
    const double k0 = P.omega[om] / P.c0;
    const int msq_i = m1 * m1 + m2 * m2;
    const double msq = (double)msq_i;
    cx<R>* out = wt + (long long)om * P.m1 * N2 + nu;
    if (msq_i >= P.graz_lo[om] && msq_i <= P.graz_hi[om]) {  // grazing: excluded
      for (int k = 0; k < P.m1; ++k) out[k * N2] = czero<R>();
      continue;
    }
    const double kn = 2.0 * M_PI / P.period;
    const double q = k0 * k0 - kn * kn * msq;
    const double2 kz = q >= 0.0 ? make_double2(sqrt(q), 0.0) : make_double2(0.0, sqrt(-q));
    const double g0 = 0.5 * P.omega[om] * P.omega[om] * P.hz;
    const double2 gamma = q >= 0.0 ? make_double2(0.0, -g0 / kz.x) : make_double2(-g0 / kz.y, 0.0);
    const double ztop = P.z1 + (P.m - 0.5) * P.hz;
    const cx<R>* in = vt + (long long)om * P.m * N2 + nu;
    double2 acc = make_double2(0, 0);
    for (int l = 0; l < P.m; ++l)
      acc = acc + exp_ikz(kz, ztop - (P.z1 + (l + 0.5) * P.hz)) * to_d(in[l * N2]);
    acc = gamma * acc;
    for (int k = 0; k < P.m1; ++k) out[k * N2] = from_d<R>(exp_ikz(kz, P.zy[k] - ztop) * acc);
  }
}

}  // namespace

template <typename R>
cudaError_t launch_forward_born(const Problem& P, const R* xi, cx<R>* src, cx<R>* W, const cx<R>* tw,
                                cudaStream_t s) {
  const long long N2 = (long long)P.n * P.n;
  k_source<R><<<1024, 256, 0, s>>>(P, xi, src);
  cudaError_t e = launch_fft2_dense<R>(src, src, P.n, (long long)P.n_omega * P.m, false, tw, s);
  if (e != cudaSuccess) return e;
  const long long modes = N2 * P.n_omega;
  k_apply_data<R><<<(unsigned)((modes + 255) / 256), 256, 0, s>>>(P, src, W);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_fft2_dense<R>(W, W, P.n, (long long)P.n_omega * P.m1, true, tw, s);
}

template cudaError_t launch_forward_born<double>(const Problem&, const double*, double2*, double2*,
                                                 const double2*, cudaStream_t);
template cudaError_t launch_forward_born<float>(const Problem&, const float*, float2*, float2*, const float2*,
                                                cudaStream_t);


// ---- Algorithm 1 (fixed point of eq. 6) -------------------------------------
namespace {

constexpr int FP_T = 256;  // threads per block of the fixed-point kernels

// U~0 of one frequency: N^2 exp(-i k0 z'_l) at nu = 0 (the rest is zeroed by the caller)
template <typename R>
__global__ void k_incident(Problem P, cx<R>* __restrict__ ut) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < P.m) {
    double s, c;
    sincos(-P.k0[0] * (P.z1 + (l + 0.5) * P.hz), &s, &c);
    const double n2 = (double)P.n * P.n;
    ut[(long long)l * P.n * P.n] = from_d<R>(make_double2(n2 * c, n2 * s));
  }
}

// s <- xi s, pointwise on the X grid
template <typename R>
__global__ void k_times_xi(long long count, const R* __restrict__ xi, cx<R>* __restrict__ s) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const R x = xi[e];
    const cx<R> v = s[e];
    s[e] = mk<R>(x * v.x, x * v.y);
  }
}

// One step of Algorithm 1 for every mode of one frequency: ut <- U~0 + gamma (F + B),
// F_l = q F_{l-1} + V~_l, B_l = q (B_{l+1} + V~_{l+1}) (fbuf holds F), and the block
// partial of ||U~_{n+1} - U~_n||^2 in a fixed order.  One thread per mode.
template <typename R>
__global__ void __launch_bounds__(FP_T)
k_interior(Problem P, const cx<R>* __restrict__ vt, cx<R>* __restrict__ ut, cx<R>* __restrict__ fbuf,
           double* __restrict__ partial) {
  __shared__ double red[FP_T];
  const int N = P.n, M = P.m;
  const long long N2 = (long long)N * N;
  const long long nu = blockIdx.x * (long long)FP_T + threadIdx.x;
  double d2 = 0.0;
  if (nu < N2) {
    const int i2 = (int)(nu / N), i1 = (int)(nu - (long long)i2 * N);
    const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
    const int msq = m1 * m1 + m2 * m2;
    const double k0 = P.k0[0];
    cx<R> qr = czero<R>(), gr = czero<R>();
    if (!(msq >= P.graz_lo[0] && msq <= P.graz_hi[0])) {  // grazing modes: T_nu = 0
      const double q = k0 * k0 - P.kn * P.kn * (double)msq;
      const double2 kz = q >= 0.0 ? make_double2(sqrt(q), 0.0) : make_double2(0.0, sqrt(-q));
      const double2 gamma = q >= 0.0 ? make_double2(0.0, -P.g0[0] / kz.x) : make_double2(-P.g0[0] / kz.y, 0.0);
      qr = from_d<R>(exp_ikz(kz, P.hz));
      gr = from_d<R>(gamma);
    }
    cx<R> f = czero<R>();
    for (int l = 0; l < M; ++l) {
      f = qr * f + vt[l * N2 + nu];
      fbuf[l * N2 + nu] = f;
    }
    const double n2 = (double)N2;
    cx<R> b = czero<R>();
    for (int l = M - 1; l >= 0; --l) {
      cx<R> un = gr * (fbuf[l * N2 + nu] + b);
      if (nu == 0) {
        double s, c;
        sincos(-k0 * (P.z1 + (l + 0.5) * P.hz), &s, &c);
        un = un + from_d<R>(make_double2(n2 * c, n2 * s));
      }
      const cx<R> d = un - ut[l * N2 + nu];
      d2 += (double)d.x * (double)d.x + (double)d.y * (double)d.y;
      ut[l * N2 + nu] = un;
      b = qr * (b + vt[l * N2 + nu]);
    }
  }
  red[threadIdx.x] = d2;
  __syncthreads();
  for (int h = FP_T / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

}  // namespace

template <typename R>
size_t forward_fixed_point_bytes(const Problem& P) {
  const size_t plane = sizeof(cx<R>) * (size_t)P.n * P.n;
  const int mm = P.m > P.m1 ? P.m : P.m1;
  const size_t nblk = ((size_t)P.n * P.n + FP_T - 1) / FP_T;
  return plane * ((size_t)P.m * 2 + mm) + sizeof(double) * nblk + 256;
}

template <typename R>
cudaError_t forward_fixed_point(const Problem& P, const R* xi, cx<R>* W, cx<R>* u_out, void* ws, double rtol,
                                int max_iter, const cx<R>* tw, cudaStream_t s, int* iters, int* converged) {
  const long long N2 = (long long)P.n * P.n, MN2 = (long long)P.m * N2;
  const int mm = P.m > P.m1 ? P.m : P.m1;
  cx<R>* ut = reinterpret_cast<cx<R>*>(ws);
  cx<R>* fb = ut + MN2;
  cx<R>* sc = fb + MN2;  // mm planes
  double* partial = reinterpret_cast<double*>(sc + (long long)mm * N2);
  const int nblk = (int)((N2 + FP_T - 1) / FP_T);
  std::vector<double> host(nblk);
  const double nrm0 = (double)N2 * sqrt((double)P.m);  // ||U~0||: N^2 |e^{-i k0 z}| on M planes
  const unsigned gx = (unsigned)((MN2 + FP_T - 1) / FP_T < 4096 ? (MN2 + FP_T - 1) / FP_T : 4096);
  cudaError_t e = cudaSuccess;
  for (int om = 0; om < P.n_omega; ++om) {
    Problem Q = P;  // one frequency
    Q.n_omega = 1;
    Q.omega[0] = P.omega[om];
    Q.graz_lo[0] = P.graz_lo[om];
    Q.graz_hi[0] = P.graz_hi[om];
    Q.k0[0] = P.k0[om];
    Q.g0[0] = P.g0[om];
    if ((e = cudaMemsetAsync(ut, 0, sizeof(cx<R>) * MN2, s)) != cudaSuccess) return e;
    k_incident<R><<<(P.m + 63) / 64, 64, 0, s>>>(Q, ut);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int it = 0;
    bool conv = max_iter == 0;
    while (it < max_iter) {
      ++it;
      // (the inverse transform works in place on its input: ut is copied first)
      if ((e = cudaMemcpyAsync(sc, ut, sizeof(cx<R>) * MN2, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
      if ((e = launch_fft2_dense<R>(sc, sc, P.n, P.m, true, tw, s)) != cudaSuccess) return e;
      k_times_xi<R><<<gx, FP_T, 0, s>>>(MN2, xi, sc);
      if ((e = launch_fft2_dense<R>(sc, sc, P.n, P.m, false, tw, s)) != cudaSuccess) return e;
      k_interior<R><<<nblk, FP_T, 0, s>>>(Q, sc, ut, fb, partial);
      if ((e = cudaMemcpyAsync(host.data(), partial, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess)
        return e;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
      double d2 = 0.0;
      for (int b = 0; b < nblk; ++b) d2 += host[b];
      const double diff = sqrt(d2);
      if (diff <= rtol * nrm0) {
        conv = true;
        break;
      }
      if (!(diff <= 1e30 * nrm0)) break;  // diverged (or not finite)
    }
    if (iters) iters[om] = it;
    if (converged) converged[om] = conv ? 1 : 0;
    if (!conv) return cudaSuccess;
    // eq. (7) with the converged field: u = F^-1 U~ (ut is not needed after this), V~ =
    // F_r[xi u], data planes
    cx<R>* uo = u_out ? u_out + (long long)om * MN2 : sc;
    if ((e = launch_fft2_dense<R>(ut, uo, P.n, P.m, true, tw, s)) != cudaSuccess) return e;
    if (uo != sc && (e = cudaMemcpyAsync(sc, uo, sizeof(cx<R>) * MN2, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
    k_times_xi<R><<<gx, FP_T, 0, s>>>(MN2, xi, sc);
    if ((e = launch_fft2_dense<R>(sc, sc, P.n, P.m, false, tw, s)) != cudaSuccess) return e;
    cx<R>* wo = W + (long long)om * P.m1 * N2;
    k_apply_data<R><<<(unsigned)((N2 + 255) / 256), 256, 0, s>>>(Q, sc, wo);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_fft2_dense<R>(wo, wo, P.n, P.m1, true, tw, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template size_t forward_fixed_point_bytes<double>(const Problem&);
template size_t forward_fixed_point_bytes<float>(const Problem&);
template cudaError_t forward_fixed_point<double>(const Problem&, const double*, double2*, double2*, void*, double,
                                                 int, const double2*, cudaStream_t, int*, int*);
template cudaError_t forward_fixed_point<float>(const Problem&, const float*, float2*, float2*, void*, double, int,
                                                const float2*, cudaStream_t, int*, int*);

}  // namespace fl
