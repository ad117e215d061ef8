// Forward data generator on the device, single-scattering form: Algorithm 1
// (Sec. 3) stopped before its first iteration, so U~ = U~0 and eq. (7) gives
//   V~ = F_r[xi F^-1 U~0] = F_r[xi u0],   W~_k = omega^2 sum_l h_z K_nu(z_k - z'_l) V~_l,
//   W = F^-1[W~]  on the data planes.
// The incident field is the plane wave u0 = exp(-i k0 z).  As in the solve, every
// data plane lies above X, so exp(i k_z (z_k - z'_l)) = exp(i k_z (z_k - z'_top)) *
// exp(i k_z (z'_top - z'_l)) and the sum over l is shared by all k.  Grazing modes
// (|nu| = k0) carry K = 0.
#include <math.h>

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

}  // namespace fl
