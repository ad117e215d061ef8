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

#include <complex>
#include <vector>

#include "pipeline.cuh"

namespace fl {

namespace {

__device__ __forceinline__ double2 exp_ikz(double2 kz, double d) {
  const double mag = exp(-kz.y * d);
  double s, c;
  sincos(kz.x * d, &s, &c);
  return make_double2(mag * c, mag * s);
}

// V = xi u0 on X (omega^2 sits in the kernel factor); u0 the plane wave, or the given
// incident field u0i [n_omega][M][N][N]
template <typename R>
__global__ void k_source(Problem P, const R* __restrict__ xi, const cx<R>* __restrict__ u0i, cx<R>* __restrict__ src) {
  const long long N2 = (long long)P.n * P.n;
  const long long per = (long long)P.m * N2;
  const long long total = per * P.n_omega;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int om = (int)(e / per);
    const long long r = e - om * per;
    const R x = xi[r];
    if (u0i) {
      const cx<R> u = u0i[e];
      src[e] = mk<R>(x * u.x, x * u.y);
      continue;
    }
    const int l = (int)(r / N2);
    const double k0 = P.omega[om] / P.c0;
    double s, c;
    sincos(-k0 * (P.z1 + (l + 0.5) * P.hz), &s, &c);
    src[e] = from_d<R>(make_double2((double)x * c, (double)x * s));
  }
}

// U~0 of point sources on the X planes (periodic model, Sec. 5): thread per (omega, l, nu),
// U~0 = (N^2/L^2) sum_s a_s K_nu(z'_l - z_s) e^{-i nu.(r_s - x0)}, K_nu(dz) = -i e^{i k_z|dz|}/(2 k_z),
// x0 = -L/2 (the grid's first node); zero on grazing modes
template <typename R>
__global__ void k_point_sources(Problem P, const double* __restrict__ spec, int n_src, cx<R>* __restrict__ ut) {
  const int N = P.n;
  const long long N2 = (long long)N * N;
  const long long total = (long long)P.n_omega * P.m * N2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long pl = e / N2;
    const int nu = (int)(e - pl * N2);
    const int om = (int)(pl / P.m), l = (int)(pl - (long long)om * P.m);
    const int i2 = nu / N, i1 = nu - i2 * N;
    const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
    const int msq = m1 * m1 + m2 * m2;
    double2 acc = make_double2(0.0, 0.0);
    if (!(msq >= P.graz_lo[om] && msq <= P.graz_hi[om])) {
      const double k0 = P.k0[om];
      const double q = k0 * k0 - P.kn * P.kn * (double)msq;
      const double2 kz = q >= 0.0 ? make_double2(sqrt(q), 0.0) : make_double2(0.0, sqrt(-q));
      // -i / (2 k_z): k_z real -> (0, -1/(2 k_z)); k_z = i kappa -> (-1/(2 kappa), 0)
      const double2 g = q >= 0.0 ? make_double2(0.0, -0.5 / kz.x) : make_double2(-0.5 / kz.y, 0.0);
      const double zl = P.z1 + (l + 0.5) * P.hz, x0 = -0.5 * P.period;
      const double nu1 = P.kn * m1, nu2 = P.kn * m2;
      for (int j = 0; j < n_src; ++j) {
        const double* sp = spec + 4 * j;
        const double2 ez = exp_ikz(kz, sp[2] - zl);  // sources above X: |dz| = z_s - z'_l
        double sn, cs;
        sincos(-(nu1 * (sp[0] - x0) + nu2 * (sp[1] - x0)), &sn, &cs);
        acc = acc + sp[3] * (ez * make_double2(cs, sn));
      }
      acc = (double)N2 / (P.period * P.period) * (g * acc);
    }
    ut[e] = from_d<R>(acc);
  }
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
cudaError_t launch_point_sources(const Problem& P, const double* spec, int n_src, cx<R>* u0, const cx<R>* tw,
                                 cudaStream_t s) {
  k_point_sources<R><<<2048, 256, 0, s>>>(P, spec, n_src, u0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_fft2_dense<R>(u0, u0, P.n, (long long)P.n_omega * P.m, true, tw, s);
}

template cudaError_t launch_point_sources<double>(const Problem&, const double*, int, double2*, const double2*,
                                                  cudaStream_t);
template cudaError_t launch_point_sources<float>(const Problem&, const double*, int, float2*, const float2*,
                                                 cudaStream_t);

template <typename R>
cudaError_t launch_forward_born(const Problem& P, const R* xi, const cx<R>* u0, cx<R>* src, cx<R>* W,
                                const cx<R>* tw, cudaStream_t s) {
  const long long N2 = (long long)P.n * P.n;
  k_source<R><<<1024, 256, 0, s>>>(P, xi, u0, src);
  cudaError_t e = launch_fft2_dense<R>(src, src, P.n, (long long)P.n_omega * P.m, false, tw, s);
  if (e != cudaSuccess) return e;
  const long long modes = N2 * P.n_omega;
  k_apply_data<R><<<(unsigned)((modes + 255) / 256), 256, 0, s>>>(P, src, W);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_fft2_dense<R>(W, W, P.n, (long long)P.n_omega * P.m1, true, tw, s);
}

template cudaError_t launch_forward_born<double>(const Problem&, const double*, const double2*, double2*, double2*,
                                                 const double2*, cudaStream_t);
template cudaError_t launch_forward_born<float>(const Problem&, const float*, const float2*, float2*, float2*,
                                                const float2*, cudaStream_t);


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

// omega^2 T_nu V~ for every mode of one frequency: gamma (F + B) with
// F_l = q F_{l-1} + V~_l, B_l = q (B_{l+1} + V~_{l+1}) (fbuf holds F).  One thread per mode.
// STEP (a step of Algorithm 1): ut <- U~0 + gamma (F + B) and the block partial of
// ||U~_{n+1} - U~_n||^2 in a fixed order; otherwise ut <- gamma (F + B).
// u0t (STEP only, may be null): U~0 of a given incident field on every mode; null for the
// plane wave, whose U~0 is N^2 exp(-i k0 z'_l) at nu = 0 alone
template <typename R, bool STEP>
__global__ void __launch_bounds__(FP_T)
k_interior(Problem P, const cx<R>* __restrict__ vt, cx<R>* __restrict__ ut, cx<R>* __restrict__ fbuf,
           double* __restrict__ partial, const cx<R>* __restrict__ u0t) {
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
      if (STEP && u0t) {
        un = un + u0t[l * N2 + nu];
      } else if (STEP && nu == 0) {
        double s, c;
        sincos(-k0 * (P.z1 + (l + 0.5) * P.hz), &s, &c);
        un = un + from_d<R>(make_double2(n2 * c, n2 * s));
      }
      if (STEP) {
        const cx<R> d = un - ut[l * N2 + nu];
        d2 += (double)d.x * (double)d.x + (double)d.y * (double)d.y;
      }
      ut[l * N2 + nu] = un;
      b = qr * (b + vt[l * N2 + nu]);
    }
  }
  if (!STEP) return;
  red[threadIdx.x] = d2;
  __syncthreads();
  for (int h = FP_T / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// ---- GMRES on u - omega^2 T(xi u) = u0 (the Krylov fallback) -----------------
constexpr int GM_BLOCKS = 512;  // blocks of the reduction kernels (grid-stride)

// the plane wave u0 = exp(-i k0 z'_l) on X
template <typename R>
__global__ void k_plane_wave(Problem P, cx<R>* __restrict__ u) {
  const long long N2 = (long long)P.n * P.n, count = (long long)P.m * N2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(e / N2);
    double s, c;
    sincos(-P.k0[0] * (P.z1 + (l + 0.5) * P.hz), &s, &c);
    u[e] = from_d<R>(make_double2(c, s));
  }
}

// y <- xi a
template <typename R>
__global__ void k_xi_times(long long count, const R* __restrict__ xi, const cx<R>* __restrict__ a,
                           cx<R>* __restrict__ y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const R x = xi[e];
    const cx<R> v = a[e];
    y[e] = mk<R>(x * v.x, x * v.y);
  }
}

// y <- a - b
template <typename R>
__global__ void k_sub(long long count, const cx<R>* __restrict__ a, const cx<R>* __restrict__ b,
                      cx<R>* __restrict__ y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = a[e] - b[e];
}

// block partials of <v_i, w> = sum conj(v_i) w (FP64 sums), grid (GM_BLOCKS, nv):
// partial[i * GM_BLOCKS + block]; summed on the host in a fixed order
template <typename R>
__global__ void __launch_bounds__(FP_T)
k_dots(long long count, const cx<R>* __restrict__ V, long long ld, const cx<R>* __restrict__ w,
       double2* __restrict__ partial) {
  __shared__ double2 red[FP_T];
  const cx<R>* v = V + blockIdx.y * ld;
  double2 acc = make_double2(0.0, 0.0);
  for (long long e = blockIdx.x * (long long)FP_T + threadIdx.x; e < count; e += (long long)gridDim.x * FP_T) {
    const double2 a = to_d(v[e]), b = to_d(w[e]);
    acc.x += a.x * b.x + a.y * b.y;
    acc.y += a.x * b.y - a.y * b.x;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = FP_T / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// w <- w + sign sum_{i < nv} c_i v_i  (c on the device)
template <typename R>
__global__ void k_comb(long long count, const cx<R>* __restrict__ V, long long ld, int nv,
                       const double2* __restrict__ c, double sign, cx<R>* __restrict__ w) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    double2 acc = to_d(w[e]);
    for (int i = 0; i < nv; ++i) {
      const double2 t = c[i] * to_d(V[i * ld + e]);
      acc.x += sign * t.x;
      acc.y += sign * t.y;
    }
    w[e] = from_d<R>(acc);
  }
}

// y <- s x (s real)
template <typename R>
__global__ void k_scale(long long count, const cx<R>* __restrict__ x, double s, cx<R>* __restrict__ y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 v = to_d(x[e]);
    y[e] = from_d<R>(make_double2(s * v.x, s * v.y));
  }
}

}  // namespace

namespace {

constexpr int GM_RESTART = 30;  // Krylov vectors per GMRES cycle

template <typename R> struct FwdLayout {
  long long N2, MN2;
  long long vec_elems;
  cx<R>* base;
  explicit FwdLayout(const Problem& P, void* ws) {
    N2 = (long long)P.n * P.n;
    MN2 = (long long)P.m * N2;
    // fixed point: ut, fb, sc, U~0 of a given incident field; GMRES: sc, tv, fb, x, u0,
    // GM_RESTART + 1 Krylov vectors
    const long long fp = 4 * MN2;
    const long long gm = (6 + GM_RESTART) * MN2;
    vec_elems = fp > gm ? fp : gm;
    base = reinterpret_cast<cx<R>*>(ws);
  }
  double2* reals() const { return reinterpret_cast<double2*>(base + vec_elems); }
  static size_t real_elems() { return (size_t)(GM_RESTART + 1) * GM_BLOCKS + (GM_RESTART + 1) + 1024; }
};

template <typename R>
Problem one_frequency(const Problem& P, int om) {
  Problem Q = P;
  Q.n_omega = 1;
  Q.omega[0] = P.omega[om];
  Q.graz_lo[0] = P.graz_lo[om];
  Q.graz_hi[0] = P.graz_hi[om];
  Q.k0[0] = P.k0[om];
  Q.g0[0] = P.g0[om];
  return Q;
}

// Algorithm 1 for one frequency; on convergence u (physical, M planes) is written to uo
// (which may be the scratch sc).  The stopping test is taken on the host each iteration.
// ||a||^2 of count complex values: block partials of k_dots summed on the host in a fixed order
template <typename R>
cudaError_t norm2_host(const cx<R>* a, long long count, double2* partial, cudaStream_t s, double* out);

template <typename R>
cudaError_t fixed_point_one(const Problem& Q, const R* xi, const cx<R>* u0, const FwdLayout<R>& L, const cx<R>* tw,
                            double rtol, int max_iter, cudaStream_t s, cx<R>* uo_user, cx<R>** uo, int* iters,
                            bool* conv) {
  const long long N2 = L.N2, MN2 = L.MN2;
  cx<R>* ut = L.base;
  cx<R>* fb = ut + MN2;
  cx<R>* sc = fb + MN2;
  cx<R>* u0t = u0 ? sc + MN2 : nullptr;  // U~0 of the given incident field
  double* partial = reinterpret_cast<double*>(L.reals());
  const int nblk = (int)((N2 + FP_T - 1) / FP_T);
  std::vector<double> host(nblk);
  double nrm0 = (double)N2 * sqrt((double)Q.m);  // ||U~0||: N^2 |e^{-i k0 z}| on M planes (plane wave)
  const unsigned gx = (unsigned)((MN2 + FP_T - 1) / FP_T < 4096 ? (MN2 + FP_T - 1) / FP_T : 4096);
  cudaError_t e;
  if (u0) {  // U~1 = U~0 = F_r[u0], and its norm for the stopping rule
    if ((e = launch_fft2_dense<R>(const_cast<cx<R>*>(u0), u0t, Q.n, Q.m, false, tw, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(ut, u0t, sizeof(cx<R>) * MN2, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    if ((e = norm2_host<R>(u0t, MN2, L.reals(), s, &nrm0)) != cudaSuccess) return e;
    nrm0 = sqrt(nrm0);
  } else {
    if ((e = cudaMemsetAsync(ut, 0, sizeof(cx<R>) * MN2, s)) != cudaSuccess) return e;
    k_incident<R><<<(Q.m + 63) / 64, 64, 0, s>>>(Q, ut);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  int it = 0;
  bool ok = max_iter == 0;
  while (it < max_iter) {
    ++it;
    // (the inverse transform works in place on its input: ut is copied first)
    if ((e = cudaMemcpyAsync(sc, ut, sizeof(cx<R>) * MN2, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    if ((e = launch_fft2_dense<R>(sc, sc, Q.n, Q.m, true, tw, s)) != cudaSuccess) return e;
    k_times_xi<R><<<gx, FP_T, 0, s>>>(MN2, xi, sc);
    if ((e = launch_fft2_dense<R>(sc, sc, Q.n, Q.m, false, tw, s)) != cudaSuccess) return e;
    k_interior<R, true><<<nblk, FP_T, 0, s>>>(Q, sc, ut, fb, partial, u0t);
    if ((e = cudaMemcpyAsync(host.data(), partial, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    double d2 = 0.0;
    for (int b = 0; b < nblk; ++b) d2 += host[b];
    const double diff = sqrt(d2);
    if (diff <= rtol * nrm0) {
      ok = true;
      break;
    }
    if (!(diff <= 1e30 * nrm0)) break;  // diverged (or not finite)
  }
  *iters = it;
  *conv = ok;
  if (!ok) return cudaSuccess;
  *uo = uo_user ? uo_user : sc;  // u = F^-1 U~ (ut is not needed after this)
  return launch_fft2_dense<R>(ut, *uo, Q.n, Q.m, true, tw, s);
}

template <typename R> struct Krylov {
  const Problem& Q;
  const R* xi;
  const cx<R>* tw;
  cudaStream_t s;
  long long N2, MN2;
  unsigned gx;
  cx<R> *sc, *tv, *fb;
  double2* partial;  // (GM_RESTART + 1) * GM_BLOCKS
  double2* coef;     // GM_RESTART + 1
  std::vector<double2> host;

  // y <- x - omega^2 F^-1 T_nu F_r[xi x]
  cudaError_t apply(const cx<R>* x, cx<R>* y) {
    k_xi_times<R><<<gx, FP_T, 0, s>>>(MN2, xi, x, sc);
    cudaError_t e = launch_fft2_dense<R>(sc, sc, Q.n, Q.m, false, tw, s);
    if (e != cudaSuccess) return e;
    k_interior<R, false><<<(unsigned)((N2 + FP_T - 1) / FP_T), FP_T, 0, s>>>(Q, sc, tv, fb, nullptr, nullptr);
    if ((e = launch_fft2_dense<R>(tv, tv, Q.n, Q.m, true, tw, s)) != cudaSuccess) return e;
    k_sub<R><<<gx, FP_T, 0, s>>>(MN2, x, tv, y);
    return cudaGetLastError();
  }
  // <v_i, w> for the nv vectors v_i = V + i MN2, summed on the host in a fixed order
  cudaError_t dots(const cx<R>* V, int nv, const cx<R>* w, std::vector<std::complex<double>>& out) {
    k_dots<R><<<dim3(GM_BLOCKS, nv), FP_T, 0, s>>>(MN2, V, MN2, w, partial);
    host.resize((size_t)nv * GM_BLOCKS);
    cudaError_t e = cudaMemcpyAsync(host.data(), partial, sizeof(double2) * host.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    out.assign(nv, 0.0);
    for (int i = 0; i < nv; ++i) {
      double re = 0.0, im = 0.0;
      for (int b = 0; b < GM_BLOCKS; ++b) {
        re += host[(size_t)i * GM_BLOCKS + b].x;
        im += host[(size_t)i * GM_BLOCKS + b].y;
      }
      out[i] = std::complex<double>(re, im);
    }
    return cudaSuccess;
  }
  // w <- w + sign sum_i c_i v_i
  cudaError_t comb(const cx<R>* V, const std::vector<std::complex<double>>& c, double sign, cx<R>* w) {
    std::vector<double2> ch(c.size());
    for (size_t i = 0; i < c.size(); ++i) ch[i] = make_double2(c[i].real(), c[i].imag());
    cudaError_t e = cudaMemcpyAsync(coef, ch.data(), sizeof(double2) * ch.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_comb<R><<<gx, FP_T, 0, s>>>(MN2, V, MN2, (int)c.size(), coef, sign, w);
    // the host vector must outlive the copy
    return cudaStreamSynchronize(s);
  }
};

// Restarted GMRES(GM_RESTART) with classical Gram-Schmidt applied twice and Givens
// rotations, from x = 0, to ||u0 - A x|| <= rtol ||u0|| (the residual of each cycle's
// start is computed, not estimated); iters counts the operator applications.
template <typename R>
cudaError_t norm2_host(const cx<R>* a, long long count, double2* partial, cudaStream_t s, double* out) {
  k_dots<R><<<dim3(GM_BLOCKS, 1), FP_T, 0, s>>>(count, a, count, a, partial);
  cudaError_t e = cudaGetLastError();
  std::vector<double2> h(GM_BLOCKS);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), partial, sizeof(double2) * GM_BLOCKS, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  double t = 0.0;
  for (int b = 0; b < GM_BLOCKS; ++b) t += h[b].x;
  *out = t;
  return cudaSuccess;
}

template <typename R>
cudaError_t gmres_one(const Problem& Q, const R* xi, const cx<R>* u0, const FwdLayout<R>& L, const cx<R>* tw,
                      double rtol, int max_iter, cudaStream_t s, cx<R>** uo, int* iters, bool* conv) {
  using cd = std::complex<double>;
  const long long N2 = L.N2, MN2 = L.MN2;
  Krylov<R> K{Q, xi, tw, s};
  K.N2 = N2;
  K.MN2 = MN2;
  K.gx = (unsigned)((MN2 + FP_T - 1) / FP_T < 4096 ? (MN2 + FP_T - 1) / FP_T : 4096);
  K.sc = L.base;
  K.tv = K.sc + MN2;
  K.fb = K.tv + MN2;
  cx<R>* x = K.fb + MN2;
  cx<R>* bv = x + MN2;
  cx<R>* V = bv + MN2;
  K.partial = L.reals();
  K.coef = K.partial + (size_t)(GM_RESTART + 1) * GM_BLOCKS;
  cudaError_t e;
  if (u0) {
    if ((e = cudaMemcpyAsync(bv, u0, sizeof(cx<R>) * MN2, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
  } else {
    k_plane_wave<R><<<K.gx, FP_T, 0, s>>>(Q, bv);
  }
  if ((e = cudaMemsetAsync(x, 0, sizeof(cx<R>) * MN2, s)) != cudaSuccess) return e;
  std::vector<cd> d;
  if ((e = K.dots(bv, 1, bv, d)) != cudaSuccess) return e;
  const double beta0 = sqrt(d[0].real());
  int total = 0;
  bool ok = false;
  const int R1 = GM_RESTART + 1;
  for (;;) {
    // residual r = u0 - A x in V_0
    if (total == 0) {
      e = cudaMemcpyAsync(V, bv, sizeof(cx<R>) * MN2, cudaMemcpyDeviceToDevice, s);
    } else {
      if ((e = K.apply(x, V)) != cudaSuccess) return e;
      k_sub<R><<<K.gx, FP_T, 0, s>>>(MN2, bv, V, V);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    if ((e = K.dots(V, 1, V, d)) != cudaSuccess) return e;
    const double beta = sqrt(d[0].real());
    if (beta <= rtol * beta0) {
      ok = true;
      break;
    }
    if (total >= max_iter || !(beta <= 1e30 * beta0)) break;
    k_scale<R><<<K.gx, FP_T, 0, s>>>(MN2, V, 1.0 / beta, V);
    std::vector<cd> H((size_t)R1 * GM_RESTART, 0.0), g(R1, 0.0), sn(GM_RESTART, 0.0);
    std::vector<double> cs(GM_RESTART, 0.0);
    auto h = [&](int i, int j) -> cd& { return H[(size_t)i * GM_RESTART + j]; };
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < GM_RESTART && total < max_iter; ++j) {
      cx<R>* w = V + (long long)(j + 1) * MN2;
      if ((e = K.apply(V + (long long)j * MN2, w)) != cudaSuccess) return e;
      ++total;
      for (int pass = 0; pass < 2; ++pass) {  // w -= V (V^H w), twice
        if ((e = K.dots(V, j + 1, w, d)) != cudaSuccess) return e;
        if ((e = K.comb(V, d, -1.0, w)) != cudaSuccess) return e;
        for (int i = 0; i <= j; ++i) h(i, j) += d[i];
      }
      if ((e = K.dots(w, 1, w, d)) != cudaSuccess) return e;
      const double hn = sqrt(d[0].real());
      h(j + 1, j) = hn;
      for (int i = 0; i < j; ++i) {  // earlier rotations on column j
        const cd t = cs[i] * h(i, j) + sn[i] * h(i + 1, j);
        h(i + 1, j) = -std::conj(sn[i]) * h(i, j) + cs[i] * h(i + 1, j);
        h(i, j) = t;
      }
      const cd a = h(j, j);
      const double r = std::sqrt(std::norm(a) + hn * hn);
      if (std::abs(a) == 0.0) {
        cs[j] = 0.0;
        sn[j] = 1.0;
      } else {
        cs[j] = std::abs(a) / r;
        sn[j] = (a / std::abs(a)) * hn / r;
      }
      h(j, j) = cs[j] * a + sn[j] * hn;
      h(j + 1, j) = 0.0;
      g[j + 1] = -std::conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      if (!(hn > 0.0) || std::abs(g[j + 1]) <= rtol * beta0) break;
      k_scale<R><<<K.gx, FP_T, 0, s>>>(MN2, w, 1.0 / hn, w);
    }
    std::vector<cd> y(k);
    for (int i = k - 1; i >= 0; --i) {  // H y = g, upper triangular
      cd t = g[i];
      for (int c = i + 1; c < k; ++c) t -= h(i, c) * y[c];
      y[i] = h(i, i) != 0.0 ? t / h(i, i) : cd(0.0);  // (an exactly singular H: a lucky breakdown)
    }
    if (k > 0 && (e = K.comb(V, y, 1.0, x)) != cudaSuccess) return e;
  }
  *iters = total;
  *conv = ok;
  *uo = x;
  return cudaSuccess;
}

}  // namespace

template <typename R>
size_t forward_bytes(const Problem& P) {
  FwdLayout<R> L(P, nullptr);
  return sizeof(cx<R>) * (size_t)L.vec_elems + sizeof(double2) * FwdLayout<R>::real_elems() + 256;
}

template <typename R>
cudaError_t forward_solve(const Problem& P, const R* xi, const cx<R>* incident, cx<R>* W, cx<R>* u_out, void* ws,
                          int method, double rtol, int max_iter, const cx<R>* tw, cudaStream_t s, int* iters,
                          int* converged) {
  const FwdLayout<R> L(P, ws);
  const long long N2 = L.N2, MN2 = L.MN2;
  const unsigned gx = (unsigned)((MN2 + FP_T - 1) / FP_T < 4096 ? (MN2 + FP_T - 1) / FP_T : 4096);
  cudaError_t e = cudaSuccess;
  for (int om = 0; om < P.n_omega; ++om) {
    const Problem Q = one_frequency<R>(P, om);
    cx<R>* uo_user = u_out ? u_out + (long long)om * MN2 : nullptr;
    cx<R>* u = nullptr;
    int it = 0;
    bool conv = false;
    const cx<R>* u0 = incident ? incident + (long long)om * MN2 : nullptr;
    if (method != 1) {  // Algorithm 1 (method 0, or the first try of method 2)
      if ((e = fixed_point_one<R>(Q, xi, u0, L, tw, rtol, max_iter, s, uo_user, &u, &it, &conv)) != cudaSuccess)
        return e;
    }
    if (!conv && method != 0) {  // GMRES (method 1, or the fallback of method 2)
      int it2 = 0;
      if ((e = gmres_one<R>(Q, xi, u0, L, tw, rtol, max_iter, s, &u, &it2, &conv)) != cudaSuccess) return e;
      it += it2;
      if (conv && uo_user &&
          (e = cudaMemcpyAsync(uo_user, u, sizeof(cx<R>) * MN2, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    }
    if (iters) iters[om] = it;
    if (converged) converged[om] = conv ? 1 : 0;
    if (!conv) return cudaSuccess;
    // eq. (7) with the converged field: V~ = F_r[xi u], data planes.  u is never at the
    // start of the workspace (the fixed point's U~, spent; the Krylov scratch)
    cx<R>* sc = L.base;
    k_xi_times<R><<<gx, FP_T, 0, s>>>(MN2, xi, u, sc);
    if ((e = launch_fft2_dense<R>(sc, sc, P.n, P.m, false, tw, s)) != cudaSuccess) return e;
    cx<R>* wo = W + (long long)om * P.m1 * N2;
    k_apply_data<R><<<(unsigned)((N2 + 255) / 256), 256, 0, s>>>(Q, sc, wo);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_fft2_dense<R>(wo, wo, P.n, P.m1, true, tw, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template size_t forward_bytes<double>(const Problem&);
template size_t forward_bytes<float>(const Problem&);
template cudaError_t forward_solve<double>(const Problem&, const double*, const double2*, double2*, double2*, void*,
                                           int, double, int, const double2*, cudaStream_t, int*, int*);
template cudaError_t forward_solve<float>(const Problem&, const float*, const float2*, float2*, float2*, void*, int,
                                          double, int, const float2*, cudaStream_t, int*, int*);

}  // namespace fl
