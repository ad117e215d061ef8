// Per-mode part of Algorithm 2: classification of the modes (discrepancy test)
// and, for every active mode nu, the regularised solution of the SLAE of eq. (8)
// followed by eq. (9) (Sec. 4 steps 1-2, Sec. 5.2).
//
// For every active mode one thread block:
//   1. builds A_nu[k, l] = omega^2 h_z K_nu(z_k - z'_l) with the Weyl closed form
//      K_nu(dz) = -i exp(i k_z |dz|)/(2 k_z) (horizontal Fourier transform of
//      G = -exp(i k0 rho)/(4 pi rho)); every data plane lies above X, so
//      exp(i k_z (z_k - z'_l)) is evaluated as exp(i k_z (z_k - z'_top)) *
//      exp(i k_z (z'_top - z'_l)) with both factors of modulus <= 1;
//   2. forms the dual normal matrix G = A A^H (M1 x M1, Hermitian);
//   3. reduces G to a real symmetric tridiagonal T = D^H Q^H G Q D by Householder
//      reflections (Q) and a diagonal phase scaling (D);
//   4. picks alpha by the discrepancy principle: with c = D^H Q^H b and
//      z(alpha) = (T + alpha I)^-1 c (tridiagonal LDL^T solve), the residual of the
//      Tikhonov solution is b - A A^H y = alpha y, so
//      phi(alpha) = ||A V~ - b|| = alpha ||z(alpha)||; the root of phi = delta_nu is
//      found by Newton's method in log(alpha) inside a bisection bracket
//      [alpha_floor, tr(G) delta_nu/(||b|| - delta_nu)], alpha_floor = alpha_rel tr(G);
//      phi(alpha_floor) >= delta_nu selects alpha_floor;
//   5. y = Q D z, V~ = A^H y (the Tikhonov solution (A^H A + alpha I)^-1 A^H b in
//      its dual form);
//   6. U~ = U~0 + omega^2 T_nu V~ with T_nu[l, l'] = h_z K_nu(z'_l - z'_l'): since the
//      X planes are uniform, T_nu is h_z(-i/2k_z) q^|l-l'| with q = exp(i k_z h_z),
//      applied as one forward and one backward first-order recurrence (this is
//      the z part of the zero-padded convolution u = u0 + G * w, done exactly).
// Mixed precision: steps 1-4 in FP32, alpha root-find in FP64 on the FP32
// tridiagonal, then y is refined against the FP64 residual b - A A^H y - alpha y;
// modes whose alpha/tr(G) falls below a switch are redone entirely in FP64.
#include <math.h>

#include "pipeline.cuh"

namespace fl {

namespace {

constexpr int ST = 128;  // threads per solve block

// ------------------------------------------------------------------------------
// classification: one block per frequency
// ------------------------------------------------------------------------------
constexpr int CT = 1024;

__global__ void __launch_bounds__(CT)
k_classify(Problem P, const double* __restrict__ norms, int* __restrict__ slot, int* __restrict__ act,
           int* __restrict__ cols, int* __restrict__ ncol, int* __restrict__ count,
           double* __restrict__ dnu_out, unsigned long long* __restrict__ ctr) {
  const int om = blockIdx.x;
  const int N = P.n;
  const int N2 = N * N;
  const double* nrm = norms + (long long)om * N2;
  __shared__ double red[CT];
  __shared__ int scan[CT];
  __shared__ int colflag[MAX_N];
  __shared__ unsigned cgraz[CT / 32];
  // ||W||^2 = sum_nu ||W~_nu||^2 / N^2 (Parseval, unnormalised DFT); fixed order
  double s = 0.0;
  for (int v = threadIdx.x; v < N2; v += CT) s += nrm[v];
  red[threadIdx.x] = s;
  for (int j = threadIdx.x; j < N; j += CT) colflag[j] = 0;
  __syncthreads();
  for (int h = CT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  const double wnorm = sqrt(red[0] / (double)N2);
  const double dnu = P.tau * fmax(P.delta, P.delta_floor) * wnorm;
  const double thresh = dnu * dnu;
  const double k0 = P.omega[om] / P.c0;
  const double sL = k0 * P.period / (2.0 * M_PI);
  const double s2 = sL * sL;
  // contiguous chunk per thread so the compaction keeps mode order
  const int C = (N2 + CT - 1) / CT;
  const int v0 = threadIdx.x * C, v1 = min(N2, v0 + C);
  int cnt = 0;
  unsigned ngz = 0;
  for (int v = v0; v < v1; ++v) {
    const int i2 = v / N, i1 = v - i2 * N;
    const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
    const double msq = (double)(m1 * m1 + m2 * m2);
    const bool graz = fabs(msq - s2) <= 1e-9 * s2;
    ngz += graz;
    const bool a = !graz && (P.alpha_mode == 1 || nrm[v] > thresh);
    cnt += a;
  }
  scan[threadIdx.x] = cnt;
  __syncthreads();
  for (int off = 1; off < CT; off <<= 1) {  // inclusive Hillis-Steele scan
    const int t = threadIdx.x >= off ? scan[threadIdx.x - off] : 0;
    __syncthreads();
    scan[threadIdx.x] += t;
    __syncthreads();
  }
  int pos = scan[threadIdx.x] - cnt;
  const int total = scan[CT - 1];
  for (int v = v0; v < v1; ++v) {
    const int i2 = v / N, i1 = v - i2 * N;
    const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
    const double msq = (double)(m1 * m1 + m2 * m2);
    const bool graz = fabs(msq - s2) <= 1e-9 * s2;
    const bool a = !graz && (P.alpha_mode == 1 || nrm[v] > thresh);
    if (a) {
      slot[(long long)om * N2 + v] = pos;
      act[(long long)om * N2 + pos] = v;
      colflag[i1] = 1;
      ++pos;
    } else {
      slot[(long long)om * N2 + v] = -1;
    }
  }
  for (int o = 16; o > 0; o >>= 1) ngz += __shfl_xor_sync(0xffffffffu, ngz, o);
  if ((threadIdx.x & 31) == 0) cgraz[threadIdx.x >> 5] = ngz;
  __syncthreads();
  if (threadIdx.x == 0) {
    colflag[0] = 1;  // the incident plane wave lives at nu = 0
    int nc = 0;
    for (int j = 0; j < N; ++j)
      if (colflag[j]) cols[om * N + nc++] = j;
    ncol[om] = nc;
    count[om] = total;
    dnu_out[om] = dnu;
    unsigned long long g = 0;
    for (int w = 0; w < CT / 32; ++w) g += cgraz[w];
    atomicAdd(ctr + C_MODES, (unsigned long long)N2);
    atomicAdd(ctr + C_COLUMNS, (unsigned long long)nc);
    atomicAdd(ctr + C_ACTIVE, (unsigned long long)total);
    atomicAdd(ctr + C_GRAZING, g);
    atomicAdd(ctr + C_ZEROED, (unsigned long long)(N2 - total) - g);
  }
}

// ------------------------------------------------------------------------------
// per-mode solve
// ------------------------------------------------------------------------------
template <typename B> struct Bulk {
  cx<B> A[MAX_M1][MAX_M + 1];
  cx<B> G[MAX_M1][MAX_M1 + 1];
  cx<B> V[MAX_M1][MAX_M1];  // reflector j: V[j][0 .. n-j-2]
  B beta[MAX_M1];
  cx<B> p[MAX_M1], wv[MAX_M1];
};

struct Shared {
  union { Bulk<double> d; Bulk<float> f; } u;
  double2 E[MAX_M1], Pz[MAX_M], b[MAX_M1], c[MAX_M1], y[MAX_M1], r[MAX_M1], t[MAX_M];
  double2 ph[MAX_M1], Vt[MAX_M], Ut[MAX_M], F[MAX_M], Bk[MAX_M];
  double d[MAX_M1], e[MAX_M1];
  double tr, alpha, bnorm2, dnu;
  double2 gamma, kz;
  int fallback;
};

template <typename B> __device__ __forceinline__ Bulk<B>& bulk(Shared& s);
template <> __device__ __forceinline__ Bulk<double>& bulk<double>(Shared& s) { return s.u.d; }
template <> __device__ __forceinline__ Bulk<float>& bulk<float>(Shared& s) { return s.u.f; }

__device__ __forceinline__ double2 warp_sum(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float2 warp_sum(float2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// exp(i kz d) for kz real (propagating) or purely imaginary (evanescent), d >= 0
__device__ __forceinline__ double2 exp_ikz(double2 kz, double d) {
  const double mag = exp(-kz.y * d);
  double s, c;
  sincos(kz.x * d, &s, &c);
  return make_double2(mag * c, mag * s);
}

// A_nu and G = A A^H in precision B; tr(G) in FP64.
template <typename B>
__device__ void build_gram(Shared& S, int n, int m) {
  Bulk<B>& K = bulk<B>(S);
  for (int e = threadIdx.x; e < n * m; e += ST) {
    const int k = e / m, l = e - k * m;
    K.A[k][l] = from_d<B>(S.gamma * (S.E[k] * S.Pz[l]));
  }
  __syncthreads();
  const int nt = n * (n + 1) / 2;
  for (int e = threadIdx.x; e < nt; e += ST) {
    int i = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > e) --i;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    const int j = e - i * (i + 1) / 2;
    cx<B> acc = czero<B>();
    for (int l = 0; l < m; ++l) acc = acc + mulc(K.A[i][l], K.A[j][l]);
    if (i == j) acc.y = B(0);
    K.G[i][j] = acc;
    K.G[j][i] = conjx(acc);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) t += (double)K.G[i][i].x;
    t = warp_sum(t);
    if (threadIdx.x == 0) S.tr = t;
  }
  __syncthreads();
}

// Householder reduction of the Hermitian G (lower part) to tridiagonal form, then
// d, |e| and the phases that make the off-diagonal real.
template <typename B>
__device__ void tridiagonalize(Shared& S, int n) {
  Bulk<B>& K = bulk<B>(S);
  for (int j = 0; j + 2 < n; ++j) {
    const int ml = n - j - 1;  // length of the column below the diagonal
    if (threadIdx.x < 32) {
      const int r = threadIdx.x;
      cx<B> x = (r < ml) ? K.G[j + 1 + r][j] : czero<B>();
      const B nx2 = warp_sum(abs2(x));
      const cx<B> x0 = K.G[j + 1][j];
      const B nx = sqrt(nx2);
      const B ax0 = sqrt(abs2(x0));
      B beta = B(0);
      cx<B> ah = czero<B>();
      if (nx > B(0)) {
        const cx<B> ph = ax0 > B(0) ? mk<B>(x0.x / ax0, x0.y / ax0) : mk<B>(B(1), B(0));
        ah = mk<B>(-ph.x * nx, -ph.y * nx);
        if (r == 0) x = mk<B>(ph.x * (ax0 + nx), ph.y * (ax0 + nx));
        beta = B(1) / (nx * (nx + ax0));
      }
      if (r < ml) K.V[j][r] = x;
      if (r == 0) {
        K.beta[j] = beta;
        K.G[j + 1][j] = ah;
        K.G[j][j + 1] = conjx(ah);
      }
    }
    __syncthreads();
    const B beta = K.beta[j];
    if (beta == B(0)) continue;  // uniform across the block
    // p = beta S v, S = trailing block; 4 threads per row
    {
      const int r = threadIdx.x >> 2, part = threadIdx.x & 3;
      cx<B> acc = czero<B>();
      if (r < ml)
        for (int cc = part; cc < ml; cc += 4) acc = acc + K.G[j + 1 + r][j + 1 + cc] * K.V[j][cc];
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
      if (r < ml && part == 0) K.p[r] = beta * acc;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int r = threadIdx.x;
      const cx<B> vr = r < ml ? K.V[j][r] : czero<B>();
      const cx<B> pr = r < ml ? K.p[r] : czero<B>();
      const B kk = B(0.5) * beta * warp_sum(vr.x * pr.x + vr.y * pr.y);  // (beta/2) Re(v^H p)
      if (r < ml) K.wv[r] = pr - kk * vr;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ml * ml; e += ST) {
      const int r = e / ml, cc = e - r * ml;
      const cx<B> v_r = K.V[j][r], v_c = K.V[j][cc], w_r = K.wv[r], w_c = K.wv[cc];
      K.G[j + 1 + r][j + 1 + cc] = K.G[j + 1 + r][j + 1 + cc] - (mulc(v_r, w_c) + mulc(w_r, v_c));
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double2 ph = make_double2(1.0, 0.0);
    for (int i = 0; i < n; ++i) {
      S.d[i] = (double)K.G[i][i].x;
      S.ph[i] = ph;
      if (i + 1 < n) {
        const double2 ei = to_d(K.G[i + 1][i]);
        const double ae = sqrt(abs2(ei));
        S.e[i] = ae;
        if (ae > 0.0) ph = ph * make_double2(ei.x / ae, ei.y / ae);
      }
    }
  }
  __syncthreads();
}

// out = D^H Q^H in (forward reflectors, ascending j), FP64 arithmetic, warp 0.
template <typename B>
__device__ void apply_QH(Shared& S, int n, const double2* in, double2* out) {
  Bulk<B>& K = bulk<B>(S);
  if (threadIdx.x < 32) {
    const int r = threadIdx.x;
    double2 x = r < n ? in[r] : make_double2(0, 0);
    for (int j = 0; j + 2 < n; ++j) {
      const double beta = (double)K.beta[j];
      if (beta == 0.0) continue;
      const int ml = n - j - 1;
      const bool mine = r > j && r - j - 1 < ml;
      const double2 v = mine ? to_d(K.V[j][r - j - 1]) : make_double2(0, 0);
      const double2 dot = warp_sum(cmul_conj_a(v, x));  // v^H x
      if (mine) x = x - beta * (v * dot);
    }
    if (r < n) out[r] = cmul_conj_a(S.ph[r], x);
  }
  __syncwarp();
}

// out = Q D in (reflectors applied in descending j), warp 0.
template <typename B>
__device__ void apply_Q(Shared& S, int n, const double2* in, double2* out) {
  Bulk<B>& K = bulk<B>(S);
  if (threadIdx.x < 32) {
    const int r = threadIdx.x;
    double2 x = r < n ? S.ph[r] * in[r] : make_double2(0, 0);
    for (int j = n - 3; j >= 0; --j) {
      const double beta = (double)K.beta[j];
      if (beta == 0.0) continue;
      const int ml = n - j - 1;
      const bool mine = r > j && r - j - 1 < ml;
      const double2 v = mine ? to_d(K.V[j][r - j - 1]) : make_double2(0, 0);
      const double2 dot = warp_sum(cmul_conj_a(v, x));
      if (mine) x = x - beta * (v * dot);
    }
    if (r < n) out[r] = x;
  }
  __syncwarp();
}

// (T + a I) z = rhs, T real symmetric tridiagonal (d, e); single thread.
__device__ void tri_solve(const double* d, const double* e, int n, double a, const double2* rhs,
                          double2* z) {
  double lp[MAX_M1], mu[MAX_M1];
  lp[0] = d[0] + a;
  mu[0] = 0.0;
  for (int i = 1; i < n; ++i) {
    mu[i] = e[i - 1] / lp[i - 1];
    lp[i] = d[i] + a - mu[i] * e[i - 1];
  }
  z[0] = rhs[0];
  for (int i = 1; i < n; ++i) z[i] = rhs[i] - mu[i] * z[i - 1];
  for (int i = 0; i < n; ++i) z[i] = (1.0 / lp[i]) * z[i];
  for (int i = n - 2; i >= 0; --i) z[i] = z[i] - mu[i + 1] * z[i + 1];
}

// Discrepancy root in log(alpha); thread 0.  Returns alpha, sets flags.
__device__ double find_alpha(Shared& S, int n, const Problem& P, int om, bool& floor_case,
                             bool& capped) {
  double2 z[MAX_M1], sv[MAX_M1];
  floor_case = false;
  capped = false;
  if (P.alpha_mode == 1) return P.alpha_given[om];
  const double lo_a = P.alpha_rel * S.tr;
  const double target = S.dnu * S.dnu;
  tri_solve(S.d, S.e, n, lo_a, S.c, z);
  double zz = 0.0;
  for (int i = 0; i < n; ++i) zz += abs2(z[i]);
  if (lo_a * lo_a * zz >= target) { floor_case = true; return lo_a; }
  const double bn = sqrt(S.bnorm2);
  const double hi_a = fmax(S.tr * S.dnu / (bn - S.dnu), lo_a);
  double tl = log(lo_a), th = log(hi_a);
  double t = 0.5 * (tl + th);
  const double lt = log(target);
  int it = 0;
  for (; it < P.max_iter; ++it) {
    const double a = exp(t);
    tri_solve(S.d, S.e, n, a, S.c, z);
    zz = 0.0;
    for (int i = 0; i < n; ++i) zz += abs2(z[i]);
    const double fa = a * a * zz;
    const double g = log(fa) - lt;
    if (g > 0) th = t; else tl = t;
    if (fabs(g) < 1e-14 || th - tl < 1e-15 * fmax(1.0, fabs(t))) break;
    tri_solve(S.d, S.e, n, a, z, sv);
    double zs = 0.0;
    for (int i = 0; i < n; ++i) zs += z[i].x * sv[i].x + z[i].y * sv[i].y;
    const double df = 2.0 * a * zz - 2.0 * a * a * zs;
    const double gp = a * df / fa;
    double tn = (gp > 0.0) ? t - g / gp : 0.5 * (tl + th);
    if (!(tn > tl && tn < th)) tn = 0.5 * (tl + th);
    t = tn;
  }
  capped = (it == P.max_iter);
  return exp(t);
}

// x = A^H y (FP64, A rebuilt from E, Pz) for l < m; all threads.
__device__ __forceinline__ double2 a_entry(const Shared& S, int k, int l) {
  return S.gamma * (S.E[k] * S.Pz[l]);
}

// residual r = b - A (A^H y) - alpha y in FP64 (mixed-precision refinement)
__device__ void residual_fp64(Shared& S, int n, int m) {
  for (int l = threadIdx.x; l < m; l += ST) {
    double2 acc = make_double2(0, 0);
    for (int k = 0; k < n; ++k) acc = acc + cmul_conj_a(a_entry(S, k, l), S.y[k]);
    S.t[l] = acc;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += ST) {
    double2 acc = make_double2(0, 0);
    for (int l = 0; l < m; ++l) acc = acc + a_entry(S, k, l) * S.t[l];
    S.r[k] = S.b[k] - acc - S.alpha * S.y[k];
  }
  __syncthreads();
}

template <typename B>
__device__ void factor_and_root(Shared& S, int n, int m, const Problem& P, int om,
                                unsigned long long* ctr) {
  build_gram<B>(S, n, m);
  tridiagonalize<B>(S, n);
  apply_QH<B>(S, n, S.b, S.c);
  __syncthreads();
  if (threadIdx.x == 0) {
    bool fl, cap;
    S.alpha = find_alpha(S, n, P, om, fl, cap);
    if (fl) atomicAdd(ctr + C_ALPHA_FLOOR, 1ull);
    if (cap) atomicAdd(ctr + C_ROOT_CAPPED, 1ull);
  }
  __syncthreads();
}

// y = Q D (T + alpha I)^-1 D^H Q^H rhs  (rhs, y in shared memory)
template <typename B>
__device__ void tikhonov_apply(Shared& S, int n, const double2* rhs, double2* y) {
  apply_QH<B>(S, n, rhs, S.c);
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 z[MAX_M1];
    tri_solve(S.d, S.e, n, S.alpha, S.c, z);
    for (int i = 0; i < n; ++i) S.r[i] = z[i];
  }
  __syncthreads();
  apply_Q<B>(S, n, S.r, y);
  __syncthreads();
}

template <typename B, bool MIXED>
__global__ void __launch_bounds__(ST)
k_solve(Problem P, const cx<B>* __restrict__ wt, const int* __restrict__ act,
        const int* __restrict__ count, const double* __restrict__ dnu_arr,
        cx<B>* __restrict__ prof, double* __restrict__ alpha_out, unsigned long long* __restrict__ ctr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared& S = *reinterpret_cast<Shared*>(smem_raw);
  const int N = P.n, n = P.m1, m = P.m;
  const long long N2 = (long long)N * N;
  long long total = 0;
  for (int w = 0; w < P.n_omega; ++w) total += count[w];
  for (long long item = blockIdx.x; item < total; item += gridDim.x) {
    int om = 0;
    long long i = item;
    while (i >= count[om]) { i -= count[om]; ++om; }
    const int nu = act[om * N2 + i];
    const int i2 = nu / N, i1 = nu - i2 * N;
    const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
    const double k0 = P.omega[om] / P.c0;
    const double om2 = P.omega[om] * P.omega[om];
    const double kn = 2.0 * M_PI / P.period;
    const double q = k0 * k0 - kn * kn * (double)(m1 * m1 + m2 * m2);
    const double2 kz = q >= 0.0 ? make_double2(sqrt(q), 0.0) : make_double2(0.0, sqrt(-q));
    // gamma = omega^2 h_z (-i / (2 k_z))
    const double g0 = 0.5 * om2 * P.hz;
    const double2 gamma = q >= 0.0 ? make_double2(0.0, -g0 / kz.x) : make_double2(-g0 / kz.y, 0.0);
    const double ztop = P.z1 + (m - 0.5) * P.hz;
    if (threadIdx.x == 0) {
      S.kz = kz;
      S.gamma = gamma;
      S.dnu = dnu_arr[om];
      S.fallback = 0;
    }
    for (int k = threadIdx.x; k < n; k += ST) {
      S.b[k] = to_d(wt[((long long)om * n + k) * N2 + nu]);
      S.E[k] = exp_ikz(kz, P.zy[k] - ztop);
    }
    for (int l = threadIdx.x; l < m; l += ST) S.Pz[l] = exp_ikz(kz, ztop - (P.z1 + (l + 0.5) * P.hz));
    __syncthreads();
    if (threadIdx.x < 32) {
      double bb = 0.0;
      for (int k = threadIdx.x; k < n; k += 32) bb += abs2(S.b[k]);
      bb = warp_sum(bb);
      if (threadIdx.x == 0) S.bnorm2 = bb;
    }
    __syncthreads();
    factor_and_root<B>(S, n, m, P, om, ctr);
    bool fp64_path = !MIXED;
    if (MIXED) {
      if (S.alpha < P.fp64_switch * S.tr) {
        fp64_path = true;
        if (threadIdx.x == 0) atomicAdd(ctr + C_FP64_FALLBACK, 1ull);
        factor_and_root<double>(S, n, m, P, om, ctr);
      }
    }
    if (fp64_path) {
      tikhonov_apply<double>(S, n, S.b, S.y);
    } else {
      tikhonov_apply<B>(S, n, S.b, S.y);
      for (int it = 0; it < P.refine_iters; ++it) {
        residual_fp64(S, n, m);
        tikhonov_apply<B>(S, n, S.r, S.F);  // correction in S.F
        for (int k = threadIdx.x; k < n; k += ST) S.y[k] = S.y[k] + S.F[k];
        __syncthreads();
      }
      if (threadIdx.x == 0) atomicAdd(ctr + C_REFINE_ITERS, (unsigned long long)P.refine_iters);
    }
    // V~ = A^H y
    for (int l = threadIdx.x; l < m; l += ST) {
      double2 acc = make_double2(0, 0);
      for (int k = 0; k < n; ++k) acc = acc + cmul_conj_a(a_entry(S, k, l), S.y[k]);
      S.Vt[l] = acc;
    }
    __syncthreads();
    // U~ = U~0 + gamma (F + B): forward/backward sweeps of T_nu's geometric kernel
    if (threadIdx.x == 0 || threadIdx.x == 32) {
      const double2 qz = exp_ikz(kz, P.hz);
      if (threadIdx.x == 0) {
        double2 f = make_double2(0, 0);
        for (int l = 0; l < m; ++l) { f = qz * f + S.Vt[l]; S.F[l] = f; }
      } else {
        double2 bk = make_double2(0, 0);
        S.Bk[m - 1] = bk;
        for (int l = m - 2; l >= 0; --l) { bk = qz * (bk + S.Vt[l + 1]); S.Bk[l] = bk; }
      }
    }
    __syncthreads();
    cx<B>* out = prof + ((long long)om * N2 + i) * 2 * m;
    for (int l = threadIdx.x; l < m; l += ST) {
      double2 u = S.gamma * (S.F[l] + S.Bk[l]);
      if (nu == 0) {
        double s, c;
        sincos(-k0 * (P.z1 + (l + 0.5) * P.hz), &s, &c);
        u = u + make_double2((double)N2 * c, (double)N2 * s);
      }
      out[l] = from_d<B>(S.Vt[l]);
      out[m + l] = from_d<B>(u);
    }
    if (threadIdx.x == 0 && alpha_out) alpha_out[om * N2 + nu] = S.alpha;
    __syncthreads();
  }
}

int solve_grid() {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = 3 * (sms > 0 ? sms : 152);
  }
  return grid;
}

template <typename B, bool MIXED>
cudaError_t solve_impl(const Problem& P, const Work<B>& w, cudaStream_t s) {
  const size_t smem = sizeof(Shared);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_solve<B, MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_solve<B, MIXED><<<solve_grid(), ST, smem, s>>>(P, w.wt, w.act, w.count, w.dnu, w.prof, w.alpha_out,
                                                   w.ctr);
  return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_classify(const Problem& P, const Work<R>& w, cudaStream_t s) {
  k_classify<<<P.n_omega, CT, 0, s>>>(P, w.norms, w.slot, w.act, w.cols, w.ncol, w.count, w.dnu, w.ctr);
  return cudaGetLastError();
}
template cudaError_t launch_classify<double>(const Problem&, const Work<double>&, cudaStream_t);
template cudaError_t launch_classify<float>(const Problem&, const Work<float>&, cudaStream_t);

cudaError_t launch_solve_fp64(const Problem& P, const Work<double>& w, cudaStream_t s) {
  return solve_impl<double, false>(P, w, s);
}
cudaError_t launch_solve_mixed(const Problem& P, const Work<float>& w, cudaStream_t s) {
  return solve_impl<float, true>(P, w, s);
}

}  // namespace fl
