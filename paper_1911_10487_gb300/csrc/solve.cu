// Per-mode part of Algorithm 2: classification of the modes (discrepancy test)
// and, for every active mode nu, the regularised solution of the SLAE of eq. (8)
// followed by eq. (9) (Sec. 4 steps 1-2, Sec. 5.2).
//
// For every active mode one thread block:
//   1. builds A_nu[k, l] = omega^2 h_z K_nu(z_k - z'_l) (FP64) with the Weyl closed
//      form K_nu(dz) = -i exp(i k_z |dz|)/(2 k_z) (horizontal Fourier transform of
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
//      applied as one forward and one backward first-order recurrence (the z part
//      of the zero-padded convolution u = u0 + G * w, done exactly).
//
// Cost model on this GPU: a dependent FP64 operation costs ~64 cycles and an FP64
// division ~640, while FP32 runs at 64x the FP64 rate.  So every sequential chain
// (Householder scalars, tridiagonal solves, the root-find) runs in FP32 wherever
// the precision allows, and FP64 is kept to parallel matrix-vector products.
//  FS_FP64 : steps 2-3 in FP64; the root is seeded by an FP32 root-find on T and
//            finished by FP64 Newton steps (reciprocals by Newton-Raphson from an
//            FP32 seed instead of FP64 division).
//  FS_MIXED: steps 2-4 in FP32; y is refined against the FP64 residual
//            b - A (A^H y) - alpha y, and alpha gets one FP64 Newton correction
//            from the refined residual.  Modes whose alpha/tr(G) falls below
//            fp64_switch (where the FP32 factorisation no longer converges the
//            refinement) take the FS_FP64 route.
#include <math.h>

#include "pipeline.cuh"

namespace fl {

namespace {

constexpr int ST = 128;  // threads per solve block (>= 2 MAX_M and >= 4 MAX_M1)
static_assert(ST >= 2 * MAX_M && ST >= 4 * MAX_M1, "solve block too small");

// ------------------------------------------------------------------------------
// classification: one block per frequency, integer arithmetic only
// ------------------------------------------------------------------------------
constexpr int CT = 1024;

__global__ void __launch_bounds__(CT)
k_classify(Problem P, const double* __restrict__ norms, const double* __restrict__ partial, int n_partial,
           int* __restrict__ slot, int* __restrict__ act, int* __restrict__ cols, int* __restrict__ ncol,
           int* __restrict__ count, double* __restrict__ dnu_out, unsigned long long* __restrict__ ctr) {
  const int om = blockIdx.x;
  const int N = P.n;
  const int N2 = N * N;
  const double* nrm = norms + (long long)om * N2;
  __shared__ int scan[CT];
  __shared__ int colflag[MAX_N];
  __shared__ unsigned cgraz[CT / 32];
  __shared__ long long thr_bits;
  for (int j = threadIdx.x; j < N; j += CT) colflag[j] = 0;
  if (threadIdx.x == 0) {
    // ||W||^2 = sum_nu ||W~_nu||^2 / N^2 (Parseval); partial sums in a fixed order
    double s = 0.0;
    for (int i = 0; i < n_partial; ++i) s += partial[(long long)om * n_partial + i];
    const double wnorm = sqrt(s / (double)N2);
    const double dnu = P.tau * fmax(P.delta, P.delta_floor) * wnorm;
    dnu_out[om] = dnu;
    thr_bits = __double_as_longlong(dnu * dnu);
  }
  __syncthreads();
  // non-negative doubles order like their bit patterns: the test nrm > dnu^2 is
  // an integer comparison (no FP64 pipe on a single SM)
  const long long tb = thr_bits;
  const int glo = P.graz_lo[om], ghi = P.graz_hi[om];
  const int C = (N2 + CT - 1) / CT;
  const int v0 = threadIdx.x * C, v1 = min(N2, v0 + C);
  const long long* nb = reinterpret_cast<const long long*>(nrm);
  int cnt = 0;
  unsigned ngz = 0;
  for (int v = v0; v < v1; ++v) {
    const int i2 = v / N, i1 = v - i2 * N;
    const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
    const int msq = m1 * m1 + m2 * m2;
    const bool graz = msq >= glo && msq <= ghi;
    ngz += graz;
    cnt += !graz && (P.alpha_mode == 1 || nb[v] > tb);
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
    const int msq = m1 * m1 + m2 * m2;
    const bool graz = msq >= glo && msq <= ghi;
    if (!graz && (P.alpha_mode == 1 || nb[v] > tb)) {
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
  if (threadIdx.x < 32) {  // compact the column list in order, one warp
    colflag[0] = 1;  // the incident plane wave lives at nu = 0
    int base = 0;
    for (int j0 = 0; j0 < N; j0 += 32) {
      const int j = j0 + threadIdx.x;
      const bool f = j < N && colflag[j];
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (f) cols[om * N + base + __popc(bal & ((1u << threadIdx.x) - 1u))] = j;
      base += __popc(bal);
    }
    if (threadIdx.x == 0) {
      ncol[om] = base;
      count[om] = total;
      unsigned long long g = 0;
      for (int w = 0; w < CT / 32; ++w) g += cgraz[w];
      atomicAdd(ctr + C_MODES, (unsigned long long)N2);
      atomicAdd(ctr + C_COLUMNS, (unsigned long long)base);
      atomicAdd(ctr + C_ACTIVE, (unsigned long long)total);
      atomicAdd(ctr + C_GRAZING, g);
      atomicAdd(ctr + C_ZEROED, (unsigned long long)(N2 - total) - g);
    }
  }
}

// ------------------------------------------------------------------------------
// scalar helpers
// ------------------------------------------------------------------------------

// Reciprocal of a normal double by Newton-Raphson (y <- y (2 - x y), quadratic
// convergence) from an FP32 seed of the mantissa; two steps take the 24-bit seed
// past 53 bits.  Exponent handled on the bit pattern.  Four dependent FP64
// operations instead of a full FP64 division.
__device__ __forceinline__ double rcp64(double x) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  if (ex == 0 || ex == 0x7ff) return 1.0 / x;  // zero, subnormal, inf, nan
  const double m = __longlong_as_double((bits & ~(0x7ffLL << 52)) | (1023LL << 52));  // [1,2), sign kept
  double y = (double)(1.0f / (float)m);
  double t = fma(-m, y, 1.0);
  y = fma(y, t, y);
  t = fma(-m, y, 1.0);
  y = fma(y, t, y);
  // y ~ 1/m in (0.5, 1]; scale by 2^-(ex-1023) through the exponent field
  const long long yb = __double_as_longlong(y);
  const int ey = (int)((yb >> 52) & 0x7ff) - (ex - 1023);
  if (ey <= 0 || ey >= 0x7ff) return 1.0 / x;
  return __longlong_as_double((yb & ~(0x7ffLL << 52)) | ((long long)ey << 52));
}

template <typename T> __device__ __forceinline__ T rcp(T x);
template <> __device__ __forceinline__ float rcp<float>(float x) { return __fdividef(1.0f, x); }  // ~2 ulp
template <> __device__ __forceinline__ double rcp<double>(double x) { return rcp64(x); }

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

// ------------------------------------------------------------------------------
// shared state of one block
// ------------------------------------------------------------------------------
template <typename B> struct Bulk {
  cx<B> G[MAX_M1][MAX_M1 + 1];
  cx<B> V[MAX_M1][MAX_M1];  // reflector j: V[j][0 .. n-j-2]
  B beta[MAX_M1];
  cx<B> p[MAX_M1], wv[MAX_M1];
};
struct BulkF : Bulk<float> {
  float2 A[MAX_M1][MAX_M + 1];   // A_nu / sqrt(tr G) in FP32 (mixed precision)
  float2 Q[MAX_M1][MAX_M1 + 1];  // Q D formed explicitly (mixed precision)
};

struct Shared {
  double2 A[MAX_M1][MAX_M + 1];  // A_nu in FP64
  union { Bulk<double> d; BulkF f; } u;
  double2 E[MAX_M1], Pz[MAX_M], b[MAX_M1], c[MAX_M1], y[MAX_M1], r[MAX_M1], z[MAX_M1];
  double2 ph[MAX_M1], Vt[MAX_M], t[MAX_M], F[MAX_M], Bk[MAX_M];
  double d[MAX_M1], e[MAX_M1];     // tridiagonal T (FP64 route: of G; scaled by 1/tr after the factor)
  float d32[MAX_M1], e32[MAX_M1];  // T / tr in FP32
  float2 c32[MAX_M1], cz[MAX_M1];
  double tr, sb, inv_sb, dnu, lo, hi, a_s, red[8];  // a_s = alpha / tr
  int fp64;
};

template <typename B> __device__ __forceinline__ Bulk<B>& bulk(Shared& s);
template <> __device__ __forceinline__ Bulk<double>& bulk<double>(Shared& s) { return s.u.d; }
template <> __device__ __forceinline__ Bulk<float>& bulk<float>(Shared& s) { return s.u.f; }

// G = A A^H in precision B: FP64 from S.A, or FP32 from the scaled copy (G / tr)
template <typename B>
__device__ void gram(Shared& S, int n, int m) {
  Bulk<B>& K = bulk<B>(S);
  const int nt = n * (n + 1) / 2;
  for (int e = threadIdx.x; e < nt; e += ST) {
    int i = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    while (i * (i + 1) / 2 > e) --i;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    const int j = e - i * (i + 1) / 2;
    cx<B> acc = czero<B>();
    if constexpr (sizeof(B) == 8) {
      for (int l = 0; l < m; ++l) acc = acc + mulc(S.A[i][l], S.A[j][l]);
    } else {
      for (int l = 0; l < m; ++l) acc = acc + mulc(S.u.f.A[i][l], S.u.f.A[j][l]);
    }
    if (i == j) acc.y = B(0);
    K.G[i][j] = acc;
    K.G[j][i] = conjx(acc);
  }
  __syncthreads();
}

// Householder reduction of the Hermitian G to tridiagonal form, then d, |e| and
// the phases D (prefix products of e_i/|e_i|) that make the off-diagonal real.
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
      const B ax02 = abs2(x0);
      B beta = B(0);
      cx<B> ah = czero<B>();
      if (nx2 > B(0)) {
        const B nx = sqrt(nx2);
        const B ax0 = sqrt(ax02);
        const B inv = ax0 > B(0) ? rcp<B>(ax0) : B(0);
        const cx<B> ph = ax0 > B(0) ? mk<B>(x0.x * inv, x0.y * inv) : mk<B>(B(1), B(0));
        ah = mk<B>(-ph.x * nx, -ph.y * nx);
        if (r == 0) x = mk<B>(ph.x * (ax0 + nx), ph.y * (ax0 + nx));
        beta = rcp<B>(nx * (nx + ax0));
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
    {  // p = beta S v, S = trailing block; 4 threads per row
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
    // S -= v w^H + w v^H on the lower triangle, mirrored to the upper one
    const int nl = ml * (ml + 1) / 2;
    for (int e = threadIdx.x; e < nl; e += ST) {
      int r = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
      while (r * (r + 1) / 2 > e) --r;
      while ((r + 1) * (r + 2) / 2 <= e) ++r;
      const int cc = e - r * (r + 1) / 2;
      const cx<B> v_r = K.V[j][r], v_c = K.V[j][cc], w_r = K.wv[r], w_c = K.wv[cc];
      cx<B> g = K.G[j + 1 + r][j + 1 + cc] - (mulc(v_r, w_c) + mulc(w_r, v_c));
      if (r == cc) g.y = B(0);
      K.G[j + 1 + r][j + 1 + cc] = g;
      K.G[j + 1 + cc][j + 1 + r] = conjx(g);
    }
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    const int i = threadIdx.x;
    cx<B> u = mk<B>(B(1), B(0));
    B ae = B(0);
    if (i < n) {
      S.d[i] = (double)K.G[i][i].x;
      if (sizeof(B) == 4) S.d32[i] = (float)K.G[i][i].x;
    }
    if (i + 1 < n) {
      const cx<B> ei = K.G[i + 1][i];
      ae = sqrt(abs2(ei));
      if (ae > B(0)) {
        const B inv = rcp<B>(ae);
        u = mk<B>(ei.x * inv, ei.y * inv);
      }
      S.e[i] = (double)ae;
      if (sizeof(B) == 4) S.e32[i] = (float)ae;
    }
    // inclusive prefix product of u over the lanes: ph[i+1] = u_0 ... u_i
    for (int off = 1; off < 32; off <<= 1) {
      const B ox = __shfl_up_sync(0xffffffffu, u.x, off);
      const B oy = __shfl_up_sync(0xffffffffu, u.y, off);
      if (i >= off) u = mk<B>(ox, oy) * u;
    }
    if (i + 1 < n) S.ph[i + 1] = to_d(u);
    if (i == 0) S.ph[0] = make_double2(1.0, 0.0);
  }
  __syncthreads();
}

// out = s * D^H Q^H in  (reflectors, ascending), warp 0, arithmetic in W.
template <typename B, typename W>
__device__ void apply_QH(Shared& S, int n, const double2* in, double s, cx<W>* out) {
  Bulk<B>& K = bulk<B>(S);
  if (threadIdx.x < 32) {
    const int r = threadIdx.x;
    cx<W> x = r < n ? from_d<W>(s * in[r]) : czero<W>();
    for (int j = 0; j + 2 < n; ++j) {
      const W beta = (W)K.beta[j];
      if (beta == W(0)) continue;
      const bool mine = r > j && r < n;  // lanes of the reflector's rows only
      const cx<W> v = mine ? from_d<W>(to_d(K.V[j][r - j - 1])) : czero<W>();
      const cx<W> dot = warp_sum(cmul_conj_a(v, x));  // v^H x
      if (mine) x = x - beta * (v * dot);
    }
    if (r < n) out[r] = cmul_conj_a(from_d<W>(S.ph[r]), x);
  }
  __syncwarp();
}

// out = s * Q D in  (reflectors, descending), warp 0, arithmetic in W.
template <typename B, typename W>
__device__ void apply_Q(Shared& S, int n, const cx<W>* in, double s, double2* out) {
  Bulk<B>& K = bulk<B>(S);
  if (threadIdx.x < 32) {
    const int r = threadIdx.x;
    cx<W> x = r < n ? from_d<W>(S.ph[r]) * in[r] : czero<W>();
    for (int j = n - 3; j >= 0; --j) {
      const W beta = (W)K.beta[j];
      if (beta == W(0)) continue;
      const bool mine = r > j && r < n;  // lanes of the reflector's rows only
      const cx<W> v = mine ? from_d<W>(to_d(K.V[j][r - j - 1])) : czero<W>();
      const cx<W> dot = warp_sum(cmul_conj_a(v, x));
      if (mine) x = x - beta * (v * dot);
    }
    if (r < n) out[r] = s * to_d(x);
  }
  __syncwarp();
}

// Q D formed explicitly in FP32 (mixed precision): backward accumulation of the
// reflectors on the identity, 4 threads per column, then column c times ph_c.
__device__ void form_QD(Shared& S, int n) {
  BulkF& K = S.u.f;
  const int col = threadIdx.x >> 2, part = threadIdx.x & 3;
  for (int e = threadIdx.x; e < n * n; e += ST) {
    const int r = e / n, c = e - r * n;
    K.Q[r][c] = make_float2(r == c ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  for (int j = n - 3; j >= 0; --j) {
    const float beta = K.beta[j];
    if (beta == 0.f) continue;
    const int ml = n - j - 1;
    float2 acc = make_float2(0.f, 0.f);
    if (col < n)
      for (int r = part; r < ml; r += 4) acc = acc + cmul_conj_a(K.V[j][r], K.Q[j + 1 + r][col]);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
    if (col < n)
      for (int r = part; r < ml; r += 4) K.Q[j + 1 + r][col] = K.Q[j + 1 + r][col] - beta * (K.V[j][r] * acc);
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += ST) {
    const int r = e / n, c = e - r * n;
    const double2 p = S.ph[c];
    K.Q[r][c] = K.Q[r][c] * make_float2((float)p.x, (float)p.y);
  }
  __syncthreads();
}

// out = s * (QD)^H in  (FP32 dense matvec, 4 threads per output)
__device__ void qd_h(Shared& S, int n, const double2* in, double s, float2* out) {
  const int k = threadIdx.x >> 2, part = threadIdx.x & 3;
  float2 acc = make_float2(0.f, 0.f);
  if (k < n)
    for (int j = part; j < n; j += 4) {
      const double2 v = s * in[j];
      acc = acc + cmul_conj_a(S.u.f.Q[j][k], make_float2((float)v.x, (float)v.y));
    }
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
  if (k < n && part == 0) out[k] = acc;
  __syncthreads();
}

// out = s * (QD) in
__device__ void qd(Shared& S, int n, const float2* in, double s, double2* out) {
  const int j = threadIdx.x >> 2, part = threadIdx.x & 3;
  float2 acc = make_float2(0.f, 0.f);
  if (j < n)
    for (int k = part; k < n; k += 4) acc = acc + S.u.f.Q[j][k] * in[k];
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
  if (j < n && part == 0) out[j] = s * to_d(acc);
  __syncthreads();
}

// (T + a I) z = rhs, T real symmetric tridiagonal (d, e); single thread.
// Returns false if a pivot is not positive (T + a I not numerically SPD).
template <typename T>
__device__ bool tri_solve(const T* d, const T* e, int n, T a, const cx<T>* rhs, cx<T>* z) {
  T mu[MAX_M1], il[MAX_M1];
  T lp = d[0] + a;
  if (!(lp > T(0))) return false;
  il[0] = rcp<T>(lp);
  mu[0] = T(0);
  z[0] = rhs[0];
  for (int i = 1; i < n; ++i) {
    mu[i] = e[i - 1] * il[i - 1];
    lp = d[i] + a - mu[i] * e[i - 1];
    if (!(lp > T(0))) return false;
    il[i] = rcp<T>(lp);
    z[i] = rhs[i] - mu[i] * z[i - 1];
  }
  for (int i = 0; i < n; ++i) z[i] = il[i] * z[i];
  for (int i = n - 2; i >= 0; --i) z[i] = z[i] - mu[i + 1] * z[i + 1];
  return true;
}

__device__ __forceinline__ float exp_t(float t) { return expf(t); }
__device__ __forceinline__ double exp_t(double t) { return exp(t); }
__device__ __forceinline__ float log_t(float t) { return logf(t); }
__device__ __forceinline__ double log_t(double t) { return log(t); }

// Safeguarded Newton in t = log(a) on g(t) = log(a^2 ||(T + a I)^-1 c||^2) - log(target),
// on the scaled problem (T = G / tr, c = D^H Q^H b / ||b||, a = alpha / tr), single
// thread.  [lo, hi] brackets the root (g(lo) < 0 < g(hi)); t0 is the start.
// Returns t; gp = dg/dt at the last point; ok = false on a breakdown.
template <typename T>
__device__ double newton_log_alpha(const T* d, const T* e, const cx<T>* c, int n, double lo, double hi,
                                   double target, double t0, double tol, int max_iter, double& gp_out,
                                   bool& ok, int& iters) {
  cx<T> z[MAX_M1], s[MAX_M1];
  T tl = log_t((T)lo), th = log_t((T)hi), t = (T)t0;
  const T lt = log_t((T)target);
  const T eps_t = sizeof(T) == 8 ? T(1e-15) : T(1e-7);
  gp_out = 0.0;
  ok = true;
  int it = 0;
  for (; it < max_iter; ++it) {
    const T a = exp_t(t);
    if (!tri_solve<T>(d, e, n, a, c, z)) { ok = false; break; }
    T zz = T(0);
    for (int i = 0; i < n; ++i) zz += abs2(z[i]);
    const T g = log_t(a * a * zz) - lt;
    if (g > T(0)) th = t; else tl = t;
    if (!tri_solve<T>(d, e, n, a, z, s)) { ok = false; break; }
    T zs = T(0);
    for (int i = 0; i < n; ++i) zs += z[i].x * s[i].x + z[i].y * s[i].y;
    const T gp = T(2) - T(2) * a * zs * rcp<T>(zz);  // d log(a^2 ||z||^2) / d log a
    gp_out = (double)gp;
    if (fabs(g) < (T)tol || th - tl < eps_t * fmax(T(1), fabs(t))) break;
    T tn = (gp > T(0)) ? t - g * rcp<T>(gp) : T(0.5) * (tl + th);
    if (!(tn > tl && tn < th)) tn = T(0.5) * (tl + th);
    t = tn;
  }
  iters = it;
  return (double)t;
}

// a^2 ||(T + a I)^-1 c||^2 in precision T; single thread.
template <typename T>
__device__ double phi2(const T* d, const T* e, const cx<T>* c, int n, double a, bool& ok) {
  cx<T> z[MAX_M1];
  ok = tri_solve<T>(d, e, n, (T)a, c, z);
  T zz = T(0);
  for (int i = 0; i < n; ++i) zz += abs2(z[i]);
  return a * a * (double)zz;
}

// r = b - A (A^H y) - alpha y in FP64 (S.t = A^H y as scratch); all threads
__device__ void residual_fp64(Shared& S, int n, int m, double alpha) {
  {  // 2 threads per column l (2 M <= blockDim); every lane reaches the shuffles
    const int l = threadIdx.x >> 1, h = threadIdx.x & 1;
    double2 acc = make_double2(0, 0);
    if (l < m)
      for (int k = h; k < n; k += 2) acc = acc + cmul_conj_a(S.A[k][l], S.y[k]);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
    if (l < m && h == 0) S.t[l] = acc;
  }
  __syncthreads();
  {  // 4 threads per row k
    const int k = threadIdx.x >> 2, h = threadIdx.x & 3;
    double2 acc = make_double2(0, 0);
    if (k < n)
      for (int l = h; l < m; l += 4) acc = acc + S.A[k][l] * S.t[l];
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
    if (k < n && h == 0) S.r[k] = S.b[k] - acc - alpha * S.y[k];
  }
  __syncthreads();
}

// block-wide sum of one double per thread (all threads get it)
__device__ double block_sum(Shared& S, double v) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) S.red[threadIdx.x >> 5] = v;
  __syncthreads();
  return (S.red[0] + S.red[1]) + (S.red[2] + S.red[3]);
}

// mixed precision: y += (QD)(T/tr + a_s I)^-1 (QD)^H r / tr, returns ||dy||^2/||y||^2
__device__ double refine_step(Shared& S, int n) {
  qd_h(S, n, S.r, S.inv_sb, S.c32);
  if (threadIdx.x == 0 && !tri_solve<float>(S.d32, S.e32, n, (float)S.a_s, S.c32, S.cz)) S.fp64 = 1;
  __syncthreads();
  if (S.fp64) return 0.0;  // FP32 model not positive definite here: caller takes the FP64 route
  qd(S, n, S.cz, S.sb / S.tr, S.z);
  double dd = 0.0, yy = 0.0;
  if (threadIdx.x < n) {
    S.y[threadIdx.x] = S.y[threadIdx.x] + S.z[threadIdx.x];
    dd = abs2(S.z[threadIdx.x]);
    yy = abs2(S.y[threadIdx.x]);
  }
  if (threadIdx.x < 32) {
    dd = warp_sum(dd);
    yy = warp_sum(yy);
    if (threadIdx.x == 0) S.red[4] = yy > 0.0 ? dd / yy : 0.0;
  }
  __syncthreads();
  return S.red[4];
}

// FP64 route: FP64 factorisation, FP32-seeded root on the scaled tridiagonal,
// FP64 Newton to full accuracy, y = Q D (T + alpha I)^-1 D^H Q^H b.
__device__ void solve_fp64(Shared& S, int n, int m, const Problem& P, int om, unsigned long long* ctr) {
  gram<double>(S, n, m);
  tridiagonalize<double>(S, n);
  const double inv_sb = rcp64(S.sb), inv_tr = rcp64(S.tr);
  apply_QH<double, double>(S, n, S.b, inv_sb, S.c);  // scaled: c = D^H Q^H b / ||b||
  __syncthreads();
  if (threadIdx.x < n) {  // scaled tridiagonal T / tr, and FP32 copies for the seed
    const int i = threadIdx.x;
    S.d[i] *= inv_tr;
    if (i + 1 < n) S.e[i] *= inv_tr;
    S.d32[i] = (float)S.d[i];
    if (i + 1 < n) S.e32[i] = (float)S.e[i];
    S.c32[i] = make_float2((float)S.c[i].x, (float)S.c[i].y);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double target = (S.dnu * inv_sb) * (S.dnu * inv_sb);
    const double lo = P.alpha_rel, hi = S.hi * inv_tr;
    bool ok = true;
    double a;
    if (P.alpha_mode == 1) {
      a = P.alpha_given[om] * inv_tr;
    } else if (phi2<double>(S.d, S.e, S.c, n, lo, ok) >= target) {
      a = lo;
      atomicAdd(ctr + C_ALPHA_FLOOR, 1ull);
    } else {
      double gp;
      bool ok32;
      int it32, it64;
      const double t_mid = 0.5 * (log(lo) + log(hi));
      double t = newton_log_alpha<float>(S.d32, S.e32, S.c32, n, lo, hi, target, t_mid, 1e-5, P.max_iter, gp,
                                         ok32, it32);
      if (!ok32 || !(t > log(lo) && t < log(hi))) t = t_mid;
      t = newton_log_alpha<double>(S.d, S.e, S.c, n, lo, hi, target, t, 1e-14, P.max_iter, gp, ok, it64);
      if (it64 >= P.max_iter) atomicAdd(ctr + C_ROOT_CAPPED, 1ull);
      a = exp(t);
    }
    S.a_s = a;
    tri_solve<double>(S.d, S.e, n, a, S.c, S.z);
  }
  __syncthreads();
  apply_Q<double, double>(S, n, S.z, S.sb * inv_tr, S.y);
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
    for (int k = threadIdx.x; k < n; k += ST) {
      S.b[k] = to_d(wt[((long long)om * n + k) * N2 + nu]);
      S.E[k] = gamma * exp_ikz(kz, P.zy[k] - ztop);
    }
    for (int l = threadIdx.x; l < m; l += ST) S.Pz[l] = exp_ikz(kz, ztop - (P.z1 + (l + 0.5) * P.hz));
    __syncthreads();
    // A (FP64), ||A||_F^2 = tr(G), ||b||^2
    double tr_part = 0.0;
    for (int e = threadIdx.x; e < n * m; e += ST) {
      const int k = e / m, l = e - k * m;
      const double2 a = S.E[k] * S.Pz[l];
      S.A[k][l] = a;
      tr_part += abs2(a);
    }
    const double tr = block_sum(S, tr_part);
    const double bb = block_sum(S, threadIdx.x < n ? abs2(S.b[threadIdx.x]) : 0.0);
    if (!(tr > 0.0)) {  // A_nu underflowed to zero: the mode carries no information, V~ = 0
      if (threadIdx.x == 0) {
        atomicAdd(ctr + C_ACTIVE, ~0ull);  // -1: counted as zeroed instead
        atomicAdd(ctr + C_ZEROED, 1ull);
        if (alpha_out) alpha_out[om * N2 + nu] = INFINITY;
      }
      cx<B>* out0 = prof + ((long long)om * N2 + i) * 2 * m;
      for (int l = threadIdx.x; l < m; l += ST) {
        double2 u = make_double2(0, 0);
        if (nu == 0) {
          double s0, c0;
          sincos(-k0 * (P.z1 + (l + 0.5) * P.hz), &s0, &c0);
          u = make_double2((double)N2 * c0, (double)N2 * s0);
        }
        out0[l] = czero<B>();
        out0[m + l] = from_d<B>(u);
      }
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) {
      S.tr = tr;
      S.sb = sqrt(bb);
      S.inv_sb = 1.0 / S.sb;
      S.dnu = dnu_arr[om];
      S.lo = P.alpha_rel * tr;
      S.hi = fmax(tr * S.dnu / (S.sb - S.dnu), S.lo);
      S.fp64 = MIXED ? 0 : 1;
    }
    __syncthreads();
    if (MIXED) {
      const double sa = rsqrt(tr);  // scaled in FP64 so that tiny tr(G) cannot underflow FP32
      for (int e = threadIdx.x; e < n * m; e += ST) {
        const int k = e / m, l = e - k * m;
        const double2 a = sa * S.A[k][l];
        S.u.f.A[k][l] = make_float2((float)a.x, (float)a.y);
      }
      __syncthreads();
      gram<float>(S, n, m);
      tridiagonalize<float>(S, n);
      form_QD(S, n);
      qd_h(S, n, S.b, S.inv_sb, S.c32);
      if (threadIdx.x == 0) {
        const double target = (S.dnu / S.sb) * (S.dnu / S.sb);
        const double lo = P.alpha_rel, hi = S.hi / S.tr;
        bool ok = true;
        int it;
        double a = 0.0, gp = 0.0;
        if (P.alpha_mode == 1) {
          a = P.alpha_given[om] / S.tr;
        } else {
          const double f_lo = phi2<float>(S.d32, S.e32, S.c32, n, lo, ok);
          if (ok && f_lo < target) {
            const double t_mid = 0.5 * (log(lo) + log(hi));
            const double t = newton_log_alpha<float>(S.d32, S.e32, S.c32, n, lo, hi, target, t_mid, 1e-6,
                                                     P.max_iter, gp, ok, it);
            a = exp(t);
          } else {
            ok = false;  // floor case (or FP32 breakdown): decided in FP64
          }
        }
        S.a_s = a;
        S.fp64 = (!ok || a < P.fp64_switch) ? 1 : 0;
        if (S.fp64) atomicAdd(ctr + C_FP64_FALLBACK, 1ull);
      }
      __syncthreads();
      if (!S.fp64) {
        // y by refinement against the FP64 residual, to ||dy|| <= 1e-9 ||y||
        for (int k = threadIdx.x; k < n; k += ST) { S.y[k] = make_double2(0, 0); S.r[k] = S.b[k]; }
        __syncthreads();
        const double alpha = S.a_s * S.tr;
        int sweeps = 0;
        for (double rel = 1.0; sweeps < P.refine_iters && rel > 1e-18 && !S.fp64; ++sweeps) {
          if (sweeps) residual_fp64(S, n, m, alpha);
          rel = refine_step(S, n);
        }
        if (threadIdx.x == 0) {
          atomicAdd(ctr + C_REFINE_ITERS, (unsigned long long)sweeps);
          if (S.fp64) atomicAdd(ctr + C_FP64_FALLBACK, 1ull);
        }
      }
    }
    if (S.fp64) solve_fp64(S, n, m, P, om, ctr);
    // V~ = A^H y (FP64), 2 threads per column
    {
      const int l = threadIdx.x >> 1, h = threadIdx.x & 1;
      double2 acc = make_double2(0, 0);
      if (l < m)
        for (int k = h; k < n; k += 2) acc = acc + cmul_conj_a(S.A[k][l], S.y[k]);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      if (l < m && h == 0) S.Vt[l] = acc;
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
      double2 u = gamma * (S.F[l] + S.Bk[l]);
      if (nu == 0) {
        double s, c;
        sincos(-k0 * (P.z1 + (l + 0.5) * P.hz), &s, &c);
        u = u + make_double2((double)N2 * c, (double)N2 * s);
      }
      out[l] = from_d<B>(S.Vt[l]);
      out[m + l] = from_d<B>(u);
    }
    if (threadIdx.x == 0 && alpha_out) alpha_out[om * N2 + nu] = S.a_s * S.tr;
    __syncthreads();
  }
}

int solve_grid() {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = 2 * (sms > 0 ? sms : 152);
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
  k_classify<<<P.n_omega, CT, 0, s>>>(P, w.norms, w.partial, w.n_partial, w.slot, w.act, w.cols, w.ncol,
                                      w.count, w.dnu, w.ctr);
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
