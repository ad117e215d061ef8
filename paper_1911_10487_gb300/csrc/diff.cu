// Derivatives of the reconstruction at a fixed Tikhonov parameter alpha_omega
// per frequency (Algorithm 2, Sec. 4, without the discrepancy search):
//
//   (W, log alpha) -> (xi, Phi),   Phi_omega = sum_nu ||A_nu V~_nu - W~_nu||^2.
//
// Per mode nu of frequency omega the matrix of eq. (8) is assembled as
// A_kl = E_k P_l (E_k = gamma e^{i k_z (z_k - z_top)}, P_l = e^{i k_z (z_top - z'_l)})
// and scaled to unit Frobenius norm, A^ = A / sqrt(tr), tr = ||A||_F^2:
//
//   G^ = A^ A^^H                      dense, FP64; depends on geometry and omega only,
//                                     computed once per plan (k_diff_gram)
//   H^ = G^ + alpha' I = L L^H        alpha' = alpha / tr; Cholesky per alpha (saved)
//   y' = H^^-1 b,  V~ = A^^H y' / sqrt(tr)     (= A^H (A A^H + alpha I)^-1 b, the
//                                     normal solution of Sec. 4 comment b, dual form)
//   U~ = U~0 + omega^2 T V~           eq. (9), two affine scans over the planes
//   Phi_nu = alpha'^2 ||y'||^2        (dual residual identity b - A V~ = alpha y)
//
// then V = F^-1[V~], u = F^-1[U~] and xi = Re(sum conj(u) V) / sum |u|^2 (step 3).
// The VJP and JVP reuse the saved factor L and y'; in scaled form
//   b-bar   = H^^-1 (A^ t / sqrt(tr) + 2 alpha'^2 Phi-bar y'),
//             t = V~-bar + (omega^2 T)^H U~-bar
//   lnalpha-bar = -alpha' Re(b-bar^H y') + 2 Phi-bar alpha'^2 ||y'||^2
//   y-dot'  = H^^-1 (b-dot - lnalpha-dot alpha' y'),  V~-dot = A^^H y-dot' / sqrt(tr)
//   Phi-dot = 2 alpha'^2 (lnalpha-dot ||y'||^2 + Re y'^H y-dot').
// Modes with no solution (grazing, or a matrix that underflowed, or alpha' beyond
// AP_MAX where V~ is zero in FP64) keep V~ = 0; their tape slot holds b, their
// residual.  Gradients use grad z = dL/dRe z + i dL/dIm z.
//
// The per-mode kernels run one warp per mode: lane k owns row k of H (and of L),
// the triangular solves broadcast the pivot value with a shuffle, and the
// Toeplitz kernel of eq. (9) is the warp scan of modes.cuh.  Per-frequency sums
// (Phi, lnalpha-bar, Phi-dot) go to per-block partials reduced in a fixed order,
// so results do not depend on scheduling.
#include <math.h>

#include "diff.cuh"
#include "modes.cuh"

namespace fl {

namespace {

constexpr int DW = 4;             // warps (modes in flight) per block
constexpr int GT = 128;           // threads of the normal-matrix kernel
constexpr double AP_MAX = 1e290;  // alpha' above this: H^ = alpha' I to FP64, V~ = 0

struct WarpMem {
  double2 H[DENSE_M1][DENSE_M1 + 1];  // H^ (lower triangle) -> Cholesky factor L
  double2 E[DENSE_M1];              // E_k / sqrt(sum |E|^2)
  double2 Pz[DENSE_M];              // P_l / sqrt(sum |P|^2)
  double2 v[DENSE_M], t[DENSE_M], F[DENSE_M], B[DENSE_M];
  double dinv[DENSE_M1];            // 1 / L_jj
};

struct ModeGeo {
  double2 gamma, q;  // omega^2 h_z (-i / 2 k_z);  e^{i k_z h_z}
  double tr, rs;     // ||A||_F^2, 1 / sqrt(tr)
  bool usable;
};

// Wavenumber, kernel factors and the scaled E, P of mode nu (one full warp).
__device__ ModeGeo mode_setup(const Problem& P, int om, long long nu, double2* E, double2* Pz) {
  const int lane = threadIdx.x & 31;
  const int N = P.n, n = P.m1, m = P.m;
  const int i2 = (int)(nu / N), i1 = (int)(nu - (long long)i2 * N);
  const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
  const int msq = m1 * m1 + m2 * m2;
  ModeGeo g;
  const bool grazing = msq >= P.graz_lo[om] && msq <= P.graz_hi[om];
  const double k0 = P.omega[om] / P.c0;
  const double kn = 2.0 * M_PI / P.period;
  const double qq = k0 * k0 - kn * kn * (double)msq;
  double2 kz = qq >= 0.0 ? make_double2(sqrt(qq), 0.0) : make_double2(0.0, sqrt(-qq));
  const double g0 = 0.5 * P.omega[om] * P.omega[om] * P.hz;
  if (grazing) {
    kz = make_double2(1.0, 0.0);  // k_z = 0: excluded; placeholder keeps the arithmetic finite
    g.gamma = make_double2(0.0, 0.0);
  } else {
    g.gamma = qq >= 0.0 ? make_double2(0.0, -g0 / kz.x) : make_double2(-g0 / kz.y, 0.0);
  }
  const double ztop = P.z1 + (m - 0.5) * P.hz;
  const double2 e = lane < n ? g.gamma * exp_ikz(kz, P.zy[lane] - ztop) : make_double2(0, 0);
  const int l0 = lane, l1 = lane + 32;
  const double2 p0 = l0 < m ? exp_ikz(kz, ztop - (P.z1 + (l0 + 0.5) * P.hz)) : make_double2(0, 0);
  const double2 p1 = l1 < m ? exp_ikz(kz, ztop - (P.z1 + (l1 + 0.5) * P.hz)) : make_double2(0, 0);
  const double sE = warp_sum(abs2(e));
  const double sP = warp_sum(abs2(p0) + abs2(p1));
  g.tr = sE * sP;
  g.usable = !grazing && g.tr > 0.0;
  g.rs = g.usable ? 1.0 / sqrt(g.tr) : 0.0;
  if (g.usable) {
    const double re = 1.0 / sqrt(sE), rp = 1.0 / sqrt(sP);
    if (lane < n) E[lane] = re * e;
    if (l0 < m) Pz[l0] = rp * p0;
    if (l1 < m) Pz[l1] = rp * p1;
  }
  g.q = exp_ikz(kz, P.hz);
  __syncwarp();
  return g;
}

__device__ __forceinline__ long long col_off(int j, int n) { return (long long)j * n - (long long)j * (j - 1) / 2; }

// packed lower triangle (column-major: column j holds rows j..n-1) <-> S.H
__device__ __forceinline__ void load_lower(WarpMem& S, const double2* __restrict__ src, int n, int lane) {
  for (int j = 0; j < n; ++j)
    if (lane < n - j) S.H[j + lane][j] = src[col_off(j, n) + lane];
  __syncwarp();
}
__device__ __forceinline__ void store_lower(double2* __restrict__ dst, const WarpMem& S, int n, int lane) {
  for (int j = 0; j < n; ++j)
    if (lane < n - j) dst[col_off(j, n) + lane] = S.H[j + lane][j];
}

// (row, column) of the packed lower triangle in column-major order (column j holds
// rows j..n-1), one entry per element, for the trailing updates of the Cholesky
// factorisation; built once per block for the problem's M1.
constexpr int MAX_P1 = DENSE_M1 * (DENSE_M1 + 1) / 2;
__device__ void build_rc(unsigned short* rc, int n) {
  const int P1 = n * (n + 1) / 2;
  for (int e = threadIdx.x; e < P1; e += blockDim.x) {
    int j = 0;
    while (col_off(j + 1, n) <= e) ++j;
    const int r = j + (int)(e - col_off(j, n));
    rc[e] = (unsigned short)(r << 8 | j);
  }
}

// In-place Cholesky H = L L^H of the lower triangle (right-looking).  The pivot
// column is scaled by lane (lane k, row k); the trailing update of step j -- the
// entries (r, c), j < c <= r, a contiguous suffix of the packed order -- is dealt
// evenly over the 32 lanes, so the FP64 pipe is not spent on idle lanes.  A pivot
// that is not positive (H not positive definite to rounding) is replaced by the
// smallest positive double and reported through `bad`.
__device__ void cholesky(WarpMem& S, int n, int lane, const unsigned short* rc, bool& bad) {
  const int P1 = n * (n + 1) / 2;
  for (int j = 0; j < n; ++j) {
    double d = S.H[j][j].x;
    if (!(d > 0.0)) { bad = true; d = 2.2250738585072014e-308; }
    const double ljj = sqrt(d), inv = rcp64(ljj);
    __syncwarp();
    if (lane == j) { S.H[j][j] = make_double2(ljj, 0.0); S.dinv[j] = inv; }
    if (lane > j && lane < n) S.H[lane][j] = inv * S.H[lane][j];
    __syncwarp();
    for (int e = (int)col_off(j + 1, n) + lane; e < P1; e += 32) {
      const int r = rc[e] >> 8, c = rc[e] & 255;
      S.H[r][c] = S.H[r][c] - mulc(S.H[r][j], S.H[c][j]);
    }
    __syncwarp();
  }
}

__device__ void set_dinv(WarpMem& S, int n, int lane) {
  if (lane < n) S.dinv[lane] = rcp64(S.H[lane][lane].x);
  __syncwarp();
}

// x = (L L^H)^-1 r, lane k holding r_k (zero for lanes >= n) and returning x_k
__device__ double2 chol_solve(const WarpMem& S, int n, int lane, double2 r) {
  for (int j = 0; j < n; ++j) {
    double2 zj = make_double2(__shfl_sync(0xffffffffu, r.x, j), __shfl_sync(0xffffffffu, r.y, j));
    zj = S.dinv[j] * zj;
    if (lane == j) r = zj;
    if (lane > j && lane < n) r = r - S.H[lane][j] * zj;
  }
  for (int j = n - 1; j >= 0; --j) {
    double2 xj = make_double2(__shfl_sync(0xffffffffu, r.x, j), __shfl_sync(0xffffffffu, r.y, j));
    xj = S.dinv[j] * xj;
    if (lane == j) r = xj;
    if (lane < j) r = r - cmul_conj_a(S.H[j][lane], xj);
  }
  return r;
}

// v_l = rs sum_k conj(A^_kl) y_k for l = lane, lane + 32 (A^_kl = E_k P_l)
__device__ void apply_AH(const WarpMem& S, int n, int m, int lane, double2 y, double rs, double2& v0, double2& v1) {
  const double2 p0 = lane < m ? S.Pz[lane] : make_double2(0, 0);
  const double2 p1 = lane + 32 < m ? S.Pz[lane + 32] : make_double2(0, 0);
  double2 a0 = make_double2(0, 0), a1 = make_double2(0, 0);
  for (int k = 0; k < n; ++k) {
    const double2 yk = make_double2(__shfl_sync(0xffffffffu, y.x, k), __shfl_sync(0xffffffffu, y.y, k));
    const double2 ek = S.E[k];
    a0 = a0 + cmul_conj_a(ek * p0, yk);
    a1 = a1 + cmul_conj_a(ek * p1, yk);
  }
  v0 = rs * a0;
  v1 = rs * a1;
}

// s_k = rs sum_l A^_kl t_l, t in S.t (lane k < n)
__device__ double2 apply_A(const WarpMem& S, int n, int m, int lane, double rs) {
  const double2 ek = lane < n ? S.E[lane] : make_double2(0, 0);
  double2 acc = make_double2(0, 0);
  for (int l = 0; l < m; ++l) acc = acc + (ek * S.Pz[l]) * S.t[l];
  return rs * acc;
}

// g (F + B) with F_l = sum_{l' <= l} q^(l-l') x_l', B_l = sum_{l' > l} q^(l'-l) x_l',
// x in S.v; returns the entries l = lane, lane + 32.  Full warp.
__device__ void toeplitz(WarpMem& S, int m, int lane, double2 q, double2 g, double2& o0, double2& o1) {
  affine_scan64(S.v, m, q, S.F);
  for (int r = lane; r < m; r += 32) S.t[r] = r == 0 ? make_double2(0, 0) : q * S.v[m - r];
  __syncwarp();
  affine_scan64(S.t, m, q, S.B);
  __syncwarp();
  o0 = lane < m ? g * (S.F[lane] + S.B[m - 1 - lane]) : make_double2(0, 0);
  o1 = lane + 32 < m ? g * (S.F[lane + 32] + S.B[m - 33 - lane]) : make_double2(0, 0);
  __syncwarp();
}

__device__ __forceinline__ void put_v(WarpMem& S, int m, int lane, double2 v0, double2 v1) {
  if (lane < m) S.v[lane] = v0;
  if (lane + 32 < m) S.v[lane + 32] = v1;
  __syncwarp();
}

// incident field of mode 0: U~0_l = N^2 e^{-i k0 z'_l}
__device__ __forceinline__ double2 incident(const Problem& P, int om, int l) {
  double s, c;
  sincos(-(P.omega[om] / P.c0) * (P.z1 + (l + 0.5) * P.hz), &s, &c);
  const double n2 = (double)P.n * P.n;
  return make_double2(n2 * c, n2 * s);
}

// block sum of one double per warp (lane 0's value) -> partial[slot]
__device__ __forceinline__ void block_partial(double v, double* red, double* partial, long long slot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < DW; ++w) s += red[w];
    partial[slot] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// normal matrices G^ = A^ A^^H, one block per mode (A^ staged in shared memory)
// ---------------------------------------------------------------------------
struct GramMem {
  double2 A[DENSE_M1][DENSE_M + 1];
  double2 E[DENSE_M1], Pz[DENSE_M];  // filled by warp 0 (mode_setup)
  int usable;
};

__global__ void __launch_bounds__(GT) k_diff_gram(Problem P, double2* __restrict__ gram) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GramMem& S = *reinterpret_cast<GramMem*>(smem_raw);
  const int n = P.m1, m = P.m;
  const int P1 = n * (n + 1) / 2;
  const long long N2 = (long long)P.n * P.n, total = N2 * P.n_omega;
  for (long long item = blockIdx.x; item < total; item += gridDim.x) {
    const int om = (int)(item / N2);
    const long long nu = item - (long long)om * N2;
    if (threadIdx.x < 32) {
      const ModeGeo g = mode_setup(P, om, nu, S.E, S.Pz);
      if (threadIdx.x == 0) S.usable = g.usable;
    }
    __syncthreads();
    const bool usable = S.usable;
    if (usable)
      for (int e = threadIdx.x; e < n * m; e += GT) {
        const int k = e / m, l = e - k * m;
        S.A[k][l] = S.E[k] * S.Pz[l];
      }
    __syncthreads();
    double2* out = gram + item * P1;
    for (int e = threadIdx.x; e < P1; e += GT) {
      int j = 0;
      while (col_off(j + 1, n) <= e) ++j;
      const int k = j + (int)(e - col_off(j, n));
      double2 acc = make_double2(0, 0);
      if (usable) {
        for (int l = 0; l < m; ++l) acc = acc + mulc(S.A[k][l], S.A[j][l]);
        if (k == j) acc.y = 0.0;
      }
      out[e] = acc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// forward: factor, solve, eq. (9); tape <- L, y' (or b), V~/U~ planes
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(DW * 32)
k_diff_forward(Problem P, const double2* __restrict__ gram, const cx<R>* __restrict__ wt,
               const double* __restrict__ log_alpha, double2* __restrict__ Ls, double2* __restrict__ ys,
               cx<R>* __restrict__ vt, cx<R>* __restrict__ ut, double* __restrict__ partial,
               unsigned long long* __restrict__ ctr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[DW];
  __shared__ unsigned short rc[MAX_P1];
  WarpMem& S = reinterpret_cast<WarpMem*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int om = blockIdx.y, n = P.m1, m = P.m;
  const int P1 = n * (n + 1) / 2;
  const long long N2 = (long long)P.n * P.n;
  const double alpha = exp(log_alpha[om]);
  build_rc(rc, n);
  __syncthreads();
  double phi = 0.0;
  bool bad = false;
  for (long long nu = (long long)blockIdx.x * DW + warp; nu < N2; nu += (long long)gridDim.x * DW) {
    const long long mode = om * N2 + nu;
    const ModeGeo g = mode_setup(P, om, nu, S.E, S.Pz);
    const double2 b = lane < n ? to_d(wt[((long long)om * n + lane) * N2 + nu]) : make_double2(0, 0);
    const double ap = alpha * g.rs * g.rs;
    double2 v0 = make_double2(0, 0), v1 = make_double2(0, 0), u0 = v0, u1 = v0;
    if (g.usable && ap < AP_MAX) {
      load_lower(S, gram + mode * P1, n, lane);
      if (lane < n) S.H[lane][lane].x += ap;
      __syncwarp();
      cholesky(S, n, lane, rc, bad);
      store_lower(Ls + mode * P1, S, n, lane);
      const double2 y = chol_solve(S, n, lane, b);
      if (lane < n) ys[mode * n + lane] = y;
      phi += ap * ap * warp_sum(abs2(y));
      apply_AH(S, n, m, lane, y, g.rs, v0, v1);
      put_v(S, m, lane, v0, v1);
      toeplitz(S, m, lane, g.q, g.gamma, u0, u1);
    } else {
      if (lane < n) ys[mode * n + lane] = b;
      phi += warp_sum(abs2(b));
    }
    if (nu == 0) {
      if (lane < m) u0 = u0 + incident(P, om, lane);
      if (lane + 32 < m) u1 = u1 + incident(P, om, lane + 32);
    }
    if (lane < m) {
      vt[((long long)om * m + lane) * N2 + nu] = from_d<R>(v0);
      ut[((long long)om * m + lane) * N2 + nu] = from_d<R>(u0);
    }
    if (lane + 32 < m) {
      vt[((long long)om * m + lane + 32) * N2 + nu] = from_d<R>(v1);
      ut[((long long)om * m + lane + 32) * N2 + nu] = from_d<R>(u1);
    }
  }
  if (bad && lane == 0) atomicAdd(ctr + C_NONFINITE, 1ull);
  block_partial(phi, red, partial, (long long)om * gridDim.x + blockIdx.x);
}

// ---------------------------------------------------------------------------
// VJP: b-bar per mode (written as N^2 b-bar for the inverse transform) and the
// lnalpha-bar partials.  vbt/ubt (the forward transforms of V-bar, u-bar) may
// be null when xi carries no cotangent; wbt may be null when W needs no gradient.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(DW * 32)
k_diff_vjp(Problem P, const double2* __restrict__ Ls, const double2* __restrict__ ys,
           const cx<R>* __restrict__ vbt, const cx<R>* __restrict__ ubt, const double* __restrict__ log_alpha,
           const double* __restrict__ grad_phi, cx<R>* __restrict__ wbt, double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[DW];
  WarpMem& S = reinterpret_cast<WarpMem*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int om = blockIdx.y, n = P.m1, m = P.m;
  const int P1 = n * (n + 1) / 2;
  const long long N2 = (long long)P.n * P.n;
  const double inv_n2 = 1.0 / (double)N2;
  const double alpha = exp(log_alpha[om]);
  const double gphi = grad_phi ? grad_phi[om] : 0.0;
  double lbar = 0.0;
  for (long long nu = (long long)blockIdx.x * DW + warp; nu < N2; nu += (long long)gridDim.x * DW) {
    const long long mode = om * N2 + nu;
    const ModeGeo g = mode_setup(P, om, nu, S.E, S.Pz);
    const double2 y = lane < n ? ys[mode * n + lane] : make_double2(0, 0);
    const double ap = alpha * g.rs * g.rs;
    double2 bb;
    if (g.usable && ap < AP_MAX) {
      load_lower(S, Ls + mode * P1, n, lane);
      set_dinv(S, n, lane);
      double2 s = make_double2(0, 0);
      if (vbt) {
        // t = V~-bar + conj(gamma) (scans with conj(q)) of U~-bar;  F^-1 adjoint = F / N^2
        double2 a0 = make_double2(0, 0), a1 = a0;
        if (lane < m) a0 = inv_n2 * to_d(ubt[((long long)om * m + lane) * N2 + nu]);
        if (lane + 32 < m) a1 = inv_n2 * to_d(ubt[((long long)om * m + lane + 32) * N2 + nu]);
        put_v(S, m, lane, a0, a1);
        double2 t0, t1;
        toeplitz(S, m, lane, conjx(g.q), conjx(g.gamma), t0, t1);
        if (lane < m) S.t[lane] = t0 + inv_n2 * to_d(vbt[((long long)om * m + lane) * N2 + nu]);
        if (lane + 32 < m) S.t[lane + 32] = t1 + inv_n2 * to_d(vbt[((long long)om * m + lane + 32) * N2 + nu]);
        __syncwarp();
        s = apply_A(S, n, m, lane, g.rs);
        __syncwarp();
      }
      s = s + (2.0 * ap * ap * gphi) * y;
      bb = chol_solve(S, n, lane, s);
      lbar += -ap * warp_sum(bb.x * y.x + bb.y * y.y) + 2.0 * gphi * ap * ap * warp_sum(abs2(y));
    } else {
      bb = (2.0 * gphi) * y;  // the slot holds b: Phi_nu = ||b||^2
    }
    if (wbt && lane < n) wbt[((long long)om * n + lane) * N2 + nu] = from_d<R>((double)N2 * bb);
  }
  block_partial(lbar, red, partial, (long long)om * gridDim.x + blockIdx.x);
}

// ---------------------------------------------------------------------------
// JVP for nd <= JVP_CHUNK directions at once (L loaded once per mode)
// dwt: [nd][n_omega][M1][N2]; dvt, dut: [nd][n_omega][M][N2]
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(DW * 32)
k_diff_jvp(Problem P, int nd, const double2* __restrict__ Ls, const double2* __restrict__ ys,
           const cx<R>* __restrict__ dwt, const double* __restrict__ log_alpha,
           const double* __restrict__ dlog_alpha, cx<R>* __restrict__ dvt, cx<R>* __restrict__ dut,
           double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[DW];
  WarpMem& S = reinterpret_cast<WarpMem*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int om = blockIdx.y, n = P.m1, m = P.m, F = P.n_omega;
  const int P1 = n * (n + 1) / 2;
  const long long N2 = (long long)P.n * P.n;
  const double alpha = exp(log_alpha[om]);
  __shared__ double acc[DW][JVP_CHUNK];  // per-warp Phi-dot sums (lane 0 adds)
  if (lane < JVP_CHUNK) acc[warp][lane] = 0.0;
  __syncwarp();
  for (long long nu = (long long)blockIdx.x * DW + warp; nu < N2; nu += (long long)gridDim.x * DW) {
    const long long mode = om * N2 + nu;
    const ModeGeo g = mode_setup(P, om, nu, S.E, S.Pz);
    const double2 y = lane < n ? ys[mode * n + lane] : make_double2(0, 0);
    const double ap = alpha * g.rs * g.rs;
    const bool solve = g.usable && ap < AP_MAX;
    double yy = 0.0;
    if (solve) {
      load_lower(S, Ls + mode * P1, n, lane);
      set_dinv(S, n, lane);
      yy = warp_sum(abs2(y));
    }
#pragma unroll 1
    for (int d = 0; d < nd; ++d) {
      const double2 db =
          lane < n ? to_d(dwt[(((long long)d * F + om) * n + lane) * N2 + nu]) : make_double2(0, 0);
      const double dla = dlog_alpha ? dlog_alpha[d * F + om] : 0.0;
      double2 v0 = make_double2(0, 0), v1 = v0, u0 = v0, u1 = v0;
      double dp;
      if (solve) {
        const double2 dy = chol_solve(S, n, lane, db - (dla * ap) * y);
        dp = 2.0 * ap * ap * (dla * yy + warp_sum(y.x * dy.x + y.y * dy.y));
        apply_AH(S, n, m, lane, dy, g.rs, v0, v1);
        put_v(S, m, lane, v0, v1);
        toeplitz(S, m, lane, g.q, g.gamma, u0, u1);
      } else {
        dp = 2.0 * warp_sum(y.x * db.x + y.y * db.y);  // Phi_nu = ||b||^2
      }
      if (lane == 0) acc[warp][d] += dp;
      const long long base = ((long long)d * F + om) * m;
      if (lane < m) {
        dvt[(base + lane) * N2 + nu] = from_d<R>(v0);
        dut[(base + lane) * N2 + nu] = from_d<R>(u0);
      }
      if (lane + 32 < m) {
        dvt[(base + lane + 32) * N2 + nu] = from_d<R>(v1);
        dut[(base + lane + 32) * N2 + nu] = from_d<R>(u1);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < nd) {
    double t = 0.0;
    for (int w = 0; w < DW; ++w) t += acc[w][threadIdx.x];
    partial[((long long)threadIdx.x * F + om) * gridDim.x + blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------
// step 3 and its derivatives, one thread per voxel (X planes), arrays
// [n_omega][M N^2] (fields) and [M N^2] (xi)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_diff_combine(Problem P, const cx<R>* __restrict__ Vx, const cx<R>* __restrict__ ux,
                               R* __restrict__ xi, R* __restrict__ c, R* __restrict__ xis) {
  const long long MN2 = (long long)P.m * P.n * P.n;
  const R guard2 = (R)(P.eps_u * P.eps_u * P.n_omega);
  const R ic2 = (R)(1.0 / (P.c0 * P.c0));
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < MN2; p += (long long)gridDim.x * blockDim.x) {
    R num = 0, D = 0;
    for (int om = 0; om < P.n_omega; ++om) {
      const cx<R> u = ux[om * MN2 + p], V = Vx[om * MN2 + p];
      num += u.x * V.x + u.y * V.y;
      D += u.x * u.x + u.y * u.y;
    }
    const R x = D < guard2 ? R(0) : num / D;
    xi[p] = x;
    xis[p] = x;
    if (c) c[p] = x < ic2 ? R(1) / sqrt(ic2 - x) : R(NAN);
  }
}

template <typename R>
__global__ void k_diff_vjp_point(Problem P, const R* __restrict__ gxi, const cx<R>* __restrict__ Vx,
                                 const cx<R>* __restrict__ ux, const R* __restrict__ xis, cx<R>* __restrict__ Vb,
                                 cx<R>* __restrict__ ub) {
  const long long MN2 = (long long)P.m * P.n * P.n;
  const R guard2 = (R)(P.eps_u * P.eps_u * P.n_omega);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < MN2; p += (long long)gridDim.x * blockDim.x) {
    R D = 0;
    for (int om = 0; om < P.n_omega; ++om) D += abs2(ux[om * MN2 + p]);
    const R gx = D < guard2 ? R(0) : gxi[p] / D;
    const R x2 = R(2) * xis[p];
    for (int om = 0; om < P.n_omega; ++om) {
      const cx<R> u = ux[om * MN2 + p], V = Vx[om * MN2 + p];
      Vb[om * MN2 + p] = gx * u;
      ub[om * MN2 + p] = gx * (V - x2 * u);
    }
  }
}

// dVx, dux: [nd][n_omega][M N^2];  dxi: [nd][M N^2]
template <typename R>
__global__ void k_diff_jvp_point(Problem P, int nd, const cx<R>* __restrict__ Vx, const cx<R>* __restrict__ ux,
                                 const R* __restrict__ xis, const cx<R>* __restrict__ dVx,
                                 const cx<R>* __restrict__ dux, R* __restrict__ dxi) {
  const long long MN2 = (long long)P.m * P.n * P.n;
  const int F = P.n_omega;
  const R guard2 = (R)(P.eps_u * P.eps_u * F);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < MN2; p += (long long)gridDim.x * blockDim.x) {
    R D = 0;
    for (int om = 0; om < F; ++om) D += abs2(ux[om * MN2 + p]);
    const R x = xis[p];
    for (int d = 0; d < nd; ++d) {
      R num = 0, dD = 0;
      for (int om = 0; om < F; ++om) {
        const cx<R> u = ux[om * MN2 + p], V = Vx[om * MN2 + p];
        const cx<R> du = dux[((long long)d * F + om) * MN2 + p], dV = dVx[((long long)d * F + om) * MN2 + p];
        num += du.x * V.x + du.y * V.y + u.x * dV.x + u.y * dV.y;
        dD += R(2) * (u.x * du.x + u.y * du.y);
      }
      dxi[(long long)d * MN2 + p] = D < guard2 ? R(0) : (num - x * dD) / D;
    }
  }
}

// out[r] = sum_c partial[r cols + c], fixed order
__global__ void k_reduce_rows(const double* __restrict__ partial, int rows, int cols, double* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double s = 0.0;
  for (int c = 0; c < cols; ++c) s += partial[(long long)r * cols + c];
  out[r] = s;
}

// opt in to more than 48 KB of dynamic shared memory, once per kernel and device
// (the flag is per call site: each caller below launches a distinct kernel)
template <typename K> cudaError_t allow_smem(K kernel, size_t bytes, SmemOptIn& flag) {
  return opt_in_smem(flag, (const void*)kernel, bytes);
}

unsigned point_grid(long long n) {
  const long long b = (n + 255) / 256;
  const long long cap = 8LL * sm_count();
  return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

int diff_blocks_per_omega(int n, int n_omega) {
  const long long N2 = (long long)n * n;
  const long long want = (N2 + DW - 1) / DW;
  long long cap = (3LL * sm_count() + n_omega - 1) / n_omega;
  if (cap < 1) cap = 1;
  return (int)(want < cap ? want : cap);
}

cudaError_t launch_diff_gram(const Problem& P, double2* gram, cudaStream_t s) {
  const size_t smem = sizeof(GramMem);
  static SmemOptIn done;
  cudaError_t e = allow_smem(k_diff_gram, smem, done);
  if (e != cudaSuccess) return e;
  const long long total = (long long)P.n * P.n * P.n_omega;
  const long long cap = 4LL * sm_count();
  k_diff_gram<<<(unsigned)(total < cap ? total : cap), GT, smem, s>>>(P, gram);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_diff_forward(const Problem& P, int gb, const double2* gram, const cx<R>* wt,
                                const double* log_alpha, double2* Ls, double2* ys, cx<R>* vt, cx<R>* ut,
                                double* partial, unsigned long long* ctr, cudaStream_t s) {
  const size_t smem = sizeof(WarpMem) * DW;
  static SmemOptIn done;
  cudaError_t e = allow_smem(k_diff_forward<R>, smem, done);
  if (e != cudaSuccess) return e;
  k_diff_forward<R><<<dim3(gb, P.n_omega), DW * 32, smem, s>>>(P, gram, wt, log_alpha, Ls, ys, vt, ut, partial, ctr);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_diff_vjp(const Problem& P, int gb, const double2* Ls, const double2* ys, const cx<R>* vbt,
                            const cx<R>* ubt, const double* log_alpha, const double* grad_phi, cx<R>* wbt,
                            double* partial, cudaStream_t s) {
  const size_t smem = sizeof(WarpMem) * DW;
  static SmemOptIn done;
  cudaError_t e = allow_smem(k_diff_vjp<R>, smem, done);
  if (e != cudaSuccess) return e;
  k_diff_vjp<R><<<dim3(gb, P.n_omega), DW * 32, smem, s>>>(P, Ls, ys, vbt, ubt, log_alpha, grad_phi, wbt, partial);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_diff_jvp(const Problem& P, int gb, int nd, const double2* Ls, const double2* ys,
                            const cx<R>* dwt, const double* log_alpha, const double* dlog_alpha, cx<R>* dvt,
                            cx<R>* dut, double* partial, cudaStream_t s) {
  if (nd < 1 || nd > JVP_CHUNK) return cudaErrorInvalidValue;
  const size_t smem = sizeof(WarpMem) * DW;
  static SmemOptIn done;
  cudaError_t e = allow_smem(k_diff_jvp<R>, smem, done);
  if (e != cudaSuccess) return e;
  k_diff_jvp<R><<<dim3(gb, P.n_omega), DW * 32, smem, s>>>(P, nd, Ls, ys, dwt, log_alpha, dlog_alpha, dvt, dut,
                                                          partial);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_diff_combine(const Problem& P, const cx<R>* Vx, const cx<R>* ux, R* xi, R* c, R* xis,
                                cudaStream_t s) {
  k_diff_combine<R><<<point_grid((long long)P.m * P.n * P.n), 256, 0, s>>>(P, Vx, ux, xi, c, xis);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_diff_vjp_point(const Problem& P, const R* gxi, const cx<R>* Vx, const cx<R>* ux, const R* xis,
                                  cx<R>* Vb, cx<R>* ub, cudaStream_t s) {
  k_diff_vjp_point<R><<<point_grid((long long)P.m * P.n * P.n), 256, 0, s>>>(P, gxi, Vx, ux, xis, Vb, ub);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_diff_jvp_point(const Problem& P, int nd, const cx<R>* Vx, const cx<R>* ux, const R* xis,
                                  const cx<R>* dVx, const cx<R>* dux, R* dxi, cudaStream_t s) {
  k_diff_jvp_point<R><<<point_grid((long long)P.m * P.n * P.n), 256, 0, s>>>(P, nd, Vx, ux, xis, dVx, dux, dxi);
  return cudaGetLastError();
}

cudaError_t launch_reduce_rows(const double* partial, int rows, int cols, double* out, cudaStream_t s) {
  k_reduce_rows<<<(rows + 127) / 128, 128, 0, s>>>(partial, rows, cols, out);
  return cudaGetLastError();
}

#define FL_DIFF_INST(R)                                                                                         \
  template cudaError_t launch_diff_forward<R>(const Problem&, int, const double2*, const cx<R>*, const double*,  \
                                              double2*, double2*, cx<R>*, cx<R>*, double*, unsigned long long*,  \
                                              cudaStream_t);                                                    \
  template cudaError_t launch_diff_vjp<R>(const Problem&, int, const double2*, const double2*, const cx<R>*,     \
                                          const cx<R>*, const double*, const double*, cx<R>*, double*,          \
                                          cudaStream_t);                                                        \
  template cudaError_t launch_diff_jvp<R>(const Problem&, int, int, const double2*, const double2*,             \
                                          const cx<R>*, const double*, const double*, cx<R>*, cx<R>*, double*,  \
                                          cudaStream_t);                                                        \
  template cudaError_t launch_diff_combine<R>(const Problem&, const cx<R>*, const cx<R>*, R*, R*, R*,            \
                                              cudaStream_t);                                                    \
  template cudaError_t launch_diff_vjp_point<R>(const Problem&, const R*, const cx<R>*, const cx<R>*, const R*,  \
                                                cx<R>*, cx<R>*, cudaStream_t);                                  \
  template cudaError_t launch_diff_jvp_point<R>(const Problem&, int, const cx<R>*, const cx<R>*, const R*,       \
                                                const cx<R>*, const cx<R>*, R*, cudaStream_t);
FL_DIFF_INST(double)
FL_DIFF_INST(float)
#undef FL_DIFF_INST

}  // namespace fl
