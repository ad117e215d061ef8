// Rank-one closed form of the per-mode problem (fs_options.solve_form = 1).
//
// Every data plane lies above X, so the Weyl kernel of eq. (8) factors,
// K_nu(z_k - z'_l) ~ e^{i k_z z_k} e^{-i k_z z'_l}, and the matrix of the SLAE is
// exactly rank one:
//   A_kl = E_k P_l,  E_k = omega^2 h_z (-i/(2 k_z)) e^{i k_z (z_k - z_top)},
//                    P_l = e^{i k_z (z_top - z'_l)}
// (both factors of modulus <= 1).  Then A A^H = ||P||^2 E E^H, tr = ||E||^2 ||P||^2 is
// the only nonzero eigenvalue, and with beta = E^H b the normal solutions of Sec. 4
// comment b are
//   Tikhonov:  V~ = A^H (A A^H + alpha I)^-1 b = conj(P) beta / (tr + alpha)
//   TSVD:      V~ = A^+ b                       = conj(P) beta / tr
// (TSVD keeps the one nonzero singular value: the discrepancy principle never
// truncates to rank zero on an active mode, whose ||b|| exceeds delta_nu).  The
// discrepancy is phi^2(alpha) = (alpha/(tr + alpha))^2 c + p with c = |beta|^2/||E||^2
// (the part of ||b||^2 in the range of A) and p = ||b||^2 - c (the rest), so the
// root of phi = delta_nu is
//   alpha = tr t/(1 - t),  t = sqrt((delta_nu^2 - p)/c),
// floored at alpha_rel tr, which is also taken when phi(alpha_floor) >= delta_nu.
// The dense form reaches the same values through the normal matrix; the two agree
// to rounding.  Cost O(M1 + M) per mode, one warp per mode; eq. (9) and the output
// layout are those of the dense solve.  It holds no matrix, so it serves layers up
// to the global limits (M, M1 <= 128), beyond those of the dense form.
#include <math.h>

#include "modes.cuh"
#include "pipeline.cuh"

namespace fl {

namespace {

constexpr int RW = 4;  // warps (modes) per block

// RKE data planes and RK X planes per lane: (1, 2) for up to 32 data and 64 X planes,
// (4, 4) up to 128 of each; the register arrays and per-warp shared memory are sized by them
template <int RK> struct Rank1Mem {
  double2 v[32 * RK], t[32 * RK], F[32 * RK], B[32 * RK];
};

// The factors E_k and P_l: FP64 exponentials in the FP64 path; in the mixed path the
// phase reduced in FP64 and the exponentials taken in FP32 (exp_ikz32), a relative
// error of ~1e-7, the precision of the FP32 data, instead of FP64 exponentials at the
// FP64 rate (the bulk of this kernel otherwise).  A = E P^T from the rounded factors
// is still exactly rank one, so the closed form below stays exact for that A.
template <typename R> __device__ __forceinline__ double2 exp_mode(double2 kz, double d) {
  if constexpr (sizeof(R) == 4) return exp_ikz32(kz, d);
  else return exp_ikz_inline(kz, d);
}

template <typename R, int RKE, int RK>
__global__ void __launch_bounds__(RW * 32)
k_solve_rank1(Problem P, const cx<R>* __restrict__ wt, const double2* __restrict__ wt64,
              const int* __restrict__ act, const int* __restrict__ count,
              const double* __restrict__ dnu_arr, cx<R>* __restrict__ prof, double* __restrict__ alpha_out,
              unsigned long long* __restrict__ ctr) {
  pdl_wait();
  pdl_trigger();
  __shared__ Rank1Mem<RK> mem[RW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Rank1Mem<RK>& S = mem[warp];
  const int N = P.n, n = P.m1, m = P.m;
  const long long N2 = (long long)N * N;
  long long total = 0;
  for (int w = 0; w < P.n_omega; ++w) total += count[w];
  unsigned long long n_floor = 0, n_zeroed = 0, n_bad = 0;
  // item w G + b on warp w of block b (G = gridDim.x): consecutive modes on different
  // blocks, so that a few active modes spread over the SMs instead of filling the
  // warps of the first blocks
  for (long long item = (long long)warp * gridDim.x + blockIdx.x; item < total; item += (long long)gridDim.x * RW) {
    int om = 0;
    long long i = item;
    while (i >= count[om]) { i -= count[om]; ++om; }
    const int nu = act[om * N2 + i];
    const int i2 = nu / N, i1 = nu - i2 * N;
    const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
    const double k0 = P.k0[om], kn = P.kn;
    const double q = k0 * k0 - kn * kn * (double)(m1 * m1 + m2 * m2);
    const double rq = rsqrt64(fabs(q));  // active modes are never grazing: q != 0
    const double2 kz = q >= 0.0 ? make_double2(fabs(q) * rq, 0.0) : make_double2(0.0, fabs(q) * rq);
    const double g0 = P.g0[om];
    const double2 gamma = q >= 0.0 ? make_double2(0.0, -g0 * rq) : make_double2(-g0 * rq, 0.0);
    const double ztop = P.z1 + (m - 0.5) * P.hz;
    // E_k, b_k on lanes k mod 32 and P_l on lanes l mod 32 (M1, M <= 128): the sums
    // sum |E|^2, sum |b|^2, E^H b and sum |P|^2, P kept in registers (slot l / 32)
    double sE = 0.0, bb = 0.0, sP = 0.0;
    double2 beta = make_double2(0, 0);
    double2 ek[RKE], bk[RKE];  // E_k and b_k of k = lane + 32 j
#pragma unroll
    for (int j = 0; j < RKE; ++j) {
      const int k = lane + 32 * j;
      ek[j] = make_double2(0, 0);
      bk[j] = make_double2(0, 0);
      if (k < n) {
        ek[j] = gamma * exp_mode<R>(kz, P.zy[k] - ztop);
        const long long at = ((long long)om * n + k) * N2 + nu;
        bk[j] = wt64 ? wt64[at] : to_d(wt[at]);  // W~ in FP64 on the mixed truncated-SVD route
      }
      sE += abs2(ek[j]);
      bb += abs2(bk[j]);
      beta = beta + cmul_conj_a(ek[j], bk[j]);
    }
    double2 pl[RK];
#pragma unroll
    for (int j = 0; j < RK; ++j) {
      const int l = lane + 32 * j;
      pl[j] = l < m ? exp_mode<R>(kz, ztop - (P.z1 + (l + 0.5) * P.hz)) : make_double2(0, 0);
      sP += abs2(pl[j]);
    }
    sE = warp_sum(sE);
    sP = warp_sum(sP);
    bb = warp_sum(bb);
    beta = warp_sum(beta);  // E^H b
    const double tr = sE * sP;
    const double dnu = dnu_arr[om];
    // ||b - E (E^H b)/||E||^2||^2, the part of ||b||^2 outside the range of A, as the norm
    // of that residual (not ||b||^2 - |E^H b|^2/||E||^2, whose rounding of order
    // eps ||b||^2 decides alpha when delta_nu << ||b||)
    double p = 0.0;
    if (tr > 0.0) {
      const double2 pr = rcp64(sE) * beta;
#pragma unroll
      for (int j = 0; j < RKE; ++j) p += abs2(bk[j] - ek[j] * pr);
      p = warp_sum(p);
    }
    double2 coef = make_double2(0, 0);  // V~_l = conj(P_l) coef
    const bool zeroed = !(tr > 0.0) || (P.alpha_mode == 0 && !(bb > dnu * dnu));
    double alpha = INFINITY;
    if (!zeroed) {
      if (P.regularizer == 1) {
        alpha = 0.0;
        coef = rcp64(tr) * beta;
      } else {
        if (P.alpha_mode == 1) {
          alpha = P.alpha_given[om];
        } else {
          const double c = abs2(beta) * rcp64(sE);  // |u^H b|^2, u = E / ||E||
          const double afl = P.alpha_rel * tr;
          const double rf = afl * rcp64(tr + afl);
          if (rf * rf * c + p >= dnu * dnu) {
            alpha = afl;
            ++n_floor;
          } else {
            const double t = sqrt((dnu * dnu - p) * rcp64(c));
            alpha = fmax(tr * t * rcp64(1.0 - t), afl);
          }
        }
        coef = rcp64(tr + alpha) * beta;
      }
    } else {
      ++n_zeroed;
    }
    // V~ and eq. (9): U~ = U~0 + gamma (F + B) over the X planes (two affine scans)
    double2 qz = make_double2(0, 0);  // P_{m-2} = e^{i k_z h_z}: the plane-to-plane factor
#pragma unroll
    for (int j = 0; j < RK; ++j) {
      const int l = lane + 32 * j;
      if (l < m) S.v[l] = cmul_conj_a(pl[j], coef);
      if (m >= 2 && j == (m - 2) >> 5) qz = pl[j];
    }
    if (m >= 2) {
      const int src = (m - 2) & 31;
      qz = make_double2(__shfl_sync(0xffffffffu, qz.x, src), __shfl_sync(0xffffffffu, qz.y, src));
    }
    __syncwarp();
    affine_scan_lanes<RK>(S.v, m, qz, S.F);
    for (int r = lane; r < m; r += 32) S.t[r] = r == 0 ? make_double2(0, 0) : qz * S.v[m - r];
    __syncwarp();
    affine_scan_lanes<RK>(S.t, m, qz, S.B);
    __syncwarp();
    cx<R>* out = prof + ((long long)om * N2 + i) * 2 * m;
    const double n2 = (double)N2;
    bool overflow = false;  // a profile beyond the range of R (FP32 in the mixed path)
    for (int l = lane; l < m; l += 32) {
      double2 u = gamma * (S.F[l] + S.B[m - 1 - l]);
      if (nu == 0 && !P.incident) {
        double s0, c0;
        sincos(-k0 * (P.z1 + (l + 0.5) * P.hz), &s0, &c0);
        u = u + make_double2(n2 * c0, n2 * s0);
      }
      const cx<R> vo = from_d<R>(S.v[l]), uo = from_d<R>(u);
      overflow |= !(isfinite(vo.x) && isfinite(vo.y) && isfinite(uo.x) && isfinite(uo.y));
      out[l] = vo;
      out[m + l] = uo;
    }
    if (__any_sync(0xffffffffu, overflow)) ++n_bad;
    if (lane == 0 && alpha_out) alpha_out[om * N2 + nu] = zeroed ? INFINITY : alpha;
    __syncwarp();
  }
  if (lane == 0) {
    if (n_floor) atomicAdd(ctr + C_ALPHA_FLOOR, n_floor);
    if (n_bad) atomicAdd(ctr + C_NONFINITE, n_bad);  // profiles beyond the range of R
    if (n_zeroed) {
      atomicAdd(ctr + C_ACTIVE, (unsigned long long)(-(long long)n_zeroed));
      atomicAdd(ctr + C_ZEROED, n_zeroed);
    }
  }
}

}  // namespace

template <typename R>
cudaError_t launch_solve_rank1(const Problem& P, const Work<R>& w, cudaStream_t s) {
  const int sms = sm_count();
  const long long modes = (long long)P.n_omega * P.n * P.n;
  const long long want = (modes + RW - 1) / RW;
  const long long cap = 8LL * sms;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  if (P.m <= 64 && P.m1 <= 32)
    return launch_pdl(k_solve_rank1<R, 1, 2>, dim3(grid), dim3(RW * 32), 0, s, P, (const cx<R>*)w.wt,
                      (const double2*)w.wt64, (const int*)w.act, (const int*)w.count, (const double*)w.dnu, w.prof,
                      w.alpha_out, w.ctr);
  return launch_pdl(k_solve_rank1<R, 4, 4>, dim3(grid), dim3(RW * 32), 0, s, P, (const cx<R>*)w.wt,
                    (const double2*)w.wt64, (const int*)w.act, (const int*)w.count, (const double*)w.dnu, w.prof,
                    w.alpha_out, w.ctr);
}

template cudaError_t launch_solve_rank1<double>(const Problem&, const Work<double>&, cudaStream_t);
template cudaError_t launch_solve_rank1<float>(const Problem&, const Work<float>&, cudaStream_t);

}  // namespace fl
