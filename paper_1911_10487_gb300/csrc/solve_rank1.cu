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
#include "twofloat.cuh"

namespace fl {

namespace {

constexpr int RW = 4;  // warps (modes) per block

// RKE data planes and RK X planes per lane: (1, 2) for up to 32 data and 64 X planes,
// (4, 4) up to 128 of each; the register arrays and per-warp shared memory are sized by them
template <int RK> struct Rank1Mem {
  double2 v[32 * RK], t[32 * RK], F[32 * RK], B[32 * RK];
};

// The FP64 path (k_solve_rank1_mixed below is the mixed one).
template <int RKE, int RK>
__global__ void __launch_bounds__(RW * 32)
k_solve_rank1(Problem P, const double2* __restrict__ wt, const int* __restrict__ act, const int* __restrict__ count,
              const double* __restrict__ dnu_arr, double2* __restrict__ prof, double* __restrict__ alpha_out,
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
        ek[j] = gamma * exp_ikz_inline(kz, P.zy[k] - ztop);
        bk[j] = wt[((long long)om * n + k) * N2 + nu];
      }
      sE += abs2(ek[j]);
      bb += abs2(bk[j]);
      beta = beta + cmul_conj_a(ek[j], bk[j]);
    }
    double2 pl[RK];
#pragma unroll
    for (int j = 0; j < RK; ++j) {
      const int l = lane + 32 * j;
      pl[j] = l < m ? exp_ikz_inline(kz, ztop - (P.z1 + (l + 0.5) * P.hz)) : make_double2(0, 0);
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
    double2* out = prof + ((long long)om * N2 + i) * 2 * m;
    const double n2 = (double)N2;
    bool overflow = false;  // a profile beyond the FP64 range
    for (int l = lane; l < m; l += 32) {
      double2 u = gamma * (S.F[l] + S.B[m - 1 - l]);
      if (nu == 0 && !P.incident) {
        double s0, c0;
        sincos(-k0 * (P.z1 + (l + 0.5) * P.hz), &s0, &c0);
        u = u + make_double2(n2 * c0, n2 * s0);
      }
      overflow |= !(isfinite(S.v[l].x) && isfinite(S.v[l].y) && isfinite(u.x) && isfinite(u.y));
      out[l] = S.v[l];
      out[m + l] = u;
    }
    if (__any_sync(0xffffffffu, overflow)) ++n_bad;
    if (lane == 0 && alpha_out) alpha_out[om * N2 + nu] = zeroed ? INFINITY : alpha;
    __syncwarp();
  }
  if (lane == 0) {
    if (n_floor) atomicAdd(ctr + C_ALPHA_FLOOR, n_floor);
    if (n_bad) atomicAdd(ctr + C_NONFINITE, n_bad);  // profiles beyond the FP64 range
    if (n_zeroed) {
      atomicAdd(ctr + C_ACTIVE, (unsigned long long)(-(long long)n_zeroed));
      atomicAdd(ctr + C_ZEROED, n_zeroed);
    }
  }
}

// ---- the mixed path: two-float arithmetic on the FP32 pipe ---------------------
// The same closed form with the factors rounded to FP32, every sum, the discrepancy
// root and V~ in two-float arithmetic (about 48 bits, the exponent range of FP32), and
// eq. (9) in closed form (below) in FP32, the precision of the output.  To keep that range, E is written as
//   E_k = s gn e_k,  e_k = e^{i k_z (z_k - z_min)}  (|e_k| <= 1, 1 on the lowest data
//   plane z_min),  s gn = gamma e^{i k_z (z_min - z_top)},  s > 0,  |gn| = 1,
// and the problem is solved for the scaled unknown: with tr_n = ||e||^2 ||p||^2
// (tr = s^2 tr_n), beta_n = conj(gn) e^H b (beta = s beta_n) and alpha = s^2 alpha_n,
//   V~ = conj(p) beta_n / (s (tr_n + alpha_n)),
// and the discrepancy root t (of c = |e^H b|^2 / ||e||^2 and the residual part p,
// which s and gn leave unchanged) gives alpha_n = tr_n t / (1 - t).  s, a decay of up
// to e^-(k_z (z_min - z_top)) on evanescent modes, is kept as an FP32 mantissa and a
// power of two.  k_z, |gamma|, the phases and s come from two-float copies of the
// problem's constants; FP64 is left to the conversion of delta_nu and to alpha as an
// output: at the FP64 rate of this GPU (one warp instruction per 64 cycles) the FP64
// form of this kernel spends most of its time on FP64 set-up, sums, root and scans.
// cos and sin of y, |y| <= pi/4 (+ rounding): their Taylor series to y^10 and y^9
// (truncation below 2e-9), Horner form
__device__ __forceinline__ float2 cos_sin_octant(float y) {
  const float y2 = y * y;
  const float c = fmaf(y2, fmaf(y2, fmaf(y2, fmaf(y2, fmaf(y2, -2.75573192e-7f, 2.48015873e-5f), -1.38888889e-3f),
                                       4.16666667e-2f), -0.5f), 1.f);
  const float sn = y * fmaf(y2, fmaf(y2, fmaf(y2, fmaf(y2, 2.75573192e-6f, -1.98412698e-4f), 8.33333333e-3f),
                                     -1.66666667e-1f), 1.f);
  return make_float2(c, sn);
}

// e^{i k_z d} from two-float |k_z| and d: propagating, the phase x = |k_z| d less the
// nearest multiple q of pi/2 in two-float (Cody-Waite with a two-float pi/2), the
// octant's cosine and sine by their series, then the quarter turns q; evanescent,
// e^{-|k_z| d} from the FP32 exponential of the leading part and the first order of
// the trailing part.  Short straight-line code: each of the kernel's calls is inlined
// and runs once per mode, so its size matters (instruction fetch).
__device__ __forceinline__ float2 exp_mode_ff(bool prop, ff kz, ff d) {
  const ff x = ff_mul(kz, d);
  if (prop) {
    const float q = rintf(x.hi * 0.636619772f);  // 2 / pi
    const ff red = ff_sub(ff_sub(x, two_prod(q, 1.57079637f)), two_prod(q, -4.37113883e-8f));
    const float2 cs = cos_sin_octant(red.hi + red.lo);
    switch ((int)q & 3) {
      case 0: return cs;
      case 1: return make_float2(-cs.y, cs.x);
      case 2: return make_float2(-cs.x, -cs.y);
      default: return make_float2(cs.y, -cs.x);
    }
  }
  return make_float2(expf(-x.hi) * (1.f - x.lo), 0.f);
}


template <int RKE, int RK>
__global__ void __launch_bounds__(RW * 32)
k_solve_rank1_mixed(Problem P, const float2* __restrict__ wt, const double2* __restrict__ wt64,
                    const int* __restrict__ act, const int* __restrict__ count, const double* __restrict__ dnu_arr,
                    float2* __restrict__ prof, double* __restrict__ alpha_out, unsigned long long* __restrict__ ctr) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int N = P.n, n = P.m1, m = P.m;
  const long long N2 = (long long)N * N;
  long long total = 0;
  for (int w = 0; w < P.n_omega; ++w) total += count[w];
  unsigned long long n_floor = 0, n_zeroed = 0, n_bad = 0;
  // item w G + b on warp w of block b, as in k_solve_rank1
  for (long long item = (long long)warp * gridDim.x + blockIdx.x; item < total; item += (long long)gridDim.x * RW) {
    int om = 0;
    long long i = item;
    while (i >= count[om]) { i -= count[om]; ++om; }
    const int nu = act[om * N2 + i];
    const int i2 = nu / N, i1 = nu - i2 * N;
    const int m1 = i1 < N / 2 ? i1 : i1 - N, m2 = i2 < N / 2 ? i2 : i2 - N;
    // k_z, |gamma| and the scale s of E = s gn e in two-float (the FP32 pipe)
    const ff k2 = ff_sub(ff{P.k0sq_f[om].x, P.k0sq_f[om].y},
                         ff_mul_f(ff{P.knsq_f.x, P.knsq_f.y}, (float)(m1 * m1 + m2 * m2)));  // k0^2 - |nu|^2
    const bool prop = k2.hi >= 0.f;  // active modes are never grazing: k2 != 0
    const ff kz = ff_sqrt(prop ? k2 : ff_neg(k2));  // |k_z|
    const ff gdf = ff_div(ff{P.g0_f[om].x, P.g0_f[om].y}, kz);  // |gamma| = g0 / |k_z|
    const ff d0 = ff{P.d0_f.x, P.d0_f.y}, hz = ff{P.hz_f.x, P.hz_f.y};
    // propagating: s = |gamma|, gn = -i e^{i k_z d0}; evanescent: gn = -1 and
    // s = |gamma| e^{-|k_z| d0} = |gamma| 2^f 2^ns, f in [0, 1)
    float2 gn = make_float2(-1.f, 0.f);
    float smf = gdf.hi + gdf.lo;  // s 2^-ns
    int ns = 0;
    if (prop) {
      const float2 ph = exp_mode_ff(true, kz, d0);
      gn = make_float2(ph.y, -ph.x);
    } else {
      const ff y = ff_mul(ff_mul(kz, d0), ff{-1.44269502f, -1.92596299e-8f});  // -|k_z| d0 log2(e)
      const float fl = floorf(y.hi);
      ns = (int)fl;
      smf *= exp2f((y.hi - fl) + y.lo);
    }
    const float inv_s = ldexpf(1.f / smf, -ns);  // 1/s (inf beyond the FP32 range: an overflowing profile)
    // e_k, b_k on lanes k mod 32, p_l on lanes l mod 32: ||e||^2, ||b||^2, e^H b, ||p||^2
    ff se = ff{0.f, 0.f}, bb = ff{0.f, 0.f}, sp = ff{0.f, 0.f};
    ffc eb = ffc_zero();
    float2 ek[RKE];
    ffc bk[RKE];
#pragma unroll
    for (int j = 0; j < RKE; ++j) {
      const int k = lane + 32 * j;
      ek[j] = make_float2(0.f, 0.f);
      bk[j] = ffc_zero();
      if (k < n) {
        ek[j] = exp_mode_ff(prop, kz, ff{P.zyd_f[k].x, P.zyd_f[k].y});
        const long long at = ((long long)om * n + k) * N2 + nu;
        if (wt64) {
          bk[j] = ffc_from(wt64[at]);  // W~ in FP64 on the truncated-SVD route
        } else {
          const float2 w = wt[at];
          bk[j] = ffc{ff{w.x, 0.f}, ff{w.y, 0.f}};
        }
      }
      se = ff_add(se, ff_add(two_prod(ek[j].x, ek[j].x), two_prod(ek[j].y, ek[j].y)));
      bb = ff_add(bb, ffc_abs2(bk[j]));
      eb = ffc_add(eb, ffc_conj_f2_mul(ek[j], bk[j]));
    }
    float2 pl[RK];
#pragma unroll
    for (int j = 0; j < RK; ++j) {
      const int l = lane + 32 * j;
      pl[j] = l < m ? exp_mode_ff(prop, kz, ff_mul_f(hz, (float)(m - 1 - l))) : make_float2(0.f, 0.f);
      sp = ff_add(sp, ff_add(two_prod(pl[j].x, pl[j].x), two_prod(pl[j].y, pl[j].y)));
    }
    // the four warp sums together: one loop, their shuffles and additions interleaved
#pragma unroll 1
    for (int o = 16; o > 0; o >>= 1) {
      const ff a = ff_shfl_xor(se, o), b2 = ff_shfl_xor(sp, o), c2 = ff_shfl_xor(bb, o);
      const ffc d = ffc_shfl_xor(eb, o);
      se = ff_add(se, a);
      sp = ff_add(sp, b2);
      bb = ff_add(bb, c2);
      eb = ffc_add(eb, d);
    }
    const ff tr = ff_mul(se, sp);  // tr_n
    const ff dnu = ff_from(dnu_arr[om]);
    const ff dnu2 = ff_mul(dnu, dnu);
    // ||b - e (e^H b)/||e||^2||^2, the part of ||b||^2 outside the range of A, as the
    // norm of that residual (its rounding does not grow with ||b||)
    ff pres = ff{0.f, 0.f};
    if (se.hi > 0.f) {
      const ffc pr = ffc{ff_div(eb.re, se), ff_div(eb.im, se)};
#pragma unroll
      for (int j = 0; j < RKE; ++j) pres = ff_add(pres, ffc_abs2(ffc_sub(bk[j], ffc_mul_f2(pr, ek[j]))));
      pres = ff_warp_sum(pres);
    }
    ffc coef = ffc_zero();  // V~_l = conj(p_l) coef
    const bool zeroed = !(tr.hi > 0.f) || (P.alpha_mode == 0 && !ff_gt(bb, dnu2));
    ff alpha = ff{0.f, 0.f};
    if (!zeroed) {
      const ffc beta = ffc_conj_f2_mul(gn, eb);  // beta_n
      if (P.regularizer == 1) {
        coef = ffc{ff_div(beta.re, tr), ff_div(beta.im, tr)};
      } else {
        if (P.alpha_mode == 1) {
          const double s2 = ldexp((double)smf * (double)smf, 2 * ns);
          const double an = P.alpha_given[om] * rcp64(s2);  // alpha / s^2
          alpha = ff_from(an < 1e30 ? an : 1e30);  // beyond: V~ is 0 to FP32 precision
        } else {
          const ff c = ff_div(ffc_abs2(eb), se);  // |e^H b|^2 / ||e||^2
          const ff afl = ff_mul(ff{P.alpha_rel_f.x, P.alpha_rel_f.y}, tr);
          const ff rf = ff_div(afl, ff_add(tr, afl));
          if (!ff_gt(dnu2, ff_add(ff_mul(ff_mul(rf, rf), c), pres))) {
            alpha = afl;
            ++n_floor;
          } else {
            const ff t = ff_sqrt(ff_div(ff_sub(dnu2, pres), c));
            alpha = ff_div(ff_mul(tr, t), ff_sub(ff{1.f, 0.f}, t));
            if (ff_gt(afl, alpha)) alpha = afl;
          }
        }
        const ff den = ff_add(tr, alpha);
        coef = ffc{ff_div(beta.re, den), ff_div(beta.im, den)};
      }
      coef = ffc{ff_mul_f(coef.re, inv_s), ff_mul_f(coef.im, inv_s)};
    } else {
      ++n_zeroed;
    }
    // V~ and eq. (9) in closed form.  With uniform X planes p_l = q^n, n = M - 1 - l,
    // q = e^{i k_z h_z}, so v_l = conj(p_l) coef and the two sums of eq. (9),
    // F_l = sum_{l' <= l} q^(l - l') v_l' and B_l = sum_{l' > l} q^(l' - l) v_l', are
    // geometric:
    //   propagating (|q| = 1, theta = k_z h_z): F_l = (l + 1) v_l,
    //     B_l = coef q sin(n theta) / sin(theta), sin(n theta) = Im p_l;
    //   evanescent (q = e^-a, a = |k_z| h_z): F_l = v_l (1 - q^(2(l+1))) / (1 - q^2),
    //     B_l = n v_l;
    // U~_l = U~0_l + gamma (F_l + B_l), evaluated in FP32 (the precision of the output).
    float2 qz = make_float2(1.f, 0.f);  // p_{M-2} = q
#pragma unroll
    for (int j = 0; j < RK; ++j)
      if (m >= 2 && j == (m - 2) >> 5) qz = pl[j];
    if (m >= 2) {
      const int src = (m - 2) & 31;
      qz = make_float2(__shfl_sync(0xffffffffu, qz.x, src), __shfl_sync(0xffffffffu, qz.y, src));
    }
    const float2 cf = ffc_to_f2(coef);
    const float gf = gdf.hi + gdf.lo;
    const float a2 = 2.f * ((kz.hi + kz.lo) * (hz.hi + hz.lo));  // evanescent: 2a
    const float den_e = prop ? 1.f : expm1f(-a2);  // q^2 - 1
    float2* out = prof + ((long long)om * N2 + i) * 2 * m;
    const float n2 = (float)N2;
    bool overflow = false;  // a profile beyond the FP32 range
#pragma unroll
    for (int j = 0; j < RK; ++j) {
      const int l = lane + 32 * j;
      if (l < m) {
        const float2 p = pl[j];
        const float2 v = make_float2(p.x * cf.x + p.y * cf.y, p.x * cf.y - p.y * cf.x);  // conj(p) coef
        const int nn = m - 1 - l;
        float2 x;
        if (prop) {
          const float d = nn > 0 ? p.y / qz.y : 0.f;  // sin(n theta) / sin(theta)
          const float2 cq = make_float2(cf.x * qz.x - cf.y * qz.y, cf.x * qz.y + cf.y * qz.x);
          x = make_float2((float)(l + 1) * v.x + d * cq.x, (float)(l + 1) * v.y + d * cq.y);
        } else {
          const float gsum = expm1f(-a2 * (float)(l + 1)) / den_e + (float)nn;
          x = make_float2(gsum * v.x, gsum * v.y);
        }
        // gamma x: gamma = -i g (propagating), -g (evanescent)
        float2 u = prop ? make_float2(gf * x.y, -gf * x.x) : make_float2(-gf * x.x, -gf * x.y);
        if (nu == 0 && !P.incident) {  // the plane wave's U~0 = N^2 exp(-i k0 z'_l)
          const ff zl = ff_add(ff{P.z1_f.x, P.z1_f.y}, ff_mul_f(hz, (float)l + 0.5f));
          const float2 w = exp_mode_ff(true, ff{P.k0_f[om].x, P.k0_f[om].y}, zl);  // e^{+i k0 z'_l}
          u = make_float2(u.x + n2 * w.x, u.y - n2 * w.y);
        }
        overflow |= !(isfinite(v.x) && isfinite(v.y) && isfinite(u.x) && isfinite(u.y));
        out[l] = v;
        out[m + l] = u;
      }
    }
    if (__any_sync(0xffffffffu, overflow)) ++n_bad;
    if (lane == 0 && alpha_out)
      alpha_out[om * N2 + nu] =
          zeroed ? INFINITY
                 : (P.regularizer == 1 ? 0.0 : ldexp((double)smf * (double)smf, 2 * ns) * ff_to(alpha));
  }
  if (lane == 0) {
    if (n_floor) atomicAdd(ctr + C_ALPHA_FLOOR, n_floor);
    if (n_bad) atomicAdd(ctr + C_NONFINITE, n_bad);  // profiles beyond the FP32 range
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
  // two blocks of RW warps per SM, all resident at once (the grid-stride loop takes any
  // count): the successor's launch waits for every block to start, and a grid of idle
  // blocks only delays it (64-problem batch 6.24 -> 6.16 ms against 8 blocks per SM)
  const long long cap = 2LL * sms;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  if constexpr (sizeof(R) == 4) {
    if (P.m <= 64 && P.m1 <= 32)
      return launch_pdl(k_solve_rank1_mixed<1, 2>, dim3(grid), dim3(RW * 32), 0, s, P, (const float2*)w.wt,
                        (const double2*)w.wt64, (const int*)w.act, (const int*)w.count, (const double*)w.dnu,
                        (float2*)w.prof, w.alpha_out, w.ctr);
    return launch_pdl(k_solve_rank1_mixed<4, 4>, dim3(grid), dim3(RW * 32), 0, s, P, (const float2*)w.wt,
                      (const double2*)w.wt64, (const int*)w.act, (const int*)w.count, (const double*)w.dnu,
                      (float2*)w.prof, w.alpha_out, w.ctr);
  } else {
    if (P.m <= 64 && P.m1 <= 32)
      return launch_pdl(k_solve_rank1<1, 2>, dim3(grid), dim3(RW * 32), 0, s, P, (const double2*)w.wt,
                        (const int*)w.act, (const int*)w.count, (const double*)w.dnu, (double2*)w.prof, w.alpha_out,
                        w.ctr);
    return launch_pdl(k_solve_rank1<4, 4>, dim3(grid), dim3(RW * 32), 0, s, P, (const double2*)w.wt,
                      (const int*)w.act, (const int*)w.count, (const double*)w.dnu, (double2*)w.prof, w.alpha_out,
                      w.ctr);
  }
}

template cudaError_t launch_solve_rank1<double>(const Problem&, const Work<double>&, cudaStream_t);
template cudaError_t launch_solve_rank1<float>(const Problem&, const Work<float>&, cudaStream_t);

}  // namespace fl
