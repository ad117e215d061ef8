// Device helpers shared by the per-mode kernels (the discrepancy solve and the
// fixed-alpha derivative kernels): scalar FP64 reciprocal, warp reductions, the
// vertical propagator exp(i k_z d) and the warp scan that applies the Toeplitz
// kernel of eq. (9) in O(M).
#pragma once

#include <math.h>

#include "common.cuh"

namespace fl {

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

// 1/sqrt(x) for a positive normal double by Newton-Raphson on f(y) = 1/y^2 - x
// (y <- y + y (1 - x y^2)/2, quadratic convergence) from an FP32 seed of the
// mantissa scaled to [1, 4); two steps take the ~23-bit seed past FP64
// precision.  Exponent handled on the bit pattern.  About six dependent FP64
// operations instead of an FP64 square root and division.
__device__ __forceinline__ double rsqrt64(double x) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  if (ex == 0 || ex == 0x7ff || bits < 0) return 1.0 / sqrt(x);  // zero, subnormal, inf, nan, negative
  const int e = ex - 1023, h = e >> 1;  // x = m 2^(2h), m in [1, 4)
  const double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | ((long long)(1023 + e - 2 * h) << 52));
  double y = (double)rsqrtf((float)m);
  double r = fma(-m * y, y, 1.0);
  y = fma(0.5 * y, r, y);
  r = fma(-m * y, y, 1.0);
  y = fma(0.5 * y, r, y);
  const long long yb = __double_as_longlong(y);  // y in (0.5, 1]: scale by 2^-h
  return __longlong_as_double(yb - ((long long)h << 52));
}

// 1/sqrt(x) and 1/x of a positive normal double to FP32 accuracy (~2e-7 relative)
// at any exponent: the FP32 reciprocal (square root) of the mantissa, the exponent on
// the bit pattern.  No FP64 arithmetic.
__device__ __forceinline__ double rsqrt32(double x) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  if (ex == 0 || ex == 0x7ff || bits < 0) return 1.0 / sqrt(x);  // zero, subnormal, inf, nan, negative
  const int e = ex - 1023, h = e >> 1;  // x = m 2^(2h), m in [1, 4)
  const double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | ((long long)(1023 + e - 2 * h) << 52));
  const double y = (double)rsqrtf((float)m);
  return __longlong_as_double(__double_as_longlong(y) - ((long long)h << 52));
}
__device__ __forceinline__ double rcp32(double x) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  if (ex == 0 || ex == 0x7ff) return 1.0 / x;  // zero, subnormal, inf, nan
  const double m = __longlong_as_double((bits & ~(0x7ffLL << 52)) | (1023LL << 52));  // [1,2), sign kept
  const long long yb = __double_as_longlong((double)(1.0f / (float)m));
  const int ey = (int)((yb >> 52) & 0x7ff) - (ex - 1023);
  if (ey <= 0 || ey >= 0x7ff) return 1.0 / x;
  return __longlong_as_double((yb & ~(0x7ffLL << 52)) | ((long long)ey << 52));
}

// exp(i kz d) inlined: for small kernels that evaluate several independent
// exponentials per thread, so that their FP64 chains can overlap
__device__ __forceinline__ double2 exp_ikz_inline(double2 kz, double d) {
  const double mag = exp(-kz.y * d);
  double s, c;
  sincos(kz.x * d, &s, &c);
  return make_double2(mag * c, mag * s);
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
__device__ __forceinline__ float2 warp_sum(float2 v) {
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
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// exp(i kz d) for kz real (propagating) or purely imaginary (evanescent), d >= 0.
// A real call, not inlined: the FP64 exp and sincos are long, and the per-mode
// kernels call this from several places executed by different warps, so one
// shared copy keeps the instruction footprint (and its fetch stalls) down.
static __device__ __noinline__ double2 exp_ikz(double2 kz, double d) {
  const double mag = exp(-kz.y * d);
  double s, c;
  sincos(kz.x * d, &s, &c);
  return make_double2(mag * c, mag * s);
}

// exp(i kz d) for the mixed route: the phase is reduced to [-pi, pi] in FP64
// (three FP64 operations) and the sine, cosine and exponential are taken in FP32
// (FP64 where the decay leaves the FP32 range).  Relative error ~1e-7, the
// precision of the FP32 data; A = E P^T built from the
// rounded factors is still exactly rank one, and the refinement converges to the
// solution of that A, so the rounding enters V~ at ~1e-7 without amplification.
__device__ __forceinline__ double2 exp_ikz32(double2 kz, double d) {
  if (kz.y * d > 80.0) return exp_ikz(kz, d);  // e^-80: the FP32 exponential nears underflow
  const double ph = kz.x * d;
  const double red = fma(-6.283185307179586, rint(ph * 0.15915494309189535), ph);
  float sn, cs;
  sincosf((float)red, &sn, &cs);
  const float mag = expf((float)(-kz.y * d));
  return make_double2((double)(mag * cs), (double)(mag * sn));
}


// F_l = sum_{l' <= l} q^(l - l') s_l' for l < len <= 64, one warp, lanes own two
// consecutive elements; an inclusive scan of the affine maps x -> A x + B.
__device__ __forceinline__ void affine_scan64(const double2* s, int len, double2 q, double2* out) {
  const int lane = threadIdx.x & 31;
  const int l0 = 2 * lane, l1 = l0 + 1;
  const double2 s0 = l0 < len ? s[l0] : make_double2(0, 0);
  const double2 s1 = l1 < len ? s[l1] : make_double2(0, 0);
  double2 A = q * q;
  double2 B = q * s0 + s1;
  for (int off = 1; off < 32; off <<= 1) {
    const double2 Ap = make_double2(__shfl_up_sync(0xffffffffu, A.x, off), __shfl_up_sync(0xffffffffu, A.y, off));
    const double2 Bp = make_double2(__shfl_up_sync(0xffffffffu, B.x, off), __shfl_up_sync(0xffffffffu, B.y, off));
    if (lane >= off) {
      B = A * Bp + B;
      A = A * Ap;
    }
  }
  // B = F_{l1}; F_{l0} = q F_{l0 - 1} + s0
  double2 prev = make_double2(__shfl_up_sync(0xffffffffu, B.x, 1), __shfl_up_sync(0xffffffffu, B.y, 1));
  if (lane == 0) prev = make_double2(0, 0);
  if (l0 < len) out[l0] = q * prev + s0;
  if (l1 < len) out[l1] = B;
}

// The same recurrence F_l = q F_{l-1} + s_l for l < len <= 32 EPL, lanes owning EPL
// consecutive elements: each lane composes its elements' affine maps x -> q x + s_l,
// the warp scans the composed maps (inclusive), and each lane replays its elements
// from the value the scan leaves before it.
template <int EPL>
__device__ __forceinline__ void affine_scan_lanes(const double2* s, int len, double2 q, double2* out) {
  const int lane = threadIdx.x & 31;
  const int l0 = EPL * lane;
  double2 v[EPL];
  double2 A = make_double2(1.0, 0.0), B = make_double2(0.0, 0.0);
#pragma unroll
  for (int j = 0; j < EPL; ++j) {
    v[j] = l0 + j < len ? s[l0 + j] : make_double2(0.0, 0.0);
    B = q * B + v[j];
    A = q * A;
  }
  for (int off = 1; off < 32; off <<= 1) {
    const double2 Ap = make_double2(__shfl_up_sync(0xffffffffu, A.x, off), __shfl_up_sync(0xffffffffu, A.y, off));
    const double2 Bp = make_double2(__shfl_up_sync(0xffffffffu, B.x, off), __shfl_up_sync(0xffffffffu, B.y, off));
    if (lane >= off) {
      B = A * Bp + B;
      A = A * Ap;
    }
  }
  double2 prev = make_double2(__shfl_up_sync(0xffffffffu, B.x, 1), __shfl_up_sync(0xffffffffu, B.y, 1));
  if (lane == 0) prev = make_double2(0.0, 0.0);
#pragma unroll
  for (int j = 0; j < EPL; ++j) {
    prev = q * prev + v[j];
    if (l0 + j < len) out[l0 + j] = prev;
  }
}

}  // namespace fl
