// Two-float arithmetic for the mixed-precision per-mode kernels (the dense solve's
// refinement residual and V~, the rank-one closed form's sums and root): FP64-class
// accuracy on the FP32 pipe, which this GPU runs at 64 times its FP64 rate.
#pragma once

#include "common.cuh"

namespace fl {

// ------------------------------------------------------------------------------
// two-float arithmetic: a value is hi + lo (|lo| <= ulp(hi)/2); sums and products
// use the error-free transformations TwoSum (Knuth) and TwoProd (with fma), which
// gives about 48 significant bits on the FP32 pipe.  The mixed route computes its
// refinement residual and V~ = A^H y this way: FP64-class accuracy without the
// FP64 pipe, which runs at 1/64 of the FP32 rate on this GPU.
// ------------------------------------------------------------------------------
struct ff { float hi, lo; };
struct ffc { ff re, im; };

__device__ __forceinline__ ff ff_from(double x) {
  ff r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ double ff_to(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
  ff r;
  r.hi = a + b;
  r.lo = b - (r.hi - a);
  return r;
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return fast_two_sum(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ffc ffc_from(double2 z) { return ffc{ff_from(z.x), ff_from(z.y)}; }
__device__ __forceinline__ double2 ffc_to(ffc z) { return make_double2(ff_to(z.re), ff_to(z.im)); }
__device__ __forceinline__ ffc ffc_zero() { return ffc{ff{0.f, 0.f}, ff{0.f, 0.f}}; }
__device__ __forceinline__ ffc ffc_add(ffc a, ffc b) { return ffc{ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
__device__ __forceinline__ ffc ffc_sub(ffc a, ffc b) { return ffc{ff_add(a.re, ff_neg(b.re)), ff_add(a.im, ff_neg(b.im))}; }
__device__ __forceinline__ ffc ffc_mul(ffc a, ffc b) {
  return ffc{ff_add(ff_mul(a.re, b.re), ff_neg(ff_mul(a.im, b.im))), ff_add(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}
__device__ __forceinline__ ffc ffc_conj_mul(ffc a, ffc b) {  // conj(a) b
  return ffc{ff_add(ff_mul(a.re, b.re), ff_mul(a.im, b.im)), ff_add(ff_mul(a.re, b.im), ff_neg(ff_mul(a.im, b.re)))};
}
// Compensated dot products of two-float operands (the Dot2 scheme of Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005): the rounded
// products hi*hi are summed exactly by TwoSum into s, and every rounding error (of
// those sums, of the products, and the cross terms hi*lo + lo*hi) is summed in plain
// FP32 into e.  As accurate as summing in two-float (the errors are O(u) terms summed
// with relative error O(n u)), for two thirds of the operations.
struct dot2 { float s, e; };
struct dot2c { dot2 re, im; };
__device__ __forceinline__ void dot2_add(dot2& d, float p, float ep) {  // d += p + ep
  const float t = d.s + p;
  const float bb = t - d.s;
  d.e += ((d.s - (t - bb)) + (p - bb)) + ep;
  d.s = t;
}
__device__ __forceinline__ void dot2_mac(dot2& d, ff a, ff b) {  // d += a b
  const float p = a.hi * b.hi;
  dot2_add(d, p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p))));
}
__device__ __forceinline__ void dot2_msub(dot2& d, ff a, ff b) { dot2_mac(d, ff_neg(a), b); }  // d -= a b
__device__ __forceinline__ void dot2c_conj_mac(dot2c& d, ffc a, ffc b) {  // d += conj(a) b
  dot2_mac(d.re, a.re, b.re);
  dot2_mac(d.re, a.im, b.im);
  dot2_mac(d.im, a.re, b.im);
  dot2_msub(d.im, a.im, b.re);
}
__device__ __forceinline__ void dot2c_mac(dot2c& d, ffc a, ffc b) {  // d += a b
  dot2_mac(d.re, a.re, b.re);
  dot2_msub(d.re, a.im, b.im);
  dot2_mac(d.im, a.re, b.im);
  dot2_mac(d.im, a.im, b.re);
}
__device__ __forceinline__ dot2c dot2c_zero() { return dot2c{dot2{0.f, 0.f}, dot2{0.f, 0.f}}; }
__device__ __forceinline__ ffc dot2c_ffc(dot2c d) {
  return ffc{fast_two_sum(d.re.s, d.re.e), fast_two_sum(d.im.s, d.im.e)};
}

__device__ __forceinline__ ffc ffc_shfl_xor(ffc a, int m) {
  ffc r;
  r.re.hi = __shfl_xor_sync(0xffffffffu, a.re.hi, m);
  r.re.lo = __shfl_xor_sync(0xffffffffu, a.re.lo, m);
  r.im.hi = __shfl_xor_sync(0xffffffffu, a.im.hi, m);
  r.im.lo = __shfl_xor_sync(0xffffffffu, a.im.lo, m);
  return r;
}

// exact product of two floats, and the operations of the rank-one closed form
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = a * b;
  return ff{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {  // a b
  const float p = a.hi * b;
  return fast_two_sum(p, fmaf(a.lo, b, fmaf(a.hi, b, -p)));
}
// a / b (b != 0): the FP32 quotient, then one correction from the two-float remainder
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  const float q1 = a.hi / b.hi;
  const ff r = ff_sub(a, ff_mul_f(b, q1));
  return fast_two_sum(q1, (r.hi + r.lo) / b.hi);
}
// sqrt(a), a >= 0: the FP32 root s, then s + (a - s^2) / (2 s)
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (!(a.hi > 0.f)) return ff{0.f, 0.f};
  const float s = sqrtf(a.hi);
  const ff e = ff_sub(a, two_prod(s, s));
  return fast_two_sum(s, (e.hi + e.lo) * (0.5f / s));
}
__device__ __forceinline__ bool ff_gt(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ ff ff_shfl_xor(ff a, int m) {
  return ff{__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}
__device__ __forceinline__ ff ff_warp_sum(ff a) {
  for (int o = 16; o > 0; o >>= 1) a = ff_add(a, ff_shfl_xor(a, o));
  return a;
}
__device__ __forceinline__ ffc ffc_warp_sum(ffc a) {
  for (int o = 16; o > 0; o >>= 1) a = ffc_add(a, ffc_shfl_xor(a, o));
  return a;
}
// a b, a two-float complex, b an FP32 complex
__device__ __forceinline__ ffc ffc_mul_f2(ffc a, float2 b) {
  return ffc{ff_sub(ff_mul_f(a.re, b.x), ff_mul_f(a.im, b.y)), ff_add(ff_mul_f(a.re, b.y), ff_mul_f(a.im, b.x))};
}
// conj(b) a
__device__ __forceinline__ ffc ffc_conj_f2_mul(float2 b, ffc a) {
  return ffc{ff_add(ff_mul_f(a.re, b.x), ff_mul_f(a.im, b.y)), ff_sub(ff_mul_f(a.im, b.x), ff_mul_f(a.re, b.y))};
}
__device__ __forceinline__ ff ffc_abs2(ffc a) { return ff_add(ff_mul(a.re, a.re), ff_mul(a.im, a.im)); }
__device__ __forceinline__ float2 ffc_to_f2(ffc a) { return make_float2(a.re.hi + a.re.lo, a.im.hi + a.im.lo); }

}  // namespace fl
