// Scalar double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, about 48 significant bits. Built from the error-free transformations of Knuth
// (TwoSum), Dekker (FastTwoSum) and the FMA-based exact product, as in Dekker (1971), "A floating-point
// technique for extending the available precision", and Hida, Li and Bailey (2001), "Algorithms for
// quad-double precision floating point arithmetic" (their double-double operations, here on FP32).
// Every FP32 operation is a round-to-nearest intrinsic, which the compiler never fuses or reorders.
// Used by the double-float kernels (lbm_df.cuh adds the paired lanes) and by the FP64 lanes of the node
// update for their logarithm and exponential (lbm_internal.cuh).
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// FP32 reciprocal by the hardware approximation, one MUFU operation (relative error about 2^-23;
// subnormal inputs and results flush to zero, which the positive, order-one denominators of the node
// update never reach).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct df {
  float hi, lo;
};

// Host construction from a double: hi = the nearest float, lo = the nearest float to the remainder.
__host__ __device__ __forceinline__ df df_from_double_host(double v) {
  const float h = (float)v;
  return df{h, (float)(v - (double)h)};
}

// Device conversions (run on the FP64 pipe; used only at tile loads and stores and per tile for the
// lattice parameters).
__device__ __forceinline__ df to_df(double v) {
  const float h = __double2float_rn(v);
  return df{h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double to_double(df x) { return (double)x.hi + (double)x.lo; }

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df ad(df x, df y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s, e);
}
__device__ __forceinline__ df sb(df x, df y) { return ad(x, df{-y.hi, -y.lo}); }
__device__ __forceinline__ df ml(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);  // exact error of the product
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
// x y + z with one normalisation.
__device__ __forceinline__ df fm(df x, df y, df z) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  float s, t;
  two_sum(p, z.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(e, z.lo));
  return fast_two_sum(s, t);
}
// FP32 reciprocal of a to within about an ulp: the hardware approximation and one Newton step.
__device__ __forceinline__ float rcp_f32(float a) {
  const float y = rcp_approx(a);
  return __fmaf_rn(y, __fmaf_rn(-a, y, 1.0f), y);
}

// 1/x: the FP32 reciprocal y of x.hi, then one Newton step y (1 + r) with the residual r = 1 - x y
// evaluated exactly to first order (FMA-based product error).
__device__ __forceinline__ df m_rcp(df x) {
  const float y = rcp_f32(x.hi);
  const float p = __fmul_rn(x.hi, y);
  const float e = __fmaf_rn(x.hi, y, -p);
  const float r = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), e), __fmul_rn(x.lo, y));
  return fast_two_sum(y, __fmul_rn(y, r));
}

__device__ __forceinline__ df dfc(float hi, float lo) { return df{hi, lo}; }

// log(1 + x) for |x| <= 0.3 by the series 2 atanh(z) = 2 z (1 + w/3 + w^2/5 + ...), z = x / (2 + x),
// w = z^2 <= 0.0312: the terms w^k/(2k+1) for k >= 5 (below 2.7e-9) in FP32 Horner form, the rest in
// double-float. Outside that range (or for non-finite x): FP64 log1p.
__device__ __forceinline__ df m_log1p(df x) {
  if (!(fabsf(x.hi) <= 0.3f)) return to_df(log1p(to_double(x)));
  const df z = ml(x, m_rcp(ad(df{2.0f, 0.0f}, x)));
  const df w = ml(z, z);
  const float wf = w.hi;
  float q = 1.0f / 21.0f;
  q = __fmaf_rn(q, wf, 1.0f / 19.0f);
  q = __fmaf_rn(q, wf, 1.0f / 17.0f);
  q = __fmaf_rn(q, wf, 1.0f / 15.0f);
  q = __fmaf_rn(q, wf, 1.0f / 13.0f);
  q = __fmaf_rn(q, wf, 1.0f / 11.0f);
  // 1/9, 1/7, 1/5, 1/3 to double-float precision.
  df p = fm(w, df{q, 0.0f}, dfc(0.111111112f, -8.27842295e-10f));
  p = fm(w, p, dfc(0.142857149f, -6.38621200e-09f));
  p = fm(w, p, dfc(0.200000003f, -2.98023228e-09f));
  p = fm(w, p, dfc(0.333333343f, -9.93410776e-09f));
  p = fm(w, p, df{1.0f, 0.0f});
  return ml(df{2.0f * z.hi, 2.0f * z.lo}, p);
}

// exp(x) - 1 for |x| <= 0.35 by its Taylor series x + x^2 (1/2! + x/3! + ... ): the terms from
// x^8/8! on (relative size below 2e-8) in FP32 Horner form up to x^14/14!, the rest in double-float.
// Outside that range (or for non-finite x): FP64 expm1.
__device__ __forceinline__ df m_expm1(df x) {
  if (!(fabsf(x.hi) <= 0.35f)) return to_df(expm1(to_double(x)));
  const float xf = x.hi;
  float t = 1.0f / 87178291200.0f;             // 1/14!
  t = __fmaf_rn(t, xf, 1.0f / 6227020800.0f);  // 1/13!
  t = __fmaf_rn(t, xf, 1.0f / 479001600.0f);   // 1/12!
  t = __fmaf_rn(t, xf, 1.0f / 39916800.0f);    // 1/11!
  t = __fmaf_rn(t, xf, 1.0f / 3628800.0f);     // 1/10!
  t = __fmaf_rn(t, xf, 1.0f / 362880.0f);      // 1/9!
  t = __fmaf_rn(t, xf, 1.0f / 40320.0f);       // 1/8!
  // 1/7!, 1/6!, 1/5!, 1/4!, 1/3!, 1/2! to double-float precision.
  df s = fm(x, df{t, 0.0f}, dfc(0.000198412701f, -2.72559687e-12f));
  s = fm(x, s, dfc(0.00138888892f, -3.36310944e-11f));
  s = fm(x, s, dfc(0.00833333377f, -4.34617203e-10f));
  s = fm(x, s, dfc(0.0416666679f, -1.24176347e-09f));
  s = fm(x, s, dfc(0.166666672f, -4.96705388e-09f));
  s = fm(x, s, df{0.5f, 0.0f});
  return fm(ml(x, x), s, x);
}

}  // namespace lbm
