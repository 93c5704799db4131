// Double-float lanes of the node update (the scalar arithmetic is in lbm_df_core.cuh): two
// double-floats on paired FP32 lanes, the numeric constants and per-lattice constants in both lane
// types, and the launchers of the double-float kernels.
//
// GB300 executes FP32 at 128 lanes per SM per clock and FP64 at 2 FMA per SM per clock, so the node
// update in double-float on the FP32 pipes runs several times faster than in FP64 while keeping
// FP64-class accuracy on the shifted populations (whose magnitude is far below one).
//
// The overloads ad, sb, ml, fm, m_rcp, m_log1p, m_expm1 make the lane-generic node update of
// lbm_internal.cuh (node_state_s, node_collide_s) run on df and df2 lanes.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "lbm_df_core.cuh"
#include "lbm_internal.cuh"

namespace lbm {

// ---------------------------------------------------------------------------------------------------
// Two double-floats on paired FP32 lanes: df2 holds nodes (x, y) as hi = (hi_x, hi_y), lo = (lo_x, lo_y),
// and every scalar operation of lbm_df_core.cuh runs on FFMA2 / FADD2 / FMUL2, lane by lane the same FP32 operations in the
// same order (a negation is a sign flip of each half, as in the scalar code), so a df2 result equals
// the two df results bit for bit.
struct df2 {
  float2 hi, lo;
};

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ df df2_get(const df2& v, int j) { return j ? df{v.hi.y, v.lo.y} : df{v.hi.x, v.lo.x}; }
__device__ __forceinline__ void df2_set(df2& v, int j, df a) {
  if (j) { v.hi.y = a.hi; v.lo.y = a.lo; }
  else { v.hi.x = a.hi; v.lo.x = a.lo; }
}
__device__ __forceinline__ df2 df2_of(df a, df b) {
  return df2{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)};
}

__device__ __forceinline__ void two_sum(float2 a, float2 b, float2& s, float2& e) {
  s = p_add(a, b);
  const float2 bb = p_sub(s, a);
  e = p_add(p_sub(a, p_sub(s, bb)), p_sub(b, bb));
}
// a - b: the same operations as two_sum(a, -b).
__device__ __forceinline__ void two_diff(float2 a, float2 b, float2& s, float2& e) {
  s = p_sub(a, b);
  const float2 bb = p_sub(s, a);
  e = p_sub(p_sub(a, p_sub(s, bb)), p_add(b, bb));
}
__device__ __forceinline__ df2 fast_two_sum(float2 a, float2 b) {
  const float2 s = p_add(a, b);
  return df2{s, p_sub(b, p_sub(s, a))};
}

__device__ __forceinline__ df2 ad(df2 x, df2 y) {
  float2 s, e;
  two_sum(x.hi, y.hi, s, e);
  e = p_add(e, p_add(x.lo, y.lo));
  return fast_two_sum(s, e);
}
__device__ __forceinline__ df2 sb(df2 x, df2 y) {
  float2 s, e;
  two_diff(x.hi, y.hi, s, e);
  e = p_add(e, p_sub(x.lo, y.lo));
  return fast_two_sum(s, e);
}
__device__ __forceinline__ df2 ml(df2 x, df2 y) {
  const float2 p = p_mul(x.hi, y.hi);
  float2 e = p_fma(x.hi, y.hi, p_neg(p));
  e = p_fma(x.hi, y.lo, e);
  e = p_fma(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df2 fm(df2 x, df2 y, df2 z) {
  const float2 p = p_mul(x.hi, y.hi);
  float2 e = p_fma(x.hi, y.hi, p_neg(p));
  e = p_fma(x.hi, y.lo, e);
  e = p_fma(x.lo, y.hi, e);
  float2 s, t;
  two_sum(p, z.hi, s, t);
  t = p_add(t, p_add(e, z.lo));
  return fast_two_sum(s, t);
}
__device__ __forceinline__ df2 m_rcp(df2 x) {
  float2 y = make_float2(rcp_approx(x.hi.x), rcp_approx(x.hi.y));
  y = p_fma(y, p_fma(p_neg(x.hi), y, make_float2(1.0f, 1.0f)), y);
  const float2 p = p_mul(x.hi, y);
  const float2 e = p_fma(x.hi, y, p_neg(p));
  const float2 r = p_sub(p_sub(p_sub(make_float2(1.0f, 1.0f), p), e), p_mul(x.lo, y));
  return fast_two_sum(y, p_mul(y, r));
}

__device__ __forceinline__ float2 pc(float v) { return make_float2(v, v); }
__device__ __forceinline__ df2 dfc2(float hi, float lo) { return df2{pc(hi), pc(lo)}; }

// The series of m_log1p(df) on both lanes; lanes outside |x| <= 0.3 take the FP64 fallback of the
// scalar function, lane by lane (the common case, both lanes inside, never leaves the paired path).
__device__ __forceinline__ df2 log1p_series2(df2 x) {
  const df2 z = ml(x, m_rcp(ad(dfc2(2.0f, 0.0f), x)));
  const df2 w = ml(z, z);
  const float2 wf = w.hi;
  float2 q = pc(1.0f / 21.0f);
  q = p_fma(q, wf, pc(1.0f / 19.0f));
  q = p_fma(q, wf, pc(1.0f / 17.0f));
  q = p_fma(q, wf, pc(1.0f / 15.0f));
  q = p_fma(q, wf, pc(1.0f / 13.0f));
  q = p_fma(q, wf, pc(1.0f / 11.0f));
  df2 p = fm(w, df2{q, pc(0.0f)}, dfc2(0.111111112f, -8.27842295e-10f));
  p = fm(w, p, dfc2(0.142857149f, -6.38621200e-09f));
  p = fm(w, p, dfc2(0.200000003f, -2.98023228e-09f));
  p = fm(w, p, dfc2(0.333333343f, -9.93410776e-09f));
  p = fm(w, p, dfc2(1.0f, 0.0f));
  return ml(df2{p_mul(pc(2.0f), z.hi), p_mul(pc(2.0f), z.lo)}, p);
}
__device__ __forceinline__ df2 m_log1p(df2 x) {
  const bool in0 = fabsf(x.hi.x) <= 0.3f, in1 = fabsf(x.hi.y) <= 0.3f;
  df2 r = log1p_series2(x);
  if (in0 && in1) return r;
  if (!in0) df2_set(r, 0, m_log1p(df2_get(x, 0)));
  if (!in1) df2_set(r, 1, m_log1p(df2_get(x, 1)));
  return r;
}

__device__ __forceinline__ df2 expm1_series2(df2 x) {
  const float2 xf = x.hi;
  float2 t = pc(1.0f / 87178291200.0f);
  t = p_fma(t, xf, pc(1.0f / 6227020800.0f));
  t = p_fma(t, xf, pc(1.0f / 479001600.0f));
  t = p_fma(t, xf, pc(1.0f / 39916800.0f));
  t = p_fma(t, xf, pc(1.0f / 3628800.0f));
  t = p_fma(t, xf, pc(1.0f / 362880.0f));
  t = p_fma(t, xf, pc(1.0f / 40320.0f));
  df2 s = fm(x, df2{t, pc(0.0f)}, dfc2(0.000198412701f, -2.72559687e-12f));
  s = fm(x, s, dfc2(0.00138888892f, -3.36310944e-11f));
  s = fm(x, s, dfc2(0.00833333377f, -4.34617203e-10f));
  s = fm(x, s, dfc2(0.0416666679f, -1.24176347e-09f));
  s = fm(x, s, dfc2(0.166666672f, -4.96705388e-09f));
  s = fm(x, s, dfc2(0.5f, 0.0f));
  return fm(ml(x, x), s, x);
}
__device__ __forceinline__ df2 m_expm1(df2 x) {
  const bool in0 = fabsf(x.hi.x) <= 0.35f, in1 = fabsf(x.hi.y) <= 0.35f;
  df2 r = expm1_series2(x);
  if (in0 && in1) return r;
  if (!in0) df2_set(r, 0, m_expm1(df2_get(x, 0)));
  if (!in1) df2_set(r, 1, m_expm1(df2_get(x, 1)));
  return r;
}

// The entropy source of the node update on double-float lanes. Where the increment is tiny, as on every
// smooth wave (about 1e-16 on the 2^26-node benchmark wave, 1e-10 on a 65 536-node one), it is taken in
// FP32 from the double-float differences du', dtheta rounded once: about a dozen FP32 roundings and
// the FP32 reciprocal, a relative error below 1e-6, so below 2.3e-16 of the field scale per step when
// |dt S| <= 2^-32, under the double-float rounding of the fields themselves. Elsewhere (a shock) it is
// the double-float evaluation of the generic form. Lane by lane on paired lanes, so that a pair gives
// each node the result it gets alone (the double-float form runs when either lane needs it).
constexpr float kSourceFastMax = 2.3283064e-10f;  // 2^-32
template <>
constexpr bool kSourceOverloaded<df> = true;
template <>
constexpr bool kSourceOverloaded<df2> = true;

__device__ __forceinline__ float source_fast_f32(const df& du, const df& dth, const df& rho1, const df& th,
                                                 const df& q_src, const df& inv_Pr) {
  const float ith = rcp_approx(th.hi);
  const float A = __fmaf_rn(__fmul_rn(dth.hi, dth.hi), __fmul_rn(ith, inv_Pr.hi), __fmul_rn(du.hi, du.hi));
  return __fmul_rn(__fmul_rn(__fmul_rn(q_src.hi, rho1.hi), ith), A);
}

__device__ __forceinline__ df source_update(df z, df rho1, df th, df ul, df ur, df thl, df thr, df q_src, df inv_Pr) {
  const df du = sb(ur, ul), dth = sb(thr, thl);
  const float q = source_fast_f32(du, dth, rho1, th, q_src, inv_Pr);
  if (fabsf(q) <= kSourceFastMax) return ad(z, df{q, 0.0f});
  const df ith = m_rcp(th);
  const df A = fm(ml(dth, dth), ml(ith, inv_Pr), ml(du, du));
  return fm(ml(ml(q_src, rho1), ith), A, z);
}

__device__ __forceinline__ df2 source_update(df2 z, df2 rho1, df2 th, df2 ul, df2 ur, df2 thl, df2 thr, df2 q_src,
                                             df2 inv_Pr) {
  const df2 du = sb(ur, ul), dth = sb(thr, thl);
  // The FP32 form on both lanes, the same FP32 operations as the scalar one.
  const float2 ith = make_float2(rcp_approx(th.hi.x), rcp_approx(th.hi.y));
  const float2 A = __ffma2_rn(__fmul2_rn(dth.hi, dth.hi), __fmul2_rn(ith, inv_Pr.hi), __fmul2_rn(du.hi, du.hi));
  const float2 q = __fmul2_rn(__fmul2_rn(__fmul2_rn(q_src.hi, rho1.hi), ith), A);
  const bool fx = fabsf(q.x) <= kSourceFastMax, fy = fabsf(q.y) <= kSourceFastMax;
  df2 r = ad(z, df2{q, make_float2(0.0f, 0.0f)});
  if (fx && fy) return r;
  const df2 ithd = m_rcp(th);
  const df2 Ad = fm(ml(dth, dth), ml(ithd, inv_Pr), ml(du, du));
  const df2 slow = fm(ml(ml(q_src, rho1), ithd), Ad, z);
  if (!fx) df2_set(r, 0, df2_get(slow, 0));
  if (!fy) df2_set(r, 1, df2_get(slow, 1));
  return r;
}

template <>
__device__ __forceinline__ df num<df>(double v) { return df{(float)v, (float)(v - (double)(float)v)}; }
template <>
__device__ __forceinline__ df2 num<df2>(double v) {
  const df a = num<df>(v);
  return df2{make_float2(a.hi, a.hi), make_float2(a.lo, a.lo)};
}

// Consts<df2> from Consts<df>: every double-float field on both lanes (host).
inline Consts<df2> pair_consts(const Consts<df>& c) {
  constexpr size_t n = offsetof(Consts<df>, eq_mode) / sizeof(df);
  static_assert(offsetof(Consts<df2>, eq_mode) == n * sizeof(df2), "Consts layout");
  Consts<df2> p;
  const df* s = reinterpret_cast<const df*>(&c);
  df2* t = reinterpret_cast<df2*>(&p);
  for (size_t i = 0; i < n; ++i) t[i] = df2{make_float2(s[i].hi, s[i].hi), make_float2(s[i].lo, s[i].lo)};
  p.eq_mode = c.eq_mode;
  p.source_on = c.source_on;
  return p;
}

// Step kernel in double-float (lbm_step_df.cu): FP64 storage, tiles of NT*V nodes, K steps per launch.
bool valid_df_config(int K, int NT, int V);
cudaError_t launch_step_tiles_df(const double* in, double* out, long long plane, const LatDev* lat,
                                 const int* tile_lat, int B, long long ntiles, int K, int NT, int V,
                                 const Consts<df>& c, cudaStream_t st, long long grid_cap);

// Adjoint block kernel on double-float lanes over FP64 storage (lbm_adjoint.cu).
cudaError_t launch_adjoint_block_df(const double* f0, const double* a_next, double* a_out, long long plane,
                                    const LatDev* lat, int B, long long ntiles, int K, const Consts<df>& c,
                                    double* grad_tile, cudaStream_t st);

}  // namespace lbm
