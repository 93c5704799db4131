// Internal declarations of the D1Q3Q3 CUDA library: per-lattice parameter records, the constant
// block passed to kernels, and the per-node collision of section 8 written on shifted
// populations. Used by the .cu files of this library only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_df_core.cuh"

namespace lbm {

// Bounds-checked debug build. Compiled with -DLBM_DEBUG_BOUNDS, the step, persistent, double-float and
// adjoint kernels check every global and shared-memory index they compute against the extent it must
// lie in before the access; an index outside is counted, the first one is recorded with its extent,
// and the access is skipped (a load gives zero), so the kernel runs to its end instead of faulting. The
// record is per translation unit (take_bounds_record reads and clears it); lbm_debug_bounds gathers
// them. Without the flag in_bounds is the constant true and the checks compile away.
#ifdef LBM_DEBUG_BOUNDS
static __device__ unsigned long long g_bounds_rec[3];  // violations, first index, its extent
static __device__ __noinline__ bool bounds_violation(long long i, long long n) {
  if (atomicAdd(&g_bounds_rec[0], 1ULL) == 0ULL) {
    atomicExch(&g_bounds_rec[1], (unsigned long long)i);
    atomicExch(&g_bounds_rec[2], (unsigned long long)n);
  }
  return false;
}
__device__ __forceinline__ bool in_bounds(long long i, long long n) {
  return (i >= 0 && i < n) ? true : bounds_violation(i, n);
}
static inline cudaError_t take_bounds_record(unsigned long long out[3]) {
  cudaError_t e = cudaMemcpyFromSymbol(out, g_bounds_rec, sizeof(unsigned long long) * 3);
  if (e != cudaSuccess) return e;
  const unsigned long long zero[3] = {0ULL, 0ULL, 0ULL};
  return cudaMemcpyToSymbol(g_bounds_rec, zero, sizeof(zero));
}
#else
__device__ __forceinline__ constexpr bool in_bounds(long long, long long) { return true; }
#endif
// Reads and clears the bounds record of lbm_step.cu, lbm_step_df.cu, lbm_adjoint.cu and lbm2d.cu (zeros
// when the build has no checks).
cudaError_t bounds_record_step(unsigned long long out[3]);
cudaError_t bounds_record_df(unsigned long long out[3]);
cudaError_t bounds_record_adjoint(unsigned long long out[3]);
cudaError_t bounds_record_2d(unsigned long long out[3]);
cudaError_t bounds_record_3d(unsigned long long out[3]);

// Per-lattice record on the device. tile0 is the index of the lattice's first tile for the current
// tile width; chunk0 the index of its first diagnostics chunk.
struct LatDev {
  long long offset, n, tile0, chunk0;
  double s_e, s_psi, s_eps;
  double q_src;    // sigma_e / 4: the source reads dt S = rho sigma_e/(4T) [du^2 + (c_p/Pr) dT^2 / T]
  double s0;       // reference entropy of eq. (gaz-parfait) for this lattice
  double zeta_r;   // rest-state moments removed from the stored populations: zeta_r = rho0 s0,
  double eps_r;    //   eps_r = e_r s0 (e_r = 3 p0 - 2 lambda^2 rho0)
  double wg0, wg1; // rest g populations (g0, g+ = g-)
  double s0h;      // s0 / c_p
  double lin_e0, lin_p0, lin_q0;  // constant terms of the linear equilibria in scaled moments
  int bc, pad;
  // s_e, s_psi, s_eps, q_src, s0h, lin_e0, lin_p0, lin_q0 rounded to FP32 on the host, for the FP32
  // kernels (a double-to-float conversion on the device runs on the slow FP64 pipe), and the low parts
  // v - (float)v of the same eight values for the double-float kernels (value = f32[i] + f32lo[i]).
  float f32[8];
  float f32lo[8];
};

// The per-lattice parameters of the step kernels in the arithmetic type R.
template <typename R>
struct StepParams {
  R s_e, s_psi, s_eps, q_src, s0h, lin_e0, lin_p0, lin_q0;
};
__device__ __forceinline__ StepParams<double> step_params(const LatDev& d, double) {
  return {d.s_e, d.s_psi, d.s_eps, d.q_src, d.s0h, d.lin_e0, d.lin_p0, d.lin_q0};
}
__device__ __forceinline__ StepParams<float> step_params(const LatDev& d, float) {
  return {d.f32[0], d.f32[1], d.f32[2], d.f32[3], d.f32[4], d.f32[5], d.f32[6], d.f32[7]};
}

// Constants shared by all lattices, converted on the host to the lane type X the node arithmetic
// runs in: double, float, or float2 (two nodes per lane for Blackwell's paired FP32 instructions;
// every field then holds the same value twice, so it can be an operand of a paired instruction).
template <typename X>
struct Consts {
  X rho0, lam, two_lam2;          // rho0, lambda, 2 lambda^2
  X inv_af, inv_af_l, inv_af_l2;  // 1/rho0, 1/(rho0 lambda), 1/(rho0 lambda^2)
  X af_l, af_l2;                  // rho0 lambda, rho0 lambda^2
  X ag, ag_l, ag_l2;              // rho0 c_p, rho0 c_p lambda, rho0 c_p lambda^2
  X inv_ag, inv_ag_l, inv_ag_l2;
  X gamma, inv_cp, p0, inv_r;     // gamma, 1/c_p, p0, 1/r with r = c_p (1 - 1/gamma)
  X e_r;                          // 3 p0 - 2 lambda^2 rho0
  X cp_log;                       // (1 - 1/gamma) c_p
  X cp_over_Pr;                   // c_p / Pr
  X m_two_lam2;                   // -2 lambda^2
  X one, m_one, two, m_two, three, half, m_half, third, sixth;  // numeric constants
  // Dimensionless form used by the step kernels (see node_state_s).
  X kp;        // p0 / (rho0 lambda^2)
  X kth;       // kp gamma / (gamma - 1)
  X e_rs;      // e_r / (rho0 lambda^2) = 3 kp - 2
  X one_m_ig;  // 1 - 1/gamma
  X inv_Pr;    // 1 / Pr
  // Linear equilibria (section 7) in scaled moments: x_eq = x0 (per lattice) + xR r + xJ j + xZ z.
  X leR, leJ, leZ, lpR, lpJ, lpZ, lqR, lqJ, lqZ;
  int eq_mode;   // 0 nonlinear (section 8), 1 linear (section 7)
  int source_on;
};

// Lane arithmetic: add, sub, mul, fused multiply-add, reciprocal. Adds and multiplies are the
// round-to-nearest intrinsics, which the compiler never fuses, so every fused multiply-add is an
// explicit fm() and a node's result does not depend on how its kernel instantiation was optimised
// (the tile shapes and depths give bitwise identical states).
__device__ __forceinline__ float ad(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double ad(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float2 ad(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float sb(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sb(double a, double b) { return __dsub_rn(a, b); }
// a - b as a + b * (-1): the product is exact, so this is the correctly rounded difference in one
// paired instruction (negating both halves of b would take two more).
__device__ __forceinline__ float2 sb(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float ml(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double ml(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float2 ml(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fm(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 fm(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// Reciprocals: FP32 uses the hardware approximation (rcp_approx, lbm_df_core.cuh), one MUFU operation.
// FP64 refines the same FP32 estimate by two Newton-Raphson steps in FP64, y <- y + y (1 - x y), each
// squaring the relative error (about 2^-23, then 2^-46, then below FP64 rounding): four FP64 fused
// multiply-adds, where this GPU's FP64 pipe runs 2 per SM and clock. The node update's denominators
// are positive and of order one, far inside FP32 range.
__device__ __forceinline__ float m_rcp(float x) { return rcp_approx(x); }
__device__ __forceinline__ double m_rcp(double x) {
  double y = (double)rcp_approx((float)x);
  y = fma(y, fma(-x, y, 1.0), y);
  return fma(y, fma(-x, y, 1.0), y);
}
__device__ __forceinline__ float2 m_rcp(float2 x) { return make_float2(rcp_approx(x.x), rcp_approx(x.y)); }

// log(1 + x) and exp(x) - 1. double and float use CUDA's functions. On paired lanes they are
// evaluated with textbook series in paired arithmetic:
//  - log1p(x) = m ln 2 + 2 atanh(z), z = t / (2 + t), with t = x and m = 0 for |x| <= 0.3, else
//    1 + x = 2^m (1 + t), 1 + t in [0.75, 1.5); 2 atanh(z) = 2 z (1 + w/3 + w^2/5 + ... + w^4/9),
//    w = z^2 <= 0.04 (first omitted term w^5/11 below 1e-8 relative, a sixth of an FP32 ulp);
//  - expm1(x) = 2^k expm1(r) + (2^k - 1), x = k ln 2 + r, |r| <= ln(2)/2 (k = 0 for |x| <= 0.35),
//    expm1(r) = r + r^2 (1/2! + r/3! + ... + r^5/7!) (first omitted term r^8/8! below 2e-8 of
//    expm1(r), a third of an FP32 ulp).
// FP64 lanes evaluate log1p and expm1 in double-float on the FP32 pipes (the series of
// lbm_df_core.cuh for |x| <= 0.3 and |x| <= 0.35, relative error below 2^-45, CUDA's FP64 functions
// outside), the argument split into hi + lo and the result summed back: GB300's FP32 pipes are 64 times
// wider than its FP64 pipe, where these two functions took a third of the node update's FP64 work.
__device__ __forceinline__ double m_log1p(double x) { return to_double(m_log1p(to_df(x))); }
__device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double m_expm1(double x) { return to_double(m_expm1(to_df(x))); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }

__device__ __forceinline__ float2 atanh2_series(float2 t) {  // 2 atanh(t / (2 + t)) for |t| <= 0.5
  const float2 d = __fadd2_rn(t, make_float2(2.0f, 2.0f));
  const float2 nd = __ffma2_rn(t, make_float2(-1.0f, -1.0f), make_float2(-2.0f, -2.0f));  // -d
  float2 y = m_rcp(d);
  y = __ffma2_rn(y, __ffma2_rn(nd, y, make_float2(1.0f, 1.0f)), y);  // Newton step
  const float2 z = __fmul2_rn(t, y);
  const float2 w = __fmul2_rn(z, z);
  float2 p = make_float2(1.0f / 9.0f, 1.0f / 9.0f);
  p = __ffma2_rn(p, w, make_float2(1.0f / 7.0f, 1.0f / 7.0f));
  p = __ffma2_rn(p, w, make_float2(1.0f / 5.0f, 1.0f / 5.0f));
  p = __ffma2_rn(p, w, make_float2(1.0f / 3.0f, 1.0f / 3.0f));
  const float2 z2 = __fadd2_rn(z, z);
  return __ffma2_rn(__fmul2_rn(z2, w), p, z2);
}

// 1 + x = 2^m (1 + t) with 1 + t in [0.75, 1.5) (x > -1 and finite; t = x, m = 0 when |x| <= 0.3).
__device__ __forceinline__ void log1p_reduce(float x, float& t, float& m) {
  if (fabsf(x) <= 0.3f) { t = x; m = 0.0f; return; }
  const float y = 1.0f + x;
  int e = ((__float_as_int(y) >> 23) & 0xff) - 127;             // y = 2^e * mant, mant in [1, 2)
  float mant = __int_as_float((__float_as_int(y) & 0x007fffff) | 0x3f800000);
  if (mant >= 1.5f) { mant *= 0.5f; e += 1; }
  t = mant - 1.0f;
  m = (float)e;
}

// Every lane's value depends on that lane alone (the other lane of the pair only decides whether the
// range reduction runs): a lane inside the series range reduces to t = x, m = 0, and a lane outside
// the domain takes CUDA's function.
__device__ __forceinline__ float2 m_log1p(float2 x) {
  if (fabsf(x.x) <= 0.3f && fabsf(x.y) <= 0.3f) return atanh2_series(x);
  const bool okx = x.x > -1.0f && x.x < 3.0e38f, oky = x.y > -1.0f && x.y < 3.0e38f;
  float2 t = make_float2(0.0f, 0.0f), m = make_float2(0.0f, 0.0f);
  if (okx) log1p_reduce(x.x, t.x, m.x);
  if (oky) log1p_reduce(x.y, t.y, m.y);
  const float2 a = atanh2_series(t);
  const float ln2_hi = 0.693145752f, ln2_lo = 1.42860677e-06f;  // ln 2 = hi + lo, hi with 17 bits
  float2 r = __ffma2_rn(m, make_float2(ln2_hi, ln2_hi), __ffma2_rn(m, make_float2(ln2_lo, ln2_lo), a));
  if (!okx) r.x = log1pf(x.x);  // outside the domain or non-finite
  if (!oky) r.y = log1pf(x.y);
  return r;
}

__device__ __forceinline__ float2 expm1_series(float2 x) {  // |x| <= 0.35
  float2 p = make_float2(1.0f / 5040.0f, 1.0f / 5040.0f);
  p = __ffma2_rn(p, x, make_float2(1.0f / 720.0f, 1.0f / 720.0f));
  p = __ffma2_rn(p, x, make_float2(1.0f / 120.0f, 1.0f / 120.0f));
  p = __ffma2_rn(p, x, make_float2(1.0f / 24.0f, 1.0f / 24.0f));
  p = __ffma2_rn(p, x, make_float2(1.0f / 6.0f, 1.0f / 6.0f));
  p = __ffma2_rn(p, x, make_float2(0.5f, 0.5f));
  return __ffma2_rn(__fmul2_rn(x, x), p, x);
}

__device__ __forceinline__ float2 m_expm1(float2 x) {
  if (fabsf(x.x) <= 0.35f && fabsf(x.y) <= 0.35f) return expm1_series(x);
  // k = round(x / ln 2); 0 on a lane inside the series range (2^0 expm1(x) + 0 is its series value)
  // and on a lane outside |x| <= 80 or non-finite, which takes CUDA's function.
  const bool okx = fabsf(x.x) <= 80.0f, oky = fabsf(x.y) <= 80.0f;
  const float kx = (okx && !(fabsf(x.x) <= 0.35f)) ? rintf(x.x * 1.44269504f) : 0.0f;
  const float ky = (oky && !(fabsf(x.y) <= 0.35f)) ? rintf(x.y * 1.44269504f) : 0.0f;
  const float2 k = make_float2(kx, ky);
  const float ln2_hi = 0.693145752f, ln2_lo = 1.42860677e-06f;
  float2 r = __ffma2_rn(k, make_float2(-ln2_hi, -ln2_hi), x);
  r = __ffma2_rn(k, make_float2(-ln2_lo, -ln2_lo), r);
  const float2 e = expm1_series(r);
  const float2 two_k = make_float2(__int_as_float(((int)kx + 127) << 23), __int_as_float(((int)ky + 127) << 23));
  float2 out = __ffma2_rn(two_k, e, __fadd2_rn(two_k, make_float2(-1.0f, -1.0f)));
  if (!okx) out.x = expm1f(x.x);
  if (!oky) out.y = expm1f(x.y);
  return out;
}

// Moments and thermodynamic state of one node (or node pair) from its shifted populations
// f - w (order f0, f+, f-, g0, g+, g-). Fields marked "t" (tilde) are deviations from the rest state.
template <typename X>
struct Node {
  X rt, J, et;       // rho - rho0, J, e - e_r
  X zt, psi, epst;   // zeta - zeta_r, psi, eps - eps_r
  X rho, inv_rho, u, ds, lnr, pt, T;  // rho, 1/rho, u, s - s0, log(rho/rho0), p - p0, T
};

template <typename X>
__device__ __forceinline__ void node_state(const X f[6], const Consts<X>& c, X s0, Node<X>& m) {
  // (ii) m = M f_d, eq. (M-d1q3q3), applied to the deviations from the rest populations.
  const X tf = ad(f[1], f[2]), tg = ad(f[4], f[5]);
  m.rt = ml(c.rho0, ad(tf, f[0]));
  m.J = ml(c.af_l, sb(f[1], f[2]));
  m.et = ml(c.af_l2, fm(f[0], c.m_two, tf));
  m.zt = ml(c.ag, ad(tg, f[3]));
  m.psi = ml(c.ag_l, sb(f[4], f[5]));
  m.epst = ml(c.ag_l2, fm(f[3], c.m_two, tg));
  // Thermodynamics, eq. (gaz-parfait): p = p0 (rho/rho0)^gamma exp(gamma (s - s0)/c_p), p = rho r T.
  m.rho = ad(c.rho0, m.rt);
  m.inv_rho = m_rcp(m.rho);
  m.u = ml(m.J, m.inv_rho);
  m.ds = ml(fm(m.rt, sb(X{}, s0), m.zt), m.inv_rho);  // zeta - rho s0 = zeta_t - rho_t s0
  m.lnr = m_log1p(ml(m.rt, c.inv_af));
  m.pt = ml(c.p0, m_expm1(ml(c.gamma, fm(m.ds, c.inv_cp, m.lnr))));
  m.T = ml(ml(ad(c.p0, m.pt), m.inv_rho), c.inv_r);
}

// Steps (iv)-(vii) for one node (pair): equilibria, relaxation, entropy source; returns the shifted
// post-collision populations fs = M^{-1} m* - w.
template <typename X>
__device__ __forceinline__ void node_collide(const Node<X>& m, X ul, X ur, X Tl, X Tr, X s_e, X s_psi, X s_eps,
                                             X q_src, X s0, const Consts<X>& c, X fs[6]) {
  // (iv) equilibria: e_eq (eq. energie-equilibre), psi_eq = zeta u (eq. psi-equilibre), and the
  // polytropic form of eq. (eq-energie-entropie-d1q3q3), all as deviations from the rest state.
  const X s = ad(s0, m.ds);
  const X zeta = ml(m.rho, s);
  const X e_eq_t = fm(m.rt, c.m_two_lam2, ml(c.three, fm(m.J, m.u, m.pt)));
  const X psi_eq = ml(zeta, m.u);
  const X eps_eq_t = fm(c.e_r, m.ds, fm(e_eq_t, s, ml(ml(c.two_lam2, m.rho), fm(c.cp_log, m.lnr, m.ds))));
  // (v) relaxation, eq. (relaxation-d1q3q3).
  const X es = fm(s_e, sb(e_eq_t, m.et), m.et);
  const X psis = fm(s_psi, sb(psi_eq, m.psi), m.psi);
  const X epss = fm(s_eps, sb(eps_eq_t, m.epst), m.epst);
  // (vii) entropy production of eq. (NS-rho-J-zeta) with centred differences, added to zeta.
  X zs = m.zt;
  if (c.source_on) {
    const X du = sb(ur, ul), dT = sb(Tr, Tl);
    const X inv_T = m_rcp(m.T);
    const X A = fm(ml(c.cp_over_Pr, ml(dT, dT)), inv_T, ml(du, du));
    zs = fm(ml(ml(q_src, m.rho), inv_T), A, m.zt);
  }
  // (vi) f_d* = M^{-1} m*, block by block: x0 = (r - q)/3, x+- = (2r + q)/6 +- j/2.
  {
    const X r = ml(m.rt, c.inv_af), j = ml(m.J, c.inv_af_l), q = ml(es, c.inv_af_l2);
    const X h = ml(fm(r, c.two, q), c.sixth);
    fs[0] = ml(sb(r, q), c.third);
    fs[1] = fm(j, c.half, h);
    fs[2] = fm(j, c.m_half, h);
  }
  {
    const X r = ml(zs, c.inv_ag), j = ml(psis, c.inv_ag_l), q = ml(epss, c.inv_ag_l2);
    const X h = ml(fm(r, c.two, q), c.sixth);
    fs[3] = ml(sb(r, q), c.third);
    fs[4] = fm(j, c.half, h);
    fs[5] = fm(j, c.m_half, h);
  }
}

// The same node update in dimensionless moments, used by the step kernels. With D = diag(rho0,
// rho0 lambda, rho0 c_p, rho0 lambda^2, rho0 c_p lambda, rho0 c_p lambda^2), the scaled moments
// D^{-1} m of the shifted populations are integer combinations of them:
//   r = f0 + f+ + f- = (rho - rho0)/rho0,  j = f+ - f- = J/(rho0 lambda),
//   e = f+ + f- - 2 f0 = (e - e_r)/(rho0 lambda^2),  and z, psi, eps likewise from g with rho0 c_p.
// With u' = u/lambda, sigma = (s - s0)/c_p, s' = s/c_p and theta = c_p T / lambda^2, the equation of
// state, the equilibria, the relaxation and the source of section 8 become
//   u' = j/(1 + r), sigma = (z - r s0/c_p)/(1 + r), E = expm1(gamma (log1p(r) + sigma)),
//   theta = kp gamma/(gamma - 1) (1 + E)/(1 + r), kp = p0/(rho0 lambda^2),
//   e_eq = 3 (j u' + kp E) - 2 r,  psi_eq = (1 + r) s' u',
//   eps_eq = 2 (1 + r)(sigma + (1 - 1/gamma) log1p(r)) + e_eq s' + (3 kp - 2) sigma,
//   dz = (sigma_e/4) (1 + r)/theta [du'^2 + dtheta^2 / (Pr theta)]  (dt S / (rho0 c_p)),
// and M^{-1} loses its scale factors: f0 = (r - e)/3, f+- = (2 r + e)/6 +- j/2 (same for g).
template <typename X>
struct NodeS {
  X r, j, e, z, ps, ep;   // scaled moments
  X rho1, inv, u, sg, lnr, E, th;  // 1 + r, 1/(1 + r), u', sigma, log1p(r), expm1(x), theta
};

// log1p / expm1 by their series alone on paired lanes, clearing ok where a lane is outside the
// series range (the value is then to be recomputed by m_log1p / m_expm1).
__device__ __forceinline__ float2 log1p_series_checked(float2 x, bool& ok) {
  ok = ok && fabsf(x.x) <= 0.3f && fabsf(x.y) <= 0.3f;
  return atanh2_series(x);
}
__device__ __forceinline__ float2 expm1_series_checked(float2 x, bool& ok) {
  ok = ok && fabsf(x.x) <= 0.35f && fabsf(x.y) <= 0.35f;
  return expm1_series(x);
}

// CHECKED (paired lanes only): log1p and expm1 by their series without a branch; the return value is
// false when some lane left the series ranges, and the caller then runs the unchecked form, whose
// results agree on every lane inside the ranges. FULL: the caller guarantees the nonlinear equilibria
// with the entropy source (eq_mode 0, source_on), so those tests compile away.
// Numeric constants of the node update in the lane type X, as the compiler's literals (rounded as
// the host rounds the Consts fields).
template <typename X>
__device__ __forceinline__ X num(double v);
template <>
__device__ __forceinline__ double num<double>(double v) { return v; }
template <>
__device__ __forceinline__ float num<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ float2 num<float2>(double v) { return make_float2((float)v, (float)v); }

template <typename X, bool CHECKED = false, bool FULL = false>
__device__ __forceinline__ bool node_state_s(const X f[6], const Consts<X>& c, X m_s0h, NodeS<X>& m) {
  // (ii) moments, eq. (M-d1q3q3), scaled.
  const X tf = ad(f[1], f[2]), tg = ad(f[4], f[5]);
  m.r = ad(tf, f[0]);
  m.j = sb(f[1], f[2]);
  m.e = fm(f[0], num<X>(-2.0), tf);
  m.z = ad(tg, f[3]);
  m.ps = sb(f[4], f[5]);
  m.ep = fm(f[3], num<X>(-2.0), tg);
  // Equation of state, eq. (gaz-parfait).
  m.rho1 = ad(num<X>(1.0), m.r);
  if (!FULL && c.eq_mode == 1) {  // the linear equilibria need no equation of state (and there is no source)
    m.inv = m.u = m.sg = m.lnr = m.E = m.th = X{};
    return true;
  }
  m.inv = m_rcp(m.rho1);
  m.u = ml(m.j, m.inv);
  m.sg = ml(fm(m.r, m_s0h, m.z), m.inv);
  bool ok = true;
  if constexpr (CHECKED) {
    m.lnr = log1p_series_checked(m.r, ok);
    m.E = expm1_series_checked(ml(c.gamma, ad(m.lnr, m.sg)), ok);
  } else {
    m.lnr = m_log1p(m.r);
    m.E = m_expm1(ml(c.gamma, ad(m.lnr, m.sg)));
  }
  m.th = ml(fm(c.kth, m.E, c.kth), m.inv);
  return ok;
}

// The entropy source z + dt S in scaled moments, dt S = q_src (1 + r)/theta [du'^2 + dtheta^2 / (Pr theta)]
// with the centred differences du' = u'_{j+1} - u'_{j-1}, dtheta likewise, is written out in the node
// update below for the FP32 and FP64 lanes; the double-float lanes (lbm_df.cuh) give their own
// source_update, found where the node update is instantiated.
template <typename X>
constexpr bool kSourceOverloaded = false;

template <typename X, bool FULL = false>
__device__ __forceinline__ void node_collide_s(const NodeS<X>& m, X ul, X ur, X thl, X thr, X s_e, X s_psi,
                                               X s_eps, X q_src, X s0h, const Consts<X>& c, X fs[6],
                                               X lin_e0 = X{}, X lin_p0 = X{}, X lin_q0 = X{}) {
  // (iv) equilibria (eqs. energie-equilibre, psi-equilibre, eq-energie-entropie-d1q3q3), or the
  // linear ones of eq. (equilibres-NS-linearise).
  X e_eq, ps_eq, ep_eq;
  if (!FULL && c.eq_mode == 1) {
    e_eq = fm(c.leZ, m.z, fm(c.leJ, m.j, fm(c.leR, m.r, lin_e0)));
    ps_eq = fm(c.lpZ, m.z, fm(c.lpJ, m.j, fm(c.lpR, m.r, lin_p0)));
    ep_eq = fm(c.lqZ, m.z, fm(c.lqJ, m.j, fm(c.lqR, m.r, lin_q0)));
  } else {
    const X sp = ad(s0h, m.sg);
    e_eq = fm(m.r, num<X>(-2.0), ml(num<X>(3.0), fm(m.j, m.u, ml(c.kp, m.E))));
    ps_eq = ml(ml(m.rho1, sp), m.u);
    ep_eq = fm(c.e_rs, m.sg, fm(e_eq, sp, ml(ad(m.rho1, m.rho1), fm(c.one_m_ig, m.lnr, m.sg))));
  }
  // (v) relaxation (eq. relaxation-d1q3q3).
  const X es = fm(s_e, sb(e_eq, m.e), m.e);
  const X pss = fm(s_psi, sb(ps_eq, m.ps), m.ps);
  const X eps = fm(s_eps, sb(ep_eq, m.ep), m.ep);
  // (vii) entropy production (eq. NS-rho-J-zeta), centred differences.
  X zs = m.z;
  if (FULL || c.source_on) {
    if constexpr (kSourceOverloaded<X>) {
      zs = source_update(m.z, m.rho1, m.th, ul, ur, thl, thr, q_src, c.inv_Pr);
    } else {
      const X du = sb(ur, ul), dth = sb(thr, thl);
      const X ith = m_rcp(m.th);
      const X A = fm(ml(dth, dth), ml(ith, c.inv_Pr), ml(du, du));
      zs = fm(ml(ml(q_src, m.rho1), ith), A, m.z);
    }
  }
  // (vi) back to populations.
  {
    const X h = ml(fm(m.r, num<X>(2.0), es), num<X>(1.0 / 6.0));
    fs[0] = ml(sb(m.r, es), num<X>(1.0 / 3.0));
    fs[1] = fm(m.j, num<X>(0.5), h);
    fs[2] = fm(m.j, num<X>(-0.5), h);
  }
  {
    const X h = ml(fm(zs, num<X>(2.0), eps), num<X>(1.0 / 6.0));
    fs[3] = ml(sb(zs, eps), num<X>(1.0 / 3.0));
    fs[4] = fm(pss, num<X>(0.5), h);
    fs[5] = fm(pss, num<X>(-0.5), h);
  }
}

// The constants in the scalar type R and, for FP32, also broadcast to paired lanes.
template <typename R>
struct ConstSet {
  Consts<R> s;
  Consts<float2> p;
  template <typename X>
  const Consts<X>& get() const;
};
template <>
template <>
inline const Consts<double>& ConstSet<double>::get<double>() const { return s; }
template <>
template <>
inline const Consts<float>& ConstSet<float>::get<float>() const { return s; }
template <>
template <>
inline const Consts<float2>& ConstSet<float>::get<float2>() const { return p; }

// Nodes a tile of NT threads x V nodes spans: NT V, less the ghost nodes that the warps of an FP32 tile
// of four nodes per thread share (kGhost per warp edge, see tile_body_packed). A tile stores
// tile_span - 4K of them (the halo of K steps is 2K nodes per side).
constexpr int kGhost = 4;
__host__ __device__ constexpr long long tile_span(int NT, int V, bool f32) {
  return (long long)NT * V - ((f32 && V == 4) ? 2LL * kGhost * (NT / 32 - 1) : 0LL);
}

// Host-side launchers (lbm_step.cu). A tile has NT threads of V nodes; K steps per launch.
// Only the first ntiles tiles are processed (the autotuner times partial launches).
template <typename R>
cudaError_t launch_step_tiles(const R* in, R* out, long long plane, const LatDev* lat, const int* tile_lat, int B,
                              long long ntiles, int K, int NT, int V, const ConstSet<R>& c, cudaStream_t st,
                              long long grid_cap);
// tile_lat[t] = lattice of tile t for a table of first tiles (lattice_of_tile, once per configuration).
cudaError_t launch_tile_map(const LatDev* lat, int B, long long ntiles, int* map, cudaStream_t st);
bool valid_tile_config(int K, int NT, int V, bool fp64);

// Work unit of the persistent launch: kUnitTiles consecutive tiles of one time block (at most 32).
#ifndef LBM_UNIT_TILES
#define LBM_UNIT_TILES 16
#endif
constexpr int kUnitTiles = LBM_UNIT_TILES;
static_assert(kUnitTiles >= 1 && kUnitTiles <= 32, "a work unit's tiles are checked by one warp");

// Control block of the persistent launch (device pointers).
struct PersistentCtl {
  unsigned long long* counter;  // next work unit
  int* done;                    // per work unit: number of finished time blocks
  int* status;                  // 0, or 1 once a bounded wait has expired
  long long spin_limit;         // polls (about 100 ns apart) before a wait gives up
  long long withhold;           // test hook: work unit whose first block is never published (-1: none)
};
template <typename R>
cudaError_t launch_persistent(R* buf0, R* buf1, long long plane, const LatDev* lat, const int* tile_lat, int B,
                              long long ntiles, int K, int NT, int V, long long nblocks, const PersistentCtl& ctl,
                              const ConstSet<R>& c, cudaStream_t st);

// Adjoint (lbm_adjoint.cu): K <= kAdjointMaxK reverse steps per launch from the forward state at the
// start of the block, tiles of kAdjointThreads nodes storing kAdjointThreads - 2(4K - 2) of them.
constexpr int kAdjointThreads = 256;
constexpr int kAdjointMaxK = 8;
inline int adjoint_tile_out(int K) { return kAdjointThreads - 2 * (4 * K - 2); }
template <typename R>
cudaError_t launch_adjoint_block(const R* f0, const R* a_next, R* a_out, long long plane, const LatDev* lat, int B,
                                 long long ntiles, int K, const ConstSet<R>& c, double* grad_tile, cudaStream_t st);
cudaError_t launch_reduce_rate_grads(const double* grad_tile, const LatDev* lat, int B, long long ntiles, double* out,
                                     bool accumulate, cudaStream_t st);
template <typename R>
cudaError_t launch_adjoint_init(const R* f0, const R* a0, long long plane, const LatDev* lat, int B,
                                const Consts<double>& c, double* drho, double* du, cudaStream_t st);
template <typename R>
cudaError_t launch_to_f64(const R* in, double* out, long long n, cudaStream_t st);
template <typename R>
cudaError_t launch_misfit_seed(const R* fT, const double* target, const double* rho_b, long long plane, double rho0,
                               R* aT, double* part, double* loss, cudaStream_t st);

// Device memory through the allocator installed with lbm_set_allocator (cudaMalloc/cudaFree if none),
// and the host/device test of the per-node array arguments (lbm_api.cu).
void* device_alloc(size_t bytes, cudaStream_t st);
void device_free(void* p);
bool is_device_pointer(const void* p);

}  // namespace lbm
