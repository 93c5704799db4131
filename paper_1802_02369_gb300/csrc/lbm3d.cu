// Three-dimensional coupled D3Q19-D3Q7 scheme for (rho, J, zeta) (declarations and the readings in
// include/lbm.h): one fused collide-stream kernel per time step. Each CTA owns a column of 32 x TY
// nodes and marches it along z through ZC planes.
//
// Variables. Populations are dimensionless (units of rho0) and stored shifted by those of the rest
// state (rho0, u = 0, s0); their moments, taken with the integer patterns of the moment rows, are the
// deviations of the moments scaled by rho0 lambda^k (and c_p for the entropy rows):
//   r = rho/rho0 - 1, j = J/(rho0 lambda), z = zeta/(rho0 c_p) - s0/c_p, and so on.
// With P = p/(rho0 lambda^2), P0 its rest value, sigma = (s - s0)/c_p, lr = log(1 + r),
// dP = P0 expm1(gamma (lr + sigma)), u = j/(1 + r) (in units of lambda) and the diagonal deviations
// a_k = dP + j_k u_k of Pi, the equilibrium deviations are
//   e = 19 tr - 30 r (tr = a_x + a_y + a_z), pxx = 3 a_x - tr, pww = a_y - a_z, pxy = j_x u_y, ...,
//   q = -(2/3) j, m = 0, eps = 12 r - 16 tr + 21 (2 P0 tr + A2 - 3 P0^2 r)/(1 + r)
//   (A2 = a_x a_y + a_y a_z + a_x a_z), pixx = 2 (tr - 3 a_x) + (3 P0 (2 a_x - a_y - a_z)
//   + 3 a_x (a_y + a_z) - 6 a_y a_z)/(1 + r), piww = -2 (a_y - a_z) + 3 (P0 + a_x)(a_y - a_z)/(1 + r),
//   psi = (s0/c_p + z) u, eps7 = 3 (A_x + A_y + A_z) - 6 z, xixx = 3 A_x - (A_x + A_y + A_z),
//   xiww = A_y - A_z, with A_k = (s0/c_p) a_k + sigma (P0 + a_k) + L and
//   L = (1 + r)((gamma - 1) lr + gamma sigma)/(gamma beta),
// the deviations from the rest values of the equilibria in include/lbm.h. The production, in the
// same units, is q_vis (1 + r)^2 / P (2 D:D + (div u)^2) + q_th (1 + r) |grad T'|^2 / (1 + T')^2 with
// T' = T/T0 - 1 = (dP/P0 - r)/(1 + r), the derivatives as centred differences without the 1/2,
// q_vis = sigma_e (1 - 1/gamma) / 12, q_th = sigma_e / (4 Pr).
// The D3Q19 patterns are mutually orthogonal (norms 19, 10 x3, 2394, 36, 12, 4 x3, 40 x3, 8 x3, 252,
// 72, 24), so the inverse is the transpose divided by the norms; the D3Q7 inverse is written out.
//
// The step kernel. Thread (tx, ty) of a CTA owns the nodes (x0 + tx, y0 + ty, z) of its column. For
// each plane z it loads the populations of plane z + 1 and reduces them to the velocity and temperature
// deviation, which go to a ring of four shared slots with a one-node ring around the tile (loaded and
// reduced by the first threads: the production needs the neighbours' u and T'). One barrier a plane:
// the ring has four slots, so a warp that runs ahead writes the slot of z + 2 while the others still
// read z - 1, z and z + 1. Then the node of plane z, whose populations waited across the barrier (in
// a shared buffer of the thread's own, in registers, or re-read: MODE below), collides and pushes its
// populations to the neighbours, f_i(x + c_i) = f_i*(x): each population is read once from DRAM and
// written once per step.
#include <cmath>
#include <string>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lbm_dfn.cuh"
#include "lbm_internal.cuh"

namespace {

constexpr int kQ = 26;
// Velocity components of population i (folded to constants in the unrolled loops).
__host__ __device__ constexpr int cx3(int i) {
  constexpr int v[kQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0};
  return v[i];
}
__host__ __device__ constexpr int cy3(int i) {
  constexpr int v[kQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 1, -1, 0, 0};
  return v[i];
}
__host__ __device__ constexpr int cz3(int i) {
  constexpr int v[kQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 0, 0, 0, 0, 0, 1, -1};
  return v[i];
}

struct P3 {
  double rho0, lam, cp, s0, gamma, beta, Pr;
  double P0, s0c, inv_gb, gm1, q_vis, q_th;
  double se, sq, sh, spsi, seps;
  double w[kQ];  // rest populations
  int source_on;
};

template <typename R>
struct P3T {
  R P0, s0c, inv_gb, gm1, gamma, q_vis, q_th, se, sq, sh, spsi, seps;
  int source_on;
};

template <typename R>
__host__ __device__ P3T<R> lanes3(const P3& p) {
  P3T<R> t;
  t.P0 = R(p.P0); t.s0c = R(p.s0c); t.inv_gb = R(p.inv_gb); t.gm1 = R(p.gm1); t.gamma = R(p.gamma);
  t.q_vis = R(p.q_vis); t.q_th = R(p.q_th);
  t.se = R(p.se); t.sq = R(p.sq); t.sh = R(p.sh); t.spsi = R(p.spsi); t.seps = R(p.seps);
  t.source_on = p.source_on;
  return t;
}

// The logarithm and exponential of the one-dimensional kernels (lbm_internal.cuh): FP32 CUDA's
// log1pf / expm1f, FP64 the double-float series on the FP32 pipes. Reciprocals: FP32 a division,
// FP64 an FP32 estimate refined by two FP64 Newton steps. A host build (the node update emulated on the
// CPU by the tests) takes the C library's log1p, expm1 and a division instead.
__host__ __device__ __forceinline__ float rcp3(float x) { return 1.0f / x; }
__host__ __device__ __forceinline__ double rcp3(double x) {
#ifdef __CUDA_ARCH__
  return lbm::m_rcp(x);
#else
  return 1.0 / x;
#endif
}
__host__ __device__ __forceinline__ float lg3(float x) {
#ifdef __CUDA_ARCH__
  return lbm::m_log1p(x);
#else
  return std::log1p(x);
#endif
}
__host__ __device__ __forceinline__ double lg3(double x) {
#ifdef __CUDA_ARCH__
  return lbm::m_log1p(x);
#else
  return std::log1p(x);
#endif
}
__host__ __device__ __forceinline__ float ex3(float x) {
#ifdef __CUDA_ARCH__
  return lbm::m_expm1(x);
#else
  return std::expm1(x);
#endif
}
__host__ __device__ __forceinline__ double ex3(double x) {
#ifdef __CUDA_ARCH__
  return lbm::m_expm1(x);
#else
  return std::expm1(x);
#endif
}
// LBM_F64_DF: FP64 planes, the node update in double-float (lbm_dfn.cuh).
using lbm::dfn;
__device__ __forceinline__ dfn rcp3(dfn x) { return lbm::dfn_rcp(x); }
__device__ __forceinline__ dfn lg3(dfn x) { return lbm::dfn_log1p(x); }
__device__ __forceinline__ dfn ex3(dfn x) { return lbm::dfn_expm1(x); }
// Storage. FP32 and FP64 planes hold floats and doubles; the double-float planes hold each population
// as its (hi, lo) FP32 pair (8 bytes, as a double), so that the step loads and stores them with no
// conversion on the FP64 pipe (measured: with FP64 planes the conversions at the 26 loads, the
// re-read and the ring, and the 26 stores kept that pipe 63 % busy and bounded the kernel).
__device__ __forceinline__ float st3(float x) { return x; }
__device__ __forceinline__ double st3(double x) { return x; }
__device__ __forceinline__ float2 st3(dfn x) { return make_float2(x.v.hi, x.v.lo); }
template <typename R>
__device__ __forceinline__ R ld3(float x) { return R(x); }
template <typename R>
__device__ __forceinline__ R ld3(double x) { return R(x); }
template <typename R>
__device__ __forceinline__ R ld3(float2 x) { return R(lbm::df{x.x, x.y}); }
// FP64 values of stored populations and the stored form of FP64 values (initialisation, read-out).
__host__ __device__ __forceinline__ double from_store(float x) { return (double)x; }
__host__ __device__ __forceinline__ double from_store(double x) { return x; }
__host__ __device__ __forceinline__ double from_store(float2 x) { return (double)x.x + (double)x.y; }
template <typename S>
__host__ __device__ __forceinline__ S to_store(double x) { return S(x); }
template <>
__host__ __device__ __forceinline__ float2 to_store<float2>(double x) {
  const lbm::df d = lbm::df_from_double_host(x);
  return make_float2(d.hi, d.lo);
}

// Conserved deviations of shifted populations.
template <typename R>
struct Cons3 {
  R r, jx, jy, jz, z;
};

template <typename R>
__host__ __device__ __forceinline__ Cons3<R> conserved3(const R (&f)[kQ]) {
  Cons3<R> c;
  const R ax = f[1] + f[2], ay = f[3] + f[4], az = f[5] + f[6];
  const R exy = (f[7] + f[8]) + (f[9] + f[10]), exz = (f[11] + f[12]) + (f[13] + f[14]);
  const R eyz = (f[15] + f[16]) + (f[17] + f[18]);
  c.r = (f[0] + (ax + ay + az)) + (exy + exz + eyz);
  const R d1 = f[7] - f[8], d2 = f[9] - f[10], e1 = f[11] - f[12], e2 = f[13] - f[14];
  const R g1 = f[15] - f[16], g2 = f[17] - f[18];
  c.jx = (f[1] - f[2]) + (d1 + d2) + (e1 + e2);
  c.jy = (f[3] - f[4]) + (d1 - d2) + (g1 + g2);
  c.jz = (f[5] - f[6]) + (e1 - e2) + (g1 - g2);
  c.z = (f[19] + (f[20] + f[21])) + ((f[22] + f[23]) + (f[24] + f[25]));
  return c;
}

// The thermodynamic state of a node: reciprocal density, velocity, entropy deviation, log density,
// pressure deviation.
template <typename R>
struct Thermo3 {
  R inv, ux, uy, uz, sig, lr, dP;
};

template <typename R>
__host__ __device__ __forceinline__ Thermo3<R> thermo3(const Cons3<R>& c, const P3T<R>& p) {
  Thermo3<R> t;
  t.inv = rcp3(R(1) + c.r);
  t.ux = c.jx * t.inv;
  t.uy = c.jy * t.inv;
  t.uz = c.jz * t.inv;
  t.sig = (c.z - p.s0c * c.r) * t.inv;
  t.lr = lg3(c.r);
  t.dP = p.P0 * ex3(p.gamma * (t.lr + t.sig));
  return t;
}

template <typename R>
__host__ __device__ __forceinline__ R temp_dev3(const Cons3<R>& c, const Thermo3<R>& t, const P3T<R>& p) {
  return (t.dP / p.P0 - c.r) * t.inv;
}

// Equilibrium deviations of the 21 non-conserved moments, in the order (e, pxx, pww, pxy, pyz, pxz,
// qx, qy, qz, mx, my, mz, eps, pixx, piww, psi_x, psi_y, psi_z, eps7, xixx, xiww); m = 0 is left out
// of the arithmetic by the caller (eq[9..11] are set to 0 here).
template <typename R>
__host__ __device__ __forceinline__ void equilibria3(const Cons3<R>& c, const Thermo3<R>& t, const P3T<R>& p,
                                                     R (&eq)[21]) {
  const R ax = t.dP + c.jx * t.ux, ay = t.dP + c.jy * t.uy, az = t.dP + c.jz * t.uz;
  const R tr = (ax + ay) + az;
  eq[0] = R(19) * tr - R(30) * c.r;
  eq[1] = R(3) * ax - tr;
  eq[2] = ay - az;
  eq[3] = c.jx * t.uy;
  eq[4] = c.jy * t.uz;
  eq[5] = c.jx * t.uz;
  eq[6] = R(-2.0 / 3.0) * c.jx;
  eq[7] = R(-2.0 / 3.0) * c.jy;
  eq[8] = R(-2.0 / 3.0) * c.jz;
  eq[9] = eq[10] = eq[11] = R(0);
  const R ayz = ay + az, dyz = ay - az;
  const R A2 = ax * ayz + ay * az;
  eq[12] = R(12) * c.r - R(16) * tr + R(21) * ((R(2) * p.P0 * tr + A2) - R(3) * p.P0 * p.P0 * c.r) * t.inv;
  eq[13] = R(2) * (tr - R(3) * ax) +
           (R(3) * p.P0 * (R(2) * ax - ayz) + R(3) * ax * ayz - R(6) * ay * az) * t.inv;
  eq[14] = R(-2) * dyz + R(3) * (p.P0 + ax) * dyz * t.inv;
  const R zeta = p.s0c + c.z;
  eq[15] = zeta * t.ux;
  eq[16] = zeta * t.uy;
  eq[17] = zeta * t.uz;
  const R L = (R(1) + c.r) * (p.gm1 * t.lr + p.gamma * t.sig) * p.inv_gb;
  const R base = t.sig * p.P0 + L;
  const R Ax = p.s0c * ax + t.sig * ax + base, Ay = p.s0c * ay + t.sig * ay + base;
  const R Az = p.s0c * az + t.sig * az + base;
  const R trA = (Ax + Ay) + Az;
  eq[18] = R(3) * trA - R(6) * c.z;
  eq[19] = R(3) * Ax - trA;
  eq[20] = Ay - Az;
}

// Non-conserved moment deviations of shifted populations (same order as the equilibria).
template <typename R>
__host__ __device__ __forceinline__ void nonconserved3(const R (&f)[kQ], R (&m)[21]) {
  const R Ax = f[1] + f[2], Ay = f[3] + f[4], Az = f[5] + f[6];
  const R Dx = f[1] - f[2], Dy = f[3] - f[4], Dz = f[5] - f[6];
  const R s1 = f[7] + f[8], s2 = f[9] + f[10], t1 = f[11] + f[12], t2 = f[13] + f[14];
  const R u1 = f[15] + f[16], u2 = f[17] + f[18];
  const R d1 = f[7] - f[8], d2 = f[9] - f[10], e1 = f[11] - f[12], e2 = f[13] - f[14];
  const R g1 = f[15] - f[16], g2 = f[17] - f[18];
  const R Exy = s1 + s2, Exz = t1 + t2, Eyz = u1 + u2;
  const R Aall = (Ax + Ay) + Az, Eall = (Exy + Exz) + Eyz;
  const R pxy_x = d1 + d2, pxz_x = e1 + e2;  // sum cx over the xy and xz edges
  const R pxy_y = d1 - d2, pyz_y = g1 + g2;  // sum cy over the xy and yz edges
  const R pxz_z = e1 - e2, pyz_z = g1 - g2;  // sum cz over the xz and yz edges
  const R xxe = (Exy + Exz) - R(2) * Eyz, wwe = Exy - Exz;
  m[0] = R(-30) * f[0] - R(11) * Aall + R(8) * Eall;
  m[1] = (R(2) * Ax - (Ay + Az)) + xxe;
  m[2] = (Ay - Az) + wwe;
  m[3] = s1 - s2;
  m[4] = u1 - u2;
  m[5] = t1 - t2;
  m[6] = R(-4) * Dx + (pxy_x + pxz_x);
  m[7] = R(-4) * Dy + (pxy_y + pyz_y);
  m[8] = R(-4) * Dz + (pxz_z + pyz_z);
  m[9] = pxy_x - pxz_x;
  m[10] = pyz_y - pxy_y;
  m[11] = pxz_z - pyz_z;
  m[12] = R(12) * f[0] - R(4) * Aall + Eall;
  m[13] = (R(-4) * Ax + R(2) * (Ay + Az)) + xxe;
  m[14] = R(-2) * (Ay - Az) + wwe;
  m[15] = f[20] - f[21];
  m[16] = f[22] - f[23];
  m[17] = f[24] - f[25];
  m[18] = R(-6) * f[19] - R(3) * ((f[20] + f[21]) + (f[22] + f[23]) + (f[24] + f[25]));
  const R Sx = f[20] + f[21], Sy = f[22] + f[23], Sz = f[24] + f[25];
  m[19] = R(2) * Sx - (Sy + Sz);
  m[20] = Sy - Sz;
}

// Populations from the conserved deviations and the 21 non-conserved moments: the D3Q19 inverse is
// the transpose of the patterns divided by their norms; the D3Q7 one solves zeta = g0 + S,
// eps7 = -6 g0 - 3 S (S the sum over the moving velocities), xixx = 2 S_x - S_y - S_z,
// xiww = S_y - S_z, psi_k = g_+k - g_-k.
template <typename R>
__host__ __device__ __forceinline__ void populations3(const Cons3<R>& c, const R (&m)[21], R (&f)[kQ]) {
  const R RR = c.r * R(1.0 / 19.0);
  const R JX = c.jx * R(0.1), JY = c.jy * R(0.1), JZ = c.jz * R(0.1);
  const R E = m[0] * R(1.0 / 2394.0), XX = m[1] * R(1.0 / 36.0), WW = m[2] * R(1.0 / 12.0);
  const R XY = m[3] * R(0.25), YZ = m[4] * R(0.25), XZ = m[5] * R(0.25);
  const R QX = m[6] * R(0.025), QY = m[7] * R(0.025), QZ = m[8] * R(0.025);
  const R MX = m[9] * R(0.125), MY = m[10] * R(0.125), MZ = m[11] * R(0.125);
  const R H = m[12] * R(1.0 / 252.0), PX = m[13] * R(1.0 / 72.0), PW = m[14] * R(1.0 / 24.0);
  f[0] = RR - R(30) * E + R(12) * H;
  const R axis = RR - R(11) * E - R(4) * H;
  const R ax_x = axis + R(2) * XX - R(4) * PX;
  const R ax_yz = axis - XX + R(2) * PX;
  const R ww = WW - R(2) * PW;
  const R vx = JX - R(4) * QX, vy = JY - R(4) * QY, vz = JZ - R(4) * QZ;
  f[1] = ax_x + vx;
  f[2] = ax_x - vx;
  f[3] = (ax_yz + ww) + vy;
  f[4] = (ax_yz + ww) - vy;
  f[5] = (ax_yz - ww) + vz;
  f[6] = (ax_yz - ww) - vz;
  const R edge = RR + R(8) * E + H;
  const R bxy = edge + (XX + PX) + (WW + PW), bxz = edge + (XX + PX) - (WW + PW);
  const R byz = edge - R(2) * (XX + PX);
  const R jq_x = JX + QX, jq_y = JY + QY, jq_z = JZ + QZ;
  // xy edges (cx, cy): bxy + cx cy XY + cx (jq_x + MX) + cy (jq_y - MY).
  const R pa = jq_x + MX, pb = jq_y - MY;
  f[7] = (bxy + XY) + (pa + pb);
  f[8] = (bxy + XY) - (pa + pb);
  f[9] = (bxy - XY) + (pa - pb);
  f[10] = (bxy - XY) - (pa - pb);
  // xz edges (cx, cz): bxz + cx cz XZ + cx (jq_x - MX) + cz (jq_z + MZ).
  const R qa = jq_x - MX, qb = jq_z + MZ;
  f[11] = (bxz + XZ) + (qa + qb);
  f[12] = (bxz + XZ) - (qa + qb);
  f[13] = (bxz - XZ) + (qa - qb);
  f[14] = (bxz - XZ) - (qa - qb);
  // yz edges (cy, cz): byz + cy cz YZ + cy (jq_y + MY) + cz (jq_z - MZ).
  const R ra = jq_y + MY, rb = jq_z - MZ;
  f[15] = (byz + YZ) + (ra + rb);
  f[16] = (byz + YZ) - (ra + rb);
  f[17] = (byz - YZ) + (ra - rb);
  f[18] = (byz - YZ) - (ra - rb);
  // D3Q7.
  const R g0 = -c.z - m[18] * R(1.0 / 3.0);
  const R S = c.z - g0;
  const R Sx = (S + m[19]) * R(1.0 / 3.0);
  const R Syz = S - Sx;
  const R Sy = (Syz + m[20]) * R(0.5), Sz = (Syz - m[20]) * R(0.5);
  f[19] = g0;
  f[20] = (Sx + m[15]) * R(0.5);
  f[21] = (Sx - m[15]) * R(0.5);
  f[22] = (Sy + m[16]) * R(0.5);
  f[23] = (Sy - m[16]) * R(0.5);
  f[24] = (Sz + m[17]) * R(0.5);
  f[25] = (Sz - m[17]) * R(0.5);
}

__host__ __device__ __forceinline__ long long wrap3(long long v, long long n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// One node's collision: relaxation of the 21 non-conserved moments and the production added to
// zeta; du[a][b] and dT[a] are the centred differences (without the 1/2) along axis a of u_b and T'.
template <typename R>
__host__ __device__ __forceinline__ void collide3(R (&f)[kQ], const P3T<R>& p, const R (&du)[3][3], const R (&dT)[3],
                                                     R Tn) {
  Cons3<R> c = conserved3(f);
  const Thermo3<R> t = thermo3(c, p);
  R m[21], eq[21];
  nonconserved3(f, m);
  equilibria3(c, t, p, eq);
#pragma unroll
  for (int k = 0; k < 21; ++k) {
    const R s = k < 6 ? p.se : k < 12 ? p.sq : k < 15 ? p.sh : k < 18 ? p.spsi : p.seps;
    m[k] = m[k] + s * (eq[k] - m[k]);
  }
  if (p.source_on) {
    const R sxy = du[0][1] + du[1][0], syz = du[1][2] + du[2][1], sxz = du[0][2] + du[2][0];
    const R div = (du[0][0] + du[1][1]) + du[2][2];
    // 2 D:D + (div u)^2 with D the symmetric part of the (undivided) gradient.
    const R G = R(2) * ((du[0][0] * du[0][0] + du[1][1] * du[1][1]) + du[2][2] * du[2][2]) +
                ((sxy * sxy + syz * syz) + sxz * sxz) + div * div;
    const R gT = (dT[0] * dT[0] + dT[1] * dT[1]) + dT[2] * dT[2];
    const R rho = R(1) + c.r, P = p.P0 + t.dP;
    if constexpr (sizeof(R) == 4)
      c.z = c.z + p.q_vis * rho * rho / P * G + p.q_th * rho * gT / (Tn * Tn);
    else
      c.z = c.z + p.q_vis * rho * rho * rcp3(P) * G + p.q_th * rho * gT * rcp3(Tn * Tn);
  }
  populations3(c, m, f);
}

// One time step of the columns of a 32 x TY tile over the planes [z_b, z_b + zc). su[slot][field][n]
// holds ux, uy, uz, T' of a plane for the tile and a one-node ring around it (n = (ty + 1)(TX + 2)
// + tx + 1 for thread (tx, ty)); plane z_b - 1 + k goes to slot k mod 4.
// MODE says where the owner keeps the populations of plane z across the barrier: 1 in registers;
// 2 in a shared buffer of its own (two planes, by parity: each thread reads back only what it wrote,
// so no barrier guards it); 0 nowhere: it reads them again from global memory after the barrier (the
// same thread loaded them one plane earlier; L2 serves most of them). Modes 0 and 2 halve the
// populations in registers, so that more CTAs share an SM.
template <typename S, typename R, int TY, int MODE>
__global__ void __launch_bounds__(32 * TY, MODE == 1 ? 1 : ((sizeof(R) == 4 ? 512 : 256) / (32 * TY) > 1 ? (sizeof(R) == 4 ? 512 : 256) / (32 * TY) : 1))
    step3d_kernel(const S* __restrict__ in, S* __restrict__ out, int nx, int ny, int nz, int zc, long long N,
                  P3T<R> p) {
  constexpr int TX = 32, RX = TX + 2, RY = TY + 2, NR = RX * RY, NT = TX * TY, NH = NR - NT;
  static_assert(NH <= NT, "the ring around the tile needs one thread per node");
  __shared__ R su[4][4][NR];
  constexpr int NO = MODE == 2 ? NT : 1;
  __shared__ R sown[MODE == 2 ? 2 : 1][kQ][NO];
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const long long x0 = (long long)blockIdx.x * TX, y0 = (long long)blockIdx.y * TY;
  const long long zb = (long long)blockIdx.z * zc;
  if (zb >= nz) return;
  const long long ze = zb + zc < nz ? zb + zc : nz;
  // The thread's own column (wrapped: the columns of a ragged tile past the lattice's edge are the
  // ring's neighbours on the other side) and the ring node it reduces, if any.
  const long long gx = wrap3(x0 + tx, nx), gy = wrap3(y0 + ty, ny);
  const bool owner = (x0 + tx < nx) && (y0 + ty < ny);
  const int n_own = (ty + 1) * RX + tx + 1;
  int n_h = -1;
  long long hxy = 0;
  if (threadIdx.x < NH) {
    int k = threadIdx.x, rx, ry;
    if (k < RX) {
      ry = 0;
      rx = k;
    } else if (k < 2 * RX) {
      ry = RY - 1;
      rx = k - RX;
    } else {
      k -= 2 * RX;
      ry = 1 + k / 2;
      rx = (k & 1) ? RX - 1 : 0;
    }
    n_h = ry * RX + rx;
    hxy = wrap3(y0 - 1 + ry, ny) * nx + wrap3(x0 - 1 + rx, nx);
  }
  const long long own_xy = gy * nx + gx;
  const long long plane = (long long)nx * ny;
  auto load = [&](long long g, R (&f)[kQ]) {
#pragma unroll
    for (int i = 0; i < kQ; ++i) f[i] = lbm::in_bounds(g + i * N, kQ * N) ? ld3<R>(in[g + i * N]) : R(0);
  };
  auto reduce = [&](const R (&f)[kQ], int slot, int n) {
    if (!lbm::in_bounds(n, NR)) return;
    const Cons3<R> c = conserved3(f);
    const Thermo3<R> t = thermo3(c, p);
    su[slot][0][n] = t.ux;
    su[slot][1][n] = t.uy;
    su[slot][2][n] = t.uz;
    su[slot][3][n] = temp_dev3(c, t, p);
  };
  R fc[kQ];
  {
    const long long zm = wrap3(zb - 1, nz);
    R f[kQ];
    load(zm * plane + own_xy, f);
    reduce(f, 0, n_own);
    if (n_h >= 0) {
      load(zm * plane + hxy, f);
      reduce(f, 0, n_h);
    }
    load(zb * plane + own_xy, fc);
    reduce(fc, 1, n_own);
    if constexpr (MODE == 2) {
#pragma unroll
      for (int i = 0; i < kQ; ++i) sown[1][i][threadIdx.x] = fc[i];
    }
    if (n_h >= 0) {
      load(zb * plane + hxy, f);
      reduce(f, 1, n_h);
    }
  }
  for (long long z = zb; z < ze; ++z) {
    const int k = (int)(z - zb) + 1;
    const long long zp = z + 1 < nz ? z + 1 : 0;
    R fn[kQ];
    load(zp * plane + own_xy, fn);
    reduce(fn, (k + 1) & 3, n_own);
    if constexpr (MODE == 2) {
#pragma unroll
      for (int i = 0; i < kQ; ++i) sown[(k + 1) & 1][i][threadIdx.x] = fn[i];
    }
    if (n_h >= 0) {
      R f[kQ];
      load(zp * plane + hxy, f);
      reduce(f, (k + 1) & 3, n_h);
    }
    __syncthreads();
    if constexpr (MODE == 0) {
      if (owner) load(z * plane + own_xy, fc);
    } else if constexpr (MODE == 2) {
#pragma unroll
      for (int i = 0; i < kQ; ++i) fc[i] = sown[k & 1][i][threadIdx.x];
    }
    // (n - RX and n + RX bound every shared index of the node: n +- 1 lie between them.)
    if (owner && lbm::in_bounds(n_own - RX, NR) && lbm::in_bounds(n_own + RX, NR)) {
      const int sm = (k - 1) & 3, s0 = k & 3, sp = (k + 1) & 3, n = n_own;
      R du[3][3], dT[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        du[0][b] = su[s0][b][n + 1] - su[s0][b][n - 1];
        du[1][b] = su[s0][b][n + RX] - su[s0][b][n - RX];
        du[2][b] = su[sp][b][n] - su[sm][b][n];
      }
      dT[0] = su[s0][3][n + 1] - su[s0][3][n - 1];
      dT[1] = su[s0][3][n + RX] - su[s0][3][n - RX];
      dT[2] = su[sp][3][n] - su[sm][3][n];
      const R Tn = R(1) + su[s0][3][n];
      collide3(fc, p, du, dT, Tn);
      // Push: population i goes to the node x + c_i of the next state.
      const long long xm = gx == 0 ? nx - 1 : gx - 1, xp = gx == nx - 1 ? 0 : gx + 1;
      const long long ym = gy == 0 ? ny - 1 : gy - 1, yp = gy == ny - 1 ? 0 : gy + 1;
      const long long zm = z == 0 ? nz - 1 : z - 1;
      const long long xs[3] = {xm, gx, xp}, ys[3] = {ym * nx, gy * nx, yp * nx};
      const long long zs[3] = {zm * plane, z * plane, zp * plane};
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const long long g = zs[cz3(i) + 1] + ys[cy3(i) + 1] + xs[cx3(i) + 1] + i * N;
        if (lbm::in_bounds(g, kQ * N)) out[g] = st3(fc[i]);
      }
    }
    if constexpr (MODE == 1) {
#pragma unroll
      for (int i = 0; i < kQ; ++i) fc[i] = fn[i];
    }
  }
}

// Equilibrium populations from the physical fields, in FP64, stored shifted in S.
template <typename S>
__global__ void init3d_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                              const double* __restrict__ uy, const double* __restrict__ uz,
                              const double* __restrict__ s, S* __restrict__ st, long long n, P3 p) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const P3T<double> q = lanes3<double>(p);
  Cons3<double> c;
  c.r = rho[i] / p.rho0 - 1.0;
  c.jx = rho[i] * ux[i] / (p.rho0 * p.lam);
  c.jy = rho[i] * uy[i] / (p.rho0 * p.lam);
  c.jz = rho[i] * uz[i] / (p.rho0 * p.lam);
  c.z = (rho[i] * s[i] - p.rho0 * p.s0) / (p.rho0 * p.cp);
  const Thermo3<double> t = thermo3(c, q);
  double eq[21], f[kQ];
  equilibria3(c, t, q, eq);
  populations3(c, eq, f);
#pragma unroll
  for (int k = 0; k < kQ; ++k) st[k * n + i] = to_store<S>(f[k]);
}

// Populations, node-major and unshifted, in FP64.
template <typename S>
__global__ void pops3d_kernel(const S* __restrict__ st, double* __restrict__ out, long long n, P3 p) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int k = 0; k < kQ; ++k) out[kQ * i + k] = from_store(st[k * n + i]) + p.w[k];
}

template <typename S>
__global__ void fields3d_kernel(const S* __restrict__ st, long long n, P3 p, double* rho, double* ux, double* uy,
                                double* uz, double* s) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[kQ];
#pragma unroll
  for (int k = 0; k < kQ; ++k) f[k] = from_store(st[k * n + i]);
  const Cons3<double> c = conserved3(f);
  const double r1 = 1.0 + c.r;
  if (rho) rho[i] = p.rho0 * r1;
  if (ux) ux[i] = p.lam * c.jx / r1;
  if (uy) uy[i] = p.lam * c.jy / r1;
  if (uz) uz[i] = p.lam * c.jz / r1;
  if (s) s[i] = p.cp * (p.s0c + c.z) / r1;
}

}  // namespace

struct lbm3d_ctx {
  long long nx = 0, ny = 0, nz = 0;
  int precision = LBM_F64;
  cudaStream_t stream = nullptr;
  P3 p{};
  void* state[2] = {nullptr, nullptr};
  int cur = 0;
  double* d_stage = nullptr;
  bool has_state = false;
  long long steps_done = 0;
  int ty = 0, zc = 0;  // 0: default
  int keep = -1;  // where plane z waits across the barrier (step3d_kernel's MODE); -1: the default
  std::string err;
  long long n() const { return nx * ny * nz; }
  size_t elem() const { return precision == LBM_F32_SHIFTED ? sizeof(float) : sizeof(double); }
  size_t state_bytes() const { return (size_t)kQ * n() * elem(); }
};

namespace {

struct NvtxRange3 {
  explicit NvtxRange3(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange3() { nvtxRangePop(); }
};

int fail3(lbm3d_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define L3_CK(ctx, call)                                                                                      \
  do {                                                                                                        \
    cudaError_t e_ = (call);                                                                                  \
    if (e_ != cudaSuccess) return fail3(ctx, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool rate_ok3(double s) { return s > 0.0 && s < 2.0 && std::isfinite(s); }

unsigned blocks3(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int derive3(const lbm3d_params* in, P3& p) {
  if (!in) return LBM_ERR_INVALID_ARG;
  p.gamma = in->gamma;
  p.Pr = in->Pr;
  p.cp = in->cp;
  p.rho0 = in->rho0;
  p.lam = in->lambda;
  p.s0 = in->s0;
  const double dx = in->dx;
  if (!(p.gamma > 1.0) || !(p.Pr > 0.0) || !(p.cp > 0.0) || !(p.rho0 > 0.0) || !(p.lam > 0.0) || !(dx > 0.0) ||
      !std::isfinite(p.s0) || !std::isfinite(p.gamma) || !std::isfinite(p.lam) || !std::isfinite(p.cp) ||
      !std::isfinite(p.rho0) || !std::isfinite(p.Pr))
    return LBM_ERR_INVALID_ARG;
  const double p0 = in->p0 > 0.0 ? in->p0 : p.rho0 * 0.25 * p.lam * p.lam / p.gamma;
  p.beta = in->beta > 0.0 ? in->beta : 9.0;
  p.se = in->s_e;
  if (!rate_ok3(p.se) || !std::isfinite(p0) || !std::isfinite(p.beta)) return LBM_ERR_INVALID_ARG;
  const double sigma_e = 1.0 / p.se - 0.5;
  p.spsi = in->s_psi > 0.0 ? in->s_psi : 1.0 / (p.beta * (p.gamma / p.Pr) * sigma_e + 0.5);
  p.seps = in->s_eps > 0.0 ? in->s_eps : 1.0;
  p.sq = in->s_q > 0.0 ? in->s_q : 1.5;
  p.sh = in->s_h > 0.0 ? in->s_h : 1.2;
  if (!rate_ok3(p.spsi) || !rate_ok3(p.seps) || !rate_ok3(p.sq) || !rate_ok3(p.sh)) return LBM_ERR_INVALID_ARG;
  p.P0 = p0 / (p.rho0 * p.lam * p.lam);
  p.s0c = p.s0 / p.cp;
  p.inv_gb = 1.0 / (p.gamma * p.beta);
  p.gm1 = p.gamma - 1.0;
  p.q_vis = sigma_e * (1.0 - 1.0 / p.gamma) / 12.0;
  p.q_th = sigma_e / (4.0 * p.Pr);
  p.source_on = in->source_on != 0;
  // Rest populations: the inverse applied to the rest moments (rho = rho0, zeta = rho0 s0, e and eps
  // of Pi = p0 I, eps7 of E = s0 p0 I; the others zero), in units of rho0 lambda^k (c_p).
  Cons3<double> c{1.0, 0.0, 0.0, 0.0, p.s0c};
  double m[21] = {0.0};
  m[0] = 57.0 * p.P0 - 30.0;
  m[12] = 12.0 - 48.0 * p.P0 + 63.0 * p.P0 * p.P0;
  m[18] = (9.0 * p.P0 - 6.0) * p.s0c;
  populations3(c, m, p.w);
  return LBM_OK;
}

int default_ty(const lbm3d_ctx*) { return 4; }
// The shared-buffer variant for FP32 on 4-row tiles (measured fastest there), else the re-read one.
int default_keep(const lbm3d_ctx* c) {
  return c->precision == LBM_F32_SHIFTED && (c->ty > 0 ? c->ty : default_ty(c)) == 4 ? 2 : 0;
}

template <typename S, typename R, int TY, int MODE>
cudaError_t launch3(lbm3d_ctx* c) {
  const unsigned gx = (unsigned)((c->nx + 31) / 32), gy = (unsigned)((c->ny + TY - 1) / TY);
  int zc = c->zc;
  if (zc <= 0) {
    // About eight CTAs per resident slot (measured at 256^3: 24 planes per CTA 18.3 GLUPS, 52 planes
    // 17.3): the planes per CTA follow from the lattice.
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step3d_kernel<S, R, TY, MODE>, 32 * TY, 0);
    const long long target = 8LL * (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    long long chunks = (target + (long long)gx * gy - 1) / ((long long)gx * gy);
    if (chunks < 1) chunks = 1;
    if (chunks > c->nz) chunks = c->nz;
    zc = (int)((c->nz + chunks - 1) / chunks);
  }
  if (zc > c->nz) zc = (int)c->nz;
  // At most 65535 CTAs along z: a taller lattice takes more planes per CTA than asked.
  const long long zc_min = (c->nz + 65534) / 65535;
  if (zc < zc_min) zc = (int)zc_min;
  const unsigned gz = (unsigned)((c->nz + zc - 1) / zc);
  step3d_kernel<S, R, TY, MODE><<<dim3(gx, gy, gz), 32 * TY, 0, c->stream>>>(
      (const S*)c->state[c->cur], (S*)c->state[1 - c->cur], (int)c->nx, (int)c->ny, (int)c->nz, zc, c->n(),
      lanes3<R>(c->p));
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_step3k(lbm3d_ctx* c) {
  const int ty = c->ty > 0 ? c->ty : default_ty(c);
  if constexpr (MODE == 2) {
    // FP32 4-row tiles only (the shared buffer of larger tiles passes the 48 KB of static shared
    // memory); lbm3d_set_config refuses the rest.
    if (c->precision != LBM_F32_SHIFTED || ty != 4) return cudaErrorInvalidConfiguration;
    return launch3<float, float, 4, 2>(c);
  } else {
    if (c->precision == LBM_F32_SHIFTED) {
      if (ty == 4) return launch3<float, float, 4, MODE>(c);
      if (ty == 16) return launch3<float, float, 16, MODE>(c);
      return launch3<float, float, 8, MODE>(c);
    }
    if (c->precision == LBM_F64_DF) return ty == 8 ? launch3<float2, dfn, 8, MODE>(c) : launch3<float2, dfn, 4, MODE>(c);
    if (ty == 8) return launch3<double, double, 8, MODE>(c);
    return launch3<double, double, 4, MODE>(c);
  }
}

cudaError_t launch_step3(lbm3d_ctx* c) {
  const int mode = c->keep >= 0 ? c->keep : default_keep(c);
  return mode == 1 ? launch_step3k<1>(c) : mode == 2 ? launch_step3k<2>(c) : launch_step3k<0>(c);
}

int ensure_stage3(lbm3d_ctx* c) {
  if (c->d_stage) return LBM_OK;
  c->d_stage = (double*)lbm::device_alloc(sizeof(double) * kQ * c->n(), c->stream);
  if (!c->d_stage) return fail3(c, LBM_ERR_OOM, "staging buffer allocation failed");
  return LBM_OK;
}

}  // namespace

namespace lbm {
cudaError_t bounds_record_3d(unsigned long long out[3]) {
#ifdef LBM_DEBUG_BOUNDS
  return take_bounds_record(out);
#else
  out[0] = out[1] = out[2] = 0ULL;
  return cudaSuccess;
#endif
}
}  // namespace lbm

extern "C" {

int lbm3d_create(lbm3d_ctx** out, int64_t nx, int64_t ny, int64_t nz, const lbm3d_params* params, int32_t precision,
                 void* stream) {
  if (!out) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  // ny / 4 tile rows must fit the grid's second dimension (65535); x, y and z indices fit an int.
  if (nx < 3 || ny < 3 || nz < 3 || nx > (1LL << 30) || ny > 4LL * 65535 || nz > (1LL << 30) ||
      nx * ny > (1LL << 33) || nx * ny * nz > (1LL << 33))
    return LBM_ERR_INVALID_ARG;
  if (precision != LBM_F64 && precision != LBM_F32_SHIFTED && precision != LBM_F64_DF) return LBM_ERR_INVALID_ARG;
  P3 p{};
  if (int rc = derive3(params, p)) return rc;
  lbm3d_ctx* c = new lbm3d_ctx();
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->precision = precision;
  c->stream = (cudaStream_t)stream;
  c->p = p;
  c->state[0] = lbm::device_alloc(c->state_bytes(), c->stream);
  c->state[1] = lbm::device_alloc(c->state_bytes(), c->stream);
  if (!c->state[0] || !c->state[1]) {
    lbm3d_destroy(c);
    return LBM_ERR_OOM;
  }
  *out = c;
  return LBM_OK;
}

void lbm3d_destroy(lbm3d_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (void* q : {c->state[0], c->state[1], (void*)c->d_stage}) lbm::device_free(q);
  delete c;
}

const char* lbm3d_last_error(const lbm3d_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t lbm3d_steps_done(const lbm3d_ctx* c) { return c ? c->steps_done : -1; }

int lbm3d_rates(const lbm3d_ctx* c, double* rates) {
  if (!c || !rates) return LBM_ERR_INVALID_ARG;
  rates[0] = c->p.se;
  rates[1] = c->p.spsi;
  rates[2] = c->p.seps;
  rates[3] = c->p.sq;
  rates[4] = c->p.sh;
  return LBM_OK;
}

int lbm3d_set_config(lbm3d_ctx* c, int32_t ty, int32_t zc, int32_t keep) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (keep < -1 || keep > 2) return fail3(c, LBM_ERR_INVALID_ARG, "lbm3d_set_config: keep must be -1, 0, 1 or 2");
  if (keep == 2 && (c->precision != LBM_F32_SHIFTED || (ty ? ty : (c->ty > 0 ? c->ty : default_ty(c))) != 4))
    return fail3(c, LBM_ERR_INVALID_ARG, "lbm3d_set_config: keep 2 (shared buffer) takes FP32 and ty 4");
  if (keep == -1 && c->keep == 2 && ty && ty != 4)
    return fail3(c, LBM_ERR_INVALID_ARG, "lbm3d_set_config: keep 2 (shared buffer) takes ty 4");
  if (zc < 0) return fail3(c, LBM_ERR_INVALID_ARG, "lbm3d_set_config: zc < 0");
  if (ty) c->ty = ty;
  if (zc) c->zc = zc;
  if (keep >= 0) c->keep = keep;
  return LBM_OK;
}

int lbm3d_get_config(const lbm3d_ctx* c, int32_t* ty, int32_t* zc, int32_t* keep) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (ty) *ty = c->ty > 0 ? c->ty : default_ty(c);
  if (zc) *zc = c->zc;
  if (keep) *keep = c->keep >= 0 ? c->keep : default_keep(c);
  return LBM_OK;
}

int lbm3d_set_state(lbm3d_ctx* c, const double* rho, const double* ux, const double* uy, const double* uz,
                    const double* s) {
  NvtxRange3 r_("lbm3d_set_state");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!rho || !ux || !uy || !uz || !s) return fail3(c, LBM_ERR_INVALID_ARG, "lbm3d_set_state: null array");
  const bool host = !lbm::is_device_pointer(rho);
  for (const double* a : {ux, uy, uz, s})
    if (host == lbm::is_device_pointer(a))
      return fail3(c, LBM_ERR_INVALID_ARG, "lbm3d_set_state: mix of host and device arrays");
  const long long n = c->n();
  const double* d[5] = {rho, ux, uy, uz, s};
  if (host) {
    if (int rc = ensure_stage3(c)) return rc;
    for (int k = 0; k < 5; ++k) {
      L3_CK(c, cudaMemcpyAsync(c->d_stage + k * n, d[k], sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
      d[k] = c->d_stage + k * n;
    }
  }
  if (c->precision == LBM_F64_DF)
    init3d_kernel<float2><<<blocks3(n, 256), 256, 0, c->stream>>>(d[0], d[1], d[2], d[3], d[4],
                                                                   (float2*)c->state[c->cur], n, c->p);
  else if (c->precision != LBM_F32_SHIFTED)
    init3d_kernel<double><<<blocks3(n, 256), 256, 0, c->stream>>>(d[0], d[1], d[2], d[3], d[4],
                                                                   (double*)c->state[c->cur], n, c->p);
  else
    init3d_kernel<float><<<blocks3(n, 256), 256, 0, c->stream>>>(d[0], d[1], d[2], d[3], d[4],
                                                                  (float*)c->state[c->cur], n, c->p);
  L3_CK(c, cudaGetLastError());
  if (host) L3_CK(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  c->steps_done = 0;
  return LBM_OK;
}

int lbm3d_step(lbm3d_ctx* c, int64_t nsteps) {
  NvtxRange3 r_("lbm3d_step");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (nsteps < 0) return fail3(c, LBM_ERR_INVALID_ARG, "lbm3d_step: nsteps < 0");
  if (!c->has_state) return fail3(c, LBM_ERR_INVALID_ARG, "lbm3d_step: no state set");
  for (int64_t k = 0; k < nsteps; ++k) {
    const cudaError_t e = launch_step3(c);
    if (e != cudaSuccess) return fail3(c, LBM_ERR_CUDA, std::string("lbm3d step launch: ") + cudaGetErrorString(e));
    c->cur = 1 - c->cur;
    ++c->steps_done;
  }
  return LBM_OK;
}

int lbm3d_get_populations(lbm3d_ctx* c, double* f) {
  NvtxRange3 r_("lbm3d_get_populations");
  if (!c || !f) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail3(c, LBM_ERR_INVALID_ARG, "lbm3d_get_populations: no state set");
  const long long n = c->n();
  const bool host = !lbm::is_device_pointer(f);
  if (host)
    if (int rc = ensure_stage3(c)) return rc;
  double* d = host ? c->d_stage : f;
  if (c->precision == LBM_F64_DF)
    pops3d_kernel<float2><<<blocks3(n, 256), 256, 0, c->stream>>>((const float2*)c->state[c->cur], d, n, c->p);
  else if (c->precision != LBM_F32_SHIFTED)
    pops3d_kernel<double><<<blocks3(n, 256), 256, 0, c->stream>>>((const double*)c->state[c->cur], d, n, c->p);
  else
    pops3d_kernel<float><<<blocks3(n, 256), 256, 0, c->stream>>>((const float*)c->state[c->cur], d, n, c->p);
  L3_CK(c, cudaGetLastError());
  if (host) {
    L3_CK(c, cudaMemcpyAsync(f, d, sizeof(double) * kQ * n, cudaMemcpyDeviceToHost, c->stream));
    L3_CK(c, cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

int lbm3d_fields(lbm3d_ctx* c, double* rho, double* ux, double* uy, double* uz, double* s) {
  NvtxRange3 r_("lbm3d_fields");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail3(c, LBM_ERR_INVALID_ARG, "lbm3d_fields: no state set");
  const long long n = c->n();
  double* outs[5] = {rho, ux, uy, uz, s};
  bool host[5] = {false, false, false, false, false};
  bool any_host = false;
  for (int k = 0; k < 5; ++k)
    if (outs[k] && !lbm::is_device_pointer(outs[k])) host[k] = any_host = true;
  if (any_host)
    if (int rc = ensure_stage3(c)) return rc;
  double* d[5];
  for (int k = 0; k < 5; ++k) d[k] = outs[k] ? (host[k] ? c->d_stage + k * n : outs[k]) : nullptr;
  if (c->precision == LBM_F64_DF)
    fields3d_kernel<float2><<<blocks3(n, 256), 256, 0, c->stream>>>((const float2*)c->state[c->cur], n, c->p, d[0],
                                                                      d[1], d[2], d[3], d[4]);
  else if (c->precision != LBM_F32_SHIFTED)
    fields3d_kernel<double><<<blocks3(n, 256), 256, 0, c->stream>>>((const double*)c->state[c->cur], n, c->p, d[0],
                                                                      d[1], d[2], d[3], d[4]);
  else
    fields3d_kernel<float><<<blocks3(n, 256), 256, 0, c->stream>>>((const float*)c->state[c->cur], n, c->p, d[0],
                                                                     d[1], d[2], d[3], d[4]);
  L3_CK(c, cudaGetLastError());
  for (int k = 0; k < 5; ++k)
    if (host[k]) L3_CK(c, cudaMemcpyAsync(outs[k], d[k], sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  if (any_host) L3_CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

}  // extern "C"
