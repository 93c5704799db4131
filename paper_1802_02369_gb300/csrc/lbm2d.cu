// Two-dimensional coupled D2Q9-D2Q5 scheme for (rho, J, zeta) (declarations and the readings in
// include/lbm.h): one fused collide-stream kernel per time step on 32 x TY tiles (TY = 12 FP32, 4 FP64).
//
// Variables. Populations are dimensionless (units of rho0) and stored shifted by those of the rest
// state (rho0, u = 0, s0); their moments, taken with the integer patterns of the moment rows, are the
// deviations of the moments scaled by rho0 lambda^k (and c_p for the entropy rows):
//   r = rho/rho0 - 1, j = J/(rho0 lambda), z = zeta/(rho0 c_p) - s0/c_p, and so on.
// With P = p/(rho0 lambda^2), P0 its rest value, sigma = (s - s0)/c_p, lr = log(1 + r),
// dP = P0 expm1(gamma (lr + sigma)), a = dP + (1 + r) ux^2, b = dP + (1 + r) uy^2 (u in units of
// lambda), the equilibrium deviations are
//   e = 3 (a + b) - 4 r, xx = a - b, xy = jx uy, q = -j,
//   h = 4 r - 6 (a + b) + 9 (P0 (a + b) + a b - P0^2 r) / (1 + r),
//   psi = (s0/c_p + z) u, xi = (s0/c_p + z)(ux^2 - uy^2), eps = 3 (Ax + Ay) - 4 z with
//   Ax = (s0/c_p) a + sigma (P0 + a) + L, L = (1 + r)(gamma - 1) lr + gamma sigma) / (gamma beta)
//   (and Ay with b), the deviations from the rest values of the equilibria in include/lbm.h.
// The production, in the same units, is q_vis (1 + r)^2 / P (2 D:D + (div u)^2) + q_th (1 + r)
// |grad T'|^2 / (1 + T')^2 with T' = T/T0 - 1 = (dP/P0 - r)/(1 + r), the derivatives as centred
// differences without the 1/2, q_vis = sigma_e (1 - 1/gamma) / 12, q_th = sigma_e / (4 Pr).
// The moment patterns of D2Q9 are orthogonal (norms 9, 6, 6, 36, 4, 4, 12, 12, 36), so the inverse
// is the transpose divided by the norms; the D2Q5 inverse is written out.
#include <cmath>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lbm_dfn.cuh"
#include "lbm_internal.cuh"

namespace {

constexpr int kQ = 14;
__constant__ int c_cx[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1, 0, 1, 0, -1, 0};
__constant__ int c_cy[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1, 0, 0, 1, 0, -1};

struct P2 {
  double rho0, lam, cp, s0, gamma, beta, Pr;
  double P0, s0c, inv_gb, gm1, q_vis, q_th;
  double se, sq, sh, spsi, seps;
  double w[kQ];  // rest populations
  int source_on;
};

template <typename R>
struct P2T {
  R P0, s0c, inv_gb, gm1, gamma, q_vis, q_th, se, sq, sh, spsi, seps;
  int source_on;
};

template <typename R>
__host__ __device__ P2T<R> lanes(const P2& p) {
  P2T<R> t;
  t.P0 = R(p.P0); t.s0c = R(p.s0c); t.inv_gb = R(p.inv_gb); t.gm1 = R(p.gm1); t.gamma = R(p.gamma);
  t.q_vis = R(p.q_vis); t.q_th = R(p.q_th);
  t.se = R(p.se); t.sq = R(p.sq); t.sh = R(p.sh); t.spsi = R(p.spsi); t.seps = R(p.seps);
  t.source_on = p.source_on;
  return t;
}

// The logarithm and exponential are those of the one-dimensional kernels (lbm_internal.cuh): FP32
// CUDA's log1pf / expm1f, FP64 the double-float series on the FP32 pipes. Reciprocals: FP32 a plain
// division (the hardware estimate measured slower in this kernel), FP64 an FP32 estimate refined by
// two FP64 Newton steps (the FP64 pipe bounds the FP64 kernel).
__device__ __forceinline__ float rcp2d(float x) { return 1.0f / x; }
__device__ __forceinline__ double rcp2d(double x) { return lbm::m_rcp(x); }

// Double-float numbers for LBM_F64_DF (lbm_dfn.cuh).
using lbm::dfn;
__device__ __forceinline__ dfn rcp2d(dfn x) { return lbm::dfn_rcp(x); }

__device__ __forceinline__ float lg2d(float x) { return lbm::m_log1p(x); }
__device__ __forceinline__ double lg2d(double x) { return lbm::m_log1p(x); }
__device__ __forceinline__ dfn lg2d(dfn x) { return lbm::dfn_log1p(x); }
__device__ __forceinline__ float ex2d(float x) { return lbm::m_expm1(x); }
__device__ __forceinline__ double ex2d(double x) { return lbm::m_expm1(x); }
__device__ __forceinline__ dfn ex2d(dfn x) { return lbm::dfn_expm1(x); }

// Values as stored (FP32 or FP64 planes).
// The double-float planes hold each population as its (hi, lo) FP32 pair (8 bytes, as a double), so
// that the step converts nothing on the FP64 pipe at its loads and stores.
__device__ __forceinline__ float stored(float x) { return x; }
__device__ __forceinline__ double stored(double x) { return x; }
__device__ __forceinline__ float2 stored(dfn x) { return make_float2(x.v.hi, x.v.lo); }
template <typename R>
__device__ __forceinline__ R loaded(float x) { return R(x); }
template <typename R>
__device__ __forceinline__ R loaded(double x) { return R(x); }
template <typename R>
__device__ __forceinline__ R loaded(float2 x) { return R(lbm::df{x.x, x.y}); }
// FP64 values of stored populations and the stored form of FP64 values (initialisation, read-out).
__device__ __forceinline__ double from_stored(float x) { return (double)x; }
__device__ __forceinline__ double from_stored(double x) { return x; }
__device__ __forceinline__ double from_stored(float2 x) { return (double)x.x + (double)x.y; }
template <typename S>
__device__ __forceinline__ S to_stored(double x) { return S(x); }
template <>
__device__ __forceinline__ float2 to_stored<float2>(double x) {
  const lbm::df d = lbm::df_from_double_host(x);
  return make_float2(d.hi, d.lo);
}

// Conserved deviations of shifted populations.
template <typename R>
struct Cons {
  R r, jx, jy, z;
};

template <typename R>
__device__ __forceinline__ Cons<R> conserved(const R (&f)[kQ]) {
  Cons<R> c;
  c.r = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  c.jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  c.jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
  c.z = ((f[9] + f[10]) + (f[11] + f[12])) + f[13];
  return c;
}

// The thermodynamic state of a node: velocity, entropy deviation, log density, pressure deviation.
template <typename R>
struct Thermo {
  R inv, ux, uy, sig, lr, dP;
};

template <typename R>
__device__ __forceinline__ Thermo<R> thermo(const Cons<R>& c, const P2T<R>& p) {
  Thermo<R> t;
  t.inv = rcp2d(R(1) + c.r);
  t.ux = c.jx * t.inv;
  t.uy = c.jy * t.inv;
  t.sig = (c.z - p.s0c * c.r) * t.inv;
  t.lr = lg2d(c.r);
  t.dP = p.P0 * ex2d(p.gamma * (t.lr + t.sig));
  return t;
}

template <typename R>
__device__ __forceinline__ R temp_dev(const Cons<R>& c, const Thermo<R>& t, const P2T<R>& p) {
  return (t.dP / p.P0 - c.r) * t.inv;
}

// Equilibrium deviations of the ten non-conserved moments (e, xx, xy, qx, qy, h, psi_x, psi_y, eps, xi).
template <typename R>
__device__ __forceinline__ void equilibria(const Cons<R>& c, const Thermo<R>& t, const P2T<R>& p, R (&eq)[10]) {
  const R a = t.dP + c.jx * t.ux, b = t.dP + c.jy * t.uy;
  const R apb = a + b;
  eq[0] = R(3) * apb - R(4) * c.r;
  eq[1] = a - b;
  eq[2] = c.jx * t.uy;
  eq[3] = -c.jx;
  eq[4] = -c.jy;
  eq[5] = R(4) * c.r - R(6) * apb + R(9) * ((p.P0 * apb + a * b) - p.P0 * p.P0 * c.r) * t.inv;
  const R zeta = p.s0c + c.z;
  eq[6] = zeta * t.ux;
  eq[7] = zeta * t.uy;
  const R L = (R(1) + c.r) * (p.gm1 * t.lr + p.gamma * t.sig) * p.inv_gb;
  const R Ax = p.s0c * a + t.sig * (p.P0 + a) + L, Ay = p.s0c * b + t.sig * (p.P0 + b) + L;
  eq[8] = R(3) * (Ax + Ay) - R(4) * c.z;
  eq[9] = zeta * (t.ux * t.ux - t.uy * t.uy);
}

// Populations from the conserved deviations and the ten non-conserved moments.
template <typename R>
__device__ __forceinline__ void populations(const Cons<R>& c, const R (&m)[10], R (&f)[kQ]) {
  const R R9 = c.r * R(1.0 / 9.0), JX = c.jx * R(1.0 / 6.0), JY = c.jy * R(1.0 / 6.0);
  const R E = m[0] * R(1.0 / 36.0), XX = m[1] * R(0.25), XY = m[2] * R(0.25);
  const R QX = m[3] * R(1.0 / 12.0), QY = m[4] * R(1.0 / 12.0), H = m[5] * R(1.0 / 36.0);
  const R base_axis = R9 - E - R(2) * H, base_diag = R9 + R(2) * E + H;
  f[0] = R9 - R(4) * E + R(4) * H;
  f[1] = base_axis + XX + (JX - R(2) * QX);
  f[3] = base_axis + XX - (JX - R(2) * QX);
  f[2] = base_axis - XX + (JY - R(2) * QY);
  f[4] = base_axis - XX - (JY - R(2) * QY);
  const R px = JX + QX, py = JY + QY;
  f[5] = base_diag + XY + (px + py);
  f[7] = base_diag + XY - (px + py);
  f[6] = base_diag - XY + (py - px);
  f[8] = base_diag - XY - (py - px);
  // D2Q5: zeta = sum g, psi = (g1 - g3, g2 - g4), eps = -4 g0 - (g1 + g2 + g3 + g4), xi = g1 - g2 + g3 - g4.
  const R g0 = -(c.z + m[8]) * R(1.0 / 3.0);
  const R S = c.z - g0;
  const R A = (S + m[9]) * R(0.5), B = (S - m[9]) * R(0.5);
  f[9] = g0;
  f[10] = (A + m[6]) * R(0.5);
  f[12] = (A - m[6]) * R(0.5);
  f[11] = (B + m[7]) * R(0.5);
  f[13] = (B - m[7]) * R(0.5);
}

// Non-conserved moment deviations of shifted populations.
template <typename R>
__device__ __forceinline__ void nonconserved(const R (&f)[kQ], R (&m)[10]) {
  const R ax = f[1] + f[3], ay = f[2] + f[4], axis = ax + ay;
  const R diag = (f[5] + f[7]) + (f[6] + f[8]);
  m[0] = R(-4) * f[0] - axis + R(2) * diag;
  m[1] = ax - ay;
  m[2] = (f[5] + f[7]) - (f[6] + f[8]);
  m[3] = R(-2) * (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
  m[4] = R(-2) * (f[2] - f[4]) + ((f[5] + f[6]) - (f[7] + f[8]));
  m[5] = R(4) * f[0] - R(2) * axis + diag;
  m[6] = f[10] - f[12];
  m[7] = f[11] - f[13];
  m[8] = R(-4) * f[9] - ((f[10] + f[11]) + (f[12] + f[13]));
  m[9] = (f[10] + f[12]) - (f[11] + f[13]);
}

__device__ __forceinline__ long long wrap(long long v, long long n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// One time step of a 32 x TY tile: the tile and a halo of 2 nodes are read into shared memory with
// their velocity and temperature deviation; the tile and a ring of 1 node collide (the production
// needs the neighbours' u and T'); the tile pulls its populations from the collided neighbours.
// S is the storage type of the planes, R the arithmetic (float, double, or dfn over planes of FP32 pairs).
template <typename S, typename R, int TY, bool REUSE>
__global__ void __launch_bounds__(32 * TY) step2d_kernel(const S* __restrict__ in, S* __restrict__ out, int nx, int ny,
                                                         long long plane, P2T<R> p) {
  constexpr int TX = 32, RX = TX + 4, RY = TY + 4, NR = RX * RY, NT = TX * TY;
  __shared__ R sf[kQ][NR];
  // Per node: u, T' (the neighbours' values of the production) and the rest of the thermodynamic
  // state, computed once for the tile and its halo and reused by the collision.
  constexpr int NS = REUSE ? NR : 1;
  __shared__ R su[NR], sv[NR], sT[NR], sinv[NS], ssig[NS], slr[NS], sdP[NS];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  for (int k = threadIdx.x; k < NR; k += NT) {
    const int ry = k / RX, rx = k - ry * RX;
    const long long gx = wrap((long long)x0 - 2 + rx, nx), gy = wrap((long long)y0 - 2 + ry, ny);
    const long long g = gy * nx + gx;
    R f[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      f[i] = lbm::in_bounds(g + i * plane, kQ * plane) ? loaded<R>(in[g + i * plane]) : R(0);
      sf[i][k] = f[i];
    }
    const Cons<R> c = conserved(f);
    const Thermo<R> t = thermo(c, p);
    su[k] = t.ux;
    sv[k] = t.uy;
    sT[k] = temp_dev(c, t, p);
    if constexpr (REUSE) {
      sinv[k] = t.inv;
      ssig[k] = t.sig;
      slr[k] = t.lr;
      sdP[k] = t.dP;
    }
  }
  __syncthreads();
  constexpr int IX = RX - 2, NI = IX * (RY - 2);
  for (int k = threadIdx.x; k < NI; k += NT) {
    const int iy = k / IX;
    const int n = (iy + 1) * RX + (k - iy * IX) + 1;
    R f[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) f[i] = sf[i][n];
    Cons<R> c = conserved(f);
    const Thermo<R> t = [&]() {
      if constexpr (REUSE) {
        Thermo<R> k;
        k.inv = sinv[n];
        k.ux = su[n];
        k.uy = sv[n];
        k.sig = ssig[n];
        k.lr = slr[n];
        k.dP = sdP[n];
        return k;
      } else {
        return thermo(c, p);
      }
    }();
    R m[10], eq[10];
    nonconserved(f, m);
    equilibria(c, t, p, eq);
    const R rate[10] = {p.se, p.se, p.se, p.sq, p.sq, p.sh, p.spsi, p.spsi, p.seps, p.seps};
#pragma unroll
    for (int i = 0; i < 10; ++i) m[i] = m[i] + rate[i] * (eq[i] - m[i]);
    if (p.source_on) {
      const R dxu = su[n + 1] - su[n - 1], dyu = su[n + RX] - su[n - RX];
      const R dxv = sv[n + 1] - sv[n - 1], dyv = sv[n + RX] - sv[n - RX];
      const R dxT = sT[n + 1] - sT[n - 1], dyT = sT[n + RX] - sT[n - RX];
      const R shear = dyu + dxv, div = dxu + dyv;
      const R G = R(2) * (dxu * dxu + dyv * dyv) + shear * shear + div * div;  // 2 D:D + (div u)^2
      const R rho = R(1) + c.r, P = p.P0 + t.dP, Tn = R(1) + sT[n];
      if constexpr (sizeof(R) == 4)
        c.z = c.z + p.q_vis * rho * rho / P * G + p.q_th * rho * (dxT * dxT + dyT * dyT) / (Tn * Tn);
      else
        c.z = c.z + p.q_vis * rho * rho * rcp2d(P) * G + p.q_th * rho * (dxT * dxT + dyT * dyT) * rcp2d(Tn * Tn);
    }
    populations(c, m, f);
#pragma unroll
    for (int i = 0; i < kQ; ++i) sf[i][n] = f[i];
  }
  __syncthreads();
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const long long gx = (long long)x0 + tx, gy = (long long)y0 + ty;
  if (gx < nx && gy < ny) {
    const int n = (ty + 2) * RX + tx + 2;
    const long long g = gy * nx + gx;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const int src = n - c_cy[i] * RX - c_cx[i];
      if (lbm::in_bounds(g + i * plane, kQ * plane) && lbm::in_bounds(src, NR)) out[g + i * plane] = stored(sf[i][src]);
    }
  }
}

// Equilibrium populations from the physical fields, in FP64, stored shifted in R.
template <typename R>
__global__ void init2d_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                              const double* __restrict__ uy, const double* __restrict__ s, R* __restrict__ st,
                              long long n, P2 p) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const P2T<double> q = lanes<double>(p);
  Cons<double> c;
  c.r = rho[i] / p.rho0 - 1.0;
  c.jx = rho[i] * ux[i] / (p.rho0 * p.lam);
  c.jy = rho[i] * uy[i] / (p.rho0 * p.lam);
  c.z = (rho[i] * s[i] - p.rho0 * p.s0) / (p.rho0 * p.cp);
  const Thermo<double> t = thermo(c, q);
  double eq[10], f[kQ];
  equilibria(c, t, q, eq);
  populations(c, eq, f);
#pragma unroll
  for (int k = 0; k < kQ; ++k) st[k * n + i] = to_stored<R>(f[k]);
}

// Populations, node-major and unshifted, in FP64.
template <typename R>
__global__ void pops2d_kernel(const R* __restrict__ st, double* __restrict__ out, long long n, P2 p) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int k = 0; k < kQ; ++k) out[kQ * i + k] = from_stored(st[k * n + i]) + p.w[k];
}

template <typename R>
__global__ void fields2d_kernel(const R* __restrict__ st, long long n, P2 p, double* rho, double* ux, double* uy,
                                double* s) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[kQ];
#pragma unroll
  for (int k = 0; k < kQ; ++k) f[k] = from_stored(st[k * n + i]);
  const Cons<double> c = conserved(f);
  const double r1 = 1.0 + c.r;
  if (rho) rho[i] = p.rho0 * r1;
  if (ux) ux[i] = p.lam * c.jx / r1;
  if (uy) uy[i] = p.lam * c.jy / r1;
  if (s) s[i] = p.cp * (p.s0c + c.z) / r1;
}

}  // namespace

struct lbm2d_ctx {
  long long nx = 0, ny = 0;
  int precision = LBM_F64;
  cudaStream_t stream = nullptr;
  P2 p{};
  void* state[2] = {nullptr, nullptr};
  int cur = 0;
  double* d_stage = nullptr;
  bool has_state = false;
  long long steps_done = 0;
  std::string err;
  long long n() const { return nx * ny; }
  size_t state_bytes() const {
    return (size_t)kQ * n() * (precision == LBM_F32_SHIFTED ? sizeof(float) : sizeof(double));
  }
};

namespace {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int fail(lbm2d_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define L2_CK(ctx, call)                                                                                     \
  do {                                                                                                       \
    cudaError_t e_ = (call);                                                                                 \
    if (e_ != cudaSuccess) return fail(ctx, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool rate_ok(double s) { return s > 0.0 && s < 2.0 && std::isfinite(s); }

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int derive(const lbm2d_params* in, P2& p) {
  if (!in) return LBM_ERR_INVALID_ARG;
  p.gamma = in->gamma;
  p.Pr = in->Pr;
  p.cp = in->cp;
  p.rho0 = in->rho0;
  p.lam = in->lambda;
  p.s0 = in->s0;
  const double dx = in->dx;
  if (!(p.gamma > 1.0) || !(p.Pr > 0.0) || !(p.cp > 0.0) || !(p.rho0 > 0.0) || !(p.lam > 0.0) || !(dx > 0.0) ||
      !std::isfinite(p.s0) || !std::isfinite(p.gamma) || !std::isfinite(p.lam))
    return LBM_ERR_INVALID_ARG;
  const double p0 = in->p0 > 0.0 ? in->p0 : p.rho0 * 0.25 * p.lam * p.lam / p.gamma;
  p.beta = in->beta > 0.0 ? in->beta : 4.5;
  p.se = in->s_e;
  if (!rate_ok(p.se) || !std::isfinite(p0) || !std::isfinite(p.beta)) return LBM_ERR_INVALID_ARG;
  const double sigma_e = 1.0 / p.se - 0.5;
  p.spsi = in->s_psi > 0.0 ? in->s_psi : 1.0 / (p.beta * (p.gamma / p.Pr) * sigma_e + 0.5);
  p.seps = in->s_eps > 0.0 ? in->s_eps : 1.5;
  p.sq = in->s_q > 0.0 ? in->s_q : 1.5;
  p.sh = in->s_h > 0.0 ? in->s_h : 1.5;
  if (!rate_ok(p.spsi) || !rate_ok(p.seps) || !rate_ok(p.sq) || !rate_ok(p.sh)) return LBM_ERR_INVALID_ARG;
  p.P0 = p0 / (p.rho0 * p.lam * p.lam);
  p.s0c = p.s0 / p.cp;
  p.inv_gb = 1.0 / (p.gamma * p.beta);
  p.gm1 = p.gamma - 1.0;
  p.q_vis = sigma_e * (1.0 - 1.0 / p.gamma) / 12.0;
  p.q_th = sigma_e / (4.0 * p.Pr);
  p.source_on = in->source_on != 0;
  // Rest populations: D2Q9 (r = 1, e = 6 P0 - 4, h = 4 - 12 P0 + 9 P0^2 in units of rho0 lambda^k),
  // D2Q5 (zeta = s0/c_p, eps = (6 P0 - 4) s0/c_p), through the inverses of the kernel.
  const double E = (6.0 * p.P0 - 4.0) / 36.0, H = (4.0 - 12.0 * p.P0 + 9.0 * p.P0 * p.P0) / 36.0, R9 = 1.0 / 9.0;
  p.w[0] = R9 - 4.0 * E + 4.0 * H;
  for (int i = 1; i <= 4; ++i) p.w[i] = R9 - E - 2.0 * H;
  for (int i = 5; i <= 8; ++i) p.w[i] = R9 + 2.0 * E + H;
  const double z = p.s0c, eps = (6.0 * p.P0 - 4.0) * p.s0c;
  const double g0 = -(z + eps) / 3.0, S = z - g0;
  p.w[9] = g0;
  for (int i = 10; i <= 13; ++i) p.w[i] = S * 0.25;
  return LBM_OK;
}

template <typename S, typename R>
cudaError_t launch_step(lbm2d_ctx* c) {
  // Tile heights measured at 8192 x 8192: FP32 8 / 12 / 16 rows 31.0 / 31.7 / 23.6 GLUPS (16 rows raise
  // the registers and halve the CTAs per SM); FP64 4 rows, the most that fits 48 KB of shared memory.
  constexpr int TY = sizeof(S) == 4 ? 12 : 4;
  // FP64 keeps the thermodynamic state of phase 1 for the collision (its logarithm, exponential and
  // reciprocals load the FP64 pipe); FP32 recomputes it, measured faster.
  constexpr bool REUSE = sizeof(S) == 8;
  const dim3 grid((unsigned)((c->nx + 31) / 32), (unsigned)((c->ny + TY - 1) / TY));
  step2d_kernel<S, R, TY, REUSE><<<grid, 32 * TY, 0, c->stream>>>((const S*)c->state[c->cur], (S*)c->state[1 - c->cur],
                                                          (int)c->nx, (int)c->ny, c->n(), lanes<R>(c->p));
  return cudaGetLastError();
}

// One staging buffer of 14 doubles per node serves every host transfer (4 fields or 14 populations).
int ensure_stage(lbm2d_ctx* c) {
  if (c->d_stage) return LBM_OK;
  c->d_stage = (double*)lbm::device_alloc(sizeof(double) * kQ * c->n(), c->stream);
  if (!c->d_stage) return fail(c, LBM_ERR_OOM, "staging buffer allocation failed");
  return LBM_OK;
}

}  // namespace

namespace lbm {
cudaError_t bounds_record_2d(unsigned long long out[3]) {
#ifdef LBM_DEBUG_BOUNDS
  return take_bounds_record(out);
#else
  out[0] = out[1] = out[2] = 0ULL;
  return cudaSuccess;
#endif
}
}  // namespace lbm

extern "C" {

int lbm2d_create(lbm2d_ctx** out, int64_t nx, int64_t ny, const lbm2d_params* params, int32_t precision,
                 void* stream) {
  if (!out) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  // ny / 4 tile rows must fit the grid's second dimension (65535).
  if (nx < 3 || ny < 3 || nx > (1LL << 30) || ny > 4LL * 65535 || nx * ny > (1LL << 34)) return LBM_ERR_INVALID_ARG;
  if (precision != LBM_F64 && precision != LBM_F32_SHIFTED && precision != LBM_F64_DF) return LBM_ERR_INVALID_ARG;
  P2 p{};
  if (int rc = derive(params, p)) return rc;
  lbm2d_ctx* c = new lbm2d_ctx();
  c->nx = nx;
  c->ny = ny;
  c->precision = precision;
  c->stream = (cudaStream_t)stream;
  c->p = p;
  c->state[0] = lbm::device_alloc(c->state_bytes(), c->stream);
  c->state[1] = lbm::device_alloc(c->state_bytes(), c->stream);
  if (!c->state[0] || !c->state[1]) {
    lbm2d_destroy(c);
    return LBM_ERR_OOM;
  }
  *out = c;
  return LBM_OK;
}

void lbm2d_destroy(lbm2d_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (void* q : {c->state[0], c->state[1], (void*)c->d_stage}) lbm::device_free(q);
  delete c;
}

const char* lbm2d_last_error(const lbm2d_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t lbm2d_steps_done(const lbm2d_ctx* c) { return c ? c->steps_done : -1; }

int lbm2d_rates(const lbm2d_ctx* c, double* rates) {
  if (!c || !rates) return LBM_ERR_INVALID_ARG;
  rates[0] = c->p.se;
  rates[1] = c->p.spsi;
  rates[2] = c->p.seps;
  rates[3] = c->p.sq;
  rates[4] = c->p.sh;
  return LBM_OK;
}

int lbm2d_set_state(lbm2d_ctx* c, const double* rho, const double* ux, const double* uy, const double* s) {
  NvtxRange r_("lbm2d_set_state");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!rho || !ux || !uy || !s) return fail(c, LBM_ERR_INVALID_ARG, "lbm2d_set_state: null array");
  const bool host = !lbm::is_device_pointer(rho);
  for (const double* a : {ux, uy, s})
    if (host == lbm::is_device_pointer(a)) return fail(c, LBM_ERR_INVALID_ARG, "lbm2d_set_state: mix of host and device arrays");
  const long long n = c->n();
  const double *a = rho, *b = ux, *d = uy, *e = s;
  if (host) {
    if (int rc = ensure_stage(c)) return rc;
    const double* src[4] = {rho, ux, uy, s};
    for (int k = 0; k < 4; ++k)
      L2_CK(c, cudaMemcpyAsync(c->d_stage + k * n, src[k], sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    a = c->d_stage;
    b = c->d_stage + n;
    d = c->d_stage + 2 * n;
    e = c->d_stage + 3 * n;
  }
  if (c->precision == LBM_F64_DF)
    init2d_kernel<float2><<<blocks_for(n, 256), 256, 0, c->stream>>>(a, b, d, e, (float2*)c->state[c->cur], n, c->p);
  else if (c->precision != LBM_F32_SHIFTED)
    init2d_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>(a, b, d, e, (double*)c->state[c->cur], n, c->p);
  else
    init2d_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>(a, b, d, e, (float*)c->state[c->cur], n, c->p);
  L2_CK(c, cudaGetLastError());
  if (host) L2_CK(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  c->steps_done = 0;
  return LBM_OK;
}

int lbm2d_step(lbm2d_ctx* c, int64_t nsteps) {
  NvtxRange r_("lbm2d_step");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (nsteps < 0) return fail(c, LBM_ERR_INVALID_ARG, "lbm2d_step: nsteps < 0");
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "lbm2d_step: no state set");
  for (int64_t k = 0; k < nsteps; ++k) {
    const cudaError_t e = c->precision == LBM_F32_SHIFTED ? launch_step<float, float>(c)
                          : c->precision == LBM_F64_DF   ? launch_step<float2, dfn>(c)
                                                         : launch_step<double, double>(c);
    if (e != cudaSuccess) return fail(c, LBM_ERR_CUDA, std::string("lbm2d step launch: ") + cudaGetErrorString(e));
    c->cur = 1 - c->cur;
    ++c->steps_done;
  }
  return LBM_OK;
}

int lbm2d_get_populations(lbm2d_ctx* c, double* f) {
  NvtxRange r_("lbm2d_get_populations");
  if (!c || !f) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "lbm2d_get_populations: no state set");
  const long long n = c->n();
  const bool host = !lbm::is_device_pointer(f);
  if (host)
    if (int rc = ensure_stage(c)) return rc;
  double* d = host ? c->d_stage : f;
  if (c->precision == LBM_F64_DF)
    pops2d_kernel<float2><<<blocks_for(n, 256), 256, 0, c->stream>>>((const float2*)c->state[c->cur], d, n, c->p);
  else if (c->precision != LBM_F32_SHIFTED)
    pops2d_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>((const double*)c->state[c->cur], d, n, c->p);
  else
    pops2d_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>((const float*)c->state[c->cur], d, n, c->p);
  L2_CK(c, cudaGetLastError());
  if (host) {
    L2_CK(c, cudaMemcpyAsync(f, d, sizeof(double) * kQ * n, cudaMemcpyDeviceToHost, c->stream));
    L2_CK(c, cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

int lbm2d_fields(lbm2d_ctx* c, double* rho, double* ux, double* uy, double* s) {
  NvtxRange r_("lbm2d_fields");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "lbm2d_fields: no state set");
  const long long n = c->n();
  double* outs[4] = {rho, ux, uy, s};
  bool host[4] = {false, false, false, false};
  bool any_host = false;
  for (int k = 0; k < 4; ++k)
    if (outs[k] && !lbm::is_device_pointer(outs[k])) host[k] = any_host = true;
  if (any_host)
    if (int rc = ensure_stage(c)) return rc;
  double* d[4];
  for (int k = 0; k < 4; ++k) d[k] = outs[k] ? (host[k] ? c->d_stage + k * n : outs[k]) : nullptr;
  if (c->precision == LBM_F64_DF)
    fields2d_kernel<float2><<<blocks_for(n, 256), 256, 0, c->stream>>>((const float2*)c->state[c->cur], n, c->p, d[0],
                                                                         d[1], d[2], d[3]);
  else if (c->precision != LBM_F32_SHIFTED)
    fields2d_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>((const double*)c->state[c->cur], n, c->p, d[0],
                                                                         d[1], d[2], d[3]);
  else
    fields2d_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>((const float*)c->state[c->cur], n, c->p, d[0],
                                                                        d[1], d[2], d[3]);
  L2_CK(c, cudaGetLastError());
  for (int k = 0; k < 4; ++k)
    if (host[k]) L2_CK(c, cudaMemcpyAsync(outs[k], d[k], sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  if (any_host) L2_CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

}  // extern "C"
