// C-ABI of the D1Q3Q3 library (declared in include/lbm.h): context management, parameter
// derivation (step (iii) of section 8), equilibrium initialisation, moment read-back,
// deterministic FP64 diagnostics and checkpoints. The time step itself is in lbm_step.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <type_traits>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"
#include "lbm_df.cuh"

using lbm::Consts;
using lbm::LatDev;

namespace {

constexpr int kChunk = 1024;       // nodes per diagnostics chunk
constexpr int kDiagThreads = 256;  // 4 nodes per thread

lbm_alloc_fn g_alloc = nullptr;
lbm_free_fn g_free = nullptr;
void* g_user = nullptr;

// Physical constants in FP64 after defaults are applied.
struct PhysD {
  double gamma, Pr, cp, rho0, p0, s0, lam;
  int source_on;
  int eq_mode;            // 0 nonlinear (section 8), 1 linear (section 7)
  double u0_lin, s0_lin;  // state of the linearisation (eq_mode 1)
  double c02() const { return gamma * p0 / rho0; }
  // Coefficients of the linear equilibria of eq. (equilibres-NS-linearise) on rho (lambda = c_p = 1).
  double lin_a1() const { return 3.0 * (1.0 - s0_lin / cp) * c02() - 3.0 * u0_lin * u0_lin - 2.0 * lam * lam; }
  double lin_b1() const {
    return -3.0 * (s0_lin * s0_lin * c02()) - 6.0 * s0_lin * u0_lin * u0_lin + 3.0 * s0_lin * c02() + 2.0 -
           2.0 * s0_lin - 2.0 / gamma;
  }
  double r() const { return cp * (1.0 - 1.0 / gamma); }
  double e_r() const { return 3.0 * p0 - 2.0 * lam * lam * rho0; }
  double wf0() const { return 1.0 - p0 / (rho0 * lam * lam); }  // rest populations of f
  double wf1() const { return p0 / (2.0 * rho0 * lam * lam); }
};

template <typename X>
X lift(double v) {
  if constexpr (std::is_same<X, float2>::value) return make_float2((float)v, (float)v);
  else if constexpr (std::is_same<X, lbm::df>::value) return lbm::df_from_double_host(v);
  else return X(v);
}

template <typename X>
Consts<X> make_consts(const PhysD& p) {
  Consts<X> c;
  const double l = p.lam, l2 = l * l, af = p.rho0, ag = p.rho0 * p.cp;
  c.rho0 = lift<X>(p.rho0);
  c.lam = lift<X>(l);
  c.two_lam2 = lift<X>(2.0 * l2);
  c.m_two_lam2 = lift<X>(-2.0 * l2);
  c.inv_af = lift<X>(1.0 / af);
  c.inv_af_l = lift<X>(1.0 / (af * l));
  c.inv_af_l2 = lift<X>(1.0 / (af * l2));
  c.af_l = lift<X>(af * l);
  c.af_l2 = lift<X>(af * l2);
  c.ag = lift<X>(ag);
  c.ag_l = lift<X>(ag * l);
  c.ag_l2 = lift<X>(ag * l2);
  c.inv_ag = lift<X>(1.0 / ag);
  c.inv_ag_l = lift<X>(1.0 / (ag * l));
  c.inv_ag_l2 = lift<X>(1.0 / (ag * l2));
  c.gamma = lift<X>(p.gamma);
  c.inv_cp = lift<X>(1.0 / p.cp);
  c.p0 = lift<X>(p.p0);
  c.inv_r = lift<X>(1.0 / p.r());
  c.e_r = lift<X>(p.e_r());
  c.cp_log = lift<X>((1.0 - 1.0 / p.gamma) * p.cp);
  c.cp_over_Pr = lift<X>(p.cp / p.Pr);
  c.one = lift<X>(1.0);
  c.m_one = lift<X>(-1.0);
  c.two = lift<X>(2.0);
  c.m_two = lift<X>(-2.0);
  c.three = lift<X>(3.0);
  c.half = lift<X>(0.5);
  c.m_half = lift<X>(-0.5);
  c.third = lift<X>(1.0 / 3.0);
  c.sixth = lift<X>(1.0 / 6.0);
  const double kp = p.p0 / (p.rho0 * l2);
  c.kp = lift<X>(kp);
  c.kth = lift<X>(kp * p.gamma / (p.gamma - 1.0));
  c.e_rs = lift<X>(3.0 * kp - 2.0);
  c.one_m_ig = lift<X>(1.0 - 1.0 / p.gamma);
  c.inv_Pr = lift<X>(1.0 / p.Pr);
  {
    const double u0 = p.u0_lin, s0 = p.s0_lin;
    c.leR = lift<X>(p.lin_a1());
    c.leJ = lift<X>(6.0 * u0);
    c.leZ = lift<X>(3.0 * u0 * u0);
    c.lpR = lift<X>(-u0 * s0);
    c.lpJ = lift<X>(s0);
    c.lpZ = lift<X>(u0);
    c.lqR = lift<X>(p.lin_b1());
    c.lqJ = lift<X>(6.0 * u0 * s0);
    c.lqZ = lift<X>(3.0 * (u0 * u0 + s0 * p.c02()));
  }
  c.eq_mode = p.eq_mode;
  c.source_on = p.source_on;
  return c;
}

template <typename R>
lbm::ConstSet<R> make_constset(const PhysD& p) {
  lbm::ConstSet<R> k;
  k.s = make_consts<R>(p);
  k.p = make_consts<float2>(p);
  return k;
}

void* dev_alloc(size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  if (g_alloc) return g_alloc(bytes, (void*)st, g_user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void* p) {
  if (!p) return;
  if (g_free) g_free(p, g_user);
  else cudaFree(p);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of page-locked (pinned) host memory, which kernels can read and write in place
// over the CPU-GPU link (on GB300 the NVLink-C2C link to Grace); nullptr for pageable memory.
const void* mapped_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// ---------------------------------------------------------------------------------------------
// Small kernels.

__device__ __forceinline__ int lattice_of_node(const LatDev* lat, int B, long long i) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (lat[mid].offset <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct InitArgs {
  double rho0, p0, gamma, cp, lam, e_r, cp_log, wf0, wf1;
  int eq_mode;
  double u0_lin, s0_lin, a1, b1, c02;
  // Reciprocals for the initialisation: 1/rho0, 1/p0, 1/c_p, c_p/gamma, and the moment scales
  // 1/(rho0 lambda^k), 1/(rho0 c_p lambda^k), k = 0, 1, 2 (a product instead of an FP64 division).
  double inv_rho0, inv_p0, inv_cp, cp_over_gamma, inv_af[3], inv_ag[3];
};

// log1p and expm1 of the initialisation: FP64 for FP64 storage; for FP32 storage double-float on the
// FP32 pipes (about 48 significant bits, far below the rounding of the stored float; this GPU's FP64
// pipe made the FP64 functions the bulk of the kernel).
template <typename R>
__device__ __forceinline__ double init_log1p(double x) {
  if constexpr (sizeof(R) == 4) return lbm::to_double(lbm::m_log1p(lbm::to_df(x)));
  else return log1p(x);
}
template <typename R>
__device__ __forceinline__ double init_expm1(double x) {
  if constexpr (sizeof(R) == 4) return lbm::to_double(lbm::m_expm1(lbm::to_df(x)));
  else return expm1(x);
}

// Equilibrium populations from (rho, u, p) (from_p = 1) or (rho, u, s) (from_p = 0), computed in
// FP64 (the logarithms and the exponential as above) and stored shifted by the rest populations.
template <typename R>
__global__ void init_kernel(const double* __restrict__ rho_in, const double* __restrict__ u_in,
                            const double* __restrict__ x_in, int from_p, R* __restrict__ st,
                            long long plane, const LatDev* __restrict__ lat, int B, InitArgs a) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= plane) return;
  const LatDev& d = lat[lattice_of_node(lat, B, i)];
  const double rho = rho_in[i], u = u_in[i];
  const double lnr = init_log1p<R>((rho - a.rho0) * a.inv_rho0);
  const double ds = from_p ? a.cp_over_gamma * init_log1p<R>((x_in[i] - a.p0) * a.inv_p0) - a.cp * lnr : x_in[i] - d.s0;
  const double s = d.s0 + ds;
  const double pt = a.p0 * init_expm1<R>(a.gamma * (lnr + ds * a.inv_cp));
  const double rt = rho - a.rho0, J = rho * u;
  const double zeta = rho * s, zt = zeta - d.zeta_r;
  const double l2 = a.lam * a.lam;
  double e_t, psi, eps_t;
  if (a.eq_mode == 1) {
    // Eq. (equilibres-NS-linearise), lambda = c_p = 1, shifted by the rest moments.
    const double u0 = a.u0_lin, s0 = a.s0_lin;
    e_t = a.a1 * rho + 6.0 * u0 * J + 3.0 * (u0 * u0 / a.cp) * zeta - a.e_r;
    psi = -u0 * s0 * rho + s0 * J + u0 * zeta;
    eps_t = a.b1 * rho + 6.0 * u0 * s0 * J + 3.0 * (a.cp * u0 * u0 + s0 * a.c02) * zeta - a.e_r * d.s0;
  } else {
    e_t = 3.0 * (J * u + pt) - 2.0 * l2 * rt;
    psi = zeta * u;
    eps_t = 2.0 * l2 * rho * (ds + a.cp_log * lnr) + e_t * s + a.e_r * ds;
  }
  // Scaled moments, then M^-1 (eq. M-d1q3q3 inverted); the FP64 pipe of this GPU runs a division as a
  // Newton sequence, so every scale is a product with a host-computed reciprocal.
  const double third = 1.0 / 3.0, sixth = 1.0 / 6.0;
  double r = rt * a.inv_af[0], j = J * a.inv_af[1], q = e_t * a.inv_af[2];
  double h = (2.0 * r + q) * sixth;
  st[0 * plane + i] = R((r - q) * third);
  st[1 * plane + i] = R(h + 0.5 * j);
  st[2 * plane + i] = R(h - 0.5 * j);
  r = zt * a.inv_ag[0]; j = psi * a.inv_ag[1]; q = eps_t * a.inv_ag[2];
  h = (2.0 * r + q) * sixth;
  st[3 * plane + i] = R((r - q) * third);
  st[4 * plane + i] = R(h + 0.5 * j);
  st[5 * plane + i] = R(h - 0.5 * j);
}

// Moments (absolute) per node; any output may be null.
template <typename R>
__global__ void moments_kernel(const R* __restrict__ st, long long plane, const LatDev* __restrict__ lat,
                               int B, InitArgs a, double* rho, double* J, double* zeta, double* e,
                               double* psi, double* eps) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= plane) return;
  const LatDev& d = lat[lattice_of_node(lat, B, i)];
  double f[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) f[k] = (double)st[k * plane + i];
  const double l = a.lam, af = a.rho0, ag = a.rho0 * a.cp;
  if (rho) rho[i] = a.rho0 + af * (f[0] + f[1] + f[2]);
  if (J) J[i] = af * l * (f[1] - f[2]);
  if (e) e[i] = a.e_r + af * l * l * (f[1] + f[2] - 2.0 * f[0]);
  if (zeta) zeta[i] = d.zeta_r + ag * (f[3] + f[4] + f[5]);
  if (psi) psi[i] = ag * l * (f[4] - f[5]);
  if (eps) eps[i] = d.eps_r + ag * l * l * (f[4] + f[5] - 2.0 * f[3]);
}

template <typename R>
__global__ void pops_out_kernel(const R* __restrict__ st, long long plane, const LatDev* __restrict__ lat,
                                int B, double wf0, double wf1, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= plane) return;
  const LatDev& d = lat[lattice_of_node(lat, B, i)];
  const double w[6] = {wf0, wf1, wf1, d.wg0, d.wg1, d.wg1};
#pragma unroll
  for (int k = 0; k < 6; ++k) out[k * plane + i] = (double)st[k * plane + i] + w[k];
}

template <typename R>
__global__ void pops_in_kernel(R* __restrict__ st, long long plane, const LatDev* __restrict__ lat, int B,
                               double wf0, double wf1, const double* __restrict__ in) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= plane) return;
  const LatDev& d = lat[lattice_of_node(lat, B, i)];
  const double w[6] = {wf0, wf1, wf1, d.wg0, d.wg1, d.wg1};
#pragma unroll
  for (int k = 0; k < 6; ++k) st[k * plane + i] = R(in[k * plane + i] - w[k]);
}

// Diagnostics, pass 1: one block per chunk of kChunk nodes of one lattice; fixed-order reduction.
template <typename R>
__global__ void __launch_bounds__(kDiagThreads) diag_chunk_kernel(const R* __restrict__ st, long long plane,
                                                                  const LatDev* __restrict__ lat, int B, InitArgs a,
                                                                  double gamma, double inv_r,
                                                                  double* __restrict__ part,
                                                                  int* __restrict__ pflag) {
  const long long chunk = blockIdx.x;
  int L = 0;
  {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (lat[mid].chunk0 <= chunk) lo = mid; else hi = mid - 1;
    }
    L = lo;
  }
  const LatDev& d = lat[L];
  const long long base = (chunk - d.chunk0) * kChunk;
  double acc[4] = {0, 0, 0, 0};
  int fl = 0;
  const double l = a.lam, af = a.rho0, ag = a.rho0 * a.cp;
  for (int t = 0; t < kChunk / kDiagThreads; ++t) {
    const long long pos = base + t * kDiagThreads + threadIdx.x;
    if (pos >= d.n) break;
    const long long i = d.offset + pos;
    double f[6];
    for (int k = 0; k < 6; ++k) {
      f[k] = (double)st[k * plane + i];
      if (!isfinite(f[k])) fl |= 1;
    }
    const double rt = af * (f[0] + f[1] + f[2]);
    const double rho = a.rho0 + rt;
    const double J = af * l * (f[1] - f[2]);
    const double zt = ag * (f[3] + f[4] + f[5]);
    const double u = J / rho;
    const double ds = (zt - rt * d.s0) / rho;
    const double p = a.p0 * exp(gamma * (log(rho / a.rho0) + ds / a.cp));
    const double T = p / rho * inv_r;
    if (!(rho > 0.0)) fl |= 2;
    if (!(T > 0.0) || !isfinite(T)) fl |= 4;
    acc[0] += rho;
    acc[1] += J;
    acc[2] += d.zeta_r + zt;
    acc[3] += p / (gamma - 1.0) + 0.5 * rho * u * u;
  }
  __shared__ double sh[4][kDiagThreads / 32];
  __shared__ int shf[kDiagThreads / 32];
  for (int k = 0; k < 4; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = v;
  }
  int f2 = fl;
  for (int o = 16; o > 0; o >>= 1) f2 |= __shfl_down_sync(0xffffffffu, f2, o);
  if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = f2;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      double v = 0.0;
      for (int w = 0; w < kDiagThreads / 32; ++w) v += sh[k][w];
      part[chunk * 4 + k] = v;
    }
    int ff = 0;
    for (int w = 0; w < kDiagThreads / 32; ++w) ff |= shf[w];
    pflag[chunk] = ff;
  }
}

// Diagnostics, pass 2: one block per lattice sums its chunks in a fixed order.
__global__ void __launch_bounds__(256) diag_final_kernel(const double* __restrict__ part, const int* __restrict__ pflag,
                                                         const LatDev* __restrict__ lat, int B, long long nchunks,
                                                         double* __restrict__ sums, int* __restrict__ flags) {
  const int L = blockIdx.x;
  const long long c0 = lat[L].chunk0;
  const long long c1 = (L + 1 < B) ? lat[L + 1].chunk0 : nchunks;
  double acc[4] = {0, 0, 0, 0};
  int fl = 0;
  for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    for (int k = 0; k < 4; ++k) acc[k] += part[c * 4 + k];
    fl |= pflag[c];
  }
  __shared__ double sh[4][8];
  __shared__ int shf[8];
  for (int k = 0; k < 4; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = v;
  }
  int f2 = fl;
  for (int o = 16; o > 0; o >>= 1) f2 |= __shfl_down_sync(0xffffffffu, f2, o);
  if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = f2;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      double v = 0.0;
      for (int w = 0; w < 8; ++w) v += sh[k][w];
      sums[L * 4 + k] = v;
    }
    int ff = 0;
    for (int w = 0; w < 8; ++w) ff |= shf[w];
    flags[L] = ff;
  }
}

}  // namespace

namespace lbm {
void* device_alloc(size_t bytes, cudaStream_t st) { return dev_alloc(bytes, st); }
void device_free(void* p) { dev_free(p); }
bool is_device_pointer(const void* p) { return is_device_ptr(p); }
}  // namespace lbm

// ---------------------------------------------------------------------------------------------
// Context.

struct lbm_ctx {
  int B = 0;
  long long Ntot = 0;
  int precision = LBM_F64;
  PhysD ph{};
  cudaStream_t stream = nullptr;
  std::vector<long long> N, offset;
  std::vector<lbm_rates> rates;
  std::vector<int> bc;
  std::vector<double> s0;
  std::vector<LatDev> host_lat;     // tile0 of table k (k = 0..3 for depth 1, 2, 4, 8) lives in
  std::vector<LatDev> host_tabs;    //   host_tabs[k * B .. k * B + B - 1]
  LatDev* d_lat = nullptr;          // 4 * B records on the device, same layout
  long long ntiles_k[4] = {0, 0, 0, 0};
  int* d_tile_lat = nullptr;        // per depth k: lattice of each tile, at d_tile_lat + k * max_tiles
  long long max_tiles = 0;
  void* state[2] = {nullptr, nullptr};
  int cur = 0;
  bool has_state = false;
  long long ntiles = 0;
  int K = 1, NT = 512, V = 1;
  long long nchunks = 0;
  double* d_part = nullptr;
  int* d_pflag = nullptr;
  double* d_sums = nullptr;
  int* d_flags = nullptr;
  double* d_stage = nullptr;
  size_t stage_bytes = 0;
  long long steps_done = 0;
  std::string err;
  // Persistent execution (lbm_set_mode).
  int mode = LBM_MODE_LAUNCH;
  int* d_done = nullptr;
  unsigned long long* d_counter = nullptr;
  int* d_status = nullptr;
  long long spin_limit = 20000000;  // about 2 s of polling per wait
  long long withhold = -1;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  long long graph_key[6] = {-1, -1, -1, -1, -1, -1};
  // Adjoint (lbm_adjoint_forward / lbm_adjoint_backward).
  long long adj_T = -1, adj_seg = 0, adj_nseg = 0;
  std::vector<void*> ckpt, stash;
  void* adj_a[2] = {nullptr, nullptr};
  int adj_K = 4;                    // reverse steps per adjoint launch (lbm_adjoint_set_config)
  LatDev* d_lat_adj = nullptr;      // per depth K = 1 .. kAdjointMaxK: B records with the adjoint tiling
  long long adj_ntiles[lbm::kAdjointMaxK] = {};
  double* d_gtile[lbm::kAdjointMaxK] = {};
  double* d_rgrad = nullptr;
  double* d_lpart = nullptr;
  double* d_loss = nullptr;

  bool f64() const { return precision != LBM_F32_SHIFTED; }  // FP64 storage (LBM_F64, LBM_F64_DF)
  size_t elem() const { return f64() ? sizeof(double) : sizeof(float); }
  size_t state_bytes() const { return 6 * (size_t)Ntot * elem(); }
};

namespace {

// NVTX range for the duration of a C-ABI call (visible in Nsight timelines; no cost without a tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int fail(lbm_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LBM_CK(ctx, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

InitArgs init_args(const lbm_ctx* c) {
  InitArgs a;
  a.rho0 = c->ph.rho0;
  a.p0 = c->ph.p0;
  a.gamma = c->ph.gamma;
  a.cp = c->ph.cp;
  a.lam = c->ph.lam;
  a.e_r = c->ph.e_r();
  a.cp_log = (1.0 - 1.0 / c->ph.gamma) * c->ph.cp;
  a.wf0 = c->ph.wf0();
  a.wf1 = c->ph.wf1();
  a.eq_mode = c->ph.eq_mode;
  a.u0_lin = c->ph.u0_lin;
  a.s0_lin = c->ph.s0_lin;
  a.a1 = c->ph.lin_a1();
  a.b1 = c->ph.lin_b1();
  a.c02 = c->ph.c02();
  a.inv_rho0 = 1.0 / c->ph.rho0;
  a.inv_p0 = 1.0 / c->ph.p0;
  a.inv_cp = 1.0 / c->ph.cp;
  a.cp_over_gamma = c->ph.cp / c->ph.gamma;
  const double af = c->ph.rho0, ag = c->ph.rho0 * c->ph.cp, l = c->ph.lam;
  a.inv_af[0] = 1.0 / af;
  a.inv_af[1] = 1.0 / (af * l);
  a.inv_af[2] = 1.0 / (af * l * l);
  a.inv_ag[0] = 1.0 / ag;
  a.inv_ag[1] = 1.0 / (ag * l);
  a.inv_ag[2] = 1.0 / (ag * l * l);
  return a;
}

inline int depth_index(int K) { return K == 1 ? 0 : K == 2 ? 1 : K == 4 ? 2 : 3; }

// For tile width NT and each depth K in {1, 2, 4, 8}: index of each lattice's first tile (tiles of
// NT - 4K output nodes); diagnostics chunk starts likewise (independent of the tiling).
void rebuild_tables(lbm_ctx* c) {
  c->host_tabs.resize(4 * (size_t)c->B);
  long long ch = 0;
  for (int b = 0; b < c->B; ++b) {
    c->host_lat[b].chunk0 = ch;
    ch += (c->N[b] + kChunk - 1) / kChunk;
  }
  c->nchunks = ch;
  for (int ki = 0; ki < 4; ++ki) {
    const long long bout = lbm::tile_span(c->NT, c->V, c->precision == LBM_F32_SHIFTED) - 4 * (1 << ki);
    long long t = 0;
    for (int b = 0; b < c->B; ++b) {
      LatDev d = c->host_lat[b];
      d.tile0 = t;
      c->host_tabs[ki * (size_t)c->B + b] = d;
      t += bout > 0 ? (c->N[b] + bout - 1) / bout : 0;
    }
    c->ntiles_k[ki] = bout > 0 ? t : 0;
  }
  c->ntiles = c->ntiles_k[depth_index(c->K)];
}

int upload_lat(lbm_ctx* c) {
  LBM_CK(c, cudaMemcpyAsync(c->d_lat, c->host_tabs.data(), sizeof(LatDev) * 4 * c->B, cudaMemcpyHostToDevice,
                            c->stream));
  if (c->d_tile_lat)
    for (int ki = 0; ki < 4; ++ki) {
      if (c->ntiles_k[ki] > c->max_tiles) return fail(c, LBM_ERR_INVALID_ARG, "tile table overflow");
      LBM_CK(c, lbm::launch_tile_map(c->d_lat + ki * (size_t)c->B, c->B, c->ntiles_k[ki],
                                     c->d_tile_lat + ki * c->max_tiles, c->stream));
    }
  LBM_CK(c, cudaStreamSynchronize(c->stream));  // host_tabs may change again before the copy runs
  return LBM_OK;
}

inline const int* tile_map_for(const lbm_ctx* c, int K);

// Device tables for depth K.
inline const LatDev* lat_for(const lbm_ctx* c, int K) { return c->d_lat + depth_index(K) * (size_t)c->B; }
inline const int* tile_map_for(const lbm_ctx* c, int K) { return c->d_tile_lat + depth_index(K) * c->max_tiles; }

int ensure_stage(lbm_ctx* c, size_t bytes) {
  if (c->stage_bytes >= bytes) return LBM_OK;
  dev_free(c->d_stage);
  c->d_stage = (double*)dev_alloc(bytes, c->stream);
  c->stage_bytes = c->d_stage ? bytes : 0;
  if (!c->d_stage) return fail(c, LBM_ERR_OOM, "staging buffer allocation failed");
  return LBM_OK;
}

bool valid_rate(double s) { return s > 0.0 && s < 2.0; }

int do_create(lbm_ctx** out, int B, const int64_t* N, double lambda, const lbm_rates* rates, const int32_t* bc,
              const double* s0, int precision, const lbm_phys* phys, void* stream) {
  if (!out) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  if (B < 1 || !N || !rates || !bc || !(lambda > 0.0) || !std::isfinite(lambda)) return LBM_ERR_INVALID_ARG;
  if (precision != LBM_F64 && precision != LBM_F32_SHIFTED && precision != LBM_F64_DF) return LBM_ERR_INVALID_ARG;
  PhysD ph;
  ph.lam = lambda;
  ph.gamma = phys ? phys->gamma : 1.4;
  ph.Pr = phys ? phys->Pr : 1.0;
  ph.cp = phys ? phys->cp : 1.0;
  ph.rho0 = phys ? phys->rho0 : 1.0;
  ph.s0 = phys ? phys->s0 : 0.0;
  ph.source_on = phys ? (phys->source_on != 0) : 1;
  ph.eq_mode = phys ? phys->equilibria : 0;
  ph.u0_lin = phys ? phys->u0_lin : 0.0;
  ph.s0_lin = phys ? phys->s0_lin : 0.0;
  const double c0 = lambda / 2.0;
  ph.p0 = (phys && phys->p0 > 0.0) ? phys->p0 : ph.rho0 * c0 * c0 / ph.gamma;
  if (!(ph.gamma > 1.0) || !(ph.Pr > 0.0) || !(ph.cp > 0.0) || !(ph.rho0 > 0.0) || !(ph.p0 > 0.0))
    return LBM_ERR_INVALID_ARG;
  if (ph.eq_mode != 0 && ph.eq_mode != 1) return LBM_ERR_INVALID_ARG;
  // The printed linear equilibria hold in lattice units lambda = c_p = 1, without the source.
  if (ph.eq_mode == 1 && (lambda != 1.0 || ph.cp != 1.0 || ph.source_on)) return LBM_ERR_INVALID_ARG;

  lbm_ctx* c = new lbm_ctx();
  c->B = B;
  c->precision = precision;
  c->ph = ph;
  c->stream = (cudaStream_t)stream;
  c->N.resize(B);
  c->offset.resize(B + 1);
  c->rates.resize(B);
  c->bc.resize(B);
  c->s0.resize(B);
  c->host_lat.resize(B);
  long long tot = 0;
  for (int b = 0; b < B; ++b) {
    if (N[b] < 3 || (bc[b] != LBM_BC_PERIODIC && bc[b] != LBM_BC_BOUNCEBACK)) { delete c; return LBM_ERR_INVALID_ARG; }
    lbm_rates r = rates[b];
    if (!valid_rate(r.s_e)) { delete c; return LBM_ERR_INVALID_ARG; }
    const double sigma_e = 1.0 / r.s_e - 0.5;
    if (!(r.s_psi > 0.0)) r.s_psi = 1.0 / (1.5 * (ph.gamma / ph.Pr) * sigma_e + 0.5);  // eq. lien-sigma-sigma
    if (!(r.s_eps > 0.0)) r.s_eps = 1.5;
    if (!valid_rate(r.s_psi) || !valid_rate(r.s_eps)) { delete c; return LBM_ERR_INVALID_ARG; }
    c->N[b] = N[b];
    c->offset[b] = tot;
    c->rates[b] = r;
    c->bc[b] = bc[b];
    c->s0[b] = s0 ? s0[b] : ph.s0;
    LatDev& d = c->host_lat[b];
    d.offset = tot;
    d.n = N[b];
    d.s_e = r.s_e;
    d.s_psi = r.s_psi;
    d.s_eps = r.s_eps;
    d.q_src = 0.25 * sigma_e;
    d.s0 = c->s0[b];
    d.zeta_r = ph.rho0 * d.s0;
    d.eps_r = ph.e_r() * d.s0;
    // Rest g populations M_g^{-1}(zeta_r, 0, eps_r).
    {
      const double r0 = d.zeta_r / (ph.rho0 * ph.cp), q0 = d.eps_r / (ph.rho0 * ph.cp * lambda * lambda);
      d.wg0 = (r0 - q0) / 3.0;
      d.wg1 = (2.0 * r0 + q0) / 6.0;
    }
    d.s0h = c->s0[b] / ph.cp;
    {
      // Constant terms of the linear equilibria in scaled shifted moments (lambda = c_p = 1):
      // x_eq = x0 + xR r + xJ j + xZ z with rho/rho0 = 1 + r, J/rho0 = j, zeta/rho0 = z + s0/c_p.
      const double u0 = ph.u0_lin, s0l = ph.s0_lin, sh = d.s0h, er = ph.e_r() / (ph.rho0 * lambda * lambda);
      d.lin_e0 = ph.lin_a1() + 3.0 * u0 * u0 * sh - er;
      d.lin_p0 = -u0 * s0l + u0 * sh;
      d.lin_q0 = ph.lin_b1() + 3.0 * (u0 * u0 + s0l * ph.c02()) * sh - er * sh;
    }
    d.bc = bc[b];
    d.pad = 0;
    {
      const double v[8] = {d.s_e, d.s_psi, d.s_eps, d.q_src, d.s0h, d.lin_e0, d.lin_p0, d.lin_q0};
      for (int i = 0; i < 8; ++i) {
        d.f32[i] = (float)v[i];  // round to nearest, as the device conversion
        d.f32lo[i] = (float)(v[i] - (double)d.f32[i]);
      }
    }
    tot += N[b];
  }
  c->offset[B] = tot;
  c->Ntot = tot;
  const bool f32 = precision == LBM_F32_SHIFTED;
  c->K = precision == LBM_F64 ? 1 : 4;
  c->adj_K = precision == LBM_F64 ? 1 : 4;  // measured fastest (FP64 is bound by its arithmetic)
  c->NT = precision == LBM_F64 ? 512 : 256;
  c->V = f32 ? 2 : 1;
  rebuild_tables(c);

  c->d_lat = (LatDev*)dev_alloc(sizeof(LatDev) * 4 * B, c->stream);
  c->state[0] = dev_alloc(c->state_bytes(), c->stream);
  c->state[1] = dev_alloc(c->state_bytes(), c->stream);
  c->d_sums = (double*)dev_alloc(sizeof(double) * 4 * B, c->stream);
  c->d_flags = (int*)dev_alloc(sizeof(int) * B, c->stream);
  c->d_part = (double*)dev_alloc(sizeof(double) * 4 * c->nchunks, c->stream);
  c->d_pflag = (int*)dev_alloc(sizeof(int) * c->nchunks, c->stream);
  {
    long long max_tiles = 0;  // narrowest tiles: 128 threads x 1 node, depth 8
    for (int b = 0; b < B; ++b) max_tiles += (c->N[b] + (128 - 32) - 1) / (128 - 32);
    c->max_tiles = max_tiles;
    c->d_done = (int*)dev_alloc(sizeof(int) * max_tiles, c->stream);
    c->d_tile_lat = (int*)dev_alloc(sizeof(int) * 4 * max_tiles, c->stream);
  }
  c->d_counter = (unsigned long long*)dev_alloc(sizeof(unsigned long long), c->stream);
  c->d_status = (int*)dev_alloc(sizeof(int), c->stream);
  if (!c->d_lat || !c->state[0] || !c->state[1] || !c->d_sums || !c->d_flags || !c->d_part || !c->d_pflag ||
      !c->d_done || !c->d_counter || !c->d_status || !c->d_tile_lat) {
    lbm_destroy(c);
    return LBM_ERR_OOM;
  }
  if (upload_lat(c) != LBM_OK || cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream) != cudaSuccess) {
    lbm_destroy(c);
    return LBM_ERR_CUDA;
  }
  *out = c;
  return LBM_OK;
}

template <typename R>
cudaError_t enqueue_persistent(lbm_ctx* c, long long nblocks, cudaStream_t st, const lbm::ConstSet<R>& k) {
  const int ki = depth_index(c->K);
  cudaError_t e = cudaMemsetAsync(c->d_done, 0, sizeof(int) * ((c->ntiles_k[ki] + lbm::kUnitTiles - 1) / lbm::kUnitTiles), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  lbm::PersistentCtl ctl{c->d_counter, c->d_done, c->d_status, c->spin_limit, c->withhold};
  return lbm::launch_persistent<R>((R*)c->state[c->cur], (R*)c->state[1 - c->cur], c->Ntot, lat_for(c, c->K),
                                   tile_map_for(c, c->K), c->B, c->ntiles_k[ki], c->K, c->NT, c->V, nblocks, ctl, k,
                                   st);
}

// Persistent launch of nblocks blocks of K steps, directly or through a cached CUDA graph.
template <typename R>
int run_persistent(lbm_ctx* c, long long nblocks, const lbm::ConstSet<R>& k) {
  if (c->mode == LBM_MODE_PERSISTENT) {
    cudaError_t e = enqueue_persistent<R>(c, nblocks, c->stream, k);
    if (e != cudaSuccess) return cuda_fail(c, e, "persistent launch");
  } else {
    const long long key[6] = {nblocks, c->cur, c->K, c->NT, c->V, c->spin_limit ^ (c->withhold << 40)};
    if (!c->graph || std::memcmp(key, c->graph_key, sizeof(key)) != 0) {
      if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
      if (!c->cap_stream) LBM_CK(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      LBM_CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = enqueue_persistent<R>(c, nblocks, c->cap_stream, k);
      cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
      if (e != cudaSuccess) return cuda_fail(c, e, "persistent capture");
      if (e2 != cudaSuccess) return cuda_fail(c, e2, "end capture");
      e = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { c->graph = nullptr; return cuda_fail(c, e, "graph instantiate"); }
      std::memcpy(c->graph_key, key, sizeof(key));
    }
    LBM_CK(c, cudaGraphLaunch(c->graph, c->stream));
  }
  if (nblocks & 1) c->cur = 1 - c->cur;
  c->steps_done += nblocks * c->K;
  return LBM_OK;
}

template <typename R>
int run_steps(lbm_ctx* c, long long nsteps) {
  const lbm::ConstSet<R> k = make_constset<R>(c->ph);
  long long left = nsteps;
  if (c->mode != LBM_MODE_LAUNCH && left >= c->K) {
    const long long nblocks = left / c->K;
    int rc = run_persistent<R>(c, nblocks, k);
    if (rc != LBM_OK) return rc;
    left -= nblocks * c->K;
  }
  while (left > 0) {
    int K = c->K;
    while (K > left) K >>= 1;  // the remainder runs with shallower launches (same arithmetic)
    const int ki = depth_index(K);
    cudaError_t e = lbm::launch_step_tiles<R>((const R*)c->state[c->cur], (R*)c->state[1 - c->cur], c->Ntot,
                                              lat_for(c, K), tile_map_for(c, K), c->B, c->ntiles_k[ki], K, c->NT,
                                              c->V, k, c->stream, 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
    c->cur = 1 - c->cur;
    left -= K;
    c->steps_done += K;
  }
  return LBM_OK;
}

// Double-float arithmetic on FP64 storage (LBM_F64_DF): one launch per K steps.
int run_steps_df(lbm_ctx* c, long long nsteps) {
  const Consts<lbm::df> k = make_consts<lbm::df>(c->ph);
  long long left = nsteps;
  while (left > 0) {
    int K = c->K;
    while (K > left) K >>= 1;
    const int ki = depth_index(K);
    cudaError_t e = lbm::launch_step_tiles_df((const double*)c->state[c->cur], (double*)c->state[1 - c->cur], c->Ntot,
                                              lat_for(c, K), tile_map_for(c, K), c->B, c->ntiles_k[ki], K, c->NT,
                                              c->V, k, c->stream, 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "double-float step kernel launch");
    c->cur = 1 - c->cur;
    left -= K;
    c->steps_done += K;
  }
  return LBM_OK;
}

bool valid_config(const lbm_ctx* c, int K, int NT, int V) {
  if (c->precision == LBM_F64_DF) return lbm::valid_df_config(K, NT, V);
  return lbm::valid_tile_config(K, NT, V, c->precision == LBM_F64);
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int set_state_impl(lbm_ctx* c, const double* rho, const double* u, const double* x, int from_p) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!rho || !u || !x) return fail(c, LBM_ERR_INVALID_ARG, "set_state: null array");
  const long long n = c->Ntot;
  const double *dr = rho, *du = u, *dx = x;
  const bool host = !is_device_ptr(rho);
  if (host != !is_device_ptr(u) || host != !is_device_ptr(x))
    return fail(c, LBM_ERR_INVALID_ARG, "set_state: mix of host and device arrays");
  const void *mr = host ? mapped_host_ptr(rho) : nullptr, *mu = host ? mapped_host_ptr(u) : nullptr;
  const void* mx = host ? mapped_host_ptr(x) : nullptr;
  if (host && mr && mu && mx) {
    // Pinned host arrays: the initialisation kernel reads them in place (no staging copy).
    dr = (const double*)mr;
    du = (const double*)mu;
    dx = (const double*)mx;
  } else if (host) {
    int rc = ensure_stage(c, 3 * sizeof(double) * n);
    if (rc) return rc;
    LBM_CK(c, cudaMemcpyAsync(c->d_stage, rho, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    LBM_CK(c, cudaMemcpyAsync(c->d_stage + n, u, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    LBM_CK(c, cudaMemcpyAsync(c->d_stage + 2 * n, x, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    dr = c->d_stage;
    du = c->d_stage + n;
    dx = c->d_stage + 2 * n;
  }
  const InitArgs a = init_args(c);
  if (c->f64())
    init_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>(dr, du, dx, from_p, (double*)c->state[c->cur], n,
                                                                    c->d_lat, c->B, a);
  else
    init_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>(dr, du, dx, from_p, (float*)c->state[c->cur], n,
                                                                   c->d_lat, c->B, a);
  LBM_CK(c, cudaGetLastError());
  if (host) LBM_CK(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  c->steps_done = 0;
  return LBM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Exported entry points.

extern "C" {

int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return LBM_ERR_INVALID_ARG;
  g_alloc = alloc;
  g_free = free_fn;
  g_user = user;
  return LBM_OK;
}

int lbm_create(lbm_ctx** out, int64_t N, double lambda, const lbm_rates* rates, int32_t bc, int32_t precision,
               const lbm_phys* phys, void* stream) {
  return do_create(out, 1, &N, lambda, rates, &bc, nullptr, precision, phys, stream);
}

int lbm_create_batch(lbm_ctx** out, int32_t B, const int64_t* N, double lambda, const lbm_rates* rates,
                     const int32_t* bc, const double* s0, int32_t precision, const lbm_phys* phys, void* stream) {
  return do_create(out, B, N, lambda, rates, bc, s0, precision, phys, stream);
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  dev_free(c->d_lat);
  dev_free(c->state[0]);
  dev_free(c->state[1]);
  dev_free(c->d_sums);
  dev_free(c->d_flags);
  dev_free(c->d_part);
  dev_free(c->d_pflag);
  dev_free(c->d_stage);
  dev_free(c->d_done);
  dev_free(c->d_tile_lat);
  dev_free(c->d_counter);
  dev_free(c->d_status);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  lbm_adjoint_release(c);
  dev_free(c->d_lat_adj);
  for (double* g : c->d_gtile) dev_free(g);
  dev_free(c->d_rgrad);
  dev_free(c->d_lpart);
  dev_free(c->d_loss);
  delete c;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : "null context"; }
int64_t lbm_total_nodes(const lbm_ctx* c) { return c ? c->Ntot : -1; }
int64_t lbm_steps_done(const lbm_ctx* c) { return c ? c->steps_done : -1; }

int lbm_set_state(lbm_ctx* c, const double* rho, const double* u, const double* p) {
  return set_state_impl(c, rho, u, p, 1);
}

int lbm_set_state_entropy(lbm_ctx* c, const double* rho, const double* u, const double* s) {
  return set_state_impl(c, rho, u, s, 0);
}

int lbm_step(lbm_ctx* c, int64_t nsteps) {
  NvtxRange r("lbm_step");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (nsteps < 0) return fail(c, LBM_ERR_INVALID_ARG, "step: nsteps < 0");
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "step: no state set");
  if (c->precision == LBM_F64_DF) return run_steps_df(c, nsteps);
  return c->precision == LBM_F64 ? run_steps<double>(c, nsteps) : run_steps<float>(c, nsteps);
}

int lbm_moments(lbm_ctx* c, double* rho, double* J, double* zeta, double* e, double* psi, double* eps) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "moments: no state set");
  double* outs[6] = {rho, J, zeta, e, psi, eps};
  int host = -1;
  for (double* p : outs) {
    if (!p) continue;
    const int h = is_device_ptr(p) ? 0 : 1;
    if (host >= 0 && h != host) return fail(c, LBM_ERR_INVALID_ARG, "moments: mix of host and device arrays");
    host = h;
  }
  if (host < 0) return LBM_OK;
  const long long n = c->Ntot;
  double* dst[6];
  bool in_place = false;  // pinned host outputs: the kernel writes them directly
  if (host) {
    in_place = true;
    for (int i = 0; i < 6; ++i) {
      dst[i] = outs[i] ? (double*)mapped_host_ptr(outs[i]) : nullptr;
      if (outs[i] && !dst[i]) in_place = false;
    }
  }
  if (host && !in_place) {
    int cnt = 0;
    for (double* p : outs) cnt += p != nullptr;
    int rc = ensure_stage(c, sizeof(double) * n * cnt);
    if (rc) return rc;
    int k = 0;
    for (int i = 0; i < 6; ++i) dst[i] = outs[i] ? c->d_stage + (k++) * n : nullptr;
  } else if (!host) {
    for (int i = 0; i < 6; ++i) dst[i] = outs[i];
  }
  const InitArgs a = init_args(c);
  if (c->f64())
    moments_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>((const double*)c->state[c->cur], n, c->d_lat, c->B,
                                                                       a, dst[0], dst[1], dst[2], dst[3], dst[4], dst[5]);
  else
    moments_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>((const float*)c->state[c->cur], n, c->d_lat, c->B,
                                                                      a, dst[0], dst[1], dst[2], dst[3], dst[4], dst[5]);
  LBM_CK(c, cudaGetLastError());
  if (host) {
    if (!in_place)
      for (int i = 0; i < 6; ++i)
        if (outs[i]) LBM_CK(c, cudaMemcpyAsync(outs[i], dst[i], sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

int lbm_get_populations(lbm_ctx* c, double* fd) {
  if (!c || !fd) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "populations: no state set");
  const long long n = c->Ntot;
  const bool host = !is_device_ptr(fd);
  double* dst = fd;
  if (host) {
    int rc = ensure_stage(c, 6 * sizeof(double) * n);
    if (rc) return rc;
    dst = c->d_stage;
  }
  const double wf0 = c->ph.wf0(), wf1 = c->ph.wf1();
  if (c->f64())
    pops_out_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>((const double*)c->state[c->cur], n, c->d_lat,
                                                                        c->B, wf0, wf1, dst);
  else
    pops_out_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>((const float*)c->state[c->cur], n, c->d_lat, c->B,
                                                                       wf0, wf1, dst);
  LBM_CK(c, cudaGetLastError());
  if (host) {
    LBM_CK(c, cudaMemcpyAsync(fd, dst, 6 * sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const double* fd) {
  if (!c || !fd) return LBM_ERR_INVALID_ARG;
  const long long n = c->Ntot;
  const bool host = !is_device_ptr(fd);
  const double* src = fd;
  if (host) {
    int rc = ensure_stage(c, 6 * sizeof(double) * n);
    if (rc) return rc;
    LBM_CK(c, cudaMemcpyAsync(c->d_stage, fd, 6 * sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    src = c->d_stage;
  }
  const double wf0 = c->ph.wf0(), wf1 = c->ph.wf1();
  if (c->f64())
    pops_in_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>((double*)c->state[c->cur], n, c->d_lat, c->B, wf0,
                                                                       wf1, src);
  else
    pops_in_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>((float*)c->state[c->cur], n, c->d_lat, c->B, wf0,
                                                                      wf1, src);
  LBM_CK(c, cudaGetLastError());
  if (host) LBM_CK(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  c->steps_done = 0;
  return LBM_OK;
}

int lbm_diagnostics(lbm_ctx* c, double* sums, int32_t* flags) {
  NvtxRange r("lbm_diagnostics");
  if (!c || !sums || !flags) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "diagnostics: no state set");
  const InitArgs a = init_args(c);
  const double inv_r = 1.0 / c->ph.r();
  if (c->nchunks > 0) {
    if (c->f64())
      diag_chunk_kernel<double><<<(unsigned)c->nchunks, kDiagThreads, 0, c->stream>>>(
          (const double*)c->state[c->cur], c->Ntot, c->d_lat, c->B, a, c->ph.gamma, inv_r, c->d_part, c->d_pflag);
    else
      diag_chunk_kernel<float><<<(unsigned)c->nchunks, kDiagThreads, 0, c->stream>>>(
          (const float*)c->state[c->cur], c->Ntot, c->d_lat, c->B, a, c->ph.gamma, inv_r, c->d_part, c->d_pflag);
    LBM_CK(c, cudaGetLastError());
  }
  diag_final_kernel<<<c->B, 256, 0, c->stream>>>(c->d_part, c->d_pflag, c->d_lat, c->B, c->nchunks, c->d_sums,
                                                   c->d_flags);
  LBM_CK(c, cudaGetLastError());
  LBM_CK(c, cudaMemcpyAsync(sums, c->d_sums, sizeof(double) * 4 * c->B, cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaMemcpyAsync(flags, c->d_flags, sizeof(int) * c->B, cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  for (int b = 0; b < c->B; ++b)
    if (flags[b]) return fail(c, LBM_ERR_UNSTABLE, "diagnostics: lattice " + std::to_string(b) + " flagged (flags=" +
                                                       std::to_string(flags[b]) + ")");
  return LBM_OK;
}

int lbm_set_config(lbm_ctx* c, int32_t k, int32_t nt, int32_t v) {
  if (!c) return LBM_ERR_INVALID_ARG;
  const int newK = k ? k : c->K, newNT = nt ? nt : c->NT, newV = v ? v : c->V;
  if (!valid_config(c, newK, newNT, newV))
    return fail(c, LBM_ERR_INVALID_ARG, "config: unsupported (steps_per_launch, block_threads, nodes_per_thread)");
  c->K = newK;
  c->NT = newNT;
  c->V = newV;
  rebuild_tables(c);
  return upload_lat(c);
}

int lbm_get_config(const lbm_ctx* c, int32_t* k, int32_t* nt, int32_t* v) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (k) *k = c->K;
  if (nt) *nt = c->NT;
  if (v) *v = c->V;
  return LBM_OK;
}

int lbm_autotune(lbm_ctx* c, int32_t trials) {
  NvtxRange r("lbm_autotune");
  if (!c || trials < 1) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "autotune: no state set");
  cudaEvent_t e0, e1;
  LBM_CK(c, cudaEventCreate(&e0));
  LBM_CK(c, cudaEventCreate(&e1));
  const int Ks[4] = {1, 2, 4, 8};
  const int NTs[6] = {32, 64, 128, 256, 512, 1024};
  const int Vs[3] = {1, 2, 4};
  double best = 1e300;
  int bestK = c->K, bestNT = c->NT, bestV = c->V;
  const long long kTrialTiles = 65536;  // 30 M nodes at 128 x 4: about 50 waves, the rest is skipped
  for (int nt : NTs)
    for (int v : Vs)
      for (int k : Ks) {
        if (!valid_config(c, k, nt, v)) continue;
        c->K = k;
        c->NT = nt;
        c->V = v;
        rebuild_tables(c);
        int rc = upload_lat(c);
        if (rc) return rc;
        const long long nt_run = std::min(c->ntiles, kTrialTiles);
        const double nodes = (double)nt_run * (lbm::tile_span(nt, v, c->precision == LBM_F32_SHIFTED) - 4 * k);
        float ms = 0.f;
        for (int t = 0; t <= trials; ++t) {  // the first launch is a warm-up
          if (t == 1) LBM_CK(c, cudaEventRecord(e0, c->stream));
          cudaError_t e;
          if (c->precision == LBM_F64_DF)
            e = lbm::launch_step_tiles_df((const double*)c->state[c->cur], (double*)c->state[1 - c->cur], c->Ntot,
                                          lat_for(c, k), tile_map_for(c, k), c->B, nt_run, k, nt, v,
                                          make_consts<lbm::df>(c->ph), c->stream, 0);
          else if (c->f64())
            e = lbm::launch_step_tiles<double>((const double*)c->state[c->cur], (double*)c->state[1 - c->cur],
                                               c->Ntot, lat_for(c, k), tile_map_for(c, k), c->B, nt_run, k, nt, v,
                                               make_constset<double>(c->ph), c->stream, 0);
          else
            e = lbm::launch_step_tiles<float>((const float*)c->state[c->cur], (float*)c->state[1 - c->cur],
                                              c->Ntot, lat_for(c, k), tile_map_for(c, k), c->B, nt_run, k, nt, v,
                                              make_constset<float>(c->ph), c->stream, 0);
          if (e != cudaSuccess) return cuda_fail(c, e, "autotune launch");
        }
        LBM_CK(c, cudaEventRecord(e1, c->stream));
        LBM_CK(c, cudaEventSynchronize(e1));
        LBM_CK(c, cudaEventElapsedTime(&ms, e0, e1));
        const double per_node_step = ms / (trials * k * nodes);
        if (per_node_step < best) { best = per_node_step; bestK = k; bestNT = nt; bestV = v; }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->K = bestK;
  c->NT = bestNT;
  c->V = bestV;
  rebuild_tables(c);
  return upload_lat(c);
}

int lbm_set_mode(lbm_ctx* c, int32_t mode) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (mode != LBM_MODE_LAUNCH && mode != LBM_MODE_PERSISTENT && mode != LBM_MODE_PERSISTENT_GRAPH)
    return fail(c, LBM_ERR_INVALID_ARG, "set_mode: unknown mode");
  if (mode != LBM_MODE_LAUNCH && c->precision == LBM_F64_DF)
    return fail(c, LBM_ERR_INVALID_ARG, "set_mode: double-float contexts run one launch per block");
  c->mode = mode;
  return LBM_OK;
}

int lbm_status(lbm_ctx* c) {
  if (!c) return LBM_ERR_INVALID_ARG;
  int st = 0;
  LBM_CK(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  if (st != 0) {
    LBM_CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return fail(c, LBM_ERR_TIMEOUT, "a bounded wait of the persistent kernel expired; the state is not valid");
  }
  return LBM_OK;
}

int lbm_debug_bounds(int64_t* violations, int64_t* first_index, int64_t* first_extent) {
  if (!violations || !first_index || !first_extent) return LBM_ERR_INVALID_ARG;
#ifdef LBM_DEBUG_BOUNDS
  if (cudaDeviceSynchronize() != cudaSuccess) return LBM_ERR_CUDA;
  unsigned long long rec[5][3];
  if (lbm::bounds_record_step(rec[0]) != cudaSuccess || lbm::bounds_record_df(rec[1]) != cudaSuccess ||
      lbm::bounds_record_adjoint(rec[2]) != cudaSuccess || lbm::bounds_record_2d(rec[3]) != cudaSuccess ||
      lbm::bounds_record_3d(rec[4]) != cudaSuccess)
    return LBM_ERR_CUDA;
  *violations = 0;
  *first_index = *first_extent = -1;
  for (auto& r : rec) {
    if (r[0] && *violations == 0) {
      *first_index = (int64_t)r[1];
      *first_extent = (int64_t)r[2];
    }
    *violations += (int64_t)r[0];
  }
#else
  *violations = -1;  // this build has no bounds checks
  *first_index = *first_extent = -1;
#endif
  return LBM_OK;
}

int lbm_debug_persistent(lbm_ctx* c, int64_t spin_limit, int64_t withhold_tile) {
  if (!c || spin_limit < 1) return LBM_ERR_INVALID_ARG;
  c->spin_limit = spin_limit;
  c->withhold = withhold_tile < 0 ? -1 : withhold_tile;
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Adjoint with sqrt(T) checkpointing.

namespace {

int adjoint_setup(lbm_ctx* c) {
  if (c->d_lat_adj) return LBM_OK;
  // Tile tables of the adjoint for every depth K (tiles store adjoint_tile_out(K) nodes).
  std::vector<LatDev> tab((size_t)lbm::kAdjointMaxK * c->B);
  for (int K = 1; K <= lbm::kAdjointMaxK; ++K) {
    const long long bout = lbm::adjoint_tile_out(K);
    long long t = 0;
    for (int b = 0; b < c->B; ++b) {
      LatDev d = c->host_lat[b];
      d.tile0 = t;
      tab[(size_t)(K - 1) * c->B + b] = d;
      t += (c->N[b] + bout - 1) / bout;
    }
    c->adj_ntiles[K - 1] = t;
    if (!c->d_gtile[K - 1]) c->d_gtile[K - 1] = (double*)dev_alloc(sizeof(double) * 2 * t, c->stream);
    if (!c->d_gtile[K - 1]) return fail(c, LBM_ERR_OOM, "adjoint: allocation failed");
  }
  if (!c->d_rgrad) c->d_rgrad = (double*)dev_alloc(sizeof(double) * 2 * c->B, c->stream);
  if (!c->d_lpart) c->d_lpart = (double*)dev_alloc(sizeof(double) * ((c->Ntot + 255) / 256), c->stream);
  if (!c->d_loss) c->d_loss = (double*)dev_alloc(sizeof(double), c->stream);
  c->d_lat_adj = (LatDev*)dev_alloc(sizeof(LatDev) * tab.size(), c->stream);
  if (!c->d_lat_adj || !c->d_rgrad || !c->d_lpart || !c->d_loss) return fail(c, LBM_ERR_OOM, "adjoint: allocation failed");
  LBM_CK(c, cudaMemcpyAsync(c->d_lat_adj, tab.data(), sizeof(LatDev) * tab.size(), cudaMemcpyHostToDevice, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

template <typename R>
int adjoint_forward_impl(lbm_ctx* c, long long T) {
  int rc = adjoint_setup(c);
  if (rc) return rc;
  lbm_adjoint_release(c);
  long long seg = (long long)std::llround(std::sqrt((double)T));
  if (seg < 1) seg = 1;
  const long long nseg = (T + seg - 1) / seg > 0 ? (T + seg - 1) / seg : 1;
  const size_t sb = c->state_bytes();
  for (long long j = 0; j < nseg; ++j) {
    void* p = dev_alloc(sb, c->stream);
    if (!p) { lbm_adjoint_release(c); return fail(c, LBM_ERR_OOM, "adjoint: checkpoint allocation failed"); }
    c->ckpt.push_back(p);
  }
  for (long long j = 0; j + 1 < seg; ++j) {
    void* p = dev_alloc(sb, c->stream);
    if (!p) { lbm_adjoint_release(c); return fail(c, LBM_ERR_OOM, "adjoint: stash allocation failed"); }
    c->stash.push_back(p);
  }
  for (int k = 0; k < 2; ++k) {
    c->adj_a[k] = dev_alloc(sb, c->stream);
    if (!c->adj_a[k]) { lbm_adjoint_release(c); return fail(c, LBM_ERR_OOM, "adjoint: buffer allocation failed"); }
  }
  const int save_mode = c->mode;
  c->mode = LBM_MODE_LAUNCH;
  for (long long j = 0; j < nseg; ++j) {
    LBM_CK(c, cudaMemcpyAsync(c->ckpt[j], c->state[c->cur], sb, cudaMemcpyDeviceToDevice, c->stream));
    const long long len = std::min(seg, T - j * seg);
    rc = c->precision == LBM_F64_DF ? run_steps_df(c, len) : run_steps<R>(c, len);
    if (rc) { c->mode = save_mode; return rc; }
  }
  c->mode = save_mode;
  c->adj_T = T;
  c->adj_seg = seg;
  c->adj_nseg = nseg;
  return LBM_OK;
}

// Reverse sweep from the seed already in adj_a[0]; leaves dL/df(0) in adj_a[res]. Each segment of
// sqrt(T) steps is split into blocks of adj_K steps: the states at the block starts are recomputed
// from the segment's checkpoint with adj_K-step launches of the step kernel, then every block runs its
// reverse steps in one launch (which recomputes the block's inner states on chip).
template <typename R>
int adjoint_reverse(lbm_ctx* c, int* res) {
  const lbm::ConstSet<R> k = make_constset<R>(c->ph);
  const Consts<lbm::df> kdf = make_consts<lbm::df>(c->ph);
  const int KA = c->adj_K;
  for (int K = 1; K <= lbm::kAdjointMaxK; ++K)
    LBM_CK(c, cudaMemsetAsync(c->d_gtile[K - 1], 0, sizeof(double) * 2 * c->adj_ntiles[K - 1], c->stream));
  int a = 0;
  for (long long j = c->adj_nseg - 1; j >= 0; --j) {
    const long long len = std::min(c->adj_seg, c->adj_T - j * c->adj_seg);
    const long long nb = (len + KA - 1) / KA;
    std::vector<const R*> st(nb);
    st[0] = (const R*)c->ckpt[j];
    for (long long b = 1; b < nb; ++b) {
      cudaError_t e;
      if constexpr (std::is_same<R, double>::value) {
        if (c->precision == LBM_F64_DF) {
          e = lbm::launch_step_tiles_df(st[b - 1], (double*)c->stash[b - 1], c->Ntot, lat_for(c, KA),
                                        tile_map_for(c, KA), c->B, c->ntiles_k[depth_index(KA)], KA, c->NT, c->V,
                                        kdf, c->stream, 0);
          if (e != cudaSuccess) return cuda_fail(c, e, "adjoint recompute");
          st[b] = (const R*)c->stash[b - 1];
          continue;
        }
      }
      e = lbm::launch_step_tiles<R>(st[b - 1], (R*)c->stash[b - 1], c->Ntot, lat_for(c, KA),
                                    tile_map_for(c, KA), c->B, c->ntiles_k[depth_index(KA)], KA, c->NT,
                                    c->V, k, c->stream, 0);
      if (e != cudaSuccess) return cuda_fail(c, e, "adjoint recompute");
      st[b] = (const R*)c->stash[b - 1];
    }
    for (long long b = nb - 1; b >= 0; --b) {
      const int Kb = (int)std::min<long long>(KA, len - b * KA);
      const LatDev* tab = c->d_lat_adj + (size_t)(Kb - 1) * c->B;
      cudaError_t e;
      if constexpr (std::is_same<R, double>::value) {
        if (c->precision == LBM_F64_DF)
          e = lbm::launch_adjoint_block_df(st[b], (const double*)c->adj_a[a], (double*)c->adj_a[1 - a], c->Ntot, tab,
                                           c->B, c->adj_ntiles[Kb - 1], Kb, kdf, c->d_gtile[Kb - 1], c->stream);
        else
          e = lbm::launch_adjoint_block<R>(st[b], (const R*)c->adj_a[a], (R*)c->adj_a[1 - a], c->Ntot, tab, c->B,
                                           c->adj_ntiles[Kb - 1], Kb, k, c->d_gtile[Kb - 1], c->stream);
      } else {
        e = lbm::launch_adjoint_block<R>(st[b], (const R*)c->adj_a[a], (R*)c->adj_a[1 - a], c->Ntot, tab, c->B,
                                         c->adj_ntiles[Kb - 1], Kb, k, c->d_gtile[Kb - 1], c->stream);
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "adjoint step");
      a = 1 - a;
    }
  }
  *res = a;
  return LBM_OK;
}

template <typename R>
int adjoint_backward_impl(lbm_ctx* c, const double* target, const double* rho_b, double* loss, double* drho0,
                          double* du0, double* drates, double* dfd0) {
  if (c->adj_T < 0) return fail(c, LBM_ERR_INVALID_ARG, "adjoint: no forward run recorded");
  const long long n = c->Ntot;
  // Inputs: stage a host target / seed on the device.
  const double* in = target ? target : rho_b;
  const bool host_in = !is_device_ptr(in);
  int rc = ensure_stage(c, sizeof(double) * n * 9);
  if (rc) return rc;
  const double* d_in = in;
  if (host_in) {
    LBM_CK(c, cudaMemcpyAsync(c->d_stage, in, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    d_in = c->d_stage;
  }
  cudaError_t e = lbm::launch_misfit_seed<R>((const R*)c->state[c->cur], target ? d_in : nullptr,
                                             target ? nullptr : d_in, n, c->ph.rho0, (R*)c->adj_a[0], c->d_lpart,
                                             c->d_loss, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint seed");
  int a = 0;
  rc = adjoint_reverse<R>(c, &a);
  if (rc) return rc;
  double* d_drho = c->d_stage + n;
  double* d_du = c->d_stage + 2 * n;
  e = lbm::launch_adjoint_init<R>((const R*)c->ckpt[0], (const R*)c->adj_a[a], n, c->d_lat, c->B,
                                  make_consts<double>(c->ph), d_drho, d_du, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint init");
  for (int K = 1; K <= lbm::kAdjointMaxK && e == cudaSuccess; ++K)  // fixed order over the depths
    e = lbm::launch_reduce_rate_grads(c->d_gtile[K - 1], c->d_lat_adj + (size_t)(K - 1) * c->B, c->B,
                                      c->adj_ntiles[K - 1], c->d_rgrad, K > 1, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint rate reduction");
  if (dfd0) {
    // dL/df(0) as float64 (the population shift is a constant and does not change the gradient).
    double* dst = is_device_ptr(dfd0) ? dfd0 : c->d_stage + 3 * n;
    e = lbm::launch_to_f64<R>((const R*)c->adj_a[a], dst, 6 * n, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint output");
    if (dst != dfd0) LBM_CK(c, cudaMemcpyAsync(dfd0, dst, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, c->stream));
  }
  if (drho0) LBM_CK(c, cudaMemcpyAsync(drho0, d_drho, sizeof(double) * n, cudaMemcpyDefault, c->stream));
  if (du0) LBM_CK(c, cudaMemcpyAsync(du0, d_du, sizeof(double) * n, cudaMemcpyDefault, c->stream));
  if (drates) LBM_CK(c, cudaMemcpyAsync(drates, c->d_rgrad, sizeof(double) * 2 * c->B, cudaMemcpyDefault, c->stream));
  if (loss && target) LBM_CK(c, cudaMemcpyAsync(loss, c->d_loss, sizeof(double), cudaMemcpyDefault, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_adjoint_forward(lbm_ctx* c, int64_t T) {
  NvtxRange r("lbm_adjoint_forward");
  if (!c || T < 1) return LBM_ERR_INVALID_ARG;
  if (c->ph.eq_mode != 0) return fail(c, LBM_ERR_INVALID_ARG, "adjoint: only the nonlinear equilibria are differentiated");
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "adjoint: no state set");
  return c->f64() ? adjoint_forward_impl<double>(c, T) : adjoint_forward_impl<float>(c, T);
}

int lbm_adjoint_backward(lbm_ctx* c, const double* dL_drho_T, double* dL_drho0, double* dL_du0, double* dL_drates,
                         double* dL_dfd0) {
  NvtxRange r("lbm_adjoint_backward");
  if (!c || !dL_drho_T) return LBM_ERR_INVALID_ARG;
  return c->f64()
             ? adjoint_backward_impl<double>(c, nullptr, dL_drho_T, nullptr, dL_drho0, dL_du0, dL_drates, dL_dfd0)
             : adjoint_backward_impl<float>(c, nullptr, dL_drho_T, nullptr, dL_drho0, dL_du0, dL_drates, dL_dfd0);
}

int lbm_adjoint(lbm_ctx* c, int64_t T, const double* rho_target, double* loss, double* dL_drho0, double* dL_du0,
                double* dL_drates) {
  if (!c || !rho_target || T < 1) return LBM_ERR_INVALID_ARG;
  int rc = lbm_adjoint_forward(c, T);
  if (rc) return rc;
  return c->f64()
             ? adjoint_backward_impl<double>(c, rho_target, nullptr, loss, dL_drho0, dL_du0, dL_drates, nullptr)
             : adjoint_backward_impl<float>(c, rho_target, nullptr, loss, dL_drho0, dL_du0, dL_drates, nullptr);
}

int lbm_adjoint_release(lbm_ctx* c) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!c->ckpt.empty() || !c->stash.empty() || c->adj_a[0] || c->adj_a[1]) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
  }
  for (void* p : c->ckpt) dev_free(p);
  for (void* p : c->stash) dev_free(p);
  c->ckpt.clear();
  c->stash.clear();
  for (int k = 0; k < 2; ++k) { dev_free(c->adj_a[k]); c->adj_a[k] = nullptr; }
  c->adj_T = -1;
  return LBM_OK;
}

int lbm_adjoint_set_config(lbm_ctx* c, int32_t steps_per_launch) {
  if (!c) return LBM_ERR_INVALID_ARG;
  const int K = steps_per_launch > 0 ? steps_per_launch : (c->precision == LBM_F64 ? 1 : 4);
  if (K != 1 && K != 2 && K != 4 && K != 8)
    return fail(c, LBM_ERR_INVALID_ARG, "adjoint_set_config: steps_per_launch must be 1, 2, 4 or 8");
  c->adj_K = K;
  return LBM_OK;
}

int lbm_adjoint_get_config(const lbm_ctx* c, int32_t* steps_per_launch) {
  if (!c || !steps_per_launch) return LBM_ERR_INVALID_ARG;
  *steps_per_launch = c->adj_K;
  return LBM_OK;
}

// Checkpoint format: magic, version, precision, B, the physical constants, per-lattice
// (N, rates, bc, s0), the step counter, then the raw state bytes (shifted populations, plane-major).
static const char kMagic[8] = {'L', 'B', 'M', 'D', '1', 'Q', '3', '3'};

int lbm_save(lbm_ctx* c, const char* path) {
  if (!c || !path) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "save: no state set");
  std::vector<char> buf(c->state_bytes());
  LBM_CK(c, cudaMemcpyAsync(buf.data(), c->state[c->cur], buf.size(), cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(c, LBM_ERR_IO, std::string("save: cannot open ") + path);
  const int32_t ver = 1, prec = c->precision, B = c->B;
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&ver, 4, 1, f) == 1 && std::fwrite(&prec, 4, 1, f) == 1 &&
            std::fwrite(&B, 4, 1, f) == 1 && std::fwrite(&c->ph, sizeof(PhysD), 1, f) == 1;
  for (int b = 0; ok && b < c->B; ++b) {
    const int64_t n = c->N[b];
    const int32_t bcv = c->bc[b];
    ok = std::fwrite(&n, 8, 1, f) == 1 && std::fwrite(&c->rates[b], sizeof(lbm_rates), 1, f) == 1 &&
         std::fwrite(&bcv, 4, 1, f) == 1 && std::fwrite(&c->s0[b], 8, 1, f) == 1;
  }
  const int64_t steps = c->steps_done;
  ok = ok && std::fwrite(&steps, 8, 1, f) == 1 && std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? LBM_OK : fail(c, LBM_ERR_IO, "save: write failed");
}

int lbm_load(lbm_ctx* c, const char* path) {
  if (!c || !path) return LBM_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(c, LBM_ERR_IO, std::string("load: cannot open ") + path);
  char magic[8];
  int32_t ver = 0, prec = -1, B = 0;
  PhysD ph;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 && std::fread(&ver, 4, 1, f) == 1 &&
            ver == 1 && std::fread(&prec, 4, 1, f) == 1 && prec == c->precision && std::fread(&B, 4, 1, f) == 1 &&
            B == c->B && std::fread(&ph, sizeof(PhysD), 1, f) == 1 && std::memcmp(&ph, &c->ph, sizeof(PhysD)) == 0;
  for (int b = 0; ok && b < c->B; ++b) {
    int64_t n;
    lbm_rates r;
    int32_t bcv;
    double s0;
    ok = std::fread(&n, 8, 1, f) == 1 && n == c->N[b] && std::fread(&r, sizeof(lbm_rates), 1, f) == 1 &&
         std::memcmp(&r, &c->rates[b], sizeof(lbm_rates)) == 0 && std::fread(&bcv, 4, 1, f) == 1 && bcv == c->bc[b] &&
         std::fread(&s0, 8, 1, f) == 1 && s0 == c->s0[b];
  }
  int64_t steps = 0;
  std::vector<char> buf(c->state_bytes());
  ok = ok && std::fread(&steps, 8, 1, f) == 1 && std::fread(buf.data(), 1, buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) return fail(c, LBM_ERR_IO, "load: file does not match this context");
  LBM_CK(c, cudaMemcpyAsync(c->state[c->cur], buf.data(), buf.size(), cudaMemcpyHostToDevice, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  c->steps_done = steps;
  return LBM_OK;
}

}  // extern "C"
