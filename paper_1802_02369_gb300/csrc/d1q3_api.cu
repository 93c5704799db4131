// C-ABI of the single-distribution D1Q3 schemes of sections 2 and 4 (lbm_d1q3_* in include/lbm.h):
// parameter derivation (the identification of kappa and s_psi of section 4), equilibrium
// initialisation, moment and population read-back, deterministic FP64 sums and the autotuner. The
// step kernel is in d1q3_step.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <type_traits>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "d1q3_internal.cuh"
#include "lbm_internal.cuh"

namespace {

constexpr int kSumChunk = 1024;  // nodes per reduction block
constexpr int kSumThreads = 256;

// Parameters after defaults, in FP64.
struct D1q3P {
  int scheme;
  double lam, scale;
  double s1, s2;       // fluid: s_e; advection-diffusion: s_psi, s_eps
  double gamma, p0;    // fluid
  double u0, alpha;    // advection-diffusion
  __host__ __device__ double kp() const { return p0 / (scale * lam * lam); }
  // Dimensionless rest-state populations (those of rho0, J = 0 or zeta0) per unit of scale:
  // f_r = M^{-1} m_r / scale with r = 1, j = j_r, q = q_r.
  __host__ __device__ double jr() const { return scheme == 0 ? 0.0 : u0 / lam; }
  __host__ __device__ double qr() const { return scheme == 0 ? 3.0 * p0 / (scale * lam * lam) - 2.0 : alpha; }
};

// Equilibrium shifted populations from (m0, m1) per node (FP64), rounded once to R.
template <typename R>
__global__ void d1q3_init_kernel(const double* __restrict__ m0, const double* __restrict__ m1, R* __restrict__ f,
                                 long long N, D1q3P p) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double r = m0[i] / p.scale - 1.0;
  double j, q;
  if (p.scheme == 0) {
    j = m1[i] / (p.scale * p.lam);
    q = 3.0 * (j * j / (1.0 + r) + p.kp() * expm1(p.gamma * log1p(r))) - 2.0 * r;
  } else {
    j = (p.u0 / p.lam) * r;
    q = p.alpha * r;
  }
  f[i] = R((r - q) / 3.0);
  f[N + i] = R((2.0 * r + q) / 6.0 + 0.5 * j);
  f[2 * N + i] = R((2.0 * r + q) / 6.0 - 0.5 * j);
}

// Absolute moments (m0, m1, m2) = M f per node; any output may be null.
template <typename R>
__global__ void d1q3_moments_kernel(const R* __restrict__ f, long long N, D1q3P p, double* m0, double* m1,
                                    double* m2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double a = (double)f[i], b = (double)f[N + i], c = (double)f[2 * N + i];
  const double s = p.scale, l = p.lam;
  if (m0) m0[i] = s * (1.0 + a + b + c);
  if (m1) m1[i] = s * l * (p.jr() + b - c);
  if (m2) m2[i] = s * l * l * (p.qr() + b + c - 2.0 * a);
}

// Absolute populations (scale removed: f = M^{-1} m with the scale of M) out / in, plane-major.
template <typename R>
__global__ void d1q3_pops_kernel(R* __restrict__ f, long long N, D1q3P p, double* __restrict__ out,
                                 const double* __restrict__ in) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double w0 = (1.0 - p.qr()) / 3.0, wp = (2.0 + p.qr()) / 6.0 + 0.5 * p.jr(), wm = (2.0 + p.qr()) / 6.0 - 0.5 * p.jr();
  const double w[3] = {w0, wp, wm};
  for (int k = 0; k < 3; ++k) {
    if (out) out[k * N + i] = (double)f[k * N + i] + w[k];
    if (in) f[k * N + i] = R(in[k * N + i] - w[k]);
  }
}

// Sums, pass 1: per block of kSumChunk nodes, fixed-order sums of m0, m1, m2 and the flag bits
// (bit 0 a non-finite population, bit 1 m0 <= 0 for the fluid scheme).
template <typename R>
__global__ void __launch_bounds__(kSumThreads) d1q3_sum_chunk_kernel(const R* __restrict__ f, long long N, D1q3P p,
                                                                     double* __restrict__ part, int* __restrict__ pflag) {
  const long long base = (long long)blockIdx.x * kSumChunk;
  double acc[3] = {0, 0, 0};
  int fl = 0;
  const double s = p.scale, l = p.lam;
  for (int t = 0; t < kSumChunk / kSumThreads; ++t) {
    const long long i = base + t * kSumThreads + threadIdx.x;
    if (i >= N) break;
    const double a = (double)f[i], b = (double)f[N + i], c = (double)f[2 * N + i];
    if (!isfinite(a) || !isfinite(b) || !isfinite(c)) fl |= 1;
    const double m0 = s * (1.0 + a + b + c);
    if (p.scheme == 0 && !(m0 > 0.0)) fl |= 2;
    acc[0] += m0;
    acc[1] += s * l * (p.jr() + b - c);
    acc[2] += s * l * l * (p.qr() + b + c - 2.0 * a);
  }
  __shared__ double sh[3][kSumThreads / 32];
  __shared__ int shf[kSumThreads / 32];
  for (int k = 0; k < 3; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = v;
  }
  int f2 = fl;
  for (int o = 16; o > 0; o >>= 1) f2 |= __shfl_down_sync(0xffffffffu, f2, o);
  if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = f2;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) {
      double v = 0.0;
      for (int q = 0; q < kSumThreads / 32; ++q) v += sh[k][q];
      part[blockIdx.x * 3LL + k] = v;
    }
    int ff = 0;
    for (int q = 0; q < kSumThreads / 32; ++q) ff |= shf[q];
    pflag[blockIdx.x] = ff;
  }
}

// Sums, pass 2: one block adds the partials in a fixed order.
__global__ void __launch_bounds__(256) d1q3_sum_final_kernel(const double* __restrict__ part,
                                                             const int* __restrict__ pflag, long long nchunks,
                                                             double* __restrict__ sums, int* __restrict__ flags) {
  double acc[3] = {0, 0, 0};
  int fl = 0;
  for (long long q = threadIdx.x; q < nchunks; q += blockDim.x) {
    for (int k = 0; k < 3; ++k) acc[k] += part[q * 3 + k];
    fl |= pflag[q];
  }
  __shared__ double sh[3][8];
  __shared__ int shf[8];
  for (int k = 0; k < 3; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = v;
  }
  int f2 = fl;
  for (int o = 16; o > 0; o >>= 1) f2 |= __shfl_down_sync(0xffffffffu, f2, o);
  if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = f2;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) {
      double v = 0.0;
      for (int q = 0; q < 8; ++q) v += sh[k][q];
      sums[k] = v;
    }
    int ff = 0;
    for (int q = 0; q < 8; ++q) ff |= shf[q];
    flags[0] = ff;
  }
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename X>
X lift(double v) {
  if constexpr (sizeof(X) == 8 && !std::is_same<X, double>::value) return make_float2((float)v, (float)v);
  else return X(v);
}

template <typename X>
lbm::D1q3Consts<X> make_consts(const D1q3P& p) {
  lbm::D1q3Consts<X> c;
  c.one = lift<X>(1.0);
  c.two = lift<X>(2.0);
  c.three = lift<X>(3.0);
  c.half = lift<X>(0.5);
  c.m_half = lift<X>(-0.5);
  c.third = lift<X>(1.0 / 3.0);
  c.sixth = lift<X>(1.0 / 6.0);
  c.m_two = lift<X>(-2.0);
  c.s1 = lift<X>(p.s1);
  c.s2 = lift<X>(p.s2);
  c.kp = lift<X>(p.kp());
  c.gamma = lift<X>(p.gamma);
  c.ul = lift<X>(p.u0 / p.lam);
  c.alpha = lift<X>(p.alpha);
  return c;
}

template <typename R>
lbm::D1q3ConstSet<R> make_set(const D1q3P& p);
template <>
lbm::D1q3ConstSet<double> make_set<double>(const D1q3P& p) {
  lbm::D1q3ConstSet<double> k;
  k.s = make_consts<double>(p);
  return k;
}
template <>
lbm::D1q3ConstSet<float> make_set<float>(const D1q3P& p) {
  lbm::D1q3ConstSet<float> k;
  k.s = make_consts<float>(p);
  k.p = make_consts<float2>(p);
  return k;
}

}  // namespace

struct lbm_d1q3_ctx {
  long long N = 0;
  int precision = LBM_F64;
  D1q3P p{};
  cudaStream_t stream = nullptr;
  void* state[2] = {nullptr, nullptr};
  int cur = 0;
  bool has_state = false;
  int K = 8, NT = 256, V = 4;
  long long steps_done = 0;
  long long nchunks = 0;
  double* d_part = nullptr;
  int* d_pflag = nullptr;
  double* d_sums = nullptr;
  int* d_flags = nullptr;
  double* d_stage = nullptr;
  std::string err;
  size_t elem() const { return precision == LBM_F64 ? sizeof(double) : sizeof(float); }
};

namespace {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int fail(lbm_d1q3_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define D1Q3_CK(ctx, call)                                                                                   \
  do {                                                                                                       \
    cudaError_t e_ = (call);                                                                                 \
    if (e_ != cudaSuccess) return fail(ctx, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int ensure_stage(lbm_d1q3_ctx* c) {
  if (c->d_stage) return LBM_OK;
  c->d_stage = (double*)lbm::device_alloc(3 * sizeof(double) * c->N, c->stream);
  if (!c->d_stage) return fail(c, LBM_ERR_OOM, "staging buffer allocation failed");
  return LBM_OK;
}

template <typename R>
int run_d1q3(lbm_d1q3_ctx* c, long long nsteps) {
  const lbm::D1q3ConstSet<R> k = make_set<R>(c->p);
  long long left = nsteps;
  while (left > 0) {
    const int K = left < c->K ? (int)left : c->K;
    cudaError_t e = lbm::launch_d1q3_step<R>((const R*)c->state[c->cur], (R*)c->state[1 - c->cur], c->N, c->p.scheme,
                                             K, c->NT, c->V, k, c->stream);
    if (e != cudaSuccess) return fail(c, LBM_ERR_CUDA, std::string("d1q3 step launch: ") + cudaGetErrorString(e));
    c->cur = 1 - c->cur;
    left -= K;
    c->steps_done += K;
  }
  return LBM_OK;
}

bool in_open_02(double s) { return s > 0.0 && s < 2.0 && std::isfinite(s); }

// Defaults and the identification of section 4: ((2 + alpha)/3 lambda^2 - u0^2)(1/s_psi - 1/2) dt = kappa
// with dt = dx / lambda and dx = 1.
int derive(const lbm_d1q3_params* in, D1q3P& p) {
  if (!in) return LBM_ERR_INVALID_ARG;
  p.scheme = in->scheme;
  p.lam = in->lambda;
  p.scale = in->scale > 0.0 ? in->scale : 1.0;
  if (!(p.lam > 0.0) || !std::isfinite(p.lam) || !std::isfinite(p.scale)) return LBM_ERR_INVALID_ARG;
  p.gamma = p.p0 = p.u0 = p.alpha = 0.0;
  if (p.scheme == LBM_D1Q3_FLUID) {
    p.s1 = in->s_e;
    p.s2 = 0.0;
    p.gamma = in->gamma > 0.0 ? in->gamma : 1.4;
    p.p0 = in->p0 > 0.0 ? in->p0 : p.scale * 0.25 * p.lam * p.lam / p.gamma;  // c0 = lambda / 2
    if (!in_open_02(p.s1) || !(p.gamma >= 1.0) || !std::isfinite(p.p0)) return LBM_ERR_INVALID_ARG;
  } else if (p.scheme == LBM_D1Q3_ADVECTION_DIFFUSION) {
    p.u0 = in->u0;
    p.alpha = in->alpha;
    p.s2 = in->s_eps > 0.0 ? in->s_eps : 1.5;
    if (in->s_psi > 0.0) {
      p.s1 = in->s_psi;
    } else {
      const double a = (2.0 + p.alpha) / 3.0 * p.lam * p.lam - p.u0 * p.u0;
      const double dt = 1.0 / p.lam;
      if (!(in->kappa > 0.0) || !(a > 0.0)) return LBM_ERR_INVALID_ARG;
      p.s1 = 1.0 / (in->kappa / (a * dt) + 0.5);
    }
    if (!in_open_02(p.s1) || !in_open_02(p.s2) || !std::isfinite(p.u0) || !std::isfinite(p.alpha))
      return LBM_ERR_INVALID_ARG;
  } else {
    return LBM_ERR_INVALID_ARG;
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_d1q3_create(lbm_d1q3_ctx** out, int64_t N, const lbm_d1q3_params* params, int32_t precision, void* stream) {
  if (!out) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  if (N < 3 || (precision != LBM_F64 && precision != LBM_F32_SHIFTED)) return LBM_ERR_INVALID_ARG;
  D1q3P p;
  if (int rc = derive(params, p)) return rc;
  lbm_d1q3_ctx* c = new lbm_d1q3_ctx();
  c->N = N;
  c->precision = precision;
  c->p = p;
  c->stream = (cudaStream_t)stream;
  c->nchunks = (N + kSumChunk - 1) / kSumChunk;
  const size_t sb = 3 * (size_t)N * c->elem();
  c->state[0] = lbm::device_alloc(sb, c->stream);
  c->state[1] = lbm::device_alloc(sb, c->stream);
  c->d_part = (double*)lbm::device_alloc(sizeof(double) * 3 * c->nchunks, c->stream);
  c->d_pflag = (int*)lbm::device_alloc(sizeof(int) * c->nchunks, c->stream);
  c->d_sums = (double*)lbm::device_alloc(sizeof(double) * 3, c->stream);
  c->d_flags = (int*)lbm::device_alloc(sizeof(int), c->stream);
  if (!c->state[0] || !c->state[1] || !c->d_part || !c->d_pflag || !c->d_sums || !c->d_flags) {
    lbm_d1q3_destroy(c);
    return LBM_ERR_OOM;
  }
  *out = c;
  return LBM_OK;
}

void lbm_d1q3_destroy(lbm_d1q3_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (void* q : {c->state[0], c->state[1], (void*)c->d_part, (void*)c->d_pflag, (void*)c->d_sums,
                  (void*)c->d_flags, (void*)c->d_stage})
    lbm::device_free(q);
  delete c;
}

const char* lbm_d1q3_last_error(const lbm_d1q3_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t lbm_d1q3_steps_done(const lbm_d1q3_ctx* c) { return c ? c->steps_done : -1; }

int lbm_d1q3_rates(const lbm_d1q3_ctx* c, double* s1, double* s2) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (s1) *s1 = c->p.s1;
  if (s2) *s2 = c->p.s2;
  return LBM_OK;
}

int lbm_d1q3_set_state(lbm_d1q3_ctx* c, const double* m0, const double* m1) {
  NvtxRange r_("lbm_d1q3_set_state");
  if (!c) return LBM_ERR_INVALID_ARG;
  const bool need_m1 = c->p.scheme == LBM_D1Q3_FLUID;
  if (!m0 || (need_m1 && !m1)) return fail(c, LBM_ERR_INVALID_ARG, "d1q3_set_state: null array");
  const bool host = !lbm::is_device_pointer(m0);
  if (need_m1 && host != !lbm::is_device_pointer(m1))
    return fail(c, LBM_ERR_INVALID_ARG, "d1q3_set_state: mix of host and device arrays");
  const long long n = c->N;
  const double *a = m0, *b = need_m1 ? m1 : m0;
  if (host) {
    if (int rc = ensure_stage(c)) return rc;
    D1Q3_CK(c, cudaMemcpyAsync(c->d_stage, m0, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    if (need_m1) D1Q3_CK(c, cudaMemcpyAsync(c->d_stage + n, m1, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    a = c->d_stage;
    b = need_m1 ? c->d_stage + n : c->d_stage;
  }
  if (c->precision == LBM_F64)
    d1q3_init_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>(a, b, (double*)c->state[c->cur], n, c->p);
  else
    d1q3_init_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>(a, b, (float*)c->state[c->cur], n, c->p);
  D1Q3_CK(c, cudaGetLastError());
  if (host) D1Q3_CK(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  c->steps_done = 0;
  return LBM_OK;
}

int lbm_d1q3_step(lbm_d1q3_ctx* c, int64_t nsteps) {
  NvtxRange r_("lbm_d1q3_step");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (nsteps < 0) return fail(c, LBM_ERR_INVALID_ARG, "d1q3_step: nsteps < 0");
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "d1q3_step: no state set");
  return c->precision == LBM_F64 ? run_d1q3<double>(c, nsteps) : run_d1q3<float>(c, nsteps);
}

int lbm_d1q3_moments(lbm_d1q3_ctx* c, double* m0, double* m1, double* m2) {
  NvtxRange r_("lbm_d1q3_moments");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "d1q3_moments: no state set");
  double* outs[3] = {m0, m1, m2};
  bool host[3] = {false, false, false};
  bool any_host = false;
  for (int k = 0; k < 3; ++k)
    if (outs[k] && !lbm::is_device_pointer(outs[k])) host[k] = any_host = true;
  if (any_host)
    if (int rc = ensure_stage(c)) return rc;
  const long long n = c->N;
  double* d[3];
  for (int k = 0; k < 3; ++k) d[k] = outs[k] ? (host[k] ? c->d_stage + k * n : outs[k]) : nullptr;
  if (c->precision == LBM_F64)
    d1q3_moments_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>((const double*)c->state[c->cur], n, c->p,
                                                                            d[0], d[1], d[2]);
  else
    d1q3_moments_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>((const float*)c->state[c->cur], n, c->p,
                                                                           d[0], d[1], d[2]);
  D1Q3_CK(c, cudaGetLastError());
  for (int k = 0; k < 3; ++k)
    if (host[k]) D1Q3_CK(c, cudaMemcpyAsync(outs[k], d[k], sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  if (any_host) D1Q3_CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

static int pops_io(lbm_d1q3_ctx* c, double* out, const double* in) {
  if (!c) return LBM_ERR_INVALID_ARG;
  const long long n = c->N;
  const double* ptr = out ? out : in;
  if (!ptr) return fail(c, LBM_ERR_INVALID_ARG, "d1q3 populations: null array");
  const bool host = !lbm::is_device_pointer(ptr);
  double* dev = out;
  const double* dev_in = in;
  if (host) {
    if (int rc = ensure_stage(c)) return rc;
    if (in) {
      D1Q3_CK(c, cudaMemcpyAsync(c->d_stage, in, 3 * sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
      dev_in = c->d_stage;
    } else {
      dev = c->d_stage;
    }
  }
  if (c->precision == LBM_F64)
    d1q3_pops_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>((double*)c->state[c->cur], n, c->p,
                                                                         in ? nullptr : dev, dev_in);
  else
    d1q3_pops_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>((float*)c->state[c->cur], n, c->p,
                                                                        in ? nullptr : dev, dev_in);
  D1Q3_CK(c, cudaGetLastError());
  if (host && out) D1Q3_CK(c, cudaMemcpyAsync(out, dev, 3 * sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  if (host) D1Q3_CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_d1q3_get_populations(lbm_d1q3_ctx* c, double* f) {
  NvtxRange r_("lbm_d1q3_get_populations");
  if (c && !c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "d1q3_get_populations: no state set");
  return pops_io(c, f, nullptr);
}

int lbm_d1q3_set_populations(lbm_d1q3_ctx* c, const double* f) {
  NvtxRange r_("lbm_d1q3_set_populations");
  const int rc = pops_io(c, nullptr, f);
  if (rc == LBM_OK) {
    c->has_state = true;
    c->steps_done = 0;
  }
  return rc;
}

int lbm_d1q3_sums(lbm_d1q3_ctx* c, double* sums, int32_t* flags) {
  NvtxRange r_("lbm_d1q3_sums");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!sums || !flags) return fail(c, LBM_ERR_INVALID_ARG, "d1q3_sums: null output");
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "d1q3_sums: no state set");
  if (c->precision == LBM_F64)
    d1q3_sum_chunk_kernel<double><<<(unsigned)c->nchunks, kSumThreads, 0, c->stream>>>(
        (const double*)c->state[c->cur], c->N, c->p, c->d_part, c->d_pflag);
  else
    d1q3_sum_chunk_kernel<float><<<(unsigned)c->nchunks, kSumThreads, 0, c->stream>>>(
        (const float*)c->state[c->cur], c->N, c->p, c->d_part, c->d_pflag);
  D1Q3_CK(c, cudaGetLastError());
  d1q3_sum_final_kernel<<<1, 256, 0, c->stream>>>(c->d_part, c->d_pflag, c->nchunks, c->d_sums, c->d_flags);
  D1Q3_CK(c, cudaGetLastError());
  D1Q3_CK(c, cudaMemcpyAsync(sums, c->d_sums, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
  D1Q3_CK(c, cudaMemcpyAsync(flags, c->d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  D1Q3_CK(c, cudaStreamSynchronize(c->stream));
  return *flags ? fail(c, LBM_ERR_UNSTABLE, "d1q3_sums: non-finite population or rho <= 0") : LBM_OK;
}

int lbm_d1q3_set_config(lbm_d1q3_ctx* c, int32_t k, int32_t nt, int32_t v) {
  if (!c) return LBM_ERR_INVALID_ARG;
  const int K = k > 0 ? k : c->K, NT = nt > 0 ? nt : c->NT, V = v > 0 ? v : c->V;
  if (!lbm::valid_d1q3_config(K, NT, V)) return fail(c, LBM_ERR_INVALID_ARG, "d1q3_set_config: unsupported configuration");
  c->K = K;
  c->NT = NT;
  c->V = V;
  return LBM_OK;
}

int lbm_d1q3_get_config(const lbm_d1q3_ctx* c, int32_t* k, int32_t* nt, int32_t* v) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (k) *k = c->K;
  if (nt) *nt = c->NT;
  if (v) *v = c->V;
  return LBM_OK;
}

int lbm_d1q3_autotune(lbm_d1q3_ctx* c, int32_t trials) {
  NvtxRange r_("lbm_d1q3_autotune");
  if (!c || trials < 1) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "d1q3_autotune: no state set");
  cudaEvent_t e0, e1;
  D1Q3_CK(c, cudaEventCreate(&e0));
  D1Q3_CK(c, cudaEventCreate(&e1));
  const int Ks[7] = {1, 2, 4, 8, 16, 32, 64};
  const int NTs[3] = {128, 256, 512};
  const int Vs[4] = {1, 2, 4, 8};
  const long long kTrialTiles = 16384;  // enough waves to be representative; the rest is skipped
  double best = 1e300;
  int bK = c->K, bNT = c->NT, bV = c->V;
  const auto kd = make_set<double>(c->p);
  const auto kf = make_set<float>(c->p);
  for (int nt : NTs)
    for (int v : Vs)
      for (int k : Ks) {
        if (!lbm::valid_d1q3_config(k, nt, v)) continue;
        const long long bout = (long long)nt * v - 2 * k;
        const long long tiles = std::min((c->N + bout - 1) / bout, kTrialTiles);
        const double nodes = std::min((double)c->N, (double)tiles * bout);
        for (int t = 0; t <= trials; ++t) {  // the first launch is a warm-up
          if (t == 1) D1Q3_CK(c, cudaEventRecord(e0, c->stream));
          cudaError_t e = c->precision == LBM_F64
              ? lbm::launch_d1q3_step<double>((const double*)c->state[c->cur], (double*)c->state[1 - c->cur], c->N,
                                              c->p.scheme, k, nt, v, kd, c->stream, kTrialTiles)
              : lbm::launch_d1q3_step<float>((const float*)c->state[c->cur], (float*)c->state[1 - c->cur], c->N,
                                             c->p.scheme, k, nt, v, kf, c->stream, kTrialTiles);
          if (e != cudaSuccess) return fail(c, LBM_ERR_CUDA, std::string("d1q3_autotune launch: ") + cudaGetErrorString(e));
        }
        D1Q3_CK(c, cudaEventRecord(e1, c->stream));
        D1Q3_CK(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        D1Q3_CK(c, cudaEventElapsedTime(&ms, e0, e1));
        const double per_node_step = ms / (trials * k * nodes);
        if (per_node_step < best) { best = per_node_step; bK = k; bNT = nt; bV = v; }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->K = bK;
  c->NT = bNT;
  c->V = bV;
  return LBM_OK;
}

}  // extern "C"
