// C-ABI of the finite-difference comparison solver of section 9 (lbm_fd_* in include/lbm.h):
// context, initial state, field read-back and deterministic FP64 diagnostics. The step kernel is in
// fd_step.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "fd_internal.cuh"
#include "lbm_internal.cuh"

namespace {

constexpr int kFdChunk = 1024;  // nodes per diagnostics block
constexpr int kFdThreads = 256;

struct FdPhysD {
  double gamma, Pr, cp, rho0, p0, s0;
  int source_on;
  __host__ __device__ double r() const { return cp * (1.0 - 1.0 / gamma); }
  __host__ __device__ double T0() const { return p0 / (rho0 * r()); }
};

// Initial state (rho - rho0, rho u, rho s - rho0 s0) from per-node rho, u, s, in FP64, rounded once.
template <typename R>
__global__ void fd_init_kernel(const double* __restrict__ rho, const double* __restrict__ u,
                               const double* __restrict__ s, R* __restrict__ w, long long N, double rho0,
                               double rho0s0) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double r = rho[i];
  w[i] = R(r - rho0);
  w[N + i] = R(r * u[i]);
  w[2 * N + i] = R(r * s[i] - rho0s0);
}

template <typename R>
__global__ void fd_fields_kernel(const R* __restrict__ w, long long N, double rho0, double rho0s0, double* rho,
                                 double* J, double* zeta) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (rho) rho[i] = rho0 + (double)w[i];
  if (J) J[i] = (double)w[N + i];
  if (zeta) zeta[i] = rho0s0 + (double)w[2 * N + i];
}

template <typename R>
__global__ void fd_raw_in_kernel(R* __restrict__ w, long long N, double rho0, double rho0s0,
                                 const double* __restrict__ W) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  w[i] = R(W[i] - rho0);
  w[N + i] = R(W[N + i]);
  w[2 * N + i] = R(W[2 * N + i] - rho0s0);
}

// Diagnostics, pass 1: per block of kFdChunk nodes, fixed-order sums of rho, J, zeta and the total
// energy p/(gamma-1) + rho u^2/2 (eq. (gaz-parfait) for p), and the flag bits.
template <typename R>
__global__ void __launch_bounds__(kFdThreads) fd_diag_chunk_kernel(const R* __restrict__ w, long long N, FdPhysD ph,
                                                                   double* __restrict__ part, int* __restrict__ pflag) {
  const long long base = (long long)blockIdx.x * kFdChunk;
  double acc[4] = {0, 0, 0, 0};
  int fl = 0;
  const double r_gas = ph.r();
  for (int t = 0; t < kFdChunk / kFdThreads; ++t) {
    const long long i = base + t * kFdThreads + threadIdx.x;
    if (i >= N) break;
    const double rt = (double)w[i], J = (double)w[N + i], zt = (double)w[2 * N + i];
    if (!isfinite(rt) || !isfinite(J) || !isfinite(zt)) fl |= 1;
    const double rho = ph.rho0 + rt, zeta = ph.rho0 * ph.s0 + zt;
    const double u = J / rho, s = zeta / rho;
    const double p = ph.p0 * pow(rho / ph.rho0, ph.gamma) * exp(ph.gamma * (s - ph.s0) / ph.cp);
    const double T = p / (rho * r_gas);
    if (!(rho > 0.0)) fl |= 2;
    if (!(T > 0.0) || !isfinite(T)) fl |= 4;
    acc[0] += rho;
    acc[1] += J;
    acc[2] += zeta;
    acc[3] += p / (ph.gamma - 1.0) + 0.5 * rho * u * u;
  }
  __shared__ double sh[4][kFdThreads / 32];
  __shared__ int shf[kFdThreads / 32];
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
      for (int q = 0; q < kFdThreads / 32; ++q) v += sh[k][q];
      part[blockIdx.x * 4LL + k] = v;
    }
    int ff = 0;
    for (int q = 0; q < kFdThreads / 32; ++q) ff |= shf[q];
    pflag[blockIdx.x] = ff;
  }
}

// Diagnostics, pass 2: one block sums the chunk partials in a fixed order.
__global__ void __launch_bounds__(256) fd_diag_final_kernel(const double* __restrict__ part,
                                                            const int* __restrict__ pflag, long long nchunks,
                                                            double* __restrict__ sums, int* __restrict__ flags) {
  double acc[4] = {0, 0, 0, 0};
  int fl = 0;
  for (long long q = threadIdx.x; q < nchunks; q += blockDim.x) {
    for (int k = 0; k < 4; ++k) acc[k] += part[q * 4 + k];
    fl |= pflag[q];
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
      for (int q = 0; q < 8; ++q) v += sh[k][q];
      sums[k] = v;
    }
    int ff = 0;
    for (int q = 0; q < 8; ++q) ff |= shf[q];
    flags[0] = ff;
  }
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct lbm_fd_ctx {
  long long N = 0;
  int precision = LBM_F64;
  FdPhysD ph{};
  double dx = 1.0, dt = 1.0, nu = 0.0;
  cudaStream_t stream = nullptr;
  void* state[2] = {nullptr, nullptr};
  int cur = 0;
  bool has_state = false;
  int K = 4, NT = 256, V = 2;
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

int fail(lbm_fd_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define FD_CK(ctx, call)                                                                         \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(ctx, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename R>
lbm::FdConsts<R> fd_consts(const lbm_fd_ctx* c) {
  const FdPhysD& p = c->ph;
  lbm::FdConsts<R> k;
  k.rho0 = R(p.rho0);
  k.inv_rho0 = R(1.0 / p.rho0);
  k.s0 = R(p.s0);
  k.rho0s0 = R(p.rho0 * p.s0);
  k.gamma = R(p.gamma);
  k.inv_cp = R(1.0 / p.cp);
  k.p0 = R(p.p0);
  k.inv_r = R(1.0 / p.r());
  k.T0 = R(p.T0());
  k.nu = R(c->nu);
  k.nu_k = R(c->nu * p.cp / p.Pr);
  k.c_adv = R(c->dt / (2.0 * c->dx));
  k.c_dif = R(c->dt / (2.0 * c->dx * c->dx));
  k.c_src = R(c->dt / (4.0 * c->dx * c->dx));
  k.source_on = p.source_on;
  return k;
}

// Host arrays are staged through a device buffer of 3N doubles (allocated on first use).
int ensure_stage(lbm_fd_ctx* c) {
  if (c->d_stage) return LBM_OK;
  c->d_stage = (double*)lbm::device_alloc(3 * sizeof(double) * c->N, c->stream);
  if (!c->d_stage) return fail(c, LBM_ERR_OOM, "staging buffer allocation failed");
  return LBM_OK;
}

template <typename R>
int run_fd(lbm_fd_ctx* c, long long nsteps) {
  const lbm::FdConsts<R> k = fd_consts<R>(c);
  long long left = nsteps;
  while (left > 0) {
    const int K = left < c->K ? (int)left : c->K;
    cudaError_t e = lbm::launch_fd_step<R>((const R*)c->state[c->cur], (R*)c->state[1 - c->cur], c->N, K, c->NT,
                                           c->V, k, c->stream);
    if (e != cudaSuccess) return fail(c, LBM_ERR_CUDA, std::string("finite-difference step launch: ") + cudaGetErrorString(e));
    c->cur = 1 - c->cur;
    left -= K;
    c->steps_done += K;
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_fd_create(lbm_fd_ctx** out, int64_t N, double dx, double dt, double nu, int32_t precision,
                  const lbm_phys* phys, void* stream) {
  if (!out) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  if (N < 3 || !(dx > 0.0) || !std::isfinite(dx) || !(dt > 0.0) || !std::isfinite(dt) || !(nu >= 0.0) ||
      !std::isfinite(nu))
    return LBM_ERR_INVALID_ARG;
  if (precision != LBM_F64 && precision != LBM_F32_SHIFTED) return LBM_ERR_INVALID_ARG;
  FdPhysD ph;
  ph.gamma = phys ? phys->gamma : 1.4;
  ph.Pr = phys ? phys->Pr : 1.0;
  ph.cp = phys ? phys->cp : 1.0;
  ph.rho0 = phys ? phys->rho0 : 1.0;
  ph.s0 = phys ? phys->s0 : 0.0;
  ph.source_on = phys ? (phys->source_on != 0) : 1;
  ph.p0 = (phys && phys->p0 > 0.0) ? phys->p0 : ph.rho0 * 0.25 / ph.gamma;  // c0 = 1/2
  if (!(ph.gamma > 1.0) || !(ph.Pr > 0.0) || !(ph.cp > 0.0) || !(ph.rho0 > 0.0) || !(ph.p0 > 0.0))
    return LBM_ERR_INVALID_ARG;
  if (phys && phys->equilibria != 0) return LBM_ERR_INVALID_ARG;  // lattice Boltzmann option only

  lbm_fd_ctx* c = new lbm_fd_ctx();
  c->N = N;
  c->precision = precision;
  c->ph = ph;
  c->dx = dx;
  c->dt = dt;
  c->nu = nu;
  c->stream = (cudaStream_t)stream;
  c->nchunks = (N + kFdChunk - 1) / kFdChunk;
  const size_t sb = 3 * (size_t)N * c->elem();
  c->state[0] = lbm::device_alloc(sb, c->stream);
  c->state[1] = lbm::device_alloc(sb, c->stream);
  c->d_part = (double*)lbm::device_alloc(sizeof(double) * 4 * c->nchunks, c->stream);
  c->d_pflag = (int*)lbm::device_alloc(sizeof(int) * c->nchunks, c->stream);
  c->d_sums = (double*)lbm::device_alloc(sizeof(double) * 4, c->stream);
  c->d_flags = (int*)lbm::device_alloc(sizeof(int), c->stream);
  if (!c->state[0] || !c->state[1] || !c->d_part || !c->d_pflag || !c->d_sums || !c->d_flags) {
    lbm_fd_destroy(c);
    return LBM_ERR_OOM;
  }
  *out = c;
  return LBM_OK;
}

void lbm_fd_destroy(lbm_fd_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  lbm::device_free(c->state[0]);
  lbm::device_free(c->state[1]);
  lbm::device_free(c->d_part);
  lbm::device_free(c->d_pflag);
  lbm::device_free(c->d_sums);
  lbm::device_free(c->d_flags);
  lbm::device_free(c->d_stage);
  delete c;
}

const char* lbm_fd_last_error(const lbm_fd_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t lbm_fd_steps_done(const lbm_fd_ctx* c) { return c ? c->steps_done : -1; }

int lbm_fd_set_state(lbm_fd_ctx* c, const double* rho, const double* u, const double* s) {
  NvtxRange r_("lbm_fd_set_state");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!rho || !u || !s) return fail(c, LBM_ERR_INVALID_ARG, "fd_set_state: null array");
  const bool host = !lbm::is_device_pointer(rho);
  if (host != !lbm::is_device_pointer(u) || host != !lbm::is_device_pointer(s))
    return fail(c, LBM_ERR_INVALID_ARG, "fd_set_state: mix of host and device arrays");
  const long long n = c->N;
  const double *dr = rho, *du = u, *ds = s;
  if (host) {
    if (int rc = ensure_stage(c)) return rc;
    FD_CK(c, cudaMemcpyAsync(c->d_stage, rho, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    FD_CK(c, cudaMemcpyAsync(c->d_stage + n, u, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    FD_CK(c, cudaMemcpyAsync(c->d_stage + 2 * n, s, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    dr = c->d_stage;
    du = c->d_stage + n;
    ds = c->d_stage + 2 * n;
  }
  const double rho0s0 = c->ph.rho0 * c->ph.s0;
  if (c->precision == LBM_F64)
    fd_init_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>(dr, du, ds, (double*)c->state[c->cur], n,
                                                                       c->ph.rho0, rho0s0);
  else
    fd_init_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>(dr, du, ds, (float*)c->state[c->cur], n,
                                                                      c->ph.rho0, rho0s0);
  FD_CK(c, cudaGetLastError());
  if (host) FD_CK(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  c->steps_done = 0;
  return LBM_OK;
}

int lbm_fd_set_fields(lbm_fd_ctx* c, const double* W) {
  NvtxRange r_("lbm_fd_set_fields");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!W) return fail(c, LBM_ERR_INVALID_ARG, "fd_set_fields: null array");
  const long long n = c->N;
  const double* dW = W;
  const bool host = !lbm::is_device_pointer(W);
  if (host) {
    if (int rc = ensure_stage(c)) return rc;
    FD_CK(c, cudaMemcpyAsync(c->d_stage, W, 3 * sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    dW = c->d_stage;
  }
  const double rho0s0 = c->ph.rho0 * c->ph.s0;
  if (c->precision == LBM_F64)
    fd_raw_in_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>((double*)c->state[c->cur], n, c->ph.rho0,
                                                                         rho0s0, dW);
  else
    fd_raw_in_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>((float*)c->state[c->cur], n, c->ph.rho0,
                                                                        rho0s0, dW);
  FD_CK(c, cudaGetLastError());
  if (host) FD_CK(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  c->steps_done = 0;
  return LBM_OK;
}

int lbm_fd_step(lbm_fd_ctx* c, int64_t nsteps) {
  NvtxRange r_("lbm_fd_step");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (nsteps < 0) return fail(c, LBM_ERR_INVALID_ARG, "fd_step: nsteps < 0");
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "fd_step: no state set");
  return c->precision == LBM_F64 ? run_fd<double>(c, nsteps) : run_fd<float>(c, nsteps);
}

int lbm_fd_fields(lbm_fd_ctx* c, double* rho, double* J, double* zeta) {
  NvtxRange r_("lbm_fd_fields");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "fd_fields: no state set");
  double* outs[3] = {rho, J, zeta};
  bool host[3] = {false, false, false};
  bool any_host = false;
  for (int k = 0; k < 3; ++k)
    if (outs[k] && !lbm::is_device_pointer(outs[k])) host[k] = any_host = true;
  if (any_host)
    if (int rc = ensure_stage(c)) return rc;
  const long long n = c->N;
  double* d[3];
  for (int k = 0; k < 3; ++k) d[k] = outs[k] ? (host[k] ? c->d_stage + k * n : outs[k]) : nullptr;
  const double rho0s0 = c->ph.rho0 * c->ph.s0;
  if (c->precision == LBM_F64)
    fd_fields_kernel<double><<<blocks_for(n, 256), 256, 0, c->stream>>>((const double*)c->state[c->cur], n,
                                                                         c->ph.rho0, rho0s0, d[0], d[1], d[2]);
  else
    fd_fields_kernel<float><<<blocks_for(n, 256), 256, 0, c->stream>>>((const float*)c->state[c->cur], n,
                                                                        c->ph.rho0, rho0s0, d[0], d[1], d[2]);
  FD_CK(c, cudaGetLastError());
  for (int k = 0; k < 3; ++k)
    if (host[k])
      FD_CK(c, cudaMemcpyAsync(outs[k], d[k], sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  if (any_host) FD_CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_fd_diagnostics(lbm_fd_ctx* c, double* sums, int32_t* flags) {
  NvtxRange r_("lbm_fd_diagnostics");
  if (!c) return LBM_ERR_INVALID_ARG;
  if (!sums || !flags) return fail(c, LBM_ERR_INVALID_ARG, "fd_diagnostics: null output");
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "fd_diagnostics: no state set");
  if (c->precision == LBM_F64)
    fd_diag_chunk_kernel<double><<<(unsigned)c->nchunks, kFdThreads, 0, c->stream>>>(
        (const double*)c->state[c->cur], c->N, c->ph, c->d_part, c->d_pflag);
  else
    fd_diag_chunk_kernel<float><<<(unsigned)c->nchunks, kFdThreads, 0, c->stream>>>(
        (const float*)c->state[c->cur], c->N, c->ph, c->d_part, c->d_pflag);
  FD_CK(c, cudaGetLastError());
  fd_diag_final_kernel<<<1, 256, 0, c->stream>>>(c->d_part, c->d_pflag, c->nchunks, c->d_sums, c->d_flags);
  FD_CK(c, cudaGetLastError());
  FD_CK(c, cudaMemcpyAsync(sums, c->d_sums, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream));
  FD_CK(c, cudaMemcpyAsync(flags, c->d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  FD_CK(c, cudaStreamSynchronize(c->stream));
  return *flags ? fail(c, LBM_ERR_UNSTABLE, "fd_diagnostics: non-finite value, rho <= 0 or T <= 0") : LBM_OK;
}

int lbm_fd_set_config(lbm_fd_ctx* c, int32_t k, int32_t nt, int32_t v) {
  if (!c) return LBM_ERR_INVALID_ARG;
  const int K = k > 0 ? k : c->K, NT = nt > 0 ? nt : c->NT, V = v > 0 ? v : c->V;
  if (!lbm::valid_fd_config(K, NT, V)) return fail(c, LBM_ERR_INVALID_ARG, "fd_set_config: unsupported configuration");
  c->K = K;
  c->NT = NT;
  c->V = V;
  return LBM_OK;
}

int lbm_fd_autotune(lbm_fd_ctx* c, int32_t trials) {
  NvtxRange r_("lbm_fd_autotune");
  if (!c || trials < 1) return LBM_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, LBM_ERR_INVALID_ARG, "fd_autotune: no state set");
  cudaEvent_t e0, e1;
  FD_CK(c, cudaEventCreate(&e0));
  FD_CK(c, cudaEventCreate(&e1));
  const int Ks[5] = {1, 2, 4, 8, 16};
  const int NTs[3] = {128, 256, 512};
  const int Vs[3] = {1, 2, 4};
  const long long kTrialTiles = 16384;  // enough waves to be representative; the rest is skipped
  double best = 1e300;
  int bK = c->K, bNT = c->NT, bV = c->V;
  for (int nt : NTs)
    for (int v : Vs)
      for (int k : Ks) {
        if (!lbm::valid_fd_config(k, nt, v)) continue;
        const long long bout = (long long)nt * v - 2 * k;
        const long long tiles = std::min((c->N + bout - 1) / bout, kTrialTiles);
        const double nodes = (double)std::min((double)c->N, (double)tiles * bout);
        for (int t = 0; t <= trials; ++t) {  // the first launch is a warm-up
          if (t == 1) FD_CK(c, cudaEventRecord(e0, c->stream));
          cudaError_t e = c->precision == LBM_F64
              ? lbm::launch_fd_step<double>((const double*)c->state[c->cur], (double*)c->state[1 - c->cur], c->N, k,
                                            nt, v, fd_consts<double>(c), c->stream, kTrialTiles)
              : lbm::launch_fd_step<float>((const float*)c->state[c->cur], (float*)c->state[1 - c->cur], c->N, k, nt,
                                           v, fd_consts<float>(c), c->stream, kTrialTiles);
          if (e != cudaSuccess) return fail(c, LBM_ERR_CUDA, std::string("fd_autotune launch: ") + cudaGetErrorString(e));
        }
        FD_CK(c, cudaEventRecord(e1, c->stream));
        FD_CK(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        FD_CK(c, cudaEventElapsedTime(&ms, e0, e1));
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

int lbm_fd_get_config(const lbm_fd_ctx* c, int32_t* k, int32_t* nt, int32_t* v) {
  if (!c) return LBM_ERR_INVALID_ARG;
  if (k) *k = c->K;
  if (nt) *nt = c->NT;
  if (v) *v = c->V;
  return LBM_OK;
}

}  // extern "C"
