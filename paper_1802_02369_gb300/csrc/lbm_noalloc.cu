// Diagnostics entry point that allocates no device memory (lbm_diagnostics_noalloc).
//
// Some callers cannot allocate device memory at all: code running inside a host callback or
// under another framework's memory pool that must not be bypassed, a process that has handed
// all device memory to its own allocator, or a caller on a fixed memory budget. For them this
// entry point computes the same per-lattice FP64 sums as lbm_diagnostics on populations the
// caller already holds, and keeps its reduction scratch in a file-scope __device__ array
// instead of calling cudaMalloc.
//
// Every GPU that loads the library holds this array (about 300 KB) until the process exits.
// All calls share it, so calls whose kernels overlap on the GPU race; one call at a time per
// device (e.g. all calls on one stream) is safe. Each call overwrites every scratch slot it
// reads, so nothing carries over from a previous call.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/lbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kNodesPerThread = 32;
constexpr long long kChunkNodes = (long long)kThreads * kNodesPerThread;  // 8192 nodes per block
constexpr long long kMaxChunks = 8192;                                     // => at most 2^26 nodes

struct Scratch {
  double part[kMaxChunks][4];
  int flag[kMaxChunks];
  double sums[4];
  int flags;
};

static __device__ __align__(256) Scratch g_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
Scratch* g_addr[kMaxDevices] = {nullptr};

struct Consts {
  double rho0, lam, cp, gamma, p0, s0, inv_r;
};

__global__ void __launch_bounds__(kThreads) chunk_kernel(const double* __restrict__ fd, long long N, Consts c,
                                                         Scratch* s) {
  const long long chunk = blockIdx.x;
  const long long base = chunk * kChunkNodes;
  double acc[4] = {0, 0, 0, 0};
  int fl = 0;
  const double af = c.rho0, ag = c.rho0 * c.cp;
  for (int t = 0; t < kNodesPerThread; ++t) {
    const long long i = base + (long long)t * kThreads + threadIdx.x;
    if (i >= N) break;
    double f[6];
    for (int k = 0; k < 6; ++k) {
      f[k] = fd[k * N + i];
      if (!isfinite(f[k])) fl |= 1;
    }
    const double rho = af * (f[0] + f[1] + f[2]);
    const double J = af * c.lam * (f[1] - f[2]);
    const double zeta = ag * (f[3] + f[4] + f[5]);
    const double u = J / rho;
    const double p = c.p0 * pow(rho / c.rho0, c.gamma) * exp(c.gamma * (zeta / rho - c.s0) / c.cp);
    const double T = p / rho * c.inv_r;
    if (!(rho > 0.0)) fl |= 2;
    if (!(T > 0.0) || !isfinite(T)) fl |= 4;
    acc[0] += rho;
    acc[1] += J;
    acc[2] += zeta;
    acc[3] += p / (c.gamma - 1.0) + 0.5 * rho * u * u;
  }
  __shared__ double sh[4][kThreads / 32];
  __shared__ int shf[kThreads / 32];
  for (int k = 0; k < 4; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = v;
  }
  for (int o = 16; o > 0; o >>= 1) fl |= __shfl_down_sync(0xffffffffu, fl, o);
  if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = fl;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      double v = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) v += sh[k][w];
      s->part[chunk][k] = v;
    }
    int ff = 0;
    for (int w = 0; w < kThreads / 32; ++w) ff |= shf[w];
    s->flag[chunk] = ff;
  }
}

// One block sums the chunk partials in a fixed order and writes the results to the scratch
// slots and, if given, to the caller's device outputs.
__global__ void __launch_bounds__(kThreads) final_kernel(long long nchunks, Scratch* s, double* sums_dev,
                                                         int* flags_dev) {
  double acc[4] = {0, 0, 0, 0};
  int fl = 0;
  for (long long c = threadIdx.x; c < nchunks; c += kThreads) {
    for (int k = 0; k < 4; ++k) acc[k] += s->part[c][k];
    fl |= s->flag[c];
  }
  __shared__ double sh[4][kThreads / 32];
  __shared__ int shf[kThreads / 32];
  for (int k = 0; k < 4; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = v;
  }
  for (int o = 16; o > 0; o >>= 1) fl |= __shfl_down_sync(0xffffffffu, fl, o);
  if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = fl;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      double v = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) v += sh[k][w];
      s->sums[k] = v;
      if (sums_dev) sums_dev[k] = v;
    }
    int ff = 0;
    for (int w = 0; w < kThreads / 32; ++w) ff |= shf[w];
    s->flags = ff;
    if (flags_dev) *flags_dev = ff;
  }
}

// Where a pointer lives: 0 host (or unknown to CUDA), 1 device memory of GPU `dev`, 2 managed memory.
int pointer_kind(const void* p, int* dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // this call's own error (no earlier error is pending: checked on entry)
    return 0;
  }
  *dev = a.device;
  if (a.type == cudaMemoryTypeDevice) return 1;
  return a.type == cudaMemoryTypeManaged ? 2 : 0;
}

// The placement rule for the pointer arguments, from their kinds (pointer_kind) and devices: fd must
// be device memory of the current device or managed memory; sums and flags must both be host, or
// both device memory of the current device / managed memory. Returns LBM_OK or LBM_ERR_INVALID_ARG and
// tells whether the outputs are on the device.
int check_placement(int cur, int k_fd, int d_fd, int k_sums, int d_sums, int k_flags, int d_flags, bool* dev_out) {
  if (k_fd == 0 || (k_fd == 1 && d_fd != cur)) return LBM_ERR_INVALID_ARG;
  if ((k_sums != 0) != (k_flags != 0)) return LBM_ERR_INVALID_ARG;
  if ((k_sums == 1 && d_sums != cur) || (k_flags == 1 && d_flags != cur)) return LBM_ERR_INVALID_ARG;
  *dev_out = k_sums != 0;
  return LBM_OK;
}

// Device address of the scratch array on the current device, looked up once per device.
int scratch_for_current_device(Scratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    Scratch* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LBM_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_diagnostics_noalloc(const double* fd, int64_t N, double lambda, const lbm_phys* phys,
                                       double* sums, int32_t* flags, void* stream) {
  if (!fd || !sums || !flags || N < 1 || !(lambda > 0.0)) return LBM_ERR_INVALID_ARG;
  if (N > kMaxChunks * kChunkNodes) return LBM_ERR_TOO_LARGE;
  // An error already pending on this thread belongs to earlier work of the caller: leave it in place
  // (it would be indistinguishable from a failed launch of this call) and refuse to run.
  if (cudaPeekAtLastError() != cudaSuccess) return LBM_ERR_CUDA;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  // Device memory must be on the current device (the scratch and the launches are); memory of
  // another GPU would be a peer access. Managed memory is reachable from any device.
  int d_fd = -1, d_sums = -1, d_flags = -1;
  const int k_fd = pointer_kind(fd, &d_fd);
  const int k_sums = pointer_kind(sums, &d_sums), k_flags = pointer_kind(flags, &d_flags);
  bool dev_out = false;
  if (check_placement(cur, k_fd, d_fd, k_sums, d_sums, k_flags, d_flags, &dev_out) != LBM_OK)
    return LBM_ERR_INVALID_ARG;
  const bool dev_sums = dev_out, dev_flags = dev_out;
  Scratch* s = nullptr;
  int rc = scratch_for_current_device(&s);
  if (rc != LBM_OK) return rc;
  Consts c;
  c.gamma = phys ? phys->gamma : 1.4;
  c.cp = phys ? phys->cp : 1.0;
  c.rho0 = phys ? phys->rho0 : 1.0;
  c.s0 = phys ? phys->s0 : 0.0;
  c.lam = lambda;
  c.p0 = (phys && phys->p0 > 0.0) ? phys->p0 : c.rho0 * (lambda / 2.0) * (lambda / 2.0) / c.gamma;
  c.inv_r = 1.0 / (c.cp * (1.0 - 1.0 / c.gamma));
  cudaStream_t st = (cudaStream_t)stream;
  const long long nchunks = (N + kChunkNodes - 1) / kChunkNodes;
  chunk_kernel<<<(unsigned)nchunks, kThreads, 0, st>>>(fd, N, c, s);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;  // this launch's error only (none was pending)
  final_kernel<<<1, kThreads, 0, st>>>(nchunks, s, dev_sums ? sums : nullptr, dev_flags ? (int*)flags : nullptr);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  if (!dev_sums) {
    if (cudaMemcpyAsync(sums, s->sums, sizeof(double) * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(flags, &s->flags, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return LBM_ERR_CUDA;
    }
    if (*flags) return LBM_ERR_UNSTABLE;
  }
  return LBM_OK;
}

// Test hook: the placement rule alone, without any CUDA call (kinds: 0 host, 1 device, 2 managed).
extern "C" int lbm_debug_noalloc_placement(int32_t current_device, int32_t fd_kind, int32_t fd_device,
                                           int32_t sums_kind, int32_t sums_device, int32_t flags_kind,
                                           int32_t flags_device) {
  bool dev_out = false;
  return check_placement(current_device, fd_kind, fd_device, sums_kind, sums_device, flags_kind, flags_device,
                         &dev_out);
}
