// Test hooks: evaluate the FP32 lane functions of the node update, and the double-float operations,
// on device arrays, so that the series can be checked against CUDA's own functions and against FP64.
#include "../../include/lbm.h"
#include "lbm_df.cuh"
#include "lbm_internal.cuh"

namespace {

__global__ void eval_kernel(const float* __restrict__ x, float* __restrict__ y, long long n, int fn) {
  const long long i = 2 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  if (i >= n) return;
  const float2 a = make_float2(x[i], i + 1 < n ? x[i + 1] : 0.0f);
  float2 r;
  switch (fn) {
    case 0: r = lbm::m_log1p(a); break;                                   // paired-lane log1p
    case 1: r = make_float2(lbm::m_log1p(a.x), lbm::m_log1p(a.y)); break;  // CUDA log1pf
    case 2: r = lbm::m_expm1(a); break;                                   // paired-lane expm1
    case 3: r = make_float2(lbm::m_expm1(a.x), lbm::m_expm1(a.y)); break;  // CUDA expm1f
    default: r = lbm::m_rcp(a); break;                                    // reciprocal
  }
  y[i] = r.x;
  if (i + 1 < n) y[i + 1] = r.y;
}

}  // namespace

extern "C" int lbm_debug_eval_f32(const float* x, float* y, int64_t n, int32_t fn, void* stream) {
  if (!x || !y || n < 1 || fn < 0 || fn > 4) return LBM_ERR_INVALID_ARG;
  const long long pairs = (n + 1) / 2;
  eval_kernel<<<(unsigned)((pairs + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y, n, fn);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// Test hook for the double-float functions of lbm_df_core.cuh: y = f(x) elementwise, computed in
// double-float from the FP64 input (split into hi + lo) and summed back to FP64 (fn 0-5); fn 6-8 the
// FP64-lane log1p, expm1 and reciprocal of the node update.
namespace {

__global__ void eval_df_kernel(const double* __restrict__ x, const double* __restrict__ x2, double* __restrict__ y,
                               long long n, int fn) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const lbm::df a = lbm::to_df(x[i]);
  lbm::df r;
  switch (fn) {
    case 0: r = lbm::m_log1p(a); break;
    case 1: r = lbm::m_expm1(a); break;
    case 2: r = lbm::m_rcp(a); break;
    case 3: r = lbm::ml(a, lbm::to_df(x2[i])); break;
    case 4: r = lbm::ad(a, lbm::to_df(x2[i])); break;
    case 5: r = lbm::fm(a, lbm::to_df(x2[i]), lbm::to_df(x2[(i + 1) % n])); break;
    // The FP64 lanes of the node update, on the FP64 input itself.
    case 6: y[i] = lbm::m_log1p(x[i]); return;
    case 7: y[i] = lbm::m_expm1(x[i]); return;
    default: y[i] = lbm::m_rcp(x[i]); return;
  }
  y[i] = lbm::to_double(r);
}

}  // namespace

extern "C" int lbm_debug_eval_df(const double* x, const double* x2, double* y, int64_t n, int32_t fn, void* stream) {
  if (!x || !y || n < 1 || fn < 0 || fn > 8 || (fn >= 3 && fn <= 5 && !x2)) return LBM_ERR_INVALID_ARG;
  eval_df_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, x2, y, n, fn);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
