// Double-float numbers for LBM_F64_DF in the two- and three-dimensional kernels: FP64 storage, the
// node update in double-float on the FP32 pipes (the operations of lbm_df_core.cuh, about 48
// significant bits), behind the operators the update is written with, so that one template of the
// update serves float, double and dfn. Construction from a double splits it into the nearest float
// and the remainder.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

struct dfn {
  df v;
  dfn() = default;
  __host__ __device__ dfn(double x) : v(df_from_double_host(x)) {}
  __device__ explicit dfn(df x) : v(x) {}
};
__device__ __forceinline__ dfn operator+(dfn a, dfn b) { return dfn(ad(a.v, b.v)); }
__device__ __forceinline__ dfn operator-(dfn a, dfn b) { return dfn(sb(a.v, b.v)); }
__device__ __forceinline__ dfn operator-(dfn a) { return dfn(df{-a.v.hi, -a.v.lo}); }
__device__ __forceinline__ dfn operator*(dfn a, dfn b) { return dfn(ml(a.v, b.v)); }
__device__ __forceinline__ dfn operator/(dfn a, dfn b) { return dfn(ml(a.v, m_rcp(b.v))); }

// The reciprocal, log1p and expm1 of a dfn, and the value it stores into an FP64 plane.
__device__ __forceinline__ dfn dfn_rcp(dfn x) { return dfn(m_rcp(x.v)); }
__device__ __forceinline__ dfn dfn_log1p(dfn x) { return dfn(m_log1p(x.v)); }
__device__ __forceinline__ dfn dfn_expm1(dfn x) { return dfn(m_expm1(x.v)); }
__device__ __forceinline__ double dfn_store(dfn x) { return to_double(x.v); }

}  // namespace lbm
