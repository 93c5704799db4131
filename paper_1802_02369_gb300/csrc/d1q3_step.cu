// Time step of the single-distribution D1Q3 schemes with temporal blocking:
//   section 2 (fluid): moments (rho, J, e) of eq. (M-d1q3); rho and J conserved; e relaxed with s_e
//     toward e_eq = 3 (rho u^2 + p) - 2 lambda^2 rho (eq. (energie-equilibre)), isentropic pressure
//     p = p0 (rho/rho0)^gamma;
//   section 4 (advection-diffusion): moments (zeta, psi, eps) of the same matrix with scale zeta0;
//     zeta conserved; psi relaxed with s_psi toward u0 zeta, eps with s_eps toward alpha lambda^2 zeta;
// then f* = M^{-1} m* and advection f0(x) = f0*(x), f+(x) = f+*(x - dx), f-(x) = f-*(x + dx).
//
// The populations are stored shifted by those of the rest state (rho0, J = 0; or zeta0), which is
// a fixed point of both schemes, so small deviations keep their relative precision in FP32. The node
// update works on the dimensionless moments r = sum f, j = f+ - f-, q = f+ + f- - 2 f0 of the shifted
// populations: for the fluid, u = lambda j / (1 + r) and the scaled equilibrium is
// q_eq = 3 (j^2 / (1 + r) + kp expm1(gamma log1p(r))) - 2 r with kp = p0 / (rho0 lambda^2); for
// advection-diffusion j_eq = (u0 / lambda) r and q_eq = alpha r. Back-transform: f0 = (r - q)/3,
// f+- = (2r + q)/6 +- j/2.
//
// Layout: three planes of N values. A CTA of NT threads owns NT*V consecutive nodes (periodic wrap);
// thread t holds nodes tV .. tV+V-1 in registers, FP32 with V >= 2 as pairs of nodes in float2 lanes
// (Blackwell's paired FP32 instructions). Only advection couples nodes, one node per step, so a tile
// advances K steps on chip and stores its NT*V - 2K interior nodes. The moving populations cross
// thread boundaries by warp shuffle and warp boundaries through shared memory (one CTA barrier per
// step; the edge buffers alternate by step parity).
#include "d1q3_internal.cuh"
#include "lbm_internal.cuh"
#include "vec_io.cuh"

namespace lbm {

namespace {

// Nodes per lane: 1 for double and float, 2 for float2.
template <typename X>
struct LaneW {
  static constexpr int value = 1;
};
template <>
struct LaneW<float2> {
  static constexpr int value = 2;
};

template <typename R, int V>
struct D1q3Lane {
  using type = R;
};
template <>
struct D1q3Lane<float, 2> {
  using type = float2;
};
template <>
struct D1q3Lane<float, 4> {
  using type = float2;
};
template <>
struct D1q3Lane<float, 8> {
  using type = float2;
};

__device__ __forceinline__ double lget(double x, int) { return x; }
__device__ __forceinline__ float lget(float x, int) { return x; }
__device__ __forceinline__ float lget(float2 x, int i) { return i ? x.y : x.x; }
__device__ __forceinline__ void lset(double& x, int, double v) { x = v; }
__device__ __forceinline__ void lset(float& x, int, float v) { x = v; }
__device__ __forceinline__ void lset(float2& x, int i, float v) {
  if (i) x.y = v;
  else x.x = v;
}

template <typename X, int SCHEME>
__device__ __forceinline__ void collide(X (&f)[3], const D1q3Consts<X>& c) {
  const X tf = ad(f[1], f[2]);
  const X r = ad(tf, f[0]);
  X j = sb(f[1], f[2]);
  X q = fm(f[0], c.m_two, tf);
  if constexpr (SCHEME == kD1q3Fluid) {
    const X inv = m_rcp(ad(c.one, r));
    const X pt = ml(c.kp, m_expm1(ml(c.gamma, m_log1p(r))));
    const X qeq = fm(c.three, fm(ml(j, j), inv, pt), ml(c.m_two, r));
    q = fm(c.s1, sb(qeq, q), q);
  } else {
    j = fm(c.s1, sb(ml(c.ul, r), j), j);
    q = fm(c.s2, sb(ml(c.alpha, r), q), q);
  }
  f[0] = ml(sb(r, q), c.third);
  const X h = ml(fm(c.two, r, q), c.sixth);
  f[1] = fm(c.half, j, h);
  f[2] = fm(c.m_half, j, h);
}

template <typename R, int NT, int V, int SCHEME>
__global__ void __launch_bounds__(NT) d1q3_step_kernel(const R* __restrict__ in, R* __restrict__ out, long long N,
                                                       long long ntiles, int K,
                                                       D1q3Consts<typename D1q3Lane<R, V>::type> c) {
  using X = typename D1q3Lane<R, V>::type;
  constexpr int W = LaneW<X>::value, NL = V / W, NW = NT / 32;
  __shared__ R edge[2][NW][2];  // per step parity and warp: f+ of its last node, f- of its first node
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long bout = (long long)NT * V - 2 * K;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long pos0 = tile * bout - K + (long long)threadIdx.x * V;
    X f[NL][3];
    if (VecIo<R, V>::ok(in, pos0, N)) {  // lanes hold consecutive nodes: vectors map onto them
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        R t[V];
        VecIo<R, V>::load(in + i * N + pos0, t);
#pragma unroll
        for (int v = 0; v < V; ++v) lset(f[v / W][i], v % W, t[v]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        long long lp = pos0 + v;
        if (lp < 0 || lp >= N) { lp %= N; if (lp < 0) lp += N; }
#pragma unroll
        for (int i = 0; i < 3; ++i) lset(f[v / W][i], v % W, in[i * N + lp]);
      }
    }
    for (int k = 0; k < K; ++k) {
#pragma unroll
      for (int l = 0; l < NL; ++l) collide<X, SCHEME>(f[l], c);
      // Advection: f+ moves one node right, f- one node left.
      const R last_p = lget(f[NL - 1][1], W - 1), first_m = lget(f[0][2], 0);
      R fpL = __shfl_up_sync(0xffffffffu, last_p, 1);
      R fmR = __shfl_down_sync(0xffffffffu, first_m, 1);
      R (*e)[2] = edge[k & 1];
      if (lane == 31) e[warp][0] = last_p;
      if (lane == 0) e[warp][1] = first_m;
      __syncthreads();
      if (lane == 0 && warp > 0) fpL = e[warp - 1][0];
      if (lane == 31 && warp < NW - 1) fmR = e[warp + 1][1];
      // (The outermost nodes of the tile take stand-ins; they are never stored.)
      R carry = fpL;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const R t = lget(f[v / W][1], v % W);
        lset(f[v / W][1], v % W, carry);
        carry = t;
      }
      carry = fmR;
#pragma unroll
      for (int v = V - 1; v >= 0; --v) {
        const R t = lget(f[v / W][2], v % W);
        lset(f[v / W][2], v % W, carry);
        carry = t;
      }
    }
    const int local0 = threadIdx.x * V;
    if (local0 >= K && local0 + V <= K + bout && VecIo<R, V>::ok(out, pos0, N)) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        R t[V];
#pragma unroll
        for (int v = 0; v < V; ++v) t[v] = lget(f[v / W][i], v % W);
        VecIo<R, V>::store(out + i * N + pos0, t);
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int local = local0 + v;
        const long long pos = pos0 + v;
        if (local >= K && local < K + bout && pos < N)
#pragma unroll
          for (int i = 0; i < 3; ++i) out[i * N + pos] = lget(f[v / W][i], v % W);
      }
    }
    __syncthreads();  // the next tile's first step rewrites the edge buffer
  }
}

template <typename R, int NT, int V, int SCHEME>
cudaError_t launch_one(const R* in, R* out, long long N, int K, const D1q3ConstSet<R>& cs, cudaStream_t st,
                       long long max_tiles) {
  const long long bout = (long long)NT * V - 2 * K;
  long long ntiles = (N + bout - 1) / bout;
  if (max_tiles > 0 && ntiles > max_tiles) ntiles = max_tiles;
  const long long grid = ntiles < 2147483647LL ? ntiles : 2147483647LL;
  using X = typename D1q3Lane<R, V>::type;
  const D1q3Consts<X>* c;
  if constexpr (sizeof(X) == 8 && sizeof(R) == 4) c = &cs.p;
  else c = &cs.s;
  d1q3_step_kernel<R, NT, V, SCHEME><<<(unsigned)grid, NT, 0, st>>>(in, out, N, ntiles, K, *c);
  return cudaGetLastError();
}

template <typename R, int SCHEME>
cudaError_t launch_scheme(const R* in, R* out, long long N, int K, int NT, int V, const D1q3ConstSet<R>& c,
                          cudaStream_t st, long long max_tiles) {
#define D1Q3_CASE(nt, v) \
  if (NT == nt && V == v) return launch_one<R, nt, v, SCHEME>(in, out, N, K, c, st, max_tiles);
  D1Q3_CASE(128, 1) D1Q3_CASE(128, 2) D1Q3_CASE(128, 4) D1Q3_CASE(128, 8)
  D1Q3_CASE(256, 1) D1Q3_CASE(256, 2) D1Q3_CASE(256, 4) D1Q3_CASE(256, 8)
  D1Q3_CASE(512, 1) D1Q3_CASE(512, 2) D1Q3_CASE(512, 4) D1Q3_CASE(512, 8)
#undef D1Q3_CASE
  return cudaErrorInvalidValue;
}

}  // namespace

bool valid_d1q3_config(int K, int NT, int V) {
  const bool nt_ok = NT == 128 || NT == 256 || NT == 512;
  const bool v_ok = V == 1 || V == 2 || V == 4 || V == 8;
  return nt_ok && v_ok && K >= 1 && K <= 64 && NT * V - 2 * K >= 32;
}

template <typename R>
cudaError_t launch_d1q3_step(const R* in, R* out, long long N, int scheme, int K, int NT, int V,
                             const D1q3ConstSet<R>& c, cudaStream_t st, long long max_tiles) {
  if (N <= 0) return cudaSuccess;
  if (!valid_d1q3_config(K, NT, V)) return cudaErrorInvalidValue;
  if (scheme == kD1q3Fluid) return launch_scheme<R, kD1q3Fluid>(in, out, N, K, NT, V, c, st, max_tiles);
  if (scheme == kD1q3AdvDiff) return launch_scheme<R, kD1q3AdvDiff>(in, out, N, K, NT, V, c, st, max_tiles);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_d1q3_step<float>(const float*, float*, long long, int, int, int, int,
                                             const D1q3ConstSet<float>&, cudaStream_t, long long);
template cudaError_t launch_d1q3_step<double>(const double*, double*, long long, int, int, int, int,
                                              const D1q3ConstSet<double>&, cudaStream_t, long long);

}  // namespace lbm
