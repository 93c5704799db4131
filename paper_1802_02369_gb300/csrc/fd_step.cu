// Time step of the finite-difference comparison solver of section 9, with temporal blocking.
//
// The paper validates its lattice Boltzmann results against a finite-difference program for the
// (rho, J, zeta) system of eq. (NS-rho-J-zeta) with second-order centred differences and explicit
// first-order time integration; it does not print the stencil. The conservation form used here
// (the same reading as the CPU oracle of this solver):
//   convective flux F = (J, rho u^2 + p, zeta u), differenced centred: (F_{j+1} - F_{j-1}) / (2 dx);
//   diffusive flux Phi = (0, rho nu d_x u, (kappa / T) d_x T) at the faces j +- 1/2, with the face
//   coefficient the mean of the two nodal ones and d_x q = (q_{j+1} - q_j) / dx, differenced over
//   the cell: (Phi_{j+1/2} - Phi_{j-1/2}) / dx;
//   entropy production S = (rho nu / T)(d_x u)^2 + (kappa / T^2)(d_x T)^2 at the node with centred
//   derivatives (the differences of step (vii) of section 8);
//   W^{n+1} = W^n + dt (-d_x F + d_x Phi + (0, 0, S)), kappa = rho nu c_p / Pr.
//
// Layout: three planes of N values (rho - rho0, J, zeta - rho0 s0). A CTA of NT threads owns a tile of
// NT*V consecutive nodes (periodic wrap at both ends of the grid); thread t holds nodes tV .. tV+V-1
// (FP32 threads of two or four nodes as pairs of nodes on paired FP32 lanes).
// The stencil reaches one node per step, so a tile advances K steps on chip and stores its
// NT*V - 2K interior nodes. Each step a node computes u, p, T and the seven values its neighbours
// need (J, the two other convective fluxes, u, T - T0, rho nu and kappa/T); neighbours read them
// from the same thread's registers, the adjacent lane (warp shuffle) or, at warp edges, shared
// memory (one CTA barrier per step).
#include "fd_internal.cuh"
#include "lbm_internal.cuh"
#include "vec_io.cuh"

namespace lbm {

namespace {

// Lanes: FP64 and one-node FP32 threads hold one node per lane value; FP32 threads of two or four
// nodes hold them in pairs (float2) for Blackwell's paired FP32 instructions, with the series log1p
// and expm1 of the lattice Boltzmann kernels (lbm_internal.cuh).
template <typename R, int V>
struct FdLane {
  using X = R;
  static constexpr int W = 1;
};
template <>
struct FdLane<float, 2> {
  using X = float2;
  static constexpr int W = 2;
};
template <>
struct FdLane<float, 4> {
  using X = float2;
  static constexpr int W = 2;
};

__device__ __forceinline__ double lget(double x, int) { return x; }
__device__ __forceinline__ float lget(float x, int) { return x; }
__device__ __forceinline__ float lget(float2 x, int j) { return j ? x.y : x.x; }
__device__ __forceinline__ void lset(double& x, int, double v) { x = v; }
__device__ __forceinline__ void lset(float& x, int, float v) { x = v; }
__device__ __forceinline__ void lset(float2& x, int j, float v) {
  if (j) x.y = v;
  else x.x = v;
}

template <typename X>
struct FdLaneConsts {
  X rho0, inv_rho0, m_s0, rho0s0, gamma, inv_cp, p0, inv_r, T0, m_T0, nu, nu_k, m_c_adv, c_dif, c_src;
  int source_on;
};

template <typename X, typename R>
__host__ FdLaneConsts<X> lane_consts(const FdConsts<R>& c) {
  auto L = [](R v) {
    if constexpr (sizeof(X) == 2 * sizeof(float) && sizeof(R) == sizeof(float)) return make_float2(v, v);
    else return X(v);
  };
  FdLaneConsts<X> k;
  k.rho0 = L(c.rho0);
  k.inv_rho0 = L(c.inv_rho0);
  k.m_s0 = L(-c.s0);
  k.rho0s0 = L(c.rho0s0);
  k.gamma = L(c.gamma);
  k.inv_cp = L(c.inv_cp);
  k.p0 = L(c.p0);
  k.inv_r = L(c.inv_r);
  k.T0 = L(c.T0);
  k.m_T0 = L(-c.T0);
  k.nu = L(c.nu);
  k.nu_k = L(c.nu_k);
  k.m_c_adv = L(-c.c_adv);
  k.c_dif = L(c.c_dif);
  k.c_src = L(c.c_src);
  k.source_on = c.source_on;
  return k;
}

constexpr int kEx = 7;  // values a node passes to its neighbours
enum { X_J = 0, X_F1, X_F2, X_U, X_TT, X_A, X_B };

// Nodal quantities of one lane from its shifted state w = (rho - rho0, J, zeta - rho0 s0):
// eq. (gaz-parfait) p = p0 (rho/rho0)^gamma exp(gamma (s - s0)/c_p), p = rho r T, written as
// p - p0 = p0 expm1(gamma (log1p((rho - rho0)/rho0) + (s - s0)/c_p)) and
// T - T0 = ((p - p0)/r - (rho - rho0) T0) / rho. Every fused multiply-add is explicit.
template <typename X>
__device__ __forceinline__ void fd_node(const X (&w)[3], const FdLaneConsts<X>& c, X (&x)[kEx], X& inv_T) {
  const X rho = ad(c.rho0, w[0]);
  const X inv_rho = m_rcp(rho);
  const X u = ml(w[1], inv_rho);
  const X ds = ml(fm(w[0], c.m_s0, w[2]), inv_rho);  // s - s0 = (zeta - rho s0) / rho
  const X lnr = m_log1p(ml(w[0], c.inv_rho0));
  const X pt = ml(c.p0, m_expm1(ml(c.gamma, fm(ds, c.inv_cp, lnr))));
  const X Tt = ml(fm(pt, c.inv_r, ml(w[0], c.m_T0)), inv_rho);
  inv_T = m_rcp(ad(c.T0, Tt));
  x[X_J] = w[1];
  x[X_F1] = fm(w[1], u, pt);          // rho u^2 + p, less the constant p0
  x[X_F2] = ml(ad(w[2], c.rho0s0), u);  // zeta u
  x[X_U] = u;
  x[X_TT] = Tt;
  x[X_A] = ml(rho, c.nu);                  // rho nu
  x[X_B] = ml(ml(rho, c.nu_k), inv_T);     // kappa / T
}

// Forward-Euler update of one lane from its own values (x0, inv_T) and its neighbours' (xl, xr).
template <typename X>
__device__ __forceinline__ void fd_update(X (&w)[3], const X (&x0)[kEx], X inv_T, const X (&xl)[kEx],
                                          const X (&xr)[kEx], const FdLaneConsts<X>& c) {
  const X dur = sb(xr[X_U], x0[X_U]), dul = sb(x0[X_U], xl[X_U]);
  const X dTr = sb(xr[X_TT], x0[X_TT]), dTl = sb(x0[X_TT], xl[X_TT]);
  const X phiJ = sb(ml(ad(x0[X_A], xr[X_A]), dur), ml(ad(xl[X_A], x0[X_A]), dul));
  const X phiZ = sb(ml(ad(x0[X_B], xr[X_B]), dTr), ml(ad(xl[X_B], x0[X_B]), dTl));
  w[0] = fm(c.m_c_adv, sb(xr[X_J], xl[X_J]), w[0]);
  w[1] = fm(c.c_dif, phiJ, fm(c.m_c_adv, sb(xr[X_F1], xl[X_F1]), w[1]));
  X z = fm(c.c_dif, phiZ, fm(c.m_c_adv, sb(xr[X_F2], xl[X_F2]), w[2]));
  if (c.source_on) {
    const X du = ad(dur, dul), dT = ad(dTr, dTl);
    z = fm(ml(c.c_src, inv_T), fm(x0[X_A], ml(du, du), ml(x0[X_B], ml(dT, dT))), z);
  }
  w[2] = z;
}

template <typename R, int NT, int V>
__global__ void __launch_bounds__(NT) fd_step_kernel(const R* __restrict__ in, R* __restrict__ out, long long N,
                                                     long long ntiles, int K,
                                                     FdLaneConsts<typename FdLane<R, V>::X> c) {
  using X = typename FdLane<R, V>::X;
  constexpr int W = FdLane<R, V>::W, NL = V / W, NW = NT / 32;
  __shared__ R edge[2][NW][2][kEx];  // per step parity, warp, side (0: its last node, 1: its first)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long bout = (long long)NT * V - 2 * K;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long pos0 = tile * bout - K + (long long)threadIdx.x * V;
    X w[NL][3];
    if (VecIo<R, V>::ok(in, pos0, N)) {  // lanes hold consecutive nodes: vectors map onto them
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        R t[V];
        VecIo<R, V>::load(in + i * N + pos0, t);
#pragma unroll
        for (int v = 0; v < V; ++v) lset(w[v / W][i], v % W, t[v]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        long long lp = pos0 + v;
        if (lp < 0 || lp >= N) { lp %= N; if (lp < 0) lp += N; }
#pragma unroll
        for (int i = 0; i < 3; ++i) lset(w[v / W][i], v % W, in[i * N + lp]);
      }
    }
    for (int k = 0; k < K; ++k) {
      X x[NL][kEx], inv_T[NL];
#pragma unroll
      for (int l = 0; l < NL; ++l) fd_node(w[l], c, x[l], inv_T[l]);
      R eL[kEx], eR[kEx];  // the neighbours of the thread's first and last node
      R (*e)[2][kEx] = edge[k & 1];
#pragma unroll
      for (int m = 0; m < kEx; ++m) {
        const R last = lget(x[NL - 1][m], W - 1), first = lget(x[0][m], 0);
        eL[m] = __shfl_up_sync(0xffffffffu, last, 1);
        eR[m] = __shfl_down_sync(0xffffffffu, first, 1);
        if (lane == 31) e[warp][0][m] = last;
        if (lane == 0) e[warp][1][m] = first;
      }
      __syncthreads();
      // The outermost nodes of the tile keep stand-in neighbours; they are never stored.
#pragma unroll
      for (int m = 0; m < kEx; ++m) {
        if (lane == 0 && warp > 0) eL[m] = e[warp - 1][0][m];
        if (lane == 31 && warp < NW - 1) eR[m] = e[warp + 1][1][m];
      }
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        X xl[kEx], xr[kEx];
#pragma unroll
        for (int m = 0; m < kEx; ++m) {
          if constexpr (W == 1) {
            xl[m] = l > 0 ? x[l - 1][m] : eL[m];
            xr[m] = l < NL - 1 ? x[l + 1][m] : eR[m];
          } else {
            xl[m] = make_float2(l > 0 ? x[l - 1][m].y : eL[m], x[l][m].x);
            xr[m] = make_float2(x[l][m].y, l < NL - 1 ? x[l + 1][m].x : eR[m]);
          }
        }
        fd_update(w[l], x[l], inv_T[l], xl, xr, c);
      }
    }
    const int local0 = threadIdx.x * V;
    if (local0 >= K && local0 + V <= K + bout && VecIo<R, V>::ok(out, pos0, N)) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        R t[V];
#pragma unroll
        for (int v = 0; v < V; ++v) t[v] = lget(w[v / W][i], v % W);
        VecIo<R, V>::store(out + i * N + pos0, t);
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int local = local0 + v;
        const long long pos = pos0 + v;
        if (local >= K && local < K + bout && pos < N)
#pragma unroll
          for (int i = 0; i < 3; ++i) out[i * N + pos] = lget(w[v / W][i], v % W);
      }
    }
    __syncthreads();  // the next tile's first step rewrites the edge buffer
  }
}

template <typename R, int NT, int V>
cudaError_t launch_nt_v(const R* in, R* out, long long N, int K, const FdConsts<R>& c, cudaStream_t st,
                        long long max_tiles) {
  const long long bout = (long long)NT * V - 2 * K;
  long long ntiles = (N + bout - 1) / bout;
  if (max_tiles > 0 && ntiles > max_tiles) ntiles = max_tiles;
  const long long grid = ntiles < 2147483647LL ? ntiles : 2147483647LL;
  using X = typename FdLane<R, V>::X;
  fd_step_kernel<R, NT, V><<<(unsigned)grid, NT, 0, st>>>(in, out, N, ntiles, K, lane_consts<X, R>(c));
  return cudaGetLastError();
}

}  // namespace

bool valid_fd_config(int K, int NT, int V) {
  const bool nt_ok = NT == 128 || NT == 256 || NT == 512;
  const bool v_ok = V == 1 || V == 2 || V == 4;
  return nt_ok && v_ok && K >= 1 && K <= 16 && NT * V - 2 * K >= 32;
}

template <typename R>
cudaError_t launch_fd_step(const R* in, R* out, long long N, int K, int NT, int V, const FdConsts<R>& c,
                           cudaStream_t st, long long max_tiles) {
  if (N <= 0) return cudaSuccess;
  if (!valid_fd_config(K, NT, V)) return cudaErrorInvalidValue;
#define FD_CASE(nt, v) \
  if (NT == nt && V == v) return launch_nt_v<R, nt, v>(in, out, N, K, c, st, max_tiles);
  FD_CASE(128, 1) FD_CASE(128, 2) FD_CASE(128, 4)
  FD_CASE(256, 1) FD_CASE(256, 2) FD_CASE(256, 4)
  FD_CASE(512, 1) FD_CASE(512, 2) FD_CASE(512, 4)
#undef FD_CASE
  return cudaErrorInvalidValue;
}

template cudaError_t launch_fd_step<float>(const float*, float*, long long, int, int, int, const FdConsts<float>&,
                                           cudaStream_t, long long);
template cudaError_t launch_fd_step<double>(const double*, double*, long long, int, int, int,
                                            const FdConsts<double>&, cudaStream_t, long long);

}  // namespace lbm
