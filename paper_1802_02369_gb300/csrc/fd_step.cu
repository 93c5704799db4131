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
// NT*V consecutive nodes (periodic wrap at both ends of the grid); thread t holds nodes tV .. tV+V-1.
// The stencil reaches one node per step, so a tile advances K steps on chip and stores its
// NT*V - 2K interior nodes. Each step a node computes u, p, T and the seven values its neighbours
// need (J, the two other convective fluxes, u, T - T0, rho nu and kappa/T); neighbours read them
// from the same thread's registers, the adjacent lane (warp shuffle) or, at warp edges, shared
// memory (one CTA barrier per step).
#include "fd_internal.cuh"

namespace lbm {

namespace {

__device__ __forceinline__ double fd_rcp(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float fd_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fd_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float fd_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double fd_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float fd_expm1(float x) { return expm1f(x); }

constexpr int kEx = 7;  // values a node passes to its neighbours
enum { X_J = 0, X_F1, X_F2, X_U, X_TT, X_A, X_B };

// Nodal quantities of one node from its shifted state w = (rho - rho0, J, zeta - rho0 s0):
// eq. (gaz-parfait) p = p0 (rho/rho0)^gamma exp(gamma (s - s0)/c_p), p = rho r T, written as
// p - p0 = p0 expm1(gamma (log1p((rho - rho0)/rho0) + (s - s0)/c_p)) and
// T - T0 = ((p - p0)/r - (rho - rho0) T0) / rho.
template <typename R>
__device__ __forceinline__ void fd_node(const R (&w)[3], const FdConsts<R>& c, R (&x)[kEx], R& inv_T) {
  const R rho = c.rho0 + w[0];
  const R inv_rho = fd_rcp(rho);
  const R u = w[1] * inv_rho;
  const R ds = (w[2] - w[0] * c.s0) * inv_rho;  // s - s0 = (zeta - rho s0) / rho
  const R lnr = fd_log1p(w[0] * c.inv_rho0);
  const R pt = c.p0 * fd_expm1(c.gamma * (lnr + ds * c.inv_cp));
  const R Tt = (pt * c.inv_r - w[0] * c.T0) * inv_rho;
  inv_T = fd_rcp(c.T0 + Tt);
  x[X_J] = w[1];
  x[X_F1] = w[1] * u + pt;       // rho u^2 + p, less the constant p0
  x[X_F2] = (w[2] + c.rho0s0) * u;  // zeta u
  x[X_U] = u;
  x[X_TT] = Tt;
  x[X_A] = rho * c.nu;               // rho nu
  x[X_B] = rho * c.nu_k * inv_T;     // kappa / T
}

// Forward-Euler update of one node from its own values (x0, inv_T) and its neighbours' (xl, xr).
template <typename R>
__device__ __forceinline__ void fd_update(R (&w)[3], const R (&x0)[kEx], R inv_T, const R* xl, const R* xr,
                                          const FdConsts<R>& c) {
  const R dur = xr[X_U] - x0[X_U], dul = x0[X_U] - xl[X_U];
  const R dTr = xr[X_TT] - x0[X_TT], dTl = x0[X_TT] - xl[X_TT];
  const R phiJ = (x0[X_A] + xr[X_A]) * dur - (xl[X_A] + x0[X_A]) * dul;
  const R phiZ = (x0[X_B] + xr[X_B]) * dTr - (xl[X_B] + x0[X_B]) * dTl;
  w[0] = w[0] - c.c_adv * (xr[X_J] - xl[X_J]);
  w[1] = w[1] - c.c_adv * (xr[X_F1] - xl[X_F1]) + c.c_dif * phiJ;
  R z = w[2] - c.c_adv * (xr[X_F2] - xl[X_F2]) + c.c_dif * phiZ;
  if (c.source_on) {
    const R du = dur + dul, dT = dTr + dTl;
    z = z + c.c_src * inv_T * (x0[X_A] * du * du + x0[X_B] * dT * dT);
  }
  w[2] = z;
}

template <typename R, int NT, int V>
__global__ void __launch_bounds__(NT) fd_step_kernel(const R* __restrict__ in, R* __restrict__ out, long long N,
                                                     long long ntiles, int K, FdConsts<R> c) {
  constexpr int NW = NT / 32;
  __shared__ R edge[2][NW][2][kEx];  // per step parity, warp, side (0: its last node, 1: its first)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long bout = (long long)NT * V - 2 * K;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long pos0 = tile * bout - K + (long long)threadIdx.x * V;
    R w[V][3];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      long long lp = pos0 + v;
      if (lp < 0 || lp >= N) { lp %= N; if (lp < 0) lp += N; }
#pragma unroll
      for (int i = 0; i < 3; ++i) w[v][i] = in[i * N + lp];
    }
    for (int k = 0; k < K; ++k) {
      R x[V][kEx], inv_T[V];
#pragma unroll
      for (int v = 0; v < V; ++v) fd_node(w[v], c, x[v], inv_T[v]);
      R xl[kEx], xr[kEx];
      R (*e)[2][kEx] = edge[k & 1];
#pragma unroll
      for (int m = 0; m < kEx; ++m) {
        xl[m] = __shfl_up_sync(0xffffffffu, x[V - 1][m], 1);
        xr[m] = __shfl_down_sync(0xffffffffu, x[0][m], 1);
        if (lane == 31) e[warp][0][m] = x[V - 1][m];
        if (lane == 0) e[warp][1][m] = x[0][m];
      }
      __syncthreads();
      // The outermost nodes of the tile keep stand-in neighbours; they are never stored.
#pragma unroll
      for (int m = 0; m < kEx; ++m) {
        if (lane == 0 && warp > 0) xl[m] = e[warp - 1][0][m];
        if (lane == 31 && warp < NW - 1) xr[m] = e[warp + 1][1][m];
      }
#pragma unroll
      for (int v = 0; v < V; ++v) fd_update(w[v], x[v], inv_T[v], v > 0 ? x[v - 1] : xl, v < V - 1 ? x[v + 1] : xr, c);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int local = threadIdx.x * V + v;
      const long long pos = pos0 + v;
      if (local >= K && local < K + bout && pos < N)
#pragma unroll
        for (int i = 0; i < 3; ++i) out[i * N + pos] = w[v][i];
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
  fd_step_kernel<R, NT, V><<<(unsigned)grid, NT, 0, st>>>(in, out, N, ntiles, K, c);
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
