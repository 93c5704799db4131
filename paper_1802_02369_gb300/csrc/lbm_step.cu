// Fused collide-stream kernel of the D1Q3Q3 scheme (section 8, steps (i)-(viii)) with temporal
// blocking: one CTA loads a tile of NT consecutive nodes of one lattice (structure-of-arrays, six
// coalesced plane loads), advances it K time steps in registers and shared memory, and stores the
// NT - 4K interior nodes whose dependency cone (radius 2 per step: the source needs u and T of
// the neighbours, streaming moves one node) stayed inside the tile.
//
// Per step and node: the moments, u and T are computed in registers; u and T go to shared memory;
// after a barrier each node reads its neighbours' u and T, collides, and writes its moving
// populations (f+, f-, g+, g-) into the neighbour's slot of four exchange arrays; after a second
// barrier each node picks up its streamed populations. f0 and g0 never leave registers.
#include "lbm_internal.cuh"

namespace lbm {

template <typename R, int NT>
__global__ void __launch_bounds__(NT) step_tiles_kernel(const R* __restrict__ in, R* __restrict__ out,
                                                        long long plane, const LatDev* __restrict__ lat,
                                                        int B, long long ntiles, int K, Consts<R> c) {
  __shared__ R su[NT];
  __shared__ R sT[NT];
  __shared__ R xfp[NT + 1];  // xfp[n] receives f+* of node n - 1
  __shared__ R xfm[NT + 1];  // xfm[n + 1] receives f-* of node n + 1
  __shared__ R xgp[NT + 1];
  __shared__ R xgm[NT + 1];
  const int n = threadIdx.x;
  if (n == 0) {
    // Edge slots no node writes: the two outermost nodes of a tile read them and are discarded.
    xfp[0] = R(0); xgp[0] = R(0); xfm[NT] = R(0); xgm[NT] = R(0);
  }
  const int halo = 2 * K;
  const int bout = NT - 2 * halo;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int L = 0;
    if (B > 1) {  // last lattice whose first tile is <= tile
      int lo = 0, hi = B - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (lat[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
      }
      L = lo;
    }
    const long long off = lat[L].offset, N = lat[L].n;
    const int bc = lat[L].bc;
    const R s_e = R(lat[L].s_e), s_psi = R(lat[L].s_psi), s_eps = R(lat[L].s_eps);
    const R q_src = R(lat[L].q_src), s0 = R(lat[L].s0);

    const long long start = (tile - lat[L].tile0) * bout;
    const long long pos = start - halo + n;  // lattice-relative position of this thread's node
    long long lp = pos;
    if (bc == 0) {
      if (lp < 0 || lp >= N) { lp %= N; if (lp < 0) lp += N; }
    } else {
      lp = lp < 0 ? 0 : (lp >= N ? N - 1 : lp);
    }
    const bool active = (bc == 0) || (pos >= 0 && pos < N);
    const bool lwall = (bc != 0) && pos == 0;
    const bool rwall = (bc != 0) && pos == N - 1;

    R f[6];
    const long long g = off + lp;
#pragma unroll
    for (int i = 0; i < 6; ++i) f[i] = in[i * plane + g];

    for (int k = 0; k < K; ++k) {
      Node<R> m;
      node_state(f, c, s0, m);
      su[n] = m.u;
      sT[n] = m.T;
      __syncthreads();
      R ul = n > 0 ? su[n - 1] : m.u, Tl = n > 0 ? sT[n - 1] : m.T;
      R ur = n < NT - 1 ? su[n + 1] : m.u, Tr = n < NT - 1 ? sT[n + 1] : m.T;
      if (lwall) { ul = -m.u; Tl = m.T; }
      if (rwall) { ur = -m.u; Tr = m.T; }
      R fs[6];
      node_collide(m, ul, ur, Tl, Tr, s_e, s_psi, s_eps, q_src, s0, c, fs);
      f[0] = fs[0];
      f[3] = fs[3];
      if (active) {
        // (viii) streaming; at a wall the outgoing population comes back reversed.
        if (rwall) { xfm[n + 1] = fs[1]; xgm[n + 1] = fs[4]; }
        else { xfp[n + 1] = fs[1]; xgp[n + 1] = fs[4]; }
        if (lwall) { xfp[n] = fs[2]; xgp[n] = fs[5]; }
        else { xfm[n] = fs[2]; xgm[n] = fs[5]; }
      }
      __syncthreads();
      f[1] = xfp[n];
      f[4] = xgp[n];
      f[2] = xfm[n + 1];
      f[5] = xgm[n + 1];
    }

    if (n >= halo && n < halo + bout && pos < N) {
      const long long o = off + pos;
#pragma unroll
      for (int i = 0; i < 6; ++i) out[i * plane + o] = f[i];
    }
  }
}

template <typename R>
cudaError_t launch_step_tiles(const R* in, R* out, long long plane, const LatDev* lat, int B,
                              long long ntiles, int K, int NT, const Consts<R>& c, cudaStream_t st,
                              int grid_cap) {
  if (ntiles <= 0) return cudaSuccess;
  long long grid = ntiles;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  switch (NT) {
    case 256: step_tiles_kernel<R, 256><<<(unsigned)grid, 256, 0, st>>>(in, out, plane, lat, B, ntiles, K, c); break;
    case 512: step_tiles_kernel<R, 512><<<(unsigned)grid, 512, 0, st>>>(in, out, plane, lat, B, ntiles, K, c); break;
    case 1024: step_tiles_kernel<R, 1024><<<(unsigned)grid, 1024, 0, st>>>(in, out, plane, lat, B, ntiles, K, c); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_step_tiles<float>(const float*, float*, long long, const LatDev*, int, long long,
                                              int, int, const Consts<float>&, cudaStream_t, int);
template cudaError_t launch_step_tiles<double>(const double*, double*, long long, const LatDev*, int, long long,
                                               int, int, const Consts<double>&, cudaStream_t, int);

}  // namespace lbm
