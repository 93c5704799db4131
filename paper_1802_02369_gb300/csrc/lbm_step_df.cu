// Fused collide-stream step of the D1Q3Q3 scheme (section 8, steps (i)-(viii)) with FP64 storage and
// double-float arithmetic on the FP32 pipes (precision LBM_F64_DF); one node per thread on scalar df
// lanes, two or four on paired df2 lanes.
//
// The same temporally blocked tile update as the step kernels of lbm_step.cu (tiles of NT*V nodes,
// thread t holding nodes tV .. tV+V-1, K steps on chip, 2K halo nodes recomputed per side), with every
// node value a double-float (lbm_df.cuh): the populations are split into hi + lo floats when the tile is
// loaded, the dimensionless node update of lbm_internal.cuh runs on df lanes, and the populations are
// summed back to FP64 when the tile is stored. Neighbour values cross threads by two shuffles (hi, lo)
// and warps through shared memory.
#include "lbm_df.cuh"
#include "lbm_internal.cuh"

namespace lbm {

namespace {

__device__ __forceinline__ df shfl_up(df v) {
  return df{__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1)};
}
__device__ __forceinline__ df shfl_down(df v) {
  return df{__shfl_down_sync(0xffffffffu, v.hi, 1), __shfl_down_sync(0xffffffffu, v.lo, 1)};
}
__device__ __forceinline__ df neg(df v) { return df{-v.hi, -v.lo}; }

template <int NT, int V, bool WALLS>
__device__ __forceinline__ void tile_body_df(const double* __restrict__ in, double* __restrict__ out,
                                             long long plane, const LatDev& d, long long start, int K,
                                             const Consts<df>& c, df (*e_ut)[4], df (*e_f)[4]) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int halo = 2 * K;
  const int bout = NT * V - 2 * halo;
  const long long off = d.offset, N = d.n;
  // Per-lattice parameters split into hi + lo on the host (no FP64-pipe conversion per tile).
  const df s_e{d.f32[0], d.f32lo[0]}, s_psi{d.f32[1], d.f32lo[1]}, s_eps{d.f32[2], d.f32lo[2]};
  const df q_src{d.f32[3], d.f32lo[3]}, s0h{d.f32[4], d.f32lo[4]}, m_s0h = neg(s0h);
  const df le0{d.f32[5], d.f32lo[5]}, lp0{d.f32[6], d.f32lo[6]}, lq0{d.f32[7], d.f32lo[7]};
  const long long pos0 = start - halo + (long long)threadIdx.x * V;

  df f[V][6];
  bool lw[V], rw[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const long long pos = pos0 + v;
    lw[v] = WALLS && pos == 0;
    rw[v] = WALLS && pos == N - 1;
    long long lp = pos;
    if (!WALLS) {
      if (lp < 0 || lp >= N) { lp %= N; if (lp < 0) lp += N; }
    } else {
      lp = lp < 0 ? 0 : (lp >= N ? N - 1 : lp);
    }
    const double* src = in + off + lp;
    const bool ok = in_bounds(lp, N) && in_bounds(off + lp, plane);
#pragma unroll
    for (int i = 0; i < 6; ++i) f[v][i] = to_df(ok ? src[i * plane] : 0.0);
  }

  for (int k = 0; k < K; ++k) {
    NodeS<df> m[V];
#pragma unroll
    for (int v = 0; v < V; ++v) node_state_s(f[v], c, m_s0h, m[v]);
    df uL = shfl_up(m[V - 1].u), TL = shfl_up(m[V - 1].th);
    df uR = shfl_down(m[0].u), TR = shfl_down(m[0].th);
    if (lane == 31) { e_ut[warp][0] = m[V - 1].u; e_ut[warp][1] = m[V - 1].th; }
    if (lane == 0) { e_ut[warp][2] = m[0].u; e_ut[warp][3] = m[0].th; }
    __syncthreads();
    if (lane == 0 && warp > 0 && in_bounds(warp - 1, NW)) { uL = e_ut[warp - 1][0]; TL = e_ut[warp - 1][1]; }
    if (lane == 31 && warp < NW - 1 && in_bounds(warp + 1, NW)) { uR = e_ut[warp + 1][2]; TR = e_ut[warp + 1][3]; }
    // (In the outermost nodes of the tile these are stand-ins; those nodes are never stored.)

    df fs[V][6];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      df ul = v > 0 ? m[v - 1].u : uL, Tl = v > 0 ? m[v - 1].th : TL;
      df ur = v < V - 1 ? m[v + 1].u : uR, Tr = v < V - 1 ? m[v + 1].th : TR;
      if (lw[v]) { ul = neg(m[v].u); Tl = m[v].th; }
      if (rw[v]) { ur = neg(m[v].u); Tr = m[v].th; }
      node_collide_s(m[v], ul, ur, Tl, Tr, s_e, s_psi, s_eps, q_src, s0h, c, fs[v], le0, lp0, lq0);
    }
    // (viii) streaming: pull f+, g+ from the left neighbour and f-, g- from the right one.
    df fpL = shfl_up(fs[V - 1][1]), gpL = shfl_up(fs[V - 1][4]);
    df fmR = shfl_down(fs[0][2]), gmR = shfl_down(fs[0][5]);
    if (lane == 31) { e_f[warp][0] = fs[V - 1][1]; e_f[warp][1] = fs[V - 1][4]; }
    if (lane == 0) { e_f[warp][2] = fs[0][2]; e_f[warp][3] = fs[0][5]; }
    __syncthreads();
    if (lane == 0 && warp > 0 && in_bounds(warp - 1, NW)) { fpL = e_f[warp - 1][0]; gpL = e_f[warp - 1][1]; }
    if (lane == 31 && warp < NW - 1 && in_bounds(warp + 1, NW)) { fmR = e_f[warp + 1][2]; gmR = e_f[warp + 1][3]; }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      f[v][0] = fs[v][0];
      f[v][3] = fs[v][3];
      f[v][1] = lw[v] ? fs[v][2] : (v > 0 ? fs[v - 1][1] : fpL);
      f[v][4] = lw[v] ? fs[v][5] : (v > 0 ? fs[v - 1][4] : gpL);
      f[v][2] = rw[v] ? fs[v][1] : (v < V - 1 ? fs[v + 1][2] : fmR);
      f[v][5] = rw[v] ? fs[v][4] : (v < V - 1 ? fs[v + 1][5] : gmR);
    }
  }

#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int local = threadIdx.x * V + v;
    const long long pos = pos0 + v;
    if (local >= halo && local < halo + bout && pos < N && in_bounds(pos, N) && in_bounds(off + pos, plane)) {
      double* dst = out + off + pos;
#pragma unroll
      for (int i = 0; i < 6; ++i) dst[i * plane] = to_double(f[v][i]);
    }
  }
}

// The same tile update with two nodes per df2 lane (V = 2 or 4 nodes per thread), so that the
// double-float arithmetic runs on Blackwell's paired FP32 instructions. Lane l of a thread holds nodes
// 2l (x) and 2l + 1 (y). Every lane of a df2 operation is the FP32 operation sequence of the scalar df
// one, so the states equal those of the one-node-per-thread kernel bit for bit.
template <int NT, int V, bool WALLS>
__device__ __forceinline__ void tile_body_df2(const double* __restrict__ in, double* __restrict__ out,
                                              long long plane, const LatDev& d, long long start, int K,
                                              const Consts<df2>& c, df (*e_ut)[4], df (*e_f)[4]) {
  constexpr int NW = NT / 32, NL = V / 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int halo = 2 * K;
  const int bout = NT * V - 2 * halo;
  const long long off = d.offset, N = d.n;
  const auto par = [&](int i) { return df2{make_float2(d.f32[i], d.f32[i]), make_float2(d.f32lo[i], d.f32lo[i])}; };
  const df2 s_e = par(0), s_psi = par(1), s_eps = par(2), q_src = par(3), s0h = par(4);
  const df2 m_s0h{p_neg(s0h.hi), p_neg(s0h.lo)};
  const df2 le0 = par(5), lp0 = par(6), lq0 = par(7);
  const long long pos0 = start - halo + (long long)threadIdx.x * V;

  df2 f[NL][6];
  bool lw[V], rw[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const long long pos = pos0 + v;
    lw[v] = WALLS && pos == 0;
    rw[v] = WALLS && pos == N - 1;
  }
  // A lane pair holds two consecutive nodes, so where the thread's V nodes lie inside the lattice at
  // an even place of even planes (a 16-byte-aligned buffer) each pair moves as one double2, loaded
  // and stored; lattice ends, odd offsets of a batch and odd halos take the per-node path.
  const auto vec_at = [&](const double* base) {
    return (((off + pos0) | plane) & 1) == 0 && pos0 >= 0 && pos0 + V <= N &&
           (reinterpret_cast<unsigned long long>(base) & 15) == 0 && in_bounds(pos0 + V - 1, N) &&
           in_bounds(off + pos0 + V - 1, plane);
  };
  if (vec_at(in)) {
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const double2 x = *reinterpret_cast<const double2*>(in + off + pos0 + 2 * l + i * plane);
        df2_set(f[l][i], 0, to_df(x.x));
        df2_set(f[l][i], 1, to_df(x.y));
      }
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      long long lp = pos0 + v;
      if (!WALLS) {
        if (lp < 0 || lp >= N) { lp %= N; if (lp < 0) lp += N; }
      } else {
        lp = lp < 0 ? 0 : (lp >= N ? N - 1 : lp);
      }
      const double* src = in + off + lp;
      const bool ok = in_bounds(lp, N) && in_bounds(off + lp, plane);
#pragma unroll
      for (int i = 0; i < 6; ++i) df2_set(f[v >> 1][i], v & 1, to_df(ok ? src[i * plane] : 0.0));
    }
  }

  for (int k = 0; k < K; ++k) {
    NodeS<df2> m[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) node_state_s(f[l], c, m_s0h, m[l]);
    df uL = shfl_up(df2_get(m[NL - 1].u, 1)), TL = shfl_up(df2_get(m[NL - 1].th, 1));
    df uR = shfl_down(df2_get(m[0].u, 0)), TR = shfl_down(df2_get(m[0].th, 0));
    if (lane == 31) { e_ut[warp][0] = df2_get(m[NL - 1].u, 1); e_ut[warp][1] = df2_get(m[NL - 1].th, 1); }
    if (lane == 0) { e_ut[warp][2] = df2_get(m[0].u, 0); e_ut[warp][3] = df2_get(m[0].th, 0); }
    __syncthreads();
    if (lane == 0 && warp > 0 && in_bounds(warp - 1, NW)) { uL = e_ut[warp - 1][0]; TL = e_ut[warp - 1][1]; }
    if (lane == 31 && warp < NW - 1 && in_bounds(warp + 1, NW)) { uR = e_ut[warp + 1][2]; TR = e_ut[warp + 1][3]; }
    // (In the outermost nodes of the tile these are stand-ins; those nodes are never stored.)

    df2 fs[NL][6];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const df ux = df2_get(m[l].u, 0), uy = df2_get(m[l].u, 1);
      const df tx = df2_get(m[l].th, 0), ty = df2_get(m[l].th, 1);
      df2 ul = df2_of(l > 0 ? df2_get(m[l - 1].u, 1) : uL, ux);
      df2 Tl = df2_of(l > 0 ? df2_get(m[l - 1].th, 1) : TL, tx);
      df2 ur = df2_of(uy, l < NL - 1 ? df2_get(m[l + 1].u, 0) : uR);
      df2 Tr = df2_of(ty, l < NL - 1 ? df2_get(m[l + 1].th, 0) : TR);
      if (lw[2 * l]) { df2_set(ul, 0, neg(ux)); df2_set(Tl, 0, tx); }
      if (lw[2 * l + 1]) { df2_set(ul, 1, neg(uy)); df2_set(Tl, 1, ty); }
      if (rw[2 * l]) { df2_set(ur, 0, neg(ux)); df2_set(Tr, 0, tx); }
      if (rw[2 * l + 1]) { df2_set(ur, 1, neg(uy)); df2_set(Tr, 1, ty); }
      node_collide_s(m[l], ul, ur, Tl, Tr, s_e, s_psi, s_eps, q_src, s0h, c, fs[l], le0, lp0, lq0);
    }
    // (viii) streaming: pull f+, g+ from the left neighbour and f-, g- from the right one.
    df fpL = shfl_up(df2_get(fs[NL - 1][1], 1)), gpL = shfl_up(df2_get(fs[NL - 1][4], 1));
    df fmR = shfl_down(df2_get(fs[0][2], 0)), gmR = shfl_down(df2_get(fs[0][5], 0));
    if (lane == 31) { e_f[warp][0] = df2_get(fs[NL - 1][1], 1); e_f[warp][1] = df2_get(fs[NL - 1][4], 1); }
    if (lane == 0) { e_f[warp][2] = df2_get(fs[0][2], 0); e_f[warp][3] = df2_get(fs[0][5], 0); }
    __syncthreads();
    if (lane == 0 && warp > 0 && in_bounds(warp - 1, NW)) { fpL = e_f[warp - 1][0]; gpL = e_f[warp - 1][1]; }
    if (lane == 31 && warp < NW - 1 && in_bounds(warp + 1, NW)) { fmR = e_f[warp + 1][2]; gmR = e_f[warp + 1][3]; }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      f[l][0] = fs[l][0];
      f[l][3] = fs[l][3];
      // f+, g+ from the left node; f-, g- from the right node; walls reflect their own.
      const df fpx = l > 0 ? df2_get(fs[l - 1][1], 1) : fpL, gpx = l > 0 ? df2_get(fs[l - 1][4], 1) : gpL;
      const df fmy = l < NL - 1 ? df2_get(fs[l + 1][2], 0) : fmR, gmy = l < NL - 1 ? df2_get(fs[l + 1][5], 0) : gmR;
      f[l][1] = df2_of(lw[2 * l] ? df2_get(fs[l][2], 0) : fpx, lw[2 * l + 1] ? df2_get(fs[l][2], 1) : df2_get(fs[l][1], 0));
      f[l][4] = df2_of(lw[2 * l] ? df2_get(fs[l][5], 0) : gpx, lw[2 * l + 1] ? df2_get(fs[l][5], 1) : df2_get(fs[l][4], 0));
      f[l][2] = df2_of(rw[2 * l] ? df2_get(fs[l][1], 0) : df2_get(fs[l][2], 1), rw[2 * l + 1] ? df2_get(fs[l][1], 1) : fmy);
      f[l][5] = df2_of(rw[2 * l] ? df2_get(fs[l][4], 0) : df2_get(fs[l][5], 1), rw[2 * l + 1] ? df2_get(fs[l][4], 1) : gmy);
    }
  }

  const int local0 = threadIdx.x * V;
  if (local0 >= halo && local0 + V <= halo + bout && vec_at(out)) {
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
      for (int i = 0; i < 6; ++i)
        *reinterpret_cast<double2*>(out + off + pos0 + 2 * l + i * plane) =
            make_double2(to_double(df2_get(f[l][i], 0)), to_double(df2_get(f[l][i], 1)));
    return;
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int local = local0 + v;
    const long long pos = pos0 + v;
    if (local >= halo && local < halo + bout && pos < N && in_bounds(pos, N) && in_bounds(off + pos, plane)) {
      double* dst = out + off + pos;
#pragma unroll
      for (int i = 0; i < 6; ++i) dst[i * plane] = to_double(df2_get(f[v >> 1][i], v & 1));
    }
  }
}

template <int NT, int V>
__global__ void __launch_bounds__(NT) step_tiles_df2_kernel(const double* __restrict__ in, double* __restrict__ out,
                                                            long long plane, const LatDev* __restrict__ lat,
                                                            const int* __restrict__ tile_lat, int B, long long ntiles,
                                                            int K, Consts<df2> c) {
  __shared__ df e_ut[NT / 32][4];
  __shared__ df e_f[NT / 32][4];
  const long long bout = NT * V - 4 * K;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int L = B > 1 ? tile_lat[tile] : 0;
    if (!in_bounds(L, B)) continue;
    const LatDev d = lat[L];
    if (d.bc == 0) tile_body_df2<NT, V, false>(in, out, plane, d, (tile - d.tile0) * bout, K, c, e_ut, e_f);
    else tile_body_df2<NT, V, true>(in, out, plane, d, (tile - d.tile0) * bout, K, c, e_ut, e_f);
    __syncthreads();  // the next tile rewrites the edge buffers
  }
}

template <int NT, int V>
__global__ void __launch_bounds__(NT) step_tiles_df_kernel(const double* __restrict__ in, double* __restrict__ out,
                                                           long long plane, const LatDev* __restrict__ lat,
                                                           const int* __restrict__ tile_lat, int B, long long ntiles,
                                                           int K, Consts<df> c) {
  __shared__ df e_ut[NT / 32][4];
  __shared__ df e_f[NT / 32][4];
  const long long bout = NT * V - 4 * K;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int L = B > 1 ? tile_lat[tile] : 0;
    if (!in_bounds(L, B)) continue;
    const LatDev d = lat[L];
    if (d.bc == 0) tile_body_df<NT, V, false>(in, out, plane, d, (tile - d.tile0) * bout, K, c, e_ut, e_f);
    else tile_body_df<NT, V, true>(in, out, plane, d, (tile - d.tile0) * bout, K, c, e_ut, e_f);
    __syncthreads();  // the next tile rewrites the edge buffers
  }
}

template <int NT, int V>
cudaError_t launch_df_nt_v(const double* in, double* out, long long plane, const LatDev* lat, const int* tile_lat,
                           int B, long long ntiles, int K, const Consts<df>& c, cudaStream_t st, long long grid) {
  if constexpr (V == 1) {
    step_tiles_df_kernel<NT, V><<<(unsigned)grid, NT, 0, st>>>(in, out, plane, lat, tile_lat, B, ntiles, K, c);
  } else {
    step_tiles_df2_kernel<NT, V><<<(unsigned)grid, NT, 0, st>>>(in, out, plane, lat, tile_lat, B, ntiles, K,
                                                                pair_consts(c));
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t bounds_record_df(unsigned long long out[3]) {
#ifdef LBM_DEBUG_BOUNDS
  return take_bounds_record(out);
#else
  out[0] = out[1] = out[2] = 0ULL;
  return cudaSuccess;
#endif
}

bool valid_df_config(int K, int NT, int V) {
  const bool nt_ok = NT == 128 || NT == 256 || NT == 512;
  const bool v_ok = V == 1 || V == 2 || V == 4;
  const bool k_ok = K == 1 || K == 2 || K == 4 || K == 8;
  return nt_ok && v_ok && k_ok && NT * V - 4 * K >= 32;
}

cudaError_t launch_step_tiles_df(const double* in, double* out, long long plane, const LatDev* lat,
                                 const int* tile_lat, int B, long long ntiles, int K, int NT, int V,
                                 const Consts<df>& c, cudaStream_t st, long long grid_cap) {
  if (ntiles <= 0) return cudaSuccess;
  long long grid = ntiles;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
#define DF_CASE(nt, v) \
  if (NT == nt && V == v) return launch_df_nt_v<nt, v>(in, out, plane, lat, tile_lat, B, ntiles, K, c, st, grid);
  DF_CASE(128, 1) DF_CASE(128, 2) DF_CASE(128, 4) DF_CASE(256, 1) DF_CASE(256, 2) DF_CASE(256, 4)
  DF_CASE(512, 1) DF_CASE(512, 2) DF_CASE(512, 4)
#undef DF_CASE
  return cudaErrorInvalidValue;
}

}  // namespace lbm
