// Fused collide-stream kernel of the D1Q3Q3 scheme (section 8, steps (i)-(viii)) with temporal
// blocking.
//
// A CTA of NT threads owns a tile of NT*V consecutive nodes of one lattice; thread t holds nodes
// t*V .. t*V + V - 1 in registers (structure-of-arrays loads of the six population planes). The
// tile advances K time steps without touching HBM and stores its NT*V - 4K interior nodes: the
// dependency radius is 2 per step (the source needs u and T of the neighbours; streaming moves one
// node), so 2K halo nodes on each side are recomputed and discarded.
//
// Per step: every node computes its moments, u and T; neighbours' u and T come from the same
// thread's registers, from the adjacent lane (warp shuffle) or, at warp edges, from two words of
// shared memory per warp. After the collision every node pulls its incoming moving populations
// (f+, g+ from the left, f-, g- from the right) the same way. f0 and g0 never move. A wall node
// (bounce-back) takes its own reflected population instead. Two CTA barriers per step (none in a
// one-warp tile, whose edges are the tile halo).
#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {

// Advances one tile K steps: reads `in`, writes the interior of the tile to `out`.
template <typename R, int NT, int V, bool WALLS>
__device__ __forceinline__ void tile_body(const R* in, R* out, long long plane, const LatDev& d, long long start,
                                          int K, const Consts<R>& c, R (*e_ut)[4], R (*e_f)[4]) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int halo = 2 * K;
  const int bout = NT * V - 2 * halo;
  const long long off = d.offset, N = d.n;
  const StepParams<R> P = step_params(d, R{});
  const R s_e = P.s_e, s_psi = P.s_psi, s_eps = P.s_eps, q_src = P.q_src, s0h = P.s0h;
  const R m_s0h = -s0h;
  const R le0 = P.lin_e0, lp0 = P.lin_p0, lq0 = P.lin_q0;
  const long long pos0 = start - halo + (long long)threadIdx.x * V;

  R f[V][6];
  bool lw[V], rw[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const long long pos = pos0 + v;
    lw[v] = WALLS && pos == 0;
    rw[v] = WALLS && pos == N - 1;
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    long long lp = pos0 + v;
    if (!WALLS) {
      if (lp < 0 || lp >= N) { lp %= N; if (lp < 0) lp += N; }
    } else {
      lp = lp < 0 ? 0 : (lp >= N ? N - 1 : lp);
    }
    const R* src = in + off + lp;
    const bool ok = in_bounds(lp, N) && in_bounds(off + lp, plane);
#pragma unroll
    for (int i = 0; i < 6; ++i) f[v][i] = ok ? src[i * plane] : R{};
  }

  for (int k = 0; k < K; ++k) {
    NodeS<R> m[V];
#pragma unroll
    for (int v = 0; v < V; ++v) node_state_s(f[v], c, m_s0h, m[v]);
    // u' and theta of the neighbours of the first and last node of this thread.
    R uL = __shfl_up_sync(0xffffffffu, m[V - 1].u, 1), TL = __shfl_up_sync(0xffffffffu, m[V - 1].th, 1);
    R uR = __shfl_down_sync(0xffffffffu, m[0].u, 1), TR = __shfl_down_sync(0xffffffffu, m[0].th, 1);
    if constexpr (NW > 1) {  // a one-warp tile has no warp edge inside it
      if (lane == 31) { e_ut[warp][0] = m[V - 1].u; e_ut[warp][1] = m[V - 1].th; }
      if (lane == 0) { e_ut[warp][2] = m[0].u; e_ut[warp][3] = m[0].th; }
      __syncthreads();
      if (lane == 0 && warp > 0 && in_bounds(warp - 1, NW)) { uL = e_ut[warp - 1][0]; TL = e_ut[warp - 1][1]; }
      if (lane == 31 && warp < NW - 1 && in_bounds(warp + 1, NW)) { uR = e_ut[warp + 1][2]; TR = e_ut[warp + 1][3]; }
    }
    // (In the outermost nodes of the tile these are stand-ins; those nodes are never stored.)

    R fs[V][6];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      R ul = v > 0 ? m[v - 1].u : uL, Tl = v > 0 ? m[v - 1].th : TL;
      R ur = v < V - 1 ? m[v + 1].u : uR, Tr = v < V - 1 ? m[v + 1].th : TR;
      if (lw[v]) { ul = -m[v].u; Tl = m[v].th; }
      if (rw[v]) { ur = -m[v].u; Tr = m[v].th; }
      node_collide_s(m[v], ul, ur, Tl, Tr, s_e, s_psi, s_eps, q_src, s0h, c, fs[v], le0, lp0, lq0);
    }
    // (viii) streaming: pull f+, g+ from the left neighbour and f-, g- from the right one.
    R fpL = __shfl_up_sync(0xffffffffu, fs[V - 1][1], 1), gpL = __shfl_up_sync(0xffffffffu, fs[V - 1][4], 1);
    R fmR = __shfl_down_sync(0xffffffffu, fs[0][2], 1), gmR = __shfl_down_sync(0xffffffffu, fs[0][5], 1);
    if constexpr (NW > 1) {
      if (lane == 31) { e_f[warp][0] = fs[V - 1][1]; e_f[warp][1] = fs[V - 1][4]; }
      if (lane == 0) { e_f[warp][2] = fs[0][2]; e_f[warp][3] = fs[0][5]; }
      __syncthreads();
      if (lane == 0 && warp > 0 && in_bounds(warp - 1, NW)) { fpL = e_f[warp - 1][0]; gpL = e_f[warp - 1][1]; }
      if (lane == 31 && warp < NW - 1 && in_bounds(warp + 1, NW)) { fmR = e_f[warp + 1][2]; gmR = e_f[warp + 1][3]; }
    }
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
      R* dst = out + off + pos;
#pragma unroll
      for (int i = 0; i < 6; ++i) dst[i * plane] = f[v][i];
    }
  }
}

// The same tile update for FP32 with two nodes per float2 lane (V = 2 or 4 nodes per thread), so
// that the node arithmetic runs on Blackwell's paired FP32 instructions. With NL = V/2 lanes, lane l
// of a thread holds nodes l (x) and l + NL (y): the left neighbours of lane l > 0 are then exactly
// lane l - 1 and the right neighbours of lane l < NL - 1 exactly lane l + 1, so only the two outer
// lanes assemble a neighbour pair from two registers.
//
// With four nodes per thread (GHOST) the warps of a tile overlap instead of exchanging their edges
// every step: warp w holds the 128 nodes starting at w * (128 - 2G), the first and last G = 4 of which
// are ghost copies of the neighbouring warps' nodes. A warp steps on shuffles alone; its outer G nodes
// lose validity at 2 nodes per step (the step's dependency radius), and every P = G / 2 steps they are
// refreshed from the neighbours' valid nodes (lane 30 of warp w - 1 and lane 1 of warp w + 1) through
// shared memory, behind one CTA barrier: K/P - 1 barriers per tile instead of two per step, for
// 2G / 128 = 6 % more node updates. A tile then spans kTileSpan(NT, V) = NT V - 2G (NT/32 - 1) nodes.
template <int NT, int V, bool WALLS, bool FULL>
__device__ __forceinline__ void tile_body_packed(const float* in, float* out, long long plane, const LatDev& d,
                                                 long long start, int K, const Consts<float2>& c,
                                                 float (*e_ut)[4], float (*e_f)[4], float2* gbuf, int tpar) {
  constexpr int NW = NT / 32, NL = V / 2;
  constexpr bool GHOST = V == 4 && NW > 1;
  constexpr int G = kGhost, P = kGhost / 2, WS = 32 * V - 2 * G;  // ghosts per side, refresh period, warp stride
  constexpr int SPAN = (int)tile_span(NT, V, true);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int halo = 2 * K;
  const int bout = SPAN - 2 * halo;
  const long long off = d.offset, N = d.n;
  const StepParams<float> P_ = step_params(d, 0.0f);
  const float2 s_e = make_float2(P_.s_e, P_.s_e), s_psi = make_float2(P_.s_psi, P_.s_psi);
  const float2 s_eps = make_float2(P_.s_eps, P_.s_eps), q_src = make_float2(P_.q_src, P_.q_src);
  const float2 s0h = make_float2(P_.s0h, P_.s0h), m_s0h = make_float2(-P_.s0h, -P_.s0h);
  const float2 le0 = make_float2(P_.lin_e0, P_.lin_e0), lp0 = make_float2(P_.lin_p0, P_.lin_p0);
  const float2 lq0 = make_float2(P_.lin_q0, P_.lin_q0);
  // First node of this thread within the tile span.
  const int local0 = GHOST ? warp * WS + lane * V : (int)threadIdx.x * V;
  const long long pos0 = start - halo + local0;
  // Ghost nodes of a warp that has a neighbour on that side: neither refreshed nor stored by this warp.
  const bool ghost_lane = GHOST && ((lane == 0 && warp > 0) || (lane == 31 && warp < NW - 1));

  // Node v of the thread sits in lane v % NL, half v / NL.
  float2 f[NL][6];
  bool lw[V], rw[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const long long pos = pos0 + v;
    lw[v] = WALLS && pos == 0;
    rw[v] = WALLS && pos == N - 1;
  }
  // A thread whose nodes lie inside the lattice loads them without the per-node wrap or wall clamp.
  if (pos0 >= 0 && pos0 + V <= N && in_bounds(off + pos0 + V - 1, plane)) {
    const float* src = in + off + pos0;
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const float x = src[v + i * plane];
        if (v >= NL) f[v - NL][i].y = x; else f[v][i].x = x;
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
      const float* src = in + off + lp;
      const bool ok = in_bounds(lp, N) && in_bounds(off + lp, plane);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const float x = ok ? src[i * plane] : 0.0f;
        if (v >= NL) f[v - NL][i].y = x; else f[v][i].x = x;
      }
    }
  }

  // Ghost exchange buffer gbuf (GS float2 slots), alternating by refresh: [side][parity][warp][lane of the
  // thread][population], side 0 = lane 30's nodes for warp + 1, side 1 = lane 1's nodes for warp - 1.
  const auto gslot = [&](int side, int par, int w, int l, int i) { return (((side * 2 + par) * NW + w) * NL + l) * 6 + i; };
  constexpr int GS = GHOST ? 2 * 2 * NW * NL * 6 : 1;

  for (int k = 0; k < K; ++k) {
    if constexpr (GHOST) {
      if (k > 0 && k % P == 0) {
        // Buffers alternate by refresh (the barrier of every refresh separates two uses of a buffer).
        // A tile of K = 8 or 4 steps has an odd number of refreshes (3 or 1), so offsetting the parity
        // by tpar, the parity of the tile's place among tiles a CTA runs back to back without a CTA
        // barrier between them (the persistent kernel's work units), keeps the alternation across
        // tiles: the first refresh of a tile never rewrites the buffer the previous tile's last refresh
        // is still being read from.
        const int par = ((k / P) + tpar) & 1;
        // Lanes 30 (for warp + 1) and 1 (for warp - 1) publish in one pass and lanes 0 and 31 take in
        // one pass, the twelve float2 of a thread as six 16-byte words (a thread's slots start at a
        // multiple of 12 float2 of the 16-byte-aligned buffer).
        if ((lane == 30 && warp < NW - 1) || (lane == 1 && warp > 0)) {
          const int base = gslot(lane == 1 ? 1 : 0, par, warp, 0, 0);
#pragma unroll
          for (int l = 0; l < NL; ++l)
#pragma unroll
            for (int i = 0; i < 6; i += 2)
              if (in_bounds(base + l * 6 + i + 1, GS))
                reinterpret_cast<float4*>(gbuf + base + l * 6 + i)[0] =
                    make_float4(f[l][i].x, f[l][i].y, f[l][i + 1].x, f[l][i + 1].y);
        }
        __syncthreads();
        if ((lane == 0 && warp > 0) || (lane == 31 && warp < NW - 1)) {
          const int src = lane == 0 ? warp - 1 : warp + 1;
          const int base = gslot(lane == 0 ? 0 : 1, par, src, 0, 0);
#pragma unroll
          for (int l = 0; l < NL; ++l)
#pragma unroll
            for (int i = 0; i < 6; i += 2)
              if (in_bounds(src, NW) && in_bounds(base + l * 6 + i + 1, GS)) {
                const float4 x = reinterpret_cast<const float4*>(gbuf + base + l * 6 + i)[0];
                f[l][i] = make_float2(x.x, x.y);
                f[l][i + 1] = make_float2(x.z, x.w);
              }
        }
      }
    }
    NodeS<float2> m[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {  // series first; a pair with a node outside their ranges is redone
      if (!node_state_s<float2, true, FULL>(f[l], c, m_s0h, m[l])) node_state_s<float2, false, FULL>(f[l], c, m_s0h, m[l]);
    }
    // Node V - 1 is lane NL - 1, half y; node 0 is lane 0, half x. (At the outer edges of a warp these
    // are stand-ins: in a ghost tile those nodes are ghosts, refreshed before they are needed; otherwise
    // they come from the neighbouring warp below, or they lie in the tile halo and are never stored.)
    float uL = __shfl_up_sync(0xffffffffu, m[NL - 1].u.y, 1), TL = __shfl_up_sync(0xffffffffu, m[NL - 1].th.y, 1);
    float uR = __shfl_down_sync(0xffffffffu, m[0].u.x, 1), TR = __shfl_down_sync(0xffffffffu, m[0].th.x, 1);
    if constexpr (NW > 1 && !GHOST) {
      if (lane == 31) { e_ut[warp][0] = m[NL - 1].u.y; e_ut[warp][1] = m[NL - 1].th.y; }
      if (lane == 0) { e_ut[warp][2] = m[0].u.x; e_ut[warp][3] = m[0].th.x; }
      __syncthreads();
      if (lane == 0 && warp > 0 && in_bounds(warp - 1, NW)) { uL = e_ut[warp - 1][0]; TL = e_ut[warp - 1][1]; }
      if (lane == 31 && warp < NW - 1 && in_bounds(warp + 1, NW)) { uR = e_ut[warp + 1][2]; TR = e_ut[warp + 1][3]; }
    }

    float2 fs[NL][6];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      float2 ul = l > 0 ? m[l - 1].u : make_float2(uL, m[NL - 1].u.x);
      float2 Tl = l > 0 ? m[l - 1].th : make_float2(TL, m[NL - 1].th.x);
      float2 ur = l < NL - 1 ? m[l + 1].u : make_float2(m[0].u.y, uR);
      float2 Tr = l < NL - 1 ? m[l + 1].th : make_float2(m[0].th.y, TR);
      if (lw[l]) { ul.x = -m[l].u.x; Tl.x = m[l].th.x; }
      if (lw[l + NL]) { ul.y = -m[l].u.y; Tl.y = m[l].th.y; }
      if (rw[l]) { ur.x = -m[l].u.x; Tr.x = m[l].th.x; }
      if (rw[l + NL]) { ur.y = -m[l].u.y; Tr.y = m[l].th.y; }
      node_collide_s<float2, FULL>(m[l], ul, ur, Tl, Tr, s_e, s_psi, s_eps, q_src, s0h, c, fs[l], le0, lp0, lq0);
    }
    float fpL = __shfl_up_sync(0xffffffffu, fs[NL - 1][1].y, 1), gpL = __shfl_up_sync(0xffffffffu, fs[NL - 1][4].y, 1);
    float fmR = __shfl_down_sync(0xffffffffu, fs[0][2].x, 1), gmR = __shfl_down_sync(0xffffffffu, fs[0][5].x, 1);
    if constexpr (NW > 1 && !GHOST) {
      if (lane == 31) { e_f[warp][0] = fs[NL - 1][1].y; e_f[warp][1] = fs[NL - 1][4].y; }
      if (lane == 0) { e_f[warp][2] = fs[0][2].x; e_f[warp][3] = fs[0][5].x; }
      __syncthreads();
      if (lane == 0 && warp > 0 && in_bounds(warp - 1, NW)) { fpL = e_f[warp - 1][0]; gpL = e_f[warp - 1][1]; }
      if (lane == 31 && warp < NW - 1 && in_bounds(warp + 1, NW)) { fmR = e_f[warp + 1][2]; gmR = e_f[warp + 1][3]; }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      // f+, g+ from the left node; f-, g- from the right node; walls reflect their own.
      float2 fp = l > 0 ? fs[l - 1][1] : make_float2(fpL, fs[NL - 1][1].x);
      float2 gp = l > 0 ? fs[l - 1][4] : make_float2(gpL, fs[NL - 1][4].x);
      float2 fm_ = l < NL - 1 ? fs[l + 1][2] : make_float2(fs[0][2].y, fmR);
      float2 gm = l < NL - 1 ? fs[l + 1][5] : make_float2(fs[0][5].y, gmR);
      if (lw[l]) { fp.x = fs[l][2].x; gp.x = fs[l][5].x; }
      if (lw[l + NL]) { fp.y = fs[l][2].y; gp.y = fs[l][5].y; }
      if (rw[l]) { fm_.x = fs[l][1].x; gm.x = fs[l][4].x; }
      if (rw[l + NL]) { fm_.y = fs[l][1].y; gm.y = fs[l][4].y; }
      f[l][0] = fs[l][0];
      f[l][3] = fs[l][3];
      f[l][1] = fp;
      f[l][4] = gp;
      f[l][2] = fm_;
      f[l][5] = gm;
    }
  }

  if (ghost_lane) return;
  // A thread whose V nodes are all stored and lie at a V-node-aligned place of V-node-aligned planes
  // stores each population as one V-wide vector (float4 / float2): one store instruction per plane
  // instead of V, whole 32-byte sectors per warp. Threads at lattice ends, in misaligned lattices of a
  // batch and at depths whose halo is not a multiple of V store node by node. (Loads stay per node:
  // the vector loads measured slower, their unpacking into the lane pairs costing registers.)
  if (local0 >= halo && local0 + V <= halo + bout && (((off + pos0) | plane) & (V - 1)) == 0 && pos0 >= 0 &&
      pos0 + V <= N && (reinterpret_cast<unsigned long long>(out) & (sizeof(float) * V - 1)) == 0 &&
      in_bounds(pos0 + V - 1, N) && in_bounds(off + pos0 + V - 1, plane)) {
    const long long g0 = off + pos0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if constexpr (V == 4) {
        *reinterpret_cast<float4*>(out + g0 + i * plane) = make_float4(f[0][i].x, f[1][i].x, f[0][i].y, f[1][i].y);
      } else {
        *reinterpret_cast<float2*>(out + g0 + i * plane) = f[0][i];
      }
    }
    return;
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int local = local0 + v;
    const long long pos = pos0 + v;
    if (local >= halo && local < halo + bout && pos < N && in_bounds(pos, N) && in_bounds(off + pos, plane)) {
      float* dst = out + off + pos;
#pragma unroll
      for (int i = 0; i < 6; ++i) dst[i * plane] = v >= NL ? f[v - NL][i].y : f[v][i].x;
    }
  }
}

__device__ __forceinline__ int lattice_of_tile(const LatDev* lat, int B, long long tile) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {  // last lattice whose first tile is <= tile
    const int mid = (lo + hi + 1) >> 1;
    if (lat[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// FP32 with two or four nodes per thread runs on paired lanes; everything else on scalar lanes.
template <typename R, int V>
struct Lanes {
  using type = R;
};
template <>
struct Lanes<float, 2> {
  using type = float2;
};
template <>
struct Lanes<float, 4> {
  using type = float2;
};

// float2 slots of the ghost exchange buffer of a tile (tile_body_packed), at least one.
template <typename R, int NT, int V>
struct GhostSlots {
  static constexpr int value = (sizeof(R) == 4 && V == 4 && NT > 32) ? 2 * 2 * (NT / 32) * (V / 2) * 6 : 1;
};

template <typename R, int NT, int V>
__device__ __forceinline__ void tile_update(const R* in, R* out, long long plane, const LatDev& d, long long start,
                                            int K, const Consts<typename Lanes<R, V>::type>& c, R (*e_ut)[4],
                                            R (*e_f)[4], float2* gbuf, int tpar) {
  // Periodic tiles take the wall-free path; bounce-back lattices the one with wall handling.
  if constexpr (std::is_same<typename Lanes<R, V>::type, float2>::value) {
    // The paper's scheme (nonlinear equilibria, entropy source) without per-node mode tests.
    const bool full = c.eq_mode == 0 && c.source_on;
    if (d.bc == 0) {
      if (full) tile_body_packed<NT, V, false, true>(in, out, plane, d, start, K, c, e_ut, e_f, gbuf, tpar);
      else tile_body_packed<NT, V, false, false>(in, out, plane, d, start, K, c, e_ut, e_f, gbuf, tpar);
    } else {
      if (full) tile_body_packed<NT, V, true, true>(in, out, plane, d, start, K, c, e_ut, e_f, gbuf, tpar);
      else tile_body_packed<NT, V, true, false>(in, out, plane, d, start, K, c, e_ut, e_f, gbuf, tpar);
    }
  } else {
    if (d.bc == 0) tile_body<R, NT, V, false>(in, out, plane, d, start, K, c, e_ut, e_f);
    else tile_body<R, NT, V, true>(in, out, plane, d, start, K, c, e_ut, e_f);
  }
}

// Lattice of every tile (one binary search per tile per configuration instead of per launch).
__global__ void tile_map_kernel(const LatDev* __restrict__ lat, int B, long long ntiles, int* __restrict__ map) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < ntiles) map[t] = lattice_of_tile(lat, B, t);
}

cudaError_t launch_tile_map(const LatDev* lat, int B, long long ntiles, int* map, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  tile_map_kernel<<<(unsigned)((ntiles + 255) / 256), 256, 0, st>>>(lat, B, ntiles, map);
  return cudaGetLastError();
}

// Minimum resident CTAs per SM for __launch_bounds__. 128 threads of four FP32 nodes: eight, i.e. at
// most 64 registers (measured faster than the 80-90 the compiler picks otherwise); one-warp tiles of
// four nodes likewise 32 warps per SM. A minimum of 0 leaves the other instances to the compiler's own
// choice (an explicit 1 lets it take far more registers).
#ifndef LBM_MINCTAS_F32_128x4
#define LBM_MINCTAS_F32_128x4 8
#endif
#ifndef LBM_MINCTAS_F32_64x4
#define LBM_MINCTAS_F32_64x4 0
#endif
template <typename R, int NT, int V>
struct MinCtas {
  static constexpr int value = sizeof(R) != 4 ? 0
                               : (NT == 128 && V == 4) ? LBM_MINCTAS_F32_128x4
                               : (NT == 64 && V == 4) ? LBM_MINCTAS_F32_64x4
                               : (NT == 32 && V == 4) ? 32
                               : 0;
};

template <typename R, int NT, int V>
__global__ void __launch_bounds__(NT, MinCtas<R, NT, V>::value) step_tiles_kernel(const R* __restrict__ in, R* __restrict__ out,
                                                        long long plane, const LatDev* __restrict__ lat,
                                                        const int* __restrict__ tile_lat, int B, long long ntiles,
                                                        int K, Consts<typename Lanes<R, V>::type> c) {
  __shared__ R e_ut[NT / 32][4];
  __shared__ R e_f[NT / 32][4];
  __shared__ __align__(16) float2 gbuf[GhostSlots<R, NT, V>::value];
  const long long bout = tile_span(NT, V, sizeof(R) == 4) - 4 * K;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int L = B > 1 ? tile_lat[tile] : 0;
    if (in_bounds(L, B)) {
      const LatDev d = lat[L];
      tile_update<R, NT, V>(in, out, plane, d, (tile - d.tile0) * bout, K, c, e_ut, e_f, gbuf, 0);
    }
    // A CTA that has another tile (a grid smaller than the tile count) waits for all its warps first:
    // the shared edge and ghost buffers are reused.
    if (tile + gridDim.x < ntiles) __syncthreads();
  }
}

template <typename R, int NT, int V>
static cudaError_t launch_nt_v(const R* in, R* out, long long plane, const LatDev* lat, const int* tile_lat, int B,
                               long long ntiles, int K, const ConstSet<R>& cs, cudaStream_t st, long long grid) {
  step_tiles_kernel<R, NT, V><<<(unsigned)grid, NT, 0, st>>>(in, out, plane, lat, tile_lat, B, ntiles, K,
                                                              cs.template get<typename Lanes<R, V>::type>());
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_step_tiles(const R* in, R* out, long long plane, const LatDev* lat, const int* tile_lat, int B,
                              long long ntiles, int K, int NT, int V, const ConstSet<R>& c, cudaStream_t st,
                              long long grid_cap) {
  if (ntiles <= 0) return cudaSuccess;
  long long grid = ntiles;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
#define LBM_CASE(nt, v) \
  if (NT == nt && V == v) return launch_nt_v<R, nt, v>(in, out, plane, lat, tile_lat, B, ntiles, K, c, st, grid);
  LBM_CASE(128, 1) LBM_CASE(128, 2) LBM_CASE(128, 4)
  LBM_CASE(256, 1) LBM_CASE(256, 2) LBM_CASE(256, 4)
  LBM_CASE(512, 1) LBM_CASE(512, 2) LBM_CASE(512, 4)
  LBM_CASE(1024, 1)
  if constexpr (sizeof(R) == 4) {
    LBM_CASE(1024, 2)
    LBM_CASE(32, 4) LBM_CASE(64, 4)
  }
#undef LBM_CASE
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------------------------
// Persistent launch over all time blocks. A work unit is (time block b of K steps, tile i); units
// are claimed from a global counter in increasing order u = b * ntiles + i. Unit (b, i) reads buffer
// b & 1 and writes buffer (b + 1) & 1, so it may start once tiles i - 1, i, i + 1 of its lattice have
// finished block b - 1: that covers both its halo reads and the reads of the region it overwrites.
// Every unit waits only on units with a smaller number, which were claimed earlier by CTAs that are
// running, so the launch cannot deadlock whatever the number of resident CTAs. Each wait is bounded:
// after spin_limit polls it sets the status word and the CTA stops; other CTAs see the status and
// stop too, so the kernel always ends.

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename R, int NT, int V>
__global__ void __launch_bounds__(NT, MinCtas<R, NT, V>::value) persistent_kernel(R* buf0, R* buf1, long long plane,
                                                        const LatDev* __restrict__ lat,
                                                        const int* __restrict__ tile_lat, int B, long long ntiles,
                                                        int K, long long nblocks, PersistentCtl ctl,
                                                        Consts<typename Lanes<R, V>::type> c) {
  __shared__ R e_ut[NT / 32][4];
  __shared__ R e_f[NT / 32][4];
  __shared__ __align__(16) float2 gbuf[GhostSlots<R, NT, V>::value];
  __shared__ long long s_next;
  __shared__ int s_go;
  constexpr int U = kUnitTiles;  // tiles per work unit
  const long long nunits = (ntiles + U - 1) / U;
  const long long total = nblocks * nunits;
  const long long bout = tile_span(NT, V, sizeof(R) == 4) - 4 * K;
  if (threadIdx.x == 0) s_next = (long long)atomicAdd(ctl.counter, 1ULL);
  __syncthreads();
  for (;;) {
    const long long u = s_next;
    __syncthreads();  // every thread has read s_next before it is overwritten
    if (u >= total) break;
    const long long b = u / nunits, k = u % nunits;
    if (threadIdx.x == 0) s_next = (long long)atomicAdd(ctl.counter, 1ULL);  // claim ahead
    if (threadIdx.x < 32) {
      // Lane l checks tile k * U + l: its own unit and the units of its lattice neighbours
      // must have finished block b - 1.
      // Every exit of this loop is warp-uniform: the status word is read by lane 0 and broadcast.
      int go = __shfl_sync(0xffffffffu, threadIdx.x == 0 ? *((volatile int*)ctl.status) : 0, 0) == 0;
      if (go && b > 0) {
        long long uL = k, uR = k;
        const long long i = k * U + threadIdx.x;
        if ((int)threadIdx.x < U && i < ntiles && in_bounds(i, ntiles)) {
          int L = B > 1 ? tile_lat[i] : 0;
          if (!in_bounds(L, B)) L = 0;
          const long long t0 = lat[L].tile0;
          const long long nt = (L + 1 < B ? lat[L + 1].tile0 : ntiles) - t0;
          const bool periodic = lat[L].bc == 0;
          const long long left = i > t0 ? i - 1 : (periodic ? t0 + nt - 1 : i);
          const long long right = i < t0 + nt - 1 ? i + 1 : (periodic ? t0 : i);
          uL = left / U;
          uR = right / U;
        }
        long long spins = 0;
        long long uk = k;
        if (!in_bounds(uk, nunits) || !in_bounds(uL, nunits) || !in_bounds(uR, nunits)) uL = uR = uk = 0;
        for (;;) {
          const bool ready = ld_acquire_gpu(ctl.done + uk) >= b && ld_acquire_gpu(ctl.done + uL) >= b &&
                             ld_acquire_gpu(ctl.done + uR) >= b;
          if (__all_sync(0xffffffffu, ready)) break;
          const int st = __shfl_sync(0xffffffffu, threadIdx.x == 0 ? *((volatile int*)ctl.status) : 0, 0);
          if (st != 0) { go = 0; break; }
          if (++spins > ctl.spin_limit) {
            if (threadIdx.x == 0) atomicExch(ctl.status, 1);
            go = 0;
            break;
          }
          __nanosleep(100);
        }
        // The acquire loads above (each one a relaxed load followed by an acquire fence) and the CTA
        // barrier below order every thread's later (ordinary, L1-cached) loads of the tiles after the
        // neighbours' released writes.
      }
      if (threadIdx.x == 0) s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const bool withheld = (b == 0 && k == ctl.withhold);
    if (!withheld) {
      R* in = (b & 1) ? buf1 : buf0;
      R* out = (b & 1) ? buf0 : buf1;
      for (long long i = k * U; i < (k + 1) * U && i < ntiles; ++i) {
        const int L = B > 1 ? tile_lat[i] : 0;
        if (!in_bounds(L, B)) continue;
        const LatDev d = lat[L];
        tile_update<R, NT, V>(in, out, plane, d, (i - d.tile0) * bout, K, c, e_ut, e_f, gbuf, (int)(i & 1));
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && !withheld && in_bounds(k, nunits)) {
      // A release store is a release fence followed by the store: with the CTA barrier above it
      // publishes every thread's stores of the unit.
      st_release_gpu(ctl.done + k, (int)(b + 1));
    }
  }
}

template <typename R, int NT, int V>
static cudaError_t launch_persistent_nt_v(R* buf0, R* buf1, long long plane, const LatDev* lat, const int* tile_lat,
                                          int B, long long ntiles, int K, long long nblocks, const PersistentCtl& ctl,
                                          const ConstSet<R>& cs, cudaStream_t st) {
  const auto c = cs.template get<typename Lanes<R, V>::type>();
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel<R, NT, V>, NT, 0);
  long long grid = (long long)nsm * (per_sm > 0 ? per_sm : 1);
  const long long total = nblocks * ((ntiles + kUnitTiles - 1) / kUnitTiles);
  if (grid > total) grid = total;
  persistent_kernel<R, NT, V><<<(unsigned)grid, NT, 0, st>>>(buf0, buf1, plane, lat, tile_lat, B, ntiles, K, nblocks,
                                                              ctl, c);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_persistent(R* buf0, R* buf1, long long plane, const LatDev* lat, const int* tile_lat, int B,
                              long long ntiles, int K, int NT, int V, long long nblocks, const PersistentCtl& ctl,
                              const ConstSet<R>& c, cudaStream_t st) {
  if (ntiles <= 0 || nblocks <= 0) return cudaSuccess;
#define LBM_CASE(nt, v)       \
  if (NT == nt && V == v) \
    return launch_persistent_nt_v<R, nt, v>(buf0, buf1, plane, lat, tile_lat, B, ntiles, K, nblocks, ctl, c, st);
  LBM_CASE(128, 1) LBM_CASE(128, 2) LBM_CASE(128, 4)
  LBM_CASE(256, 1) LBM_CASE(256, 2) LBM_CASE(256, 4)
  LBM_CASE(512, 1) LBM_CASE(512, 2) LBM_CASE(512, 4)
  LBM_CASE(1024, 1)
  if constexpr (sizeof(R) == 4) {
    LBM_CASE(1024, 2)
    LBM_CASE(32, 4) LBM_CASE(64, 4)
  }
#undef LBM_CASE
  return cudaErrorInvalidValue;
}

template cudaError_t launch_persistent<float>(float*, float*, long long, const LatDev*, const int*, int, long long,
                                              int, int, int, long long, const PersistentCtl&, const ConstSet<float>&,
                                              cudaStream_t);
template cudaError_t launch_persistent<double>(double*, double*, long long, const LatDev*, const int*, int, long long,
                                               int, int, int, long long, const PersistentCtl&,
                                               const ConstSet<double>&, cudaStream_t);

cudaError_t bounds_record_step(unsigned long long out[3]) {
#ifdef LBM_DEBUG_BOUNDS
  return take_bounds_record(out);
#else
  out[0] = out[1] = out[2] = 0ULL;
  return cudaSuccess;
#endif
}

bool valid_tile_config(int K, int NT, int V, bool fp64) {
  const bool nt_ok = NT == 128 || NT == 256 || NT == 512 || NT == 1024;
  const bool v_ok = V == 1 || V == 2 || V == 4;
  const bool k_ok = K == 1 || K == 2 || K == 4 || K == 8;
  // 1024 x 4 is not instantiated; FP64 1024 x 2 would spill at the 64-register cap of 1024 threads.
  const bool size_ok = !(NT == 1024 && V == 4) && !(fp64 && NT == 1024 && V == 2);
  // FP32 only: one-warp and two-warp tiles of four nodes per thread (one-warp tiles exchange nothing
  // through shared memory and need no CTA barrier).
  const bool f32_extra = !fp64 && k_ok && V == 4 && (NT == 32 || NT == 64);
  return ((nt_ok && v_ok && k_ok && size_ok) || f32_extra) && tile_span(NT, V, !fp64) - 4 * K >= 32;
}

template cudaError_t launch_step_tiles<float>(const float*, float*, long long, const LatDev*, const int*, int,
                                              long long, int, int, int, const ConstSet<float>&, cudaStream_t,
                                              long long);
template cudaError_t launch_step_tiles<double>(const double*, double*, long long, const LatDev*, const int*, int,
                                               long long, int, int, int, const ConstSet<double>&, cudaStream_t,
                                               long long);

}  // namespace lbm
