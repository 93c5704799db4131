// Reverse mode (adjoint) of the D1Q3Q3 time step and of the equilibrium initialisation.
//
// One adjoint step maps a_{t+1} = dL/df(t+1) to a_t = dL/df(t) at the state f(t):
//   1. transpose of the streaming of eq. (iteration-d1q3q3): the adjoint of the post-collision
//      populations of node c is a0(c), a+(c+1), a-(c-1) (a wall node takes its own reflected one);
//   2. transpose of f* = M^{-1} m*, then of the relaxation (eq. relaxation-d1q3q3), the equilibria
//      (eqs. energie-equilibre, psi-equilibre, eq-energie-entropie-d1q3q3 in its polytropic form)
//      and the entropy source of eq. (NS-rho-J-zeta); the source of node c depends on u and T of
//      c - 1 and c + 1, so those adjoint contributions are scattered to the neighbours;
//   3. transpose of the equation of state (eq. gaz-parfait) and of m = M f (eq. M-d1q3q3).
// The dependency radius is 2 (as in the forward step). A launch runs K such steps on a tile after
// recomputing the K forward states it needs from the one state at the start of the block.
#include <atomic>
#include <type_traits>

#include "lbm_df.cuh"
#include "lbm_internal.cuh"

namespace lbm {

// Lanes: a thread holds W consecutive nodes in one lane value X (W = 1: X = double, float, or df,
// the double-float of lbm_df.cuh over FP64 storage; W = 2: X = float2, two nodes on Blackwell's paired
// FP32 instructions, or df2, two double-float nodes on them). R is the storage type.
template <typename X>
struct Lane {
  using R = X;
  static constexpr int W = 1;
};
template <>
struct Lane<float2> {
  using R = float;
  static constexpr int W = 2;
};
template <>
struct Lane<df> {
  using R = double;
  static constexpr int W = 1;
};
template <>
struct Lane<df2> {
  using R = double;
  static constexpr int W = 2;
};
__device__ __forceinline__ double lget(double x, int) { return x; }
__device__ __forceinline__ float lget(float x, int) { return x; }
__device__ __forceinline__ float lget(float2 x, int j) { return j ? x.y : x.x; }
__device__ __forceinline__ double lget(df x, int) { return to_double(x); }
__device__ __forceinline__ double lget(df2 x, int j) { return to_double(df2_get(x, j)); }
__device__ __forceinline__ void lset(double& x, int, double v) { x = v; }
__device__ __forceinline__ void lset(float& x, int, float v) { x = v; }
__device__ __forceinline__ void lset(float2& x, int j, float v) {
  if (j) x.y = v;
  else x.x = v;
}
__device__ __forceinline__ void lset(df& x, int, double v) { x = to_df(v); }
__device__ __forceinline__ void lset(df2& x, int j, double v) { df2_set(x, j, to_df(v)); }
template <typename X>
__device__ __forceinline__ X lit(double v) {
  if constexpr (std::is_same<X, df2>::value) {
    const df a = df_from_double_host(v);  // folded for constants
    return df2_of(a, a);
  } else if constexpr (Lane<X>::W == 2) {
    return make_float2((float)v, (float)v);
  } else if constexpr (std::is_same<X, df>::value) {
    return df_from_double_host(v);
  } else {
    return X(v);
  }
}
template <typename X>
__device__ __forceinline__ X lit_r(typename Lane<X>::R v) {
  if constexpr (std::is_same<X, df2>::value) {
    const df a = to_df(v);
    return df2_of(a, a);
  } else if constexpr (Lane<X>::W == 2) {
    return make_float2(v, v);
  } else if constexpr (std::is_same<X, df>::value) {
    return to_df(v);
  } else {
    return v;
  }
}
// Per-lane select: lane j takes a where b[j], else keeps x.
template <typename X>
__device__ __forceinline__ X sel(const bool (&b)[Lane<X>::W], X a, X x) {
  if constexpr (Lane<X>::W == 1) {
    return b[0] ? a : x;
  } else if constexpr (std::is_same<X, df2>::value) {
#pragma unroll
    for (int j = 0; j < 2; ++j)
      if (b[j]) df2_set(x, j, df2_get(a, j));
    return x;
  } else {
#pragma unroll
    for (int j = 0; j < Lane<X>::W; ++j)
      if (b[j]) lset(x, j, lget(a, j));
    return x;
  }
}

// Shared-memory exchange buffers of one CTA of NT threads, one lane value per thread (W nodes), so a
// thread's accesses are single 4- or 8-byte words (no bank conflicts).
template <typename X, int NT>
struct AdjShared {
  X su[NT], sT[NT];                      // forward u and T (u' and theta in the recomputation)
  X sfp[NT], sgp[NT], sfm[NT], sgm[NT];  // a+ (f, g) and a- (f, g) at t + 1; moving populations forward
  X sul[NT], sur[NT], sTl[NT], sTr[NT];  // source adjoints scattered to the neighbours
  double sg[2][NT / 32];
};

// Per-node flags of a thread's W nodes.
template <int W>
struct NodeFlags {
  bool lw[W], rw[W];    // left / right wall node (bounce-back)
  bool inactive[W];     // outside the lattice (bounce-back tiles only)
};

// For every lane, the value of the node to its left (right) in the tile: the thread's own previous
// (next) lane, or the last (first) lane of the neighbouring thread from a per-thread shared array. At
// the tile edges the lane's own value stands in (those nodes are never stored).
template <typename X, int NT>
__device__ __forceinline__ X left_of(const X* arr, int t, X own) {
  if constexpr (Lane<X>::W == 1) {
    return (t > 0 && in_bounds(t - 1, NT)) ? arr[t - 1] : own;
  } else if constexpr (std::is_same<X, df2>::value) {
    const df x0 = df2_get(own, 0);
    return df2_of((t > 0 && in_bounds(t - 1, NT)) ? df2_get(arr[t - 1], 1) : x0, x0);
  } else {
    return make_float2((t > 0 && in_bounds(t - 1, NT)) ? arr[t - 1].y : own.x, own.x);
  }
}
template <typename X, int NT>
__device__ __forceinline__ X right_of(const X* arr, int t, X own) {
  if constexpr (Lane<X>::W == 1) {
    return (t < NT - 1 && in_bounds(t + 1, NT)) ? arr[t + 1] : own;
  } else if constexpr (std::is_same<X, df2>::value) {
    const df x1 = df2_get(own, 1);
    return df2_of(x1, (t < NT - 1 && in_bounds(t + 1, NT)) ? df2_get(arr[t + 1], 0) : x1);
  } else {
    return make_float2(own.y, (t < NT - 1 && in_bounds(t + 1, NT)) ? arr[t + 1].x : own.y);
  }
}

// Rate-dependent lane constants of one lattice.
template <typename X>
struct AdjRates {
  X s_e, s_psi, s_eps, one_m_se, one_m_sp, one_m_ss, q, s0, m_s0, gse;  // gse = -1/(4 s_e^2)
};

// One adjoint step of the thread's W nodes (every thread of the CTA calls it together; two CTA
// barriers): from the forward states f = f(t) and a = a(t+1) to ao = a(t) and these nodes' terms of
// dL/ds_e and dL/ds_psi. Valid where f and a are valid two nodes to each side. Every fused
// multiply-add is explicit (fm), so paired lanes use FFMA2.
template <typename X, int NT>
__device__ __forceinline__ void adjoint_node_step(const X (&f)[6], const X (&a)[6], AdjShared<X, NT>& sh, int t,
                                                  const NodeFlags<Lane<X>::W>& nf, const AdjRates<X>& rt_,
                                                  const Consts<X>& c, X (&ao)[6], X& g_se, X& g_sp) {
  const X zero = lit<X>(0.0);
  // Phase 1: forward state of these nodes and their adjoint at t + 1.
  Node<X> m;
  node_state(f, c, rt_.s0, m);
  sh.su[t] = m.u;
  sh.sT[t] = m.T;
  sh.sfp[t] = a[1]; sh.sgp[t] = a[4];
  sh.sfm[t] = a[2]; sh.sgm[t] = a[5];
  __syncthreads();

  // Phase 2: adjoint of the post-collision populations (transposed streaming): a+ from the right
  // neighbour, a- from the left one; a wall node takes its own reflected one.
  X as[6];
  as[0] = a[0];
  as[3] = a[3];
  as[1] = sel<X>(nf.rw, a[2], right_of<X, NT>(sh.sfp, t, a[1]));
  as[4] = sel<X>(nf.rw, a[5], right_of<X, NT>(sh.sgp, t, a[4]));
  as[2] = sel<X>(nf.lw, a[1], left_of<X, NT>(sh.sfm, t, a[2]));
  as[5] = sel<X>(nf.lw, a[4], left_of<X, NT>(sh.sgm, t, a[5]));
  // Transpose of M^{-1}: x0 = (r - q)/3, x+- = (2r + q)/6 +- j/2 per block.
  const X m_third = lit<X>(-1.0 / 3.0);
  const X rbf = ml(ad(ad(as[0], as[1]), as[2]), c.third);
  const X qbf = fm(as[0], m_third, ml(ad(as[1], as[2]), c.sixth));
  const X jbf = ml(c.half, sb(as[1], as[2]));
  const X rbg = ml(ad(ad(as[3], as[4]), as[5]), c.third);
  const X qbg = fm(as[3], m_third, ml(ad(as[4], as[5]), c.sixth));
  const X jbg = ml(c.half, sb(as[4], as[5]));
  X rt_b = ml(rbf, c.inv_af), J_b = ml(jbf, c.inv_af_l);
  const X es_b = ml(qbf, c.inv_af_l2);
  X zt_b = ml(rbg, c.inv_ag);
  const X psis_b = ml(jbg, c.inv_ag_l), epss_b = ml(qbg, c.inv_ag_l2);

  // Forward quantities of the collision; wall ghosts u = -u0, T = T0.
  X ul = left_of<X, NT>(sh.su, t, m.u), Tl = left_of<X, NT>(sh.sT, t, m.T);
  X ur = right_of<X, NT>(sh.su, t, m.u), Tr = right_of<X, NT>(sh.sT, t, m.T);
  const X neg_u = ml(m.u, c.m_one);
  ul = sel<X>(nf.lw, neg_u, ul);
  Tl = sel<X>(nf.lw, m.T, Tl);
  ur = sel<X>(nf.rw, neg_u, ur);
  Tr = sel<X>(nf.rw, m.T, Tr);
  const X s = ad(rt_.s0, m.ds);
  const X zeta = ml(m.rho, s);
  const X e_eq_t = fm(c.m_two_lam2, m.rt, ml(c.three, fm(m.J, m.u, m.pt)));
  const X psi_eq = ml(zeta, m.u);

  // Relaxation.
  const X et_b = ml(rt_.one_m_se, es_b);
  X e_eq_b = ml(rt_.s_e, es_b);
  const X psi_b = ml(rt_.one_m_sp, psis_b), psi_eq_b = ml(rt_.s_psi, psis_b);
  const X epst_b = ml(rt_.one_m_ss, epss_b), eps_eq_b = ml(rt_.s_eps, epss_b);
  g_se = ml(es_b, sb(e_eq_t, m.et));
  g_sp = ml(psis_b, sb(psi_eq, m.psi));

  X rho_b = zero, ds_b, lnr_b, u_b = zero, T_b = zero, pt_b, ir_b;
  X ul_b = zero, ur_b = zero, Tl_b = zero, Tr_b = zero;
  // Source: zs = zt + S, S = q rho iT (du^2 + cP dT^2 iT); so far zt_b is the adjoint of zs.
  if (c.source_on) {
    const X S_b = zt_b;
    const X du = sb(ur, ul), dT = sb(Tr, Tl);
    const X iT = m_rcp(m.T);
    const X cdT2 = ml(c.cp_over_Pr, ml(dT, dT));
    const X A = fm(cdT2, iT, ml(du, du));
    const X Sq = ml(S_b, rt_.q);
    rho_b = ml(ml(Sq, iT), A);
    const X iT_b = ml(ml(Sq, m.rho), fm(cdT2, iT, A));
    T_b = ml(ml(iT_b, iT), ml(iT, c.m_one));
    const X Sqri2 = ml(ml(Sq, m.rho), ml(iT, c.two));
    const X du_b = ml(Sqri2, du);
    const X dT_b = ml(Sqri2, ml(ml(c.cp_over_Pr, dT), iT));
    ur_b = du_b; ul_b = ml(du_b, c.m_one); Tr_b = dT_b; Tl_b = ml(dT_b, c.m_one);
    g_se = fm(ml(S_b, ml(ml(m.rho, iT), A)), rt_.gse, g_se);
  }
  // Walls: the ghosts are functions of these nodes' own u and T.
  u_b = sel<X>(nf.lw, sb(u_b, ul_b), u_b);
  T_b = sel<X>(nf.lw, ad(T_b, Tl_b), T_b);
  ul_b = sel<X>(nf.lw, zero, ul_b);
  Tl_b = sel<X>(nf.lw, zero, Tl_b);
  u_b = sel<X>(nf.rw, sb(u_b, ur_b), u_b);
  T_b = sel<X>(nf.rw, ad(T_b, Tr_b), T_b);
  ur_b = sel<X>(nf.rw, zero, ur_b);
  Tr_b = sel<X>(nf.rw, zero, Tr_b);
  // eps_eq_t = 2 lam^2 rho (ds + cp_log lnr) + e_eq_t s + e_r ds.
  const X ee2 = ml(eps_eq_b, c.two_lam2);
  rho_b = fm(ee2, fm(c.cp_log, m.lnr, m.ds), rho_b);
  ds_b = ml(eps_eq_b, ad(fm(c.two_lam2, m.rho, c.e_r), e_eq_t));
  lnr_b = ml(ee2, ml(m.rho, c.cp_log));
  e_eq_b = fm(eps_eq_b, s, e_eq_b);
  // psi_eq = zeta u with zeta = rho s.
  const X zeta_b = ml(psi_eq_b, m.u);
  u_b = fm(psi_eq_b, zeta, u_b);
  rho_b = fm(zeta_b, s, rho_b);
  ds_b = fm(zeta_b, m.rho, ds_b);
  // e_eq_t = 3 (J u + pt) - 2 lam^2 rt.
  const X e3 = ml(c.three, e_eq_b);
  J_b = fm(e3, m.u, J_b);
  u_b = fm(e3, m.J, u_b);
  pt_b = e3;
  rt_b = fm(c.m_two_lam2, e_eq_b, rt_b);

  // Scatter the neighbours' source adjoints; only nodes of the lattice contribute.
  {
    const X ulv = sel<X>(nf.inactive, zero, ul_b), urv = sel<X>(nf.inactive, zero, ur_b);
    const X Tlv = sel<X>(nf.inactive, zero, Tl_b), Trv = sel<X>(nf.inactive, zero, Tr_b);
    sh.sul[t] = ulv;
    sh.sur[t] = urv;
    sh.sTl[t] = Tlv;
    sh.sTr[t] = Trv;
    __syncthreads();
    // Phase 3: gather node i - 1's right contribution and node i + 1's left one (none across a wall).
    const X gu = ad(sel<X>(nf.lw, zero, left_of<X, NT>(sh.sur, t, urv)), sel<X>(nf.rw, zero, right_of<X, NT>(sh.sul, t, ulv)));
    const X gT = ad(sel<X>(nf.lw, zero, left_of<X, NT>(sh.sTr, t, Trv)), sel<X>(nf.rw, zero, right_of<X, NT>(sh.sTl, t, Tlv)));
    u_b = ad(u_b, gu);
    T_b = ad(T_b, gT);
  }

  // Equation of state: T = (p0 + pt) ir / r, pt = p0 expm1(x), x = gamma (lnr + ds / cp).
  const X p = ad(c.p0, m.pt);
  pt_b = fm(ml(T_b, m.inv_rho), c.inv_r, pt_b);
  ir_b = ml(ml(T_b, p), c.inv_r);
  const X x_b = ml(pt_b, p);
  lnr_b = fm(c.gamma, x_b, lnr_b);
  ds_b = fm(ml(c.gamma, c.inv_cp), x_b, ds_b);
  // lnr = log1p(rt / rho0)
  rt_b = fm(lnr_b, m.inv_rho, rt_b);
  // ds = (zt - rt s0) ir
  const X dsi = ml(ds_b, m.inv_rho);
  zt_b = ad(zt_b, dsi);
  rt_b = fm(dsi, rt_.m_s0, rt_b);
  ir_b = fm(ds_b, fm(m.rt, rt_.m_s0, m.zt), ir_b);
  // u = J ir
  J_b = fm(u_b, m.inv_rho, J_b);
  ir_b = fm(u_b, m.J, ir_b);
  // ir = 1 / rho, rho = rho0 + rt
  rho_b = sb(rho_b, ml(ml(ir_b, m.inv_rho), m.inv_rho));
  rt_b = ad(rt_b, rho_b);
  // Transpose of m = M f.
  const X m2 = lit<X>(-2.0);
  const X r0 = ml(c.rho0, rt_b), et2 = ml(c.af_l2, et_b);
  ao[0] = fm(m2, et2, r0);
  ao[1] = fm(c.af_l, J_b, ad(r0, et2));
  ao[2] = fm(ml(c.af_l, c.m_one), J_b, ad(r0, et2));
  const X z0 = ml(c.ag, zt_b), ep2 = ml(c.ag_l2, epst_b);
  ao[3] = fm(m2, ep2, z0);
  ao[4] = fm(c.ag_l, psi_b, ad(z0, ep2));
  ao[5] = fm(ml(c.ag_l, c.m_one), psi_b, ad(z0, ep2));
}

// K adjoint steps per launch: a(t0 + K) -> a(t0), from the forward state f(t0) alone.
// A CTA of NT threads owns TW = NT W consecutive nodes (W per thread). It first recomputes the forward
// states f(t0), ..., f(t0 + K - 1) of its nodes on chip (the fused collide-stream update of the step
// kernels) and keeps them in shared memory, then runs the K reverse steps. The forward step and the
// reverse step each reach two nodes, so f(t0 + k) is valid 2k nodes in from the tile edges,
// a(t0 + k) 2K + 2(K - 1 - k) nodes in, and the tile stores its TW - 2(4K - 2) central nodes. HBM
// traffic per node is one state and two adjoint reads/writes per K steps.
// The rate gradients dL/ds_e and dL/ds_psi of the stored nodes are summed per warp and step in the
// arithmetic type, accumulated over the K steps in FP64 per warp, reduced over warps in a fixed order
// and added to a per-tile accumulator only this tile's CTA touches (deterministic).
// Paired FP32 lanes: at least six CTAs of 128 threads per SM (at most 85 registers; the compiler takes
// 80 with a 20-byte spill), measured 1.6 % faster than the five CTAs its own register choice allows.
template <typename X, int NT>
__global__ void __launch_bounds__(NT, std::is_same<X, float2>::value ? 6 : 0) adjoint_block_kernel(const typename Lane<X>::R* __restrict__ f0,
                                                           const typename Lane<X>::R* __restrict__ a_next,
                                                           typename Lane<X>::R* __restrict__ a_out, long long plane,
                                                           const LatDev* __restrict__ lat, int B, long long ntiles,
                                                           int K, Consts<X> c, double* __restrict__ grad_tile) {
  using R = typename Lane<X>::R;
  constexpr int W = Lane<X>::W, TW = NT * W, NW = NT / 32;
  extern __shared__ __align__(16) unsigned char adj_dyn[];
  X* sfx = reinterpret_cast<X*>(adj_dyn);  // [K][6][NT] forward states of this tile (one lane value per thread)
  __shared__ AdjShared<X, NT> sh;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int halo = 4 * K - 2;
  const int bout = TW - 2 * halo;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int L = 0;
    if (B > 1) {
      int lo = 0, hi = B - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (lat[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
      }
      L = lo;
    }
    if (!in_bounds(L, B)) continue;
    const LatDev d = lat[L];
    const long long N = d.n, off = d.offset;
    NodeFlags<W> nf;
    long long pos[W], lp[W];
    bool owned[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const int i = t * W + j;
      pos[j] = (tile - d.tile0) * bout - halo + i;
      lp[j] = pos[j];
      if (d.bc == 0) {
        if (lp[j] < 0 || lp[j] >= N) { lp[j] %= N; if (lp[j] < 0) lp[j] += N; }
      } else {
        lp[j] = lp[j] < 0 ? 0 : (lp[j] >= N ? N - 1 : lp[j]);
      }
      const bool inside = pos[j] >= 0 && pos[j] < N;
      nf.inactive[j] = d.bc != 0 && !inside;
      nf.lw[j] = d.bc != 0 && pos[j] == 0;
      nf.rw[j] = d.bc != 0 && pos[j] == N - 1;
      owned[j] = i >= halo && i < halo + bout && inside;
    }
    const StepParams<R> P = step_params(d, R{});
    const X s_e = lit_r<X>(P.s_e), s_psi = lit_r<X>(P.s_psi), s_eps = lit_r<X>(P.s_eps);
    const X q_src = lit_r<X>(P.q_src), s0h = lit_r<X>(P.s0h), m_s0h = lit_r<X>(-P.s0h);
    const X le0 = lit_r<X>(P.lin_e0), lp0 = lit_r<X>(P.lin_p0), lq0 = lit_r<X>(P.lin_q0);
    AdjRates<X> ar;
    {
      const R s0 = R(d.s0);
      ar.s_e = s_e; ar.s_psi = s_psi; ar.s_eps = s_eps;
      ar.one_m_se = lit_r<X>(R(1) - P.s_e);
      ar.one_m_sp = lit_r<X>(R(1) - P.s_psi);
      ar.one_m_ss = lit_r<X>(R(1) - P.s_eps);
      ar.q = q_src;
      ar.s0 = lit_r<X>(s0);
      ar.m_s0 = lit_r<X>(-s0);
      ar.gse = lit_r<X>(R(-0.25) * m_rcp(P.s_e * P.s_e));
    }

    // Forward recompute: f(t0 + k) into shared memory, k = 0 .. K - 1.
    bool lp_ok[W];
#pragma unroll
    for (int j = 0; j < W; ++j) lp_ok[j] = in_bounds(lp[j], N) && in_bounds(off + lp[j], plane);
    X f[6];
#pragma unroll
    for (int q = 0; q < 6; ++q)
#pragma unroll
      for (int j = 0; j < W; ++j) lset(f[q], j, lp_ok[j] ? f0[q * plane + off + lp[j]] : R(0));
    for (int k = 0; k < K; ++k) {
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if (in_bounds((k * 6 + q) * NT + t, K * 6 * NT)) sfx[(k * 6 + q) * NT + t] = f[q];
      if (k == K - 1) break;
      NodeS<X> ms;
      node_state_s(f, c, m_s0h, ms);
      sh.su[t] = ms.u;
      sh.sT[t] = ms.th;
      __syncthreads();
      X ul = left_of<X, NT>(sh.su, t, ms.u), thl = left_of<X, NT>(sh.sT, t, ms.th);
      X ur = right_of<X, NT>(sh.su, t, ms.u), thr = right_of<X, NT>(sh.sT, t, ms.th);
      const X neg_u = ml(ms.u, c.m_one);
      ul = sel<X>(nf.lw, neg_u, ul);
      thl = sel<X>(nf.lw, ms.th, thl);
      ur = sel<X>(nf.rw, neg_u, ur);
      thr = sel<X>(nf.rw, ms.th, thr);
      X fs[6];
      node_collide_s(ms, ul, ur, thl, thr, s_e, s_psi, s_eps, q_src, s0h, c, fs, le0, lp0, lq0);
      sh.sfp[t] = fs[1]; sh.sgp[t] = fs[4];
      sh.sfm[t] = fs[2]; sh.sgm[t] = fs[5];
      __syncthreads();
      // Streaming: f+, g+ from the left node, f-, g- from the right one; walls reflect their own.
      f[0] = fs[0];
      f[3] = fs[3];
      f[1] = sel<X>(nf.lw, fs[2], left_of<X, NT>(sh.sfp, t, fs[1]));
      f[4] = sel<X>(nf.lw, fs[5], left_of<X, NT>(sh.sgp, t, fs[4]));
      f[2] = sel<X>(nf.rw, fs[1], right_of<X, NT>(sh.sfm, t, fs[2]));
      f[5] = sel<X>(nf.rw, fs[4], right_of<X, NT>(sh.sgm, t, fs[5]));
    }
    __syncthreads();  // the reverse steps rewrite the exchange buffers

    // Reverse steps t0 + K - 1 .. t0.
    X a[6];
#pragma unroll
    for (int q = 0; q < 6; ++q)
#pragma unroll
      for (int j = 0; j < W; ++j) lset(a[q], j, lp_ok[j] ? a_next[q * plane + off + lp[j]] : R(0));
    double acc_se = 0.0, acc_sp = 0.0;  // per warp (lane 0), over the K steps
    for (int k = K - 1; k >= 0; --k) {
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if (in_bounds((k * 6 + q) * NT + t, K * 6 * NT)) f[q] = sfx[(k * 6 + q) * NT + t];
      X ao[6], gx_se, gx_sp;
      adjoint_node_step<X, NT>(f, a, sh, t, nf, ar, c, ao, gx_se, gx_sp);
#pragma unroll
      for (int q = 0; q < 6; ++q) a[q] = ao[q];
      R g_se = R(0), g_sp = R(0);
#pragma unroll
      for (int j = 0; j < W; ++j)
        if (owned[j]) { g_se += lget(gx_se, j); g_sp += lget(gx_sp, j); }
      for (int o = 16; o > 0; o >>= 1) {
        g_se += __shfl_down_sync(0xffffffffu, g_se, o);
        g_sp += __shfl_down_sync(0xffffffffu, g_sp, o);
      }
      if (lane == 0) { acc_se += (double)g_se; acc_sp += (double)g_sp; }
    }
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (owned[j] && in_bounds(pos[j], N) && in_bounds(off + pos[j], plane))
#pragma unroll
        for (int q = 0; q < 6; ++q) a_out[q * plane + off + pos[j]] = lget(a[q], j);
    if (lane == 0) { sh.sg[0][warp] = acc_se; sh.sg[1][warp] = acc_sp; }
    __syncthreads();
    if (t == 0 && in_bounds(tile, ntiles)) {
      double t0 = 0.0, t1 = 0.0;
      for (int w = 0; w < NW; ++w) { t0 += sh.sg[0][w]; t1 += sh.sg[1][w]; }
      grad_tile[2 * tile] += t0;
      grad_tile[2 * tile + 1] += t1;
    }
    __syncthreads();
  }
}

// Per-lattice sum of the per-tile rate gradients (fixed order) into out[2 * L + k], or added to it.
__global__ void reduce_rate_grads_kernel(const double* __restrict__ grad_tile, const LatDev* __restrict__ lat, int B,
                                         long long ntiles, double* __restrict__ out, int accumulate) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= B) return;
  const long long t0 = lat[L].tile0, t1 = L + 1 < B ? lat[L + 1].tile0 : ntiles;
  double a = 0.0, b = 0.0;
  for (long long t = t0; t < t1; ++t) { a += grad_tile[2 * t]; b += grad_tile[2 * t + 1]; }
  out[2 * L] = accumulate ? out[2 * L] + a : a;
  out[2 * L + 1] = accumulate ? out[2 * L + 1] + b : b;
}

// Adjoint of the equilibrium initialisation f = M^{-1} m_eq(rho, J = rho u, zeta = rho s) at fixed
// specific entropy s: from a0 = dL/df(0) and the initial state (read back from its populations)
// to dL/drho(0) and dL/du(0). FP64 arithmetic.
template <typename R>
__global__ void adjoint_init_kernel(const R* __restrict__ f0, const R* __restrict__ a0, long long plane,
                                    const LatDev* __restrict__ lat, int B, Consts<double> c, double* __restrict__ drho,
                                    double* __restrict__ du) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= plane) return;
  int L = 0;
  {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (lat[mid].offset <= i) lo = mid; else hi = mid - 1;
    }
    L = lo;
  }
  const double s0 = lat[L].s0;
  double f[6], a[6];
  for (int k = 0; k < 6; ++k) { f[k] = (double)f0[k * plane + i]; a[k] = (double)a0[k * plane + i]; }
  // Initial rho, u, s from the populations.
  const double rt = c.rho0 * (f[0] + f[1] + f[2]);
  const double rho = c.rho0 + rt;
  const double J = c.af_l * (f[1] - f[2]);
  const double zt = c.ag * (f[3] + f[4] + f[5]);
  const double u = J / rho;
  const double ds = (zt - rt * s0) / rho;
  const double s = s0 + ds;
  const double lnr = log1p(rt * c.inv_af);
  const double pt = c.p0 * expm1(c.gamma * (lnr + ds * c.inv_cp));
  const double p = c.p0 + pt;
  // Transpose of M^{-1} per block.
  const double rbf = (a[0] + a[1] + a[2]) / 3.0, qbf = -a[0] / 3.0 + (a[1] + a[2]) / 6.0, jbf = 0.5 * (a[1] - a[2]);
  const double rbg = (a[3] + a[4] + a[5]) / 3.0, qbg = -a[3] / 3.0 + (a[4] + a[5]) / 6.0, jbg = 0.5 * (a[4] - a[5]);
  double rt_b = rbf * c.inv_af, J_b = jbf * c.inv_af_l, e_b = qbf * c.inv_af_l2;
  const double zt_b = rbg * c.inv_ag, psi_b = jbg * c.inv_ag_l, eps_b = qbg * c.inv_ag_l2;
  double rho_b = 0.0, u_b = 0.0, lnr_b = 0.0, p_b = 0.0;
  // eps_eq_t = 2 lam^2 rho (ds + cp_log lnr) + e_eq_t s + e_r ds  (ds fixed)
  rho_b += eps_b * c.two_lam2 * (ds + c.cp_log * lnr);
  lnr_b += eps_b * c.two_lam2 * rho * c.cp_log;
  e_b += eps_b * s;
  // psi_eq = rho s u
  rho_b += psi_b * s * u;
  u_b += psi_b * rho * s;
  // zeta_t = rho s - zeta_r
  rho_b += zt_b * s;
  // e_eq_t = 3 (J u + pt) - 2 lam^2 rt
  J_b += 3.0 * e_b * u;
  u_b += 3.0 * e_b * J;
  p_b += 3.0 * e_b;
  rt_b -= c.two_lam2 * e_b;
  // p = p0 (rho/rho0)^gamma exp(gamma ds / cp): dp/drho = gamma p / rho at fixed s
  rho_b += p_b * c.gamma * p / rho;
  rho_b += lnr_b / rho;
  // J = rho u, rt = rho - rho0
  rho_b += J_b * u;
  u_b += J_b * rho;
  rho_b += rt_b;
  drho[i] = rho_b;
  du[i] = u_b;
}

// Seed of the squared density misfit: rho_b = 2 (rho_T - rho*), a_T = (rho0 rho_b) on f, 0 on g;
// per-block partial sums of (rho_T - rho*)^2 in FP64.
template <typename R>
__global__ void __launch_bounds__(256) misfit_seed_kernel(const R* __restrict__ fT, const double* __restrict__ target,
                                                          const double* __restrict__ rho_b_in, long long plane,
                                                          double rho0, R* __restrict__ aT, double* __restrict__ part) {
  const long long i = blockIdx.x * 256LL + threadIdx.x;
  double sq = 0.0;
  if (i < plane) {
    double rb;
    if (target) {
      const double rho = rho0 + rho0 * ((double)fT[i] + (double)fT[plane + i] + (double)fT[2 * plane + i]);
      const double dlt = rho - target[i];
      sq = dlt * dlt;
      rb = 2.0 * dlt;
    } else {
      rb = rho_b_in[i];
    }
    const R v = R(rho0 * rb);
    aT[i] = v;
    aT[plane + i] = v;
    aT[2 * plane + i] = v;
    aT[3 * plane + i] = R(0);
    aT[4 * plane + i] = R(0);
    aT[5 * plane + i] = R(0);
  }
  __shared__ double sh[8];
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

__global__ void sum_parts_kernel(const double* __restrict__ part, long long n, double* __restrict__ out) {
  __shared__ double sh[8];
  double t = 0.0;
  for (long long i = threadIdx.x; i < n; i += 256) t += part[i];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sh[w];
    *out = s;
  }
}

// FP64 runs one node per thread; FP32 two per thread on paired lanes. Both tile kAdjointThreads nodes.
template <typename X>
static cudaError_t launch_block_lanes(const typename Lane<X>::R* f0, const typename Lane<X>::R* a_next,
                                      typename Lane<X>::R* a_out, long long plane, const LatDev* lat, int B,
                                      long long ntiles, int K, const Consts<X>& c, double* grad_tile, cudaStream_t st) {
  using R = typename Lane<X>::R;
  constexpr int NT = kAdjointThreads / Lane<X>::W;
  const size_t dyn = (size_t)kAdjointMaxK * 6 * kAdjointThreads * sizeof(R);
  // The shared-memory limit is an attribute of the function on each device: set it once per device.
  static std::atomic<unsigned long long> attr_set{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ULL << (dev & 63);
  if (dev >= 64 || !(attr_set.load() & bit)) {
    e = cudaFuncSetAttribute(adjoint_block_kernel<X, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    if (dev < 64) attr_set.fetch_or(bit);
  }
  const size_t use = (size_t)K * 6 * kAdjointThreads * sizeof(R);
  adjoint_block_kernel<X, NT><<<(unsigned)ntiles, NT, use, st>>>(f0, a_next, a_out, plane, lat, B, ntiles, K, c,
                                                                 grad_tile);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_block_df(const double* f0, const double* a_next, double* a_out, long long plane,
                                    const LatDev* lat, int B, long long ntiles, int K, const Consts<df>& c,
                                    double* grad_tile, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (K < 1 || K > kAdjointMaxK) return cudaErrorInvalidValue;
  // Two nodes per thread on paired FP32 lanes (df2): lane for lane the operations of one node per
  // thread, on the same 256-node tiles.
  return launch_block_lanes<df2>(f0, a_next, a_out, plane, lat, B, ntiles, K, pair_consts(c), grad_tile, st);
}

template <typename R>
cudaError_t launch_adjoint_block(const R* f0, const R* a_next, R* a_out, long long plane, const LatDev* lat, int B,
                                 long long ntiles, int K, const ConstSet<R>& c, double* grad_tile, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (K < 1 || K > kAdjointMaxK) return cudaErrorInvalidValue;
  if constexpr (sizeof(R) == 4)
    return launch_block_lanes<float2>(f0, a_next, a_out, plane, lat, B, ntiles, K, c.p, grad_tile, st);
  else
    return launch_block_lanes<double>(f0, a_next, a_out, plane, lat, B, ntiles, K, c.s, grad_tile, st);
}

cudaError_t launch_reduce_rate_grads(const double* grad_tile, const LatDev* lat, int B, long long ntiles, double* out,
                                     bool accumulate, cudaStream_t st) {
  reduce_rate_grads_kernel<<<(B + 127) / 128, 128, 0, st>>>(grad_tile, lat, B, ntiles, out, accumulate ? 1 : 0);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adjoint_init(const R* f0, const R* a0, long long plane, const LatDev* lat, int B,
                                const Consts<double>& c, double* drho, double* du, cudaStream_t st) {
  adjoint_init_kernel<R><<<(unsigned)((plane + 255) / 256), 256, 0, st>>>(f0, a0, plane, lat, B, c, drho, du);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_misfit_seed(const R* fT, const double* target, const double* rho_b, long long plane, double rho0,
                               R* aT, double* part, double* loss, cudaStream_t st) {
  const long long nb = (plane + 255) / 256;
  misfit_seed_kernel<R><<<(unsigned)nb, 256, 0, st>>>(fT, target, rho_b, plane, rho0, aT, part);
  if (target) sum_parts_kernel<<<1, 256, 0, st>>>(part, nb, loss);
  return cudaGetLastError();
}

template <typename R>
__global__ void to_f64_kernel(const R* __restrict__ in, double* __restrict__ out, long long n) {
  const long long i = blockIdx.x * 256LL + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

template <typename R>
cudaError_t launch_to_f64(const R* in, double* out, long long n, cudaStream_t st) {
  to_f64_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}
template cudaError_t launch_to_f64<float>(const float*, double*, long long, cudaStream_t);
template cudaError_t launch_to_f64<double>(const double*, double*, long long, cudaStream_t);

template cudaError_t launch_adjoint_block<float>(const float*, const float*, float*, long long, const LatDev*, int,
                                                 long long, int, const ConstSet<float>&, double*, cudaStream_t);
template cudaError_t launch_adjoint_block<double>(const double*, const double*, double*, long long, const LatDev*, int,
                                                  long long, int, const ConstSet<double>&, double*, cudaStream_t);
template cudaError_t launch_adjoint_init<float>(const float*, const float*, long long, const LatDev*, int,
                                                const Consts<double>&, double*, double*, cudaStream_t);
template cudaError_t launch_adjoint_init<double>(const double*, const double*, long long, const LatDev*, int,
                                                 const Consts<double>&, double*, double*, cudaStream_t);
template cudaError_t launch_misfit_seed<float>(const float*, const double*, const double*, long long, double, float*,
                                               double*, double*, cudaStream_t);
template cudaError_t launch_misfit_seed<double>(const double*, const double*, const double*, long long, double,
                                                double*, double*, double*, cudaStream_t);

cudaError_t bounds_record_adjoint(unsigned long long out[3]) {
#ifdef LBM_DEBUG_BOUNDS
  return take_bounds_record(out);
#else
  out[0] = out[1] = out[2] = 0ULL;
  return cudaSuccess;
#endif
}

}  // namespace lbm
