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
#include "lbm_internal.cuh"

namespace lbm {

// Shared-memory exchange buffers of one CTA of NT threads (one node per thread).
template <typename R, int NT>
struct AdjShared {
  R su[NT], sT[NT];                 // forward u and T (or u' and theta in the recompute) of each node
  R sap[NT][2], sam[NT][2];         // a+ and a- (f, g) of each node at t + 1; moving populations forward
  R sul[NT], sur[NT], sTl[NT], sTr[NT];  // source adjoints scattered to the neighbours
  double sg[2][NT / 32];
};

// One adjoint step of node n (all threads of the CTA call it together; two CTA barriers): from the
// forward state f = f(t) and a = a(t+1) of this node to ao = a(t) and this node's terms of dL/ds_e and
// dL/ds_psi. Valid where f and a are valid two nodes to each side.
template <typename R, int NT>
__device__ __forceinline__ void adjoint_node_step(const R (&f)[6], const R (&a)[6], AdjShared<R, NT>& sh, int n,
                                                  bool lw, bool rw, bool active, R s_e, R s_psi, R s_eps, R q, R s0,
                                                  const Consts<R>& c, R (&ao)[6], R& g_se, R& g_sp) {
  // Phase 1: forward state of this node, its adjoint at t + 1.
  Node<R> m;
  node_state(f, c, s0, m);
  sh.su[n] = m.u;
  sh.sT[n] = m.T;
  sh.sap[n][0] = a[1]; sh.sap[n][1] = a[4];
  sh.sam[n][0] = a[2]; sh.sam[n][1] = a[5];
  __syncthreads();

  // Phase 2: adjoint of the post-collision populations (transposed streaming).
  R as[6];
  as[0] = a[0];
  as[3] = a[3];
  as[1] = rw ? a[2] : (n < NT - 1 ? sh.sap[n + 1][0] : R(0));
  as[4] = rw ? a[5] : (n < NT - 1 ? sh.sap[n + 1][1] : R(0));
  as[2] = lw ? a[1] : (n > 0 ? sh.sam[n - 1][0] : R(0));
  as[5] = lw ? a[4] : (n > 0 ? sh.sam[n - 1][1] : R(0));
  // Transpose of M^{-1}: x0 = (r - q)/3, x+- = (2r + q)/6 +- j/2 per block.
  const R rbf = (as[0] + as[1] + as[2]) * R(1.0 / 3.0), qbf = -as[0] * R(1.0 / 3.0) + (as[1] + as[2]) * R(1.0 / 6.0);
  const R jbf = R(0.5) * (as[1] - as[2]);
  const R rbg = (as[3] + as[4] + as[5]) * R(1.0 / 3.0), qbg = -as[3] * R(1.0 / 3.0) + (as[4] + as[5]) * R(1.0 / 6.0);
  const R jbg = R(0.5) * (as[4] - as[5]);
  R rt_b = rbf * c.inv_af, J_b = jbf * c.inv_af_l;
  const R es_b = qbf * c.inv_af_l2;
  R zt_b = rbg * c.inv_ag;
  const R psis_b = jbg * c.inv_ag_l, epss_b = qbg * c.inv_ag_l2;

  // Forward quantities of the collision.
  R ul = n > 0 ? sh.su[n - 1] : m.u, Tl = n > 0 ? sh.sT[n - 1] : m.T;
  R ur = n < NT - 1 ? sh.su[n + 1] : m.u, Tr = n < NT - 1 ? sh.sT[n + 1] : m.T;
  if (lw) { ul = -m.u; Tl = m.T; }
  if (rw) { ur = -m.u; Tr = m.T; }
  const R s = s0 + m.ds;
  const R zeta = m.rho * s;
  const R e_eq_t = R(3) * (m.J * m.u + m.pt) - c.two_lam2 * m.rt;
  const R psi_eq = zeta * m.u;

  // Relaxation.
  R et_b = (R(1) - s_e) * es_b, e_eq_b = s_e * es_b;
  R psi_b = (R(1) - s_psi) * psis_b, psi_eq_b = s_psi * psis_b;
  R epst_b = (R(1) - s_eps) * epss_b, eps_eq_b = s_eps * epss_b;
  // Rate-gradient terms of this node in the arithmetic type.
  g_se = es_b * (e_eq_t - m.et);
  g_sp = psis_b * (psi_eq - m.psi);

  R rho_b = R(0), ds_b = R(0), lnr_b = R(0), u_b = R(0), T_b = R(0), pt_b = R(0), ir_b = R(0);
  R ul_b = R(0), ur_b = R(0), Tl_b = R(0), Tr_b = R(0);
  // Source: zs = zt + S, S = q rho iT (du^2 + cP dT^2 iT); so far zt_b is the adjoint of zs.
  if (c.source_on) {
    const R S_b = zt_b;
    const R du = ur - ul, dT = Tr - Tl;
    const R iT = m_rcp(m.T);
    const R A = du * du + c.cp_over_Pr * dT * dT * iT;
    rho_b += S_b * q * iT * A;
    const R iT_b = S_b * q * m.rho * (A + c.cp_over_Pr * dT * dT * iT);
    T_b -= iT_b * iT * iT;
    const R du_b = S_b * q * m.rho * iT * R(2) * du;
    const R dT_b = S_b * q * m.rho * iT * c.cp_over_Pr * R(2) * dT * iT;
    ur_b = du_b; ul_b = -du_b; Tr_b = dT_b; Tl_b = -dT_b;
    g_se += S_b * (m.rho * iT * A) * (R(-0.25) * m_rcp(s_e * s_e));
  }
  // Walls: the ghosts are functions of this node's own u and T.
  if (lw) { u_b -= ul_b; T_b += Tl_b; ul_b = R(0); Tl_b = R(0); }
  if (rw) { u_b -= ur_b; T_b += Tr_b; ur_b = R(0); Tr_b = R(0); }
  // eps_eq_t = 2 lam^2 rho (ds + cp_log lnr) + e_eq_t s + e_r ds.
  rho_b += eps_eq_b * c.two_lam2 * (m.ds + c.cp_log * m.lnr);
  ds_b += eps_eq_b * (c.two_lam2 * m.rho + c.e_r + e_eq_t);  // s = s0 + ds
  lnr_b += eps_eq_b * c.two_lam2 * m.rho * c.cp_log;
  e_eq_b += eps_eq_b * s;
  // psi_eq = zeta u with zeta = rho s.
  const R zeta_b = psi_eq_b * m.u;
  u_b += psi_eq_b * zeta;
  rho_b += zeta_b * s;
  ds_b += zeta_b * m.rho;
  // e_eq_t = 3 (J u + pt) - 2 lam^2 rt.
  J_b += R(3) * e_eq_b * m.u;
  u_b += R(3) * e_eq_b * m.J;
  pt_b += R(3) * e_eq_b;
  rt_b -= c.two_lam2 * e_eq_b;

  // Scatter the neighbours' source adjoints; only nodes of the lattice contribute.
  sh.sul[n] = active ? ul_b : R(0);
  sh.sur[n] = active ? ur_b : R(0);
  sh.sTl[n] = active ? Tl_b : R(0);
  sh.sTr[n] = active ? Tr_b : R(0);
  __syncthreads();
  // Phase 3: gather (node n - 1's right contribution and node n + 1's left one).
  if (!lw && n > 0) { u_b += sh.sur[n - 1]; T_b += sh.sTr[n - 1]; }
  if (!rw && n < NT - 1) { u_b += sh.sul[n + 1]; T_b += sh.sTl[n + 1]; }

  // Equation of state: T = (p0 + pt) ir / r, pt = p0 expm1(x), x = gamma (lnr + ds / cp).
  pt_b += T_b * m.inv_rho * c.inv_r;
  ir_b += T_b * (c.p0 + m.pt) * c.inv_r;
  const R x_b = pt_b * (c.p0 + m.pt);
  lnr_b += c.gamma * x_b;
  ds_b += c.gamma * c.inv_cp * x_b;
  // lnr = log1p(rt / rho0)
  rt_b += lnr_b * m.inv_rho;
  // ds = (zt - rt s0) ir
  zt_b += ds_b * m.inv_rho;
  rt_b -= ds_b * s0 * m.inv_rho;
  ir_b += ds_b * (m.zt - m.rt * s0);
  // u = J ir
  J_b += u_b * m.inv_rho;
  ir_b += u_b * m.J;
  // ir = 1 / rho, rho = rho0 + rt
  rho_b -= ir_b * m.inv_rho * m.inv_rho;
  rt_b += rho_b;
  // Transpose of m = M f.
  ao[0] = c.rho0 * rt_b - R(2) * c.af_l2 * et_b;
  ao[1] = c.rho0 * rt_b + c.af_l * J_b + c.af_l2 * et_b;
  ao[2] = c.rho0 * rt_b - c.af_l * J_b + c.af_l2 * et_b;
  ao[3] = c.ag * zt_b - R(2) * c.ag_l2 * epst_b;
  ao[4] = c.ag * zt_b + c.ag_l * psi_b + c.ag_l2 * epst_b;
  ao[5] = c.ag * zt_b - c.ag_l * psi_b + c.ag_l2 * epst_b;
}

// K adjoint steps per launch: a(t0 + K) -> a(t0), from the forward state f(t0) alone.
// A CTA of NT threads owns NT consecutive nodes (one per thread). It first recomputes the forward
// states f(t0), ..., f(t0 + K - 1) of its nodes on chip (the fused collide-stream update of the step
// kernels, scalar lanes) and keeps them in shared memory, then runs the K reverse steps. The forward
// step and the reverse step each reach two nodes, so f(t0 + k) is valid 2k nodes in from the tile
// edges, a(t0 + k) 2K + 2(K - 1 - k) nodes in, and the tile stores its NT - 2(4K - 2) central nodes.
// HBM traffic per node is one state and two adjoint reads/writes per K steps.
// The rate gradients dL/ds_e and dL/ds_psi of the stored nodes are summed per warp and step in the
// arithmetic type, accumulated over the K steps in FP64 per warp, reduced over warps in a fixed order
// and added to a per-tile accumulator only this tile's CTA touches (deterministic).
template <typename R, int NT>
__global__ void __launch_bounds__(NT) adjoint_block_kernel(const R* __restrict__ f0, const R* __restrict__ a_next,
                                                           R* __restrict__ a_out, long long plane,
                                                           const LatDev* __restrict__ lat, int B, long long ntiles, int K,
                                                           Consts<R> c, double* __restrict__ grad_tile) {
  extern __shared__ __align__(16) unsigned char adj_dyn[];
  R* sf = reinterpret_cast<R*>(adj_dyn);  // [K][6][NT] forward states of this tile
  __shared__ AdjShared<R, NT> sh;
  const int n = threadIdx.x, lane = n & 31, warp = n >> 5;
  const int halo = 4 * K - 2;
  const int bout = NT - 2 * halo;
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
    const LatDev d = lat[L];
    const long long N = d.n, off = d.offset;
    const long long pos = (tile - d.tile0) * bout - halo + n;
    long long lp = pos;
    if (d.bc == 0) {
      if (lp < 0 || lp >= N) { lp %= N; if (lp < 0) lp += N; }
    } else {
      lp = lp < 0 ? 0 : (lp >= N ? N - 1 : lp);
    }
    const bool inside = pos >= 0 && pos < N;
    const bool active = d.bc == 0 || inside;
    const bool lw = d.bc != 0 && pos == 0, rw = d.bc != 0 && pos == N - 1;
    const bool owned = n >= halo && n < halo + bout && inside;
    const StepParams<R> P = step_params(d, R{});
    const R m_s0h = -P.s0h, s0 = R(d.s0);

    // Forward recompute: f(t0 + k) into shared memory, k = 0 .. K - 1.
    R f[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) f[i] = f0[i * plane + off + lp];
    for (int k = 0; k < K; ++k) {
#pragma unroll
      for (int i = 0; i < 6; ++i) sf[(k * 6 + i) * NT + n] = f[i];
      if (k == K - 1) break;
      NodeS<R> ms;
      node_state_s(f, c, m_s0h, ms);
      sh.su[n] = ms.u;
      sh.sT[n] = ms.th;
      __syncthreads();
      R ul = n > 0 ? sh.su[n - 1] : ms.u, thl = n > 0 ? sh.sT[n - 1] : ms.th;
      R ur = n < NT - 1 ? sh.su[n + 1] : ms.u, thr = n < NT - 1 ? sh.sT[n + 1] : ms.th;
      if (lw) { ul = -ms.u; thl = ms.th; }
      if (rw) { ur = -ms.u; thr = ms.th; }
      R fs[6];
      node_collide_s(ms, ul, ur, thl, thr, P.s_e, P.s_psi, P.s_eps, P.q_src, P.s0h, c, fs, P.lin_e0, P.lin_p0,
                     P.lin_q0);
      sh.sap[n][0] = fs[1]; sh.sap[n][1] = fs[4];
      sh.sam[n][0] = fs[2]; sh.sam[n][1] = fs[5];
      __syncthreads();
      f[0] = fs[0];
      f[3] = fs[3];
      f[1] = lw ? fs[2] : (n > 0 ? sh.sap[n - 1][0] : fs[1]);
      f[4] = lw ? fs[5] : (n > 0 ? sh.sap[n - 1][1] : fs[4]);
      f[2] = rw ? fs[1] : (n < NT - 1 ? sh.sam[n + 1][0] : fs[2]);
      f[5] = rw ? fs[4] : (n < NT - 1 ? sh.sam[n + 1][1] : fs[5]);
    }
    __syncthreads();  // the reverse steps rewrite the exchange buffers

    // Reverse steps t0 + K - 1 .. t0.
    R a[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) a[i] = a_next[i * plane + off + lp];
    double acc_se = 0.0, acc_sp = 0.0;  // per warp (lane 0), over the K steps
    for (int k = K - 1; k >= 0; --k) {
#pragma unroll
      for (int i = 0; i < 6; ++i) f[i] = sf[(k * 6 + i) * NT + n];
      R ao[6], g_se, g_sp;
      adjoint_node_step<R, NT>(f, a, sh, n, lw, rw, active, P.s_e, P.s_psi, P.s_eps, P.q_src, s0, c, ao, g_se, g_sp);
#pragma unroll
      for (int i = 0; i < 6; ++i) a[i] = ao[i];
      if (!owned) { g_se = R(0); g_sp = R(0); }
      for (int o = 16; o > 0; o >>= 1) {
        g_se += __shfl_down_sync(0xffffffffu, g_se, o);
        g_sp += __shfl_down_sync(0xffffffffu, g_sp, o);
      }
      if (lane == 0) { acc_se += (double)g_se; acc_sp += (double)g_sp; }
    }
    if (owned)
#pragma unroll
      for (int i = 0; i < 6; ++i) a_out[i * plane + off + pos] = a[i];
    if (lane == 0) { sh.sg[0][warp] = acc_se; sh.sg[1][warp] = acc_sp; }
    __syncthreads();
    if (n == 0) {
      double t0 = 0.0, t1 = 0.0;
      for (int w = 0; w < NT / 32; ++w) { t0 += sh.sg[0][w]; t1 += sh.sg[1][w]; }
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

template <typename R>
cudaError_t launch_adjoint_block(const R* f0, const R* a_next, R* a_out, long long plane, const LatDev* lat, int B,
                                 long long ntiles, int K, const Consts<R>& c, double* grad_tile, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (K < 1 || K > kAdjointMaxK) return cudaErrorInvalidValue;
  const size_t dyn = (size_t)kAdjointMaxK * 6 * kAdjointThreads * sizeof(R);
  static bool attr_set[2] = {false, false};  // per arithmetic type, once per process (the limit is per function)
  bool& done = attr_set[sizeof(R) == 8];
  if (!done) {
    cudaError_t e = cudaFuncSetAttribute(adjoint_block_kernel<R, kAdjointThreads>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    done = true;
  }
  const size_t use = (size_t)K * 6 * kAdjointThreads * sizeof(R);
  adjoint_block_kernel<R, kAdjointThreads><<<(unsigned)ntiles, kAdjointThreads, use, st>>>(f0, a_next, a_out, plane,
                                                                                          lat, B, ntiles, K, c,
                                                                                          grad_tile);
  return cudaGetLastError();
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
                                                 long long, int, const Consts<float>&, double*, cudaStream_t);
template cudaError_t launch_adjoint_block<double>(const double*, const double*, double*, long long, const LatDev*, int,
                                                  long long, int, const Consts<double>&, double*, cudaStream_t);
template cudaError_t launch_adjoint_init<float>(const float*, const float*, long long, const LatDev*, int,
                                                const Consts<double>&, double*, double*, cudaStream_t);
template cudaError_t launch_adjoint_init<double>(const double*, const double*, long long, const LatDev*, int,
                                                 const Consts<double>&, double*, double*, cudaStream_t);
template cudaError_t launch_misfit_seed<float>(const float*, const double*, const double*, long long, double, float*,
                                               double*, double*, cudaStream_t);
template cudaError_t launch_misfit_seed<double>(const double*, const double*, const double*, long long, double,
                                                double*, double*, double*, cudaStream_t);

}  // namespace lbm
