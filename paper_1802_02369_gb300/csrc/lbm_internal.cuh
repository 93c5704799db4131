// Internal declarations of the D1Q3Q3 CUDA library: per-lattice parameter records, the constant
// block passed to kernels, and the per-node collision of section 8 written on shifted
// populations. Used by the .cu files of this library only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Per-lattice record on the device. tile0 is the index of the lattice's first tile for the current
// tile width; chunk0 the index of its first diagnostics chunk.
struct LatDev {
  long long offset, n, tile0, chunk0;
  double s_e, s_psi, s_eps;
  double q_src;    // sigma_e / 4: the source reads dt S = rho sigma_e/(4T) [du^2 + (c_p/Pr) dT^2 / T]
  double s0;       // reference entropy of eq. (gaz-parfait) for this lattice
  double zeta_r;   // rest-state moments removed from the stored populations: zeta_r = rho0 s0,
  double eps_r;    //   eps_r = e_r s0 (e_r = 3 p0 - 2 lambda^2 rho0)
  double wg0, wg1; // rest g populations (g0, g+ = g-)
  int bc, pad;
};

// Constants shared by all lattices, converted to the arithmetic type R on the host.
template <typename R>
struct Consts {
  R rho0, lam, two_lam2;          // rho0, lambda, 2 lambda^2
  R inv_af, inv_af_l, inv_af_l2;  // 1/rho0, 1/(rho0 lambda), 1/(rho0 lambda^2)
  R af_l, af_l2;                  // rho0 lambda, rho0 lambda^2
  R ag, ag_l, ag_l2;              // rho0 c_p, rho0 c_p lambda, rho0 c_p lambda^2
  R inv_ag, inv_ag_l, inv_ag_l2;
  R gamma, inv_cp, p0, inv_r;     // gamma, 1/c_p, p0, 1/r with r = c_p (1 - 1/gamma)
  R e_r;                          // 3 p0 - 2 lambda^2 rho0
  R cp_log;                       // (1 - 1/gamma) c_p
  R cp_over_Pr;                   // c_p / Pr
  int source_on;
};

__device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }

// Moments and thermodynamic state of one node from its shifted populations
// ft = f - w (order f0, f+, f-, g0, g+, g-). Everything returned is a deviation from the rest
// state where marked "t" (tilde).
template <typename R>
struct Node {
  R rt, J, et;       // rho - rho0, J, e - e_r
  R zt, psi, epst;   // zeta - zeta_r, psi, eps - eps_r
  R rho, inv_rho, u, ds, lnr, pt, T;  // rho, 1/rho, u, s - s0, log(rho/rho0), p - p0, T
};

template <typename R>
__device__ __forceinline__ void node_state(const R f[6], const Consts<R>& c, R s0, Node<R>& m) {
  // (ii) m = M f_d, eq. (M-d1q3q3), applied to the deviations from the rest populations.
  m.rt = c.rho0 * (f[0] + f[1] + f[2]);
  m.J = c.af_l * (f[1] - f[2]);
  m.et = c.af_l2 * (f[1] + f[2] - R(2) * f[0]);
  m.zt = c.ag * (f[3] + f[4] + f[5]);
  m.psi = c.ag_l * (f[4] - f[5]);
  m.epst = c.ag_l2 * (f[4] + f[5] - R(2) * f[3]);
  // Thermodynamics, eq. (gaz-parfait): p = p0 (rho/rho0)^gamma exp(gamma (s - s0)/c_p), p = rho r T.
  m.rho = c.rho0 + m.rt;
  m.inv_rho = R(1) / m.rho;
  m.u = m.J * m.inv_rho;
  m.ds = (m.zt - m.rt * s0) * m.inv_rho;  // zeta - rho s0 = zeta_t - rho_t s0
  m.lnr = m_log1p(m.rt * c.inv_af);
  m.pt = c.p0 * m_expm1(c.gamma * (m.lnr + m.ds * c.inv_cp));
  m.T = (c.p0 + m.pt) * m.inv_rho * c.inv_r;
}

// Steps (iv)-(vii) for one node: equilibria, relaxation, entropy source; returns the shifted
// post-collision populations fs = M^{-1} m* - w.
template <typename R>
__device__ __forceinline__ void node_collide(const Node<R>& m, R ul, R ur, R Tl, R Tr, R s_e, R s_psi,
                                             R s_eps, R q_src, R s0, const Consts<R>& c, R fs[6]) {
  // (iv) equilibria: e_eq (eq. energie-equilibre), psi_eq = zeta u (eq. psi-equilibre), and the
  // polytropic form of eq. (eq-energie-entropie-d1q3q3), all as deviations from the rest state.
  const R s = s0 + m.ds;
  const R zeta = m.rho * s;
  const R e_eq_t = R(3) * (m.J * m.u + m.pt) - c.two_lam2 * m.rt;
  const R psi_eq = zeta * m.u;
  const R eps_eq_t = c.two_lam2 * m.rho * (m.ds + c.cp_log * m.lnr) + e_eq_t * s + c.e_r * m.ds;
  // (v) relaxation, eq. (relaxation-d1q3q3).
  const R es = m.et + s_e * (e_eq_t - m.et);
  const R psis = m.psi + s_psi * (psi_eq - m.psi);
  const R epss = m.epst + s_eps * (eps_eq_t - m.epst);
  // (vii) entropy production of eq. (NS-rho-J-zeta) with centred differences, added to zeta.
  R zs = m.zt;
  if (c.source_on) {
    const R du = ur - ul, dT = Tr - Tl;
    const R inv_T = R(1) / m.T;
    zs += q_src * m.rho * inv_T * (du * du + c.cp_over_Pr * dT * dT * inv_T);
  }
  // (vi) f_d* = M^{-1} m*, block by block: x0 = (r - q)/3, x+- = (2r + q)/6 +- j/2.
  {
    const R r = m.rt * c.inv_af, j = m.J * c.inv_af_l, q = es * c.inv_af_l2;
    const R h = (R(2) * r + q) * R(1.0 / 6.0);
    fs[0] = (r - q) * R(1.0 / 3.0);
    fs[1] = h + R(0.5) * j;
    fs[2] = h - R(0.5) * j;
  }
  {
    const R r = zs * c.inv_ag, j = psis * c.inv_ag_l, q = epss * c.inv_ag_l2;
    const R h = (R(2) * r + q) * R(1.0 / 6.0);
    fs[3] = (r - q) * R(1.0 / 3.0);
    fs[4] = h + R(0.5) * j;
    fs[5] = h - R(0.5) * j;
  }
}

// Host-side launchers (lbm_step.cu).
template <typename R>
cudaError_t launch_step_tiles(const R* in, R* out, long long plane, const LatDev* lat, int B,
                              long long ntiles, int K, int NT, const Consts<R>& c, cudaStream_t st,
                              int grid_cap);

}  // namespace lbm
