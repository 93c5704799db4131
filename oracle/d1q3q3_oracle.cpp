// CPU oracle for the coupled D1Q3Q3 lattice Boltzmann scheme for the (rho, J, zeta)
// Navier-Stokes system (Dubois, Graille, Lallemand, "Recovering the full Navier Stokes
// equations with lattice Boltzmann schemes", sections 6 and 8).
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct reference that the
// CUDA path is checked against. Only the tests, the smoke check and the benchmark's CPU-baseline
// leg load it. It shares no code, header, table or constant with the CUDA library.
//
// Everything is FP64 (or forward-mode dual numbers built on FP64), with no FMA contraction
// (compiled with -ffp-contract=off). Each time step follows the algorithm of section 8, steps
// (i)-(viii), in that order and notation:
//   (ii)   m = M f_d with the 6x6 matrix M of eq. (M-d1q3q3), applied as a matrix-vector product;
//   (iii)  rates: s_e given, sigma_psi = (3/2)(gamma/Pr) sigma_e (eq. lien-sigma-sigma),
//          s_eps = 1.5, Henon's sigma = 1/s - 1/2 (eq. henon-d1q3q3);
//   (iv)   e_eq = 3(rho u^2 + p) - 2 lambda^2 rho        (eq. energie-equilibre),
//          psi_eq = zeta u                               (eq. psi-equilibre),
//          eps_eq = (2 rho c_p lambda^2/gamma) log(T/T0) + e_eq s  (eq. eq-energie-entropie-d1q3q3),
//          with the polytropic equation of state p(rho, s) of eq. (gaz-parfait) and p = rho r T;
//   (v)    relaxation of e, psi, eps (eq. relaxation-d1q3q3);
//   (vii)  entropy-production source of eq. (NS-rho-J-zeta), third line, with second-order centred
//          differences for d_x u and d_x T, nu = sigma_e lambda dx (eq. nu-d1q3q3),
//          kappa = rho nu c_p / Pr (definition of Pr, section 5), added to zeta;
//   (vi)   f_d* = M^{-1} m*, with M^{-1} obtained by Gauss-Jordan elimination of M;
//   (viii) streaming of eq. (iteration-d1q3q3).
// Readings where the paper is silent: the source is evaluated from the fields at time t (before
// relaxation, on the same time level for j-1, j, j+1) and added to zeta after relaxation, the
// equilibria using the un-sourced zeta; bounce-back walls (not in the paper) are halfway
// bounce-back with ghost values u_{-1} = -u_0, T_{-1} = T_0 (mirrored at the right end).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------------
// Forward-mode dual numbers with a fixed number of tangent directions.
constexpr int KD = 8;

struct Dual {
  double v;
  double d[KD];
  Dual() : v(0.0) { for (int k = 0; k < KD; ++k) d[k] = 0.0; }
  Dual(double x) : v(x) { for (int k = 0; k < KD; ++k) d[k] = 0.0; }  // NOLINT: implicit on purpose
};
inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int k = 0; k < KD; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int k = 0; k < KD; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int k = 0; k < KD; ++k) r.d[k] = -a.d[k]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int k = 0; k < KD; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  for (int k = 0; k < KD; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
  return r;
}
inline Dual operator+(const Dual& a, double b) { return a + Dual(b); }
inline Dual operator+(double a, const Dual& b) { return Dual(a) + b; }
inline Dual operator-(const Dual& a, double b) { return a - Dual(b); }
inline Dual operator-(double a, const Dual& b) { return Dual(a) - b; }
inline Dual operator*(const Dual& a, double b) { Dual r(a.v * b); for (int k = 0; k < KD; ++k) r.d[k] = a.d[k] * b; return r; }
inline Dual operator*(double a, const Dual& b) { return b * a; }
inline Dual operator/(const Dual& a, double b) { Dual r(a.v / b); for (int k = 0; k < KD; ++k) r.d[k] = a.d[k] / b; return r; }
inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }
inline Dual log(const Dual& a) { Dual r(std::log(a.v)); for (int k = 0; k < KD; ++k) r.d[k] = a.d[k] / a.v; return r; }
inline Dual exp(const Dual& a) { Dual r(std::exp(a.v)); for (int k = 0; k < KD; ++k) r.d[k] = r.v * a.d[k]; return r; }
inline Dual pow(const Dual& a, double g) { return exp(g * log(a)); }

inline double value_of(double x) { return x; }
inline double value_of(const Dual& x) { return x.v; }

// ---------------------------------------------------------------------------------------------
// Physical and lattice constants. p0 is the reference pressure of eq. (gaz-parfait).
struct Phys {
  double gamma, Pr, cp, rho0, p0, s0, lambda, dx;
  int32_t source_on;
  int32_t bc;  // 0 periodic, 1 halfway bounce-back at both ends
  // Equilibria: 0 the nonlinear ones of section 8; 1 the linear ones of eq. (equilibres-NS-linearise)
  // (section 7) around the state of velocity u0_lin and specific entropy s0_lin.
  int32_t eq_mode;
  int32_t pad;
  double u0_lin, s0_lin;
};

template <class R>
struct Rates {
  R s_e, s_psi, s_eps;
};

// Moment ordering m = (rho, J, zeta, e, psi, eps); population ordering f_d = (f0, f+, f-, g0, g+, g-).
struct Matrices {
  double M[6][6];
  double Minv[6][6];
};

// Eq. (M-d1q3q3), written entry by entry.
void build_matrices(const Phys& ph, Matrices& mm) {
  const double l = ph.lambda, c = ph.cp, r0 = ph.rho0;
  const double A[6][6] = {
      {1, 1, 1, 0, 0, 0},
      {0, l, -l, 0, 0, 0},
      {0, 0, 0, c, c, c},
      {-2 * l * l, l * l, l * l, 0, 0, 0},
      {0, 0, 0, 0, c * l, -c * l},
      {0, 0, 0, -2 * c * l * l, c * l * l, c * l * l},
  };
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) mm.M[i][j] = r0 * A[i][j];
  // Gauss-Jordan elimination with partial pivoting on [M | I].
  double a[6][12];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 12; ++j) a[i][j] = (j < 6) ? mm.M[i][j] : (j - 6 == i ? 1.0 : 0.0);
  for (int col = 0; col < 6; ++col) {
    int piv = col;
    for (int i = col + 1; i < 6; ++i)
      if (std::fabs(a[i][col]) > std::fabs(a[piv][col])) piv = i;
    if (piv != col)
      for (int j = 0; j < 12; ++j) { double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t; }
    const double inv = 1.0 / a[col][col];
    for (int j = 0; j < 12; ++j) a[col][j] *= inv;
    for (int i = 0; i < 6; ++i) {
      if (i == col) continue;
      const double f = a[i][col];
      if (f != 0.0)
        for (int j = 0; j < 12; ++j) a[i][j] -= f * a[col][j];
    }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) mm.Minv[i][j] = a[i][j + 6];
}

template <class R>
inline void matvec(const double (*A)[6], const R* x, R* y) {
  for (int i = 0; i < 6; ++i) {
    R acc(0.0);
    for (int j = 0; j < 6; ++j)
      if (A[i][j] != 0.0) acc = acc + A[i][j] * x[j];
    y[i] = acc;
  }
}

inline double gas_r(const Phys& ph) { return ph.cp * (1.0 - 1.0 / ph.gamma); }
inline double T_ref(const Phys& ph) { return ph.p0 / (ph.rho0 * gas_r(ph)); }

// Eq. (gaz-parfait): p = p0 (rho/rho0)^gamma exp(gamma (s - s0)/c_p), and p = rho r T.
template <class R>
inline void thermo(const Phys& ph, const R& rho, const R& s, R& p, R& T) {
  using std::exp;
  using std::pow;
  p = ph.p0 * pow(rho / ph.rho0, ph.gamma) * exp(ph.gamma * (s - ph.s0) / ph.cp);
  T = p / (rho * gas_r(ph));
}

// Equilibrium moments (iv) from the conserved moments and the thermodynamic state.
template <class R>
inline void equilibria(const Phys& ph, const R& rho, const R& u, const R& zeta, const R& s,
                       const R& p, const R& T, R& e_eq, R& psi_eq, R& eps_eq) {
  using std::log;
  const double l2 = ph.lambda * ph.lambda;
  if (ph.eq_mode == 1) {
    // Eq. (equilibres-NS-linearise), as printed (lattice units lambda = c_p = 1), linear in
    // (rho, J, zeta) around (rho0, u0, s0) with c0^2 = gamma p0 / rho0.
    const double u0 = ph.u0_lin, s0 = ph.s0_lin, cp = ph.cp, g = ph.gamma;
    const double c02 = g * ph.p0 / ph.rho0;
    const R J = rho * u;
    e_eq = (3.0 * (1.0 - s0 / cp) * c02 - 3.0 * u0 * u0 - 2.0 * l2) * rho + 6.0 * u0 * J + 3.0 * (u0 * u0 / cp) * zeta;
    psi_eq = -u0 * s0 * rho + s0 * J + u0 * zeta;
    eps_eq = (-3.0 * (s0 * s0 * c02) - 6.0 * s0 * u0 * u0 + 3.0 * s0 * c02 + 2.0 - 2.0 * s0 - 2.0 / g) * rho +
             6.0 * u0 * s0 * J + 3.0 * (cp * u0 * u0 + s0 * c02) * zeta;
    (void)s; (void)p; (void)T;
    return;
  }
  e_eq = 3.0 * (rho * u * u + p) - 2.0 * l2 * rho;                        // eq. energie-equilibre
  psi_eq = zeta * u;                                                      // eq. psi-equilibre
  eps_eq = (2.0 * rho * ph.cp * l2 / ph.gamma) * log(T / T_ref(ph)) + e_eq * s;  // eq. eq-energie-entropie
}

// Equilibrium initialisation: f_d = M^{-1} m_eq(rho, J = rho u, zeta = rho s).
template <class R>
void init_state(const Phys& ph, const Matrices& mm, int64_t N, const R* rho, const R* u, const R* s,
                R* fd) {
  for (int64_t j = 0; j < N; ++j) {
    R p, T;
    thermo(ph, rho[j], s[j], p, T);
    R m[6];
    m[0] = rho[j];
    m[1] = rho[j] * u[j];
    m[2] = rho[j] * s[j];
    equilibria(ph, rho[j], u[j], m[2], s[j], p, T, m[3], m[4], m[5]);
    matvec(mm.Minv, m, fd + 6 * j);
  }
}

// Runs fn(lo, hi) over [0, N) split into nthreads contiguous chunks.
template <class F>
void parallel_for(int64_t N, int nthreads, F fn) {
  if (nthreads <= 1 || N < 4096) { fn(int64_t(0), N); return; }
  std::vector<std::thread> th;
  const int64_t chunk = (N + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    const int64_t lo = t * chunk, hi = std::min<int64_t>(N, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back([=]() { fn(lo, hi); });
  }
  for (auto& x : th) x.join();
}

// One time step f_d(t) -> f_d(t + dt), node-major arrays [N][6].
template <class R>
void step(const Phys& ph, const Matrices& mm, const Rates<R>& rt, int64_t N, const R* fd, R* out,
          std::vector<R>& mbuf, std::vector<R>& ubuf, std::vector<R>& Tbuf, std::vector<R>& sbuf,
          std::vector<R>& pbuf, int nthreads) {
  const double dt = ph.dx / ph.lambda;
  // (ii) moments, then the thermodynamic state of every node at time t.
  parallel_for(N, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t j = lo; j < hi; ++j) {
      R* m = &mbuf[6 * j];
      matvec(mm.M, fd + 6 * j, m);
      const R rho = m[0], J = m[1], zeta = m[2];
      ubuf[j] = J / rho;
      sbuf[j] = zeta / rho;
      thermo(ph, rho, sbuf[j], pbuf[j], Tbuf[j]);
    }
  });
  // (iii) relaxation rates: s_e and s_psi as given (the caller applies the coupling of
  // eq. lien-sigma-sigma), nu from eq. (nu-d1q3q3).
  const R sigma_e = 1.0 / rt.s_e - 0.5;
  const R nu = sigma_e * ph.lambda * ph.dx;
  parallel_for(N, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t j = lo; j < hi; ++j) {
      const R* m = &mbuf[6 * j];
      const R rho = m[0], J = m[1], zeta = m[2], e = m[3], psi = m[4], eps = m[5];
      const R u = ubuf[j], s = sbuf[j], p = pbuf[j], T = Tbuf[j];
      (void)J;
      // (iv) equilibria.
      R e_eq, psi_eq, eps_eq;
      equilibria(ph, rho, u, zeta, s, p, T, e_eq, psi_eq, eps_eq);
      // (v) relaxation.
      R ms[6];
      ms[0] = rho;
      ms[1] = m[1];
      ms[2] = zeta;
      ms[3] = e + rt.s_e * (e_eq - e);
      ms[4] = psi + rt.s_psi * (psi_eq - psi);
      ms[5] = eps + rt.s_eps * (eps_eq - eps);
      // (vii) entropy production with centred differences of u and T at time t.
      if (ph.source_on) {
        R ul, ur, Tl, Tr;
        if (ph.bc == 0) {
          const int64_t jl = (j == 0) ? N - 1 : j - 1, jr = (j == N - 1) ? 0 : j + 1;
          ul = ubuf[jl]; ur = ubuf[jr]; Tl = Tbuf[jl]; Tr = Tbuf[jr];
        } else {
          if (j == 0) { ul = -u; Tl = T; } else { ul = ubuf[j - 1]; Tl = Tbuf[j - 1]; }
          if (j == N - 1) { ur = -u; Tr = T; } else { ur = ubuf[j + 1]; Tr = Tbuf[j + 1]; }
        }
        const R dudx = (ur - ul) / (2.0 * ph.dx);
        const R dTdx = (Tr - Tl) / (2.0 * ph.dx);
        const R kappa = rho * nu * ph.cp / ph.Pr;
        const R S = rho * nu / T * dudx * dudx + kappa / (T * T) * dTdx * dTdx;
        ms[2] = ms[2] + dt * S;
      }
      // (vi) back to particles.
      R fs[6];
      matvec(mm.Minv, ms, fs);
      // (viii) streaming: f0, g0 stay; f+, g+ move to j+1; f-, g- move to j-1.
      out[6 * j + 0] = fs[0];
      out[6 * j + 3] = fs[3];
      if (j < N - 1) { out[6 * (j + 1) + 1] = fs[1]; out[6 * (j + 1) + 4] = fs[4]; }
      else if (ph.bc == 0) { out[1] = fs[1]; out[4] = fs[4]; }
      else { out[6 * j + 2] = fs[1]; out[6 * j + 5] = fs[4]; }
      if (j > 0) { out[6 * (j - 1) + 2] = fs[2]; out[6 * (j - 1) + 5] = fs[5]; }
      else if (ph.bc == 0) { out[6 * (N - 1) + 2] = fs[2]; out[6 * (N - 1) + 5] = fs[5]; }
      else { out[6 * j + 1] = fs[2]; out[6 * j + 4] = fs[5]; }
    }
  });
}

template <class R>
void run(const Phys& ph, const Rates<R>& rt, int64_t N, int64_t nsteps, R* fd, int nthreads) {
  Matrices mm;
  build_matrices(ph, mm);
  std::vector<R> other(6 * N), mbuf(6 * N), ubuf(N), Tbuf(N), sbuf(N), pbuf(N);
  R* a = fd;
  R* b = other.data();
  for (int64_t t = 0; t < nsteps; ++t) {
    step(ph, mm, rt, N, a, b, mbuf, ubuf, Tbuf, sbuf, pbuf, nthreads);
    R* tmp = a; a = b; b = tmp;
  }
  if (a != fd) std::memcpy(fd, a, sizeof(R) * 6 * N);
}

bool valid(const Phys* ph, int64_t N) {
  if (!ph || N < 3) return false;
  if (!(ph->lambda > 0) || !(ph->dx > 0) || !(ph->gamma > 1) || !(ph->cp > 0) || !(ph->rho0 > 0) ||
      !(ph->p0 > 0) || !(ph->Pr > 0))
    return false;
  // The printed linear equilibria are consistent in units only for lambda = c_p = 1.
  if (ph->eq_mode == 1 && (ph->lambda != 1.0 || ph->cp != 1.0)) return false;
  if (ph->eq_mode != 0 && ph->eq_mode != 1) return false;
  return ph->bc == 0 || ph->bc == 1;
}

}  // namespace

extern "C" {

typedef Phys oracle_phys;

// Coupled rate of eq. (lien-sigma-sigma): sigma_psi = (3/2)(gamma/Pr) sigma_e, s = 1/(sigma + 1/2).
double oracle_coupled_s_psi(double s_e, double gamma, double Pr) {
  const double sigma_e = 1.0 / s_e - 0.5;
  const double sigma_psi = 1.5 * (gamma / Pr) * sigma_e;
  return 1.0 / (sigma_psi + 0.5);
}

// M and M^{-1} as row-major 6x6 arrays.
int oracle_matrices(const oracle_phys* ph, double* M, double* Minv) {
  if (!ph) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) { M[6 * i + j] = mm.M[i][j]; Minv[6 * i + j] = mm.Minv[i][j]; }
  return 0;
}

// Specific entropy from (rho, p) by inverting eq. (gaz-parfait).
int oracle_entropy_from_pressure(const oracle_phys* ph, int64_t N, const double* rho, const double* p,
                                 double* s) {
  if (!ph) return -1;
  for (int64_t j = 0; j < N; ++j)
    s[j] = ph->s0 + (ph->cp / ph->gamma) * std::log((p[j] / ph->p0) * std::pow(ph->rho0 / rho[j], ph->gamma));
  return 0;
}

// Equilibrium initial populations [N][6] from rho, u, s.
int oracle_init(const oracle_phys* ph, int64_t N, const double* rho, const double* u, const double* s,
                double* fd) {
  if (!valid(ph, N)) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  init_state<double>(*ph, mm, N, rho, u, s, fd);
  return 0;
}

// Equilibrium moments at every node of a state: out [N][3] = (e_eq, psi_eq, eps_eq).
int oracle_equilibria(const oracle_phys* ph, int64_t N, const double* fd, double* out) {
  if (!ph) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  for (int64_t j = 0; j < N; ++j) {
    double m[6];
    matvec(mm.M, fd + 6 * j, m);
    const double rho = m[0], u = m[1] / rho, s = m[2] / rho;
    double p, T;
    thermo(*ph, rho, s, p, T);
    equilibria(*ph, rho, u, m[2], s, p, T, out[3 * j], out[3 * j + 1], out[3 * j + 2]);
  }
  return 0;
}

// Advances fd [N][6] in place by nsteps steps. rates = (s_e, s_psi, s_eps).
int oracle_run(const oracle_phys* ph, const double* rates, int64_t N, int64_t nsteps, double* fd,
               int32_t nthreads) {
  if (!valid(ph, N) || nsteps < 0) return -1;
  Rates<double> rt{rates[0], rates[1], rates[2]};
  run<double>(*ph, rt, N, nsteps, fd, nthreads);
  return 0;
}

// Moments m = M f_d per node, [N][6] -> [N][6].
int oracle_moments(const oracle_phys* ph, int64_t N, const double* fd, double* m) {
  if (!ph) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  for (int64_t j = 0; j < N; ++j) matvec(mm.M, fd + 6 * j, m + 6 * j);
  return 0;
}

// Global sums (rho, J, zeta, total energy rho E = p/(gamma-1) + rho u^2/2) and a flag word:
// bit 0 any non-finite population, bit 1 any rho <= 0, bit 2 any T <= 0 (or non-finite).
int oracle_diagnostics(const oracle_phys* ph, int64_t N, const double* fd, double* sums, int32_t* flags) {
  if (!ph) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  double a[4] = {0, 0, 0, 0};
  int32_t fl = 0;
  for (int64_t j = 0; j < N; ++j) {
    for (int k = 0; k < 6; ++k)
      if (!std::isfinite(fd[6 * j + k])) fl |= 1;
    double m[6];
    matvec(mm.M, fd + 6 * j, m);
    const double rho = m[0], u = m[1] / rho, s = m[2] / rho;
    double p, T;
    thermo(*ph, rho, s, p, T);
    if (!(rho > 0)) fl |= 2;
    if (!(T > 0) || !std::isfinite(T)) fl |= 4;
    a[0] += m[0];
    a[1] += m[1];
    a[2] += m[2];
    a[3] += p / (ph->gamma - 1.0) + 0.5 * rho * u * u;
  }
  for (int k = 0; k < 4; ++k) sums[k] = a[k];
  *flags = fl;
  return 0;
}

// Forward-mode tangents. ndir <= 8 directions. Initial state from (rho, u) with tangents
// drho[ndir][N], du[ndir][N] at fixed specific entropy s; rates (s_e, s_psi) with tangents
// drates[ndir][2] (s_eps is not differentiated). Runs nsteps steps and returns the final
// populations fd [N][6] and their tangents dfd [ndir][N][6].
int oracle_run_tangent(const oracle_phys* ph, const double* rates, const double* drates, int32_t ndir,
                       int64_t N, int64_t nsteps, const double* rho, const double* u, const double* s,
                       const double* drho, const double* du, double* fd, double* dfd, int32_t nthreads) {
  if (!valid(ph, N) || ndir < 0 || ndir > KD || nsteps < 0) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  std::vector<Dual> r(N), v(N), sv(N), f(6 * N);
  for (int64_t j = 0; j < N; ++j) {
    r[j] = Dual(rho[j]);
    v[j] = Dual(u[j]);
    sv[j] = Dual(s[j]);
    for (int k = 0; k < ndir; ++k) { r[j].d[k] = drho[k * N + j]; v[j].d[k] = du[k * N + j]; }
  }
  init_state<Dual>(*ph, mm, N, r.data(), v.data(), sv.data(), f.data());
  Rates<Dual> rt{Dual(rates[0]), Dual(rates[1]), Dual(rates[2])};
  for (int k = 0; k < ndir; ++k) { rt.s_e.d[k] = drates[2 * k]; rt.s_psi.d[k] = drates[2 * k + 1]; }
  run<Dual>(*ph, rt, N, nsteps, f.data(), nthreads);
  for (int64_t i = 0; i < 6 * N; ++i) {
    fd[i] = f[i].v;
    for (int k = 0; k < ndir; ++k) dfd[k * 6 * N + i] = f[i].d[k];
  }
  return 0;
}

// Tangent of one step with respect to the populations: given fd [N][6] and ndir tangent
// populations dfd0 [ndir][N][6], returns the stepped state and the stepped tangents.
int oracle_step_jvp(const oracle_phys* ph, const double* rates, int32_t ndir, int64_t N, int64_t nsteps,
                    const double* fd0, const double* dfd0, double* fd, double* dfd) {
  if (!valid(ph, N) || ndir < 0 || ndir > KD) return -1;
  std::vector<Dual> f(6 * N);
  for (int64_t i = 0; i < 6 * N; ++i) {
    f[i] = Dual(fd0[i]);
    for (int k = 0; k < ndir; ++k) f[i].d[k] = dfd0[k * 6 * N + i];
  }
  Rates<Dual> rt{Dual(rates[0]), Dual(rates[1]), Dual(rates[2])};
  run<Dual>(*ph, rt, N, nsteps, f.data(), 1);
  for (int64_t i = 0; i < 6 * N; ++i) {
    fd[i] = f[i].v;
    for (int k = 0; k < ndir; ++k) dfd[k * 6 * N + i] = f[i].d[k];
  }
  return 0;
}

}  // extern "C"
