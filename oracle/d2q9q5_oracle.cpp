// CPU oracle for a two-dimensional coupled D2Q9-D2Q5 lattice Boltzmann scheme for the (rho, J, zeta)
// Navier-Stokes system: the extension that the conclusion of Dubois, Graille and Lallemand,
// "Recovering the full Navier Stokes equations with lattice Boltzmann schemes", names as the next
// step without specifying it. The readings below carry the one-dimensional scheme of sections 6 and
// 8 and its second-order analysis to two dimensions:
//   * with the coupling beta = 3/2 of eq. (lien-sigma-sigma) the scheme is, on data that do not
//     depend on y (and have J_y = 0), exactly the D1Q3Q3 scheme along x (and likewise along y);
//   * but that closure asks the D2Q5 entropy populations for a second moment of about
//     (p/rho + 2 lambda^2/3) zeta per direction, more than a D2Q5 with a non-negative rest
//     population can hold (lambda^2 zeta / 2), and the scheme is then linearly unstable at the
//     diagonal modes; the two-dimensional scheme therefore takes beta = 9/2, which keeps the
//     conductivity kappa of section 8 and puts the second moment near 0.4 lambda^2 zeta.
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct reference that the
// CUDA path is checked against. Only the tests, the smoke check and the benchmark's CPU-baseline
// leg load it. It shares no code, header, table or constant with the CUDA library.
//
// Everything is FP64 with no FMA contraction (compiled with -ffp-contract=off). Lattice: Nx x Ny
// nodes, periodic in both directions, node n = y Nx + x. Velocities v = lambda c with
//   D2Q9: c = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)     populations f0..f8
//   D2Q5: c = (0,0) (1,0) (0,1) (-1,0) (0,-1)                                 populations g0..g4
// Moments m = M f_d (the rows scaled by rho0, the entropy rows also by c_p, as in eq. M-d1q3q3):
//   rho = sum f, J = sum v f, e = sum (3|v|^2 - 4 lambda^2) f, xx = sum (vx^2 - vy^2) f,
//   xy = sum vx vy f, q = sum (3|v|^2 - 5 lambda^2) v f, h = sum (4 lambda^4 - 21/2 lambda^2 |v|^2
//   + 9/2 |v|^4) f; zeta = c_p sum g, psi = c_p sum v g, eps = c_p sum (3|v|^2 - 4 lambda^2) g,
//   xi = c_p sum (vx^2 - vy^2) g; in the order (rho, Jx, Jy, zeta, e, xx, xy, qx, qy, h, psi_x,
//   psi_y, eps, xi). M^{-1} by Gauss-Jordan elimination.
// One time step (the steps of the algorithm of section 8 in its order):
//   moments; p, T from eq. (gaz-parfait) with s = zeta / rho and p = rho r T; u = J / rho;
//   equilibria: with Pi = rho u u^T + p I and the entropy-energy tensor
//     E = s Pi + (rho c_p lambda^2 / (gamma beta)) log(T/T0) I (beta = 3/2: eq. eq-energie-entropie-d1q3q3),
//     e_eq = 3 tr Pi - 4 lambda^2 rho, xx_eq = Pi_xx - Pi_yy, xy_eq = Pi_xy,
//     q_eq = -lambda^2 J (so that sum vx vy^2 f_eq = lambda^2 Jx / 3), h_eq = 4 lambda^4 rho
//     - 6 lambda^2 tr Pi + 9 Q4 with Q4 = Pi_xx Pi_yy / rho,
//     psi_eq = zeta u, eps_eq = 3 tr E - 4 lambda^2 zeta, xi_eq = E_xx - E_yy;
//   relaxation: e, xx, xy at s_e; q at s_q; h at s_h; psi at s_psi (sigma_psi = beta (gamma/Pr)
//     sigma_e, so that sigma_psi dt (E_xx - s Pi_xx) = kappa log(T/T0) as in section 8); eps, xi at s_eps;
//   entropy-production source added to zeta: dt S with
//     S = (rho nu / (3 T)) (2 D:D + (div u)^2) + kappa |grad T|^2 / T^2,
//     D the strain rate, nu = sigma_e lambda dx (eq. nu-d1q3q3), kappa = rho nu c_p / Pr, the
//     derivatives by centred differences of u and T at time t;
//   back to populations, then streaming f_i(x + c_i dx) = f_i*(x).
// On one-dimensional data the source is the one of eq. (NS-rho-J-zeta): 2 D:D + (div u)^2 =
// 3 (d_x u)^2.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr int Q = 14;  // 9 + 5 populations per node

struct Phys2 {
  double gamma, Pr, cp, rho0, p0, s0, lambda, dx;
  double beta;  // coupling sigma_psi = beta (gamma / Pr) sigma_e; 3/2 is eq. (lien-sigma-sigma)
  int32_t source_on;
  int32_t pad;
};

struct Rates2 {
  double s_e, s_psi, s_eps, s_q, s_h;
};

const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1, /* g */ 0, 1, 0, -1, 0};
const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1, /* g */ 0, 0, 1, 0, -1};

struct Matrices {
  double M[Q][Q];
  double Minv[Q][Q];
};

void build_matrices(const Phys2& ph, Matrices& mm) {
  const double l = ph.lambda, l2 = l * l, c = ph.cp;
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) mm.M[i][j] = 0.0;
  for (int j = 0; j < 9; ++j) {
    const double vx = l * CX[j], vy = l * CY[j], v2 = vx * vx + vy * vy;
    mm.M[0][j] = 1.0;
    mm.M[1][j] = vx;
    mm.M[2][j] = vy;
    mm.M[4][j] = 3.0 * v2 - 4.0 * l2;
    mm.M[5][j] = vx * vx - vy * vy;
    mm.M[6][j] = vx * vy;
    mm.M[7][j] = (3.0 * v2 - 5.0 * l2) * vx;
    mm.M[8][j] = (3.0 * v2 - 5.0 * l2) * vy;
    mm.M[9][j] = 4.0 * l2 * l2 - 10.5 * l2 * v2 + 4.5 * v2 * v2;
  }
  for (int j = 9; j < Q; ++j) {
    const double vx = l * CX[j], vy = l * CY[j], v2 = vx * vx + vy * vy;
    mm.M[3][j] = c;
    mm.M[10][j] = c * vx;
    mm.M[11][j] = c * vy;
    mm.M[12][j] = c * (3.0 * v2 - 4.0 * l2);
    mm.M[13][j] = c * (vx * vx - vy * vy);
  }
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) mm.M[i][j] *= ph.rho0;
  // Gauss-Jordan elimination with partial pivoting on [M | I].
  double a[Q][2 * Q];
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < 2 * Q; ++j) a[i][j] = (j < Q) ? mm.M[i][j] : (j - Q == i ? 1.0 : 0.0);
  for (int col = 0; col < Q; ++col) {
    int piv = col;
    for (int i = col + 1; i < Q; ++i)
      if (std::fabs(a[i][col]) > std::fabs(a[piv][col])) piv = i;
    if (piv != col)
      for (int j = 0; j < 2 * Q; ++j) std::swap(a[col][j], a[piv][j]);
    const double inv = 1.0 / a[col][col];
    for (int j = 0; j < 2 * Q; ++j) a[col][j] *= inv;
    for (int i = 0; i < Q; ++i) {
      if (i == col) continue;
      const double f = a[i][col];
      if (f != 0.0)
        for (int j = 0; j < 2 * Q; ++j) a[i][j] -= f * a[col][j];
    }
  }
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) mm.Minv[i][j] = a[i][j + Q];
}

inline void matvec(const double (*A)[Q], const double* x, double* y) {
  for (int i = 0; i < Q; ++i) {
    double acc = 0.0;
    for (int j = 0; j < Q; ++j)
      if (A[i][j] != 0.0) acc = acc + A[i][j] * x[j];
    y[i] = acc;
  }
}

inline double gas_r(const Phys2& ph) { return ph.cp * (1.0 - 1.0 / ph.gamma); }
inline double T_ref(const Phys2& ph) { return ph.p0 / (ph.rho0 * gas_r(ph)); }

// Eq. (gaz-parfait): p = p0 (rho/rho0)^gamma exp(gamma (s - s0)/c_p), and p = rho r T.
inline void thermo(const Phys2& ph, double rho, double s, double& p, double& T) {
  p = ph.p0 * std::pow(rho / ph.rho0, ph.gamma) * std::exp(ph.gamma * (s - ph.s0) / ph.cp);
  T = p / (rho * gas_r(ph));
}

// The ten equilibrium values of the non-conserved moments, in the order of m[4..13].
inline void equilibria(const Phys2& ph, double rho, double ux, double uy, double zeta, double p, double T,
                       double* eq) {
  const double l2 = ph.lambda * ph.lambda;
  const double s = zeta / rho;
  const double Jx = rho * ux, Jy = rho * uy;
  const double Pxx = rho * ux * ux + p, Pyy = rho * uy * uy + p, Pxy = rho * ux * uy;
  const double L = (rho * ph.cp * l2 / (ph.gamma * ph.beta)) * std::log(T / T_ref(ph));
  const double Exx = s * Pxx + L, Eyy = s * Pyy + L;
  eq[0] = 3.0 * (Pxx + Pyy) - 4.0 * l2 * rho;                          // e
  eq[1] = Pxx - Pyy;                                                   // xx
  eq[2] = Pxy;                                                         // xy
  eq[3] = -l2 * Jx;                                                    // qx
  eq[4] = -l2 * Jy;                                                    // qy
  eq[5] = 4.0 * l2 * l2 * rho - 6.0 * l2 * (Pxx + Pyy) + 9.0 * Pxx * Pyy / rho;  // h
  eq[6] = zeta * ux;                                                   // psi_x
  eq[7] = zeta * uy;                                                   // psi_y
  eq[8] = 3.0 * (Exx + Eyy) - 4.0 * l2 * zeta;                         // eps
  eq[9] = Exx - Eyy;                                                   // xi
}

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

struct Work {
  std::vector<double> m, ux, uy, T;
};

void step(const Phys2& ph, const Matrices& mm, const Rates2& rt, int64_t Nx, int64_t Ny, const double* fd,
          double* out, Work& w, int nthreads) {
  const int64_t N = Nx * Ny;
  const double dt = ph.dx / ph.lambda;
  parallel_for(N, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t n = lo; n < hi; ++n) {
      double* m = &w.m[Q * n];
      matvec(mm.M, fd + Q * n, m);
      const double rho = m[0];
      w.ux[n] = m[1] / rho;
      w.uy[n] = m[2] / rho;
      double p;
      thermo(ph, rho, m[3] / rho, p, w.T[n]);
    }
  });
  const double sigma_e = 1.0 / rt.s_e - 0.5;
  const double nu = sigma_e * ph.lambda * ph.dx;
  const double rate[10] = {rt.s_e, rt.s_e, rt.s_e, rt.s_q, rt.s_q, rt.s_h, rt.s_psi, rt.s_psi, rt.s_eps, rt.s_eps};
  parallel_for(N, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t n = lo; n < hi; ++n) {
      const int64_t x = n % Nx, y = n / Nx;
      const double* m = &w.m[Q * n];
      const double rho = m[0], zeta = m[3], ux = w.ux[n], uy = w.uy[n], T = w.T[n];
      double p, Tn;
      thermo(ph, rho, zeta / rho, p, Tn);  // T = Tn, stored by the first pass
      double eq[10];
      equilibria(ph, rho, ux, uy, zeta, p, T, eq);
      double ms[Q];
      for (int k = 0; k < 4; ++k) ms[k] = m[k];
      for (int k = 0; k < 10; ++k) ms[4 + k] = m[4 + k] + rate[k] * (eq[k] - m[4 + k]);
      if (ph.source_on) {
        const int64_t xl = (x == 0) ? Nx - 1 : x - 1, xr = (x == Nx - 1) ? 0 : x + 1;
        const int64_t yd = (y == 0) ? Ny - 1 : y - 1, yu = (y == Ny - 1) ? 0 : y + 1;
        const int64_t nl = y * Nx + xl, nr = y * Nx + xr, nd = yd * Nx + x, nup = yu * Nx + x;
        const double h2 = 2.0 * ph.dx;
        const double dxux = (w.ux[nr] - w.ux[nl]) / h2, dyux = (w.ux[nup] - w.ux[nd]) / h2;
        const double dxuy = (w.uy[nr] - w.uy[nl]) / h2, dyuy = (w.uy[nup] - w.uy[nd]) / h2;
        const double dxT = (w.T[nr] - w.T[nl]) / h2, dyT = (w.T[nup] - w.T[nd]) / h2;
        const double shear = dyux + dxuy;
        const double DD = dxux * dxux + dyuy * dyuy + 0.5 * shear * shear;
        const double div = dxux + dyuy;
        const double kappa = rho * nu * ph.cp / ph.Pr;
        const double S = rho * nu / (3.0 * T) * (2.0 * DD + div * div) + kappa / (T * T) * (dxT * dxT + dyT * dyT);
        ms[3] = ms[3] + dt * S;
      }
      double fs[Q];
      matvec(mm.Minv, ms, fs);
      for (int i = 0; i < Q; ++i) {
        const int64_t xt = (x + CX[i] + Nx) % Nx, yt = (y + CY[i] + Ny) % Ny;
        out[Q * (yt * Nx + xt) + i] = fs[i];
      }
    }
  });
}

bool valid(const Phys2* ph, int64_t Nx, int64_t Ny) {
  if (!ph || Nx < 3 || Ny < 3) return false;
  return ph->lambda > 0 && ph->dx > 0 && ph->gamma > 1 && ph->cp > 0 && ph->rho0 > 0 && ph->p0 > 0 && ph->Pr > 0 &&
         ph->beta > 0;
}

}  // namespace

extern "C" {

typedef Phys2 oracle2d_phys;
typedef Rates2 oracle2d_rates;

// M and M^{-1} as row-major 14 x 14 arrays.
int oracle2d_matrices(const oracle2d_phys* ph, double* M, double* Minv) {
  if (!ph) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) { M[Q * i + j] = mm.M[i][j]; Minv[Q * i + j] = mm.Minv[i][j]; }
  return 0;
}

// Equilibrium populations f_d = M^{-1} m_eq(rho, J = rho u, zeta = rho s), node-major [N][14].
int oracle2d_init(const oracle2d_phys* ph, int64_t Nx, int64_t Ny, const double* rho, const double* ux,
                  const double* uy, const double* s, double* fd) {
  if (!valid(ph, Nx, Ny)) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  for (int64_t n = 0; n < Nx * Ny; ++n) {
    double p, T;
    thermo(*ph, rho[n], s[n], p, T);
    double m[Q];
    m[0] = rho[n];
    m[1] = rho[n] * ux[n];
    m[2] = rho[n] * uy[n];
    m[3] = rho[n] * s[n];
    equilibria(*ph, rho[n], ux[n], uy[n], m[3], p, T, m + 4);
    matvec(mm.Minv, m, fd + Q * n);
  }
  return 0;
}

// nsteps time steps in place.
int oracle2d_run(const oracle2d_phys* ph, const oracle2d_rates* rt, int64_t Nx, int64_t Ny, int64_t nsteps,
                 double* fd, int32_t nthreads) {
  if (!valid(ph, Nx, Ny) || !rt || nsteps < 0) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  const int64_t N = Nx * Ny;
  Work w;
  w.m.resize(Q * N);
  w.ux.resize(N);
  w.uy.resize(N);
  w.T.resize(N);
  std::vector<double> other(Q * N);
  double* a = fd;
  double* b = other.data();
  for (int64_t t = 0; t < nsteps; ++t) {
    step(*ph, mm, *rt, Nx, Ny, a, b, w, nthreads);
    std::swap(a, b);
  }
  if (a != fd) std::memcpy(fd, a, sizeof(double) * Q * N);
  return 0;
}

// Moments [N][14] in the order (rho, Jx, Jy, zeta, e, xx, xy, qx, qy, h, psi_x, psi_y, eps, xi).
int oracle2d_moments(const oracle2d_phys* ph, int64_t N, const double* fd, double* m) {
  if (!ph || N < 0) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  for (int64_t n = 0; n < N; ++n) matvec(mm.M, fd + Q * n, m + Q * n);
  return 0;
}

// Equilibrium values of the ten non-conserved moments [N][10] for the conserved moments of fd.
int oracle2d_equilibria(const oracle2d_phys* ph, int64_t N, const double* fd, double* eq) {
  if (!ph || N < 0) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  for (int64_t n = 0; n < N; ++n) {
    double m[Q];
    matvec(mm.M, fd + Q * n, m);
    double p, T;
    thermo(*ph, m[0], m[3] / m[0], p, T);
    equilibria(*ph, m[0], m[1] / m[0], m[2] / m[0], m[3], p, T, eq + 10 * n);
  }
  return 0;
}

}  // extern "C"
