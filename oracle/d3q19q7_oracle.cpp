// CPU oracle for a three-dimensional coupled D3Q19-D3Q7 lattice Boltzmann scheme for the (rho, J, zeta)
// Navier-Stokes system: the second extension that the conclusion of Dubois, Graille and Lallemand,
// "Recovering the full Navier Stokes equations with lattice Boltzmann schemes", names without
// specifying it. The readings are those of the two-dimensional D2Q9-D2Q5 scheme carried to three
// dimensions (the one-dimensional scheme of sections 6 and 8 and its second-order analysis):
//   * with the coupling beta = 3/2 of eq. (lien-sigma-sigma) the scheme is, on data that depend on one
//     coordinate only (the velocity along it), exactly the D1Q3Q3 scheme along that axis;
//   * the D3Q7 entropy populations hold at most lambda^2 zeta / 3 per direction with a non-negative
//     rest population, so the three-dimensional scheme takes beta = 9 (second moment about
//     0.29 lambda^2 zeta per direction at c0 = lambda / 2), keeping the conductivity kappa of section 8.
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct reference that the
// CUDA path is checked against. Only the tests, the smoke check and the benchmark's CPU-baseline
// leg load it. It shares no code, header, table or constant with the CUDA library.
//
// Everything is FP64 with no FMA contraction (compiled with -ffp-contract=off). Lattice: Nx x Ny x Nz
// nodes, periodic in all directions, node n = (z Ny + y) Nx + x. Velocities v = lambda c with
//   D3Q19: c = 0; (+-1,0,0), (0,+-1,0), (0,0,+-1) (in that order); then (1,1,0) (-1,-1,0) (1,-1,0)
//          (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1):
//          populations f0..f18;
//   D3Q7:  c = 0; (+-1,0,0), (0,+-1,0), (0,0,+-1): populations g0..g6.
// Moments m = M f_d (rows scaled by rho0, the entropy rows also by c_p, as in eq. M-d1q3q3), in the
// order (rho, Jx, Jy, Jz, zeta, e, pxx, pww, pxy, pyz, pxz, qx, qy, qz, mx, my, mz, eps, pixx, piww,
// psi_x, psi_y, psi_z, eps7, xixx, xiww), with the patterns (|c|^2 = c.c; the D3Q19 ones mutually orthogonal)
//   e = 19|c|^2 - 30, pxx = 3cx^2 - |c|^2, pww = cy^2 - cz^2, pxy = cx cy, pyz = cy cz, pxz = cx cz,
//   q = (5|c|^2 - 9) c, mx = (cy^2 - cz^2) cx, my = (cz^2 - cx^2) cy, mz = (cx^2 - cy^2) cz,
//   eps = (21|c|^4 - 53|c|^2 + 24)/2, pixx = (3|c|^2 - 5)(3cx^2 - |c|^2), piww = (3|c|^2 - 5)(cy^2 - cz^2);
//   zeta = 1, psi = c, eps7 = 3|c|^2 - 6, xixx = 3cx^2 - |c|^2, xiww = cy^2 - cz^2 on the D3Q7 set (eps7
//   is the row 3|c|^2 - 2d of the one-dimensional eps, d = 3: the production, added to zeta with the
//   other moments held, then feeds each axis as in one dimension); each times lambda^k for its
//   degree k. M^{-1} by Gauss-Jordan elimination.
// One time step (the steps of the algorithm of section 8 in its order):
//   moments; p, T from eq. (gaz-parfait) with s = zeta / rho and p = rho r T; u = J / rho;
//   equilibria, with Pi = rho u u^T + p I, Q4_ab = Pi_aa Pi_bb / rho (a != b; the Gaussian fourth
//   moment sum va^2 vb^2 f) and E = s Pi + (rho c_p lambda^2 / (gamma beta)) log(T/T0) I:
//     e = 19 tr Pi - 30 lambda^2 rho, pxx = 3 Pi_xx - tr Pi, pww = Pi_yy - Pi_zz, pab = Pi_ab,
//     q = -(2/3) lambda^2 J (so that sum va vb^2 f_eq = lambda^2 Ja / 3, b != a), m = 0,
//     eps = 12 lambda^4 rho - 16 lambda^2 tr Pi + 21 (Q4_xy + Q4_yz + Q4_xz),
//     pixx = 2 lambda^2 (tr Pi - 3 Pi_xx) + 3 (Q4_xy + Q4_xz) - 6 Q4_yz,
//     piww = -2 lambda^2 (Pi_yy - Pi_zz) + 3 (Q4_xy - Q4_xz),
//     psi = zeta u, eps7 = 3 tr E - 6 lambda^2 zeta, xixx = 3 E_xx - tr E, xiww = E_yy - E_zz;
//   relaxation: e, pxx, pww, pxy, pyz, pxz at s_e; q and m at s_q; eps, pixx, piww at s_h; psi at
//     s_psi (sigma_psi = beta (gamma/Pr) sigma_e); eps7, xixx, xiww at s_eps;
//   entropy-production source added to zeta: dt [rho nu (2 D:D + (div u)^2) / (3T) + kappa |grad T|^2/T^2],
//     nu = sigma_e lambda dx (eq. nu-d1q3q3), kappa = rho nu c_p / Pr, centred differences at time t;
//   back to populations, then streaming f_i(x + c_i dx) = f_i*(x).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr int Q = 26;  // 19 + 7 populations per node

struct Phys3 {
  double gamma, Pr, cp, rho0, p0, s0, lambda, dx;
  double beta;  // coupling sigma_psi = beta (gamma / Pr) sigma_e; 3/2 is eq. (lien-sigma-sigma)
  int32_t source_on;
  int32_t pad;
};

struct Rates3 {
  double s_e, s_psi, s_eps, s_q, s_h;
};

const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, /* g */ 0, 1, -1, 0, 0, 0, 0};
const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, /* g */ 0, 0, 0, 1, -1, 0, 0};
const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, /* g */ 0, 0, 0, 0, 0, 1, -1};

struct Matrices {
  double M[Q][Q];
  double Minv[Q][Q];
};

void build_matrices(const Phys3& ph, Matrices& mm) {
  const double l = ph.lambda, l2 = l * l, l3 = l2 * l, l4 = l2 * l2;
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) mm.M[i][j] = 0.0;
  for (int j = 0; j < 19; ++j) {
    const double cx = CX[j], cy = CY[j], cz = CZ[j], c2 = cx * cx + cy * cy + cz * cz;
    mm.M[0][j] = 1.0;
    mm.M[1][j] = l * cx;
    mm.M[2][j] = l * cy;
    mm.M[3][j] = l * cz;
    mm.M[5][j] = l2 * (19.0 * c2 - 30.0);
    mm.M[6][j] = l2 * (3.0 * cx * cx - c2);
    mm.M[7][j] = l2 * (cy * cy - cz * cz);
    mm.M[8][j] = l2 * cx * cy;
    mm.M[9][j] = l2 * cy * cz;
    mm.M[10][j] = l2 * cx * cz;
    mm.M[11][j] = l3 * (5.0 * c2 - 9.0) * cx;
    mm.M[12][j] = l3 * (5.0 * c2 - 9.0) * cy;
    mm.M[13][j] = l3 * (5.0 * c2 - 9.0) * cz;
    mm.M[14][j] = l3 * (cy * cy - cz * cz) * cx;
    mm.M[15][j] = l3 * (cz * cz - cx * cx) * cy;
    mm.M[16][j] = l3 * (cx * cx - cy * cy) * cz;
    mm.M[17][j] = l4 * (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
    mm.M[18][j] = l4 * (3.0 * c2 - 5.0) * (3.0 * cx * cx - c2);
    mm.M[19][j] = l4 * (3.0 * c2 - 5.0) * (cy * cy - cz * cz);
  }
  for (int j = 19; j < Q; ++j) {
    const double cx = CX[j], cy = CY[j], cz = CZ[j], c2 = cx * cx + cy * cy + cz * cz;
    mm.M[4][j] = ph.cp;
    mm.M[20][j] = ph.cp * l * cx;
    mm.M[21][j] = ph.cp * l * cy;
    mm.M[22][j] = ph.cp * l * cz;
    mm.M[23][j] = ph.cp * l2 * (3.0 * c2 - 6.0);
    mm.M[24][j] = ph.cp * l2 * (3.0 * cx * cx - c2);
    mm.M[25][j] = ph.cp * l2 * (cy * cy - cz * cz);
  }
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) mm.M[i][j] *= ph.rho0;
  // Gauss-Jordan elimination with partial pivoting on [M | I].
  std::vector<double> a(Q * 2 * Q);
  auto A = [&](int i, int j) -> double& { return a[i * 2 * Q + j]; };
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < 2 * Q; ++j) A(i, j) = (j < Q) ? mm.M[i][j] : (j - Q == i ? 1.0 : 0.0);
  for (int col = 0; col < Q; ++col) {
    int piv = col;
    for (int i = col + 1; i < Q; ++i)
      if (std::fabs(A(i, col)) > std::fabs(A(piv, col))) piv = i;
    if (piv != col)
      for (int j = 0; j < 2 * Q; ++j) std::swap(A(col, j), A(piv, j));
    const double inv = 1.0 / A(col, col);
    for (int j = 0; j < 2 * Q; ++j) A(col, j) *= inv;
    for (int i = 0; i < Q; ++i) {
      if (i == col) continue;
      const double f = A(i, col);
      if (f != 0.0)
        for (int j = 0; j < 2 * Q; ++j) A(i, j) -= f * A(col, j);
    }
  }
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) mm.Minv[i][j] = A(i, j + Q);
}

inline void matvec(const double (*A)[Q], const double* x, double* y) {
  for (int i = 0; i < Q; ++i) {
    double acc = 0.0;
    for (int j = 0; j < Q; ++j)
      if (A[i][j] != 0.0) acc = acc + A[i][j] * x[j];
    y[i] = acc;
  }
}

inline double gas_r(const Phys3& ph) { return ph.cp * (1.0 - 1.0 / ph.gamma); }
inline double T_ref(const Phys3& ph) { return ph.p0 / (ph.rho0 * gas_r(ph)); }

// Eq. (gaz-parfait): p = p0 (rho/rho0)^gamma exp(gamma (s - s0)/c_p), and p = rho r T.
inline void thermo(const Phys3& ph, double rho, double s, double& p, double& T) {
  p = ph.p0 * std::pow(rho / ph.rho0, ph.gamma) * std::exp(ph.gamma * (s - ph.s0) / ph.cp);
  T = p / (rho * gas_r(ph));
}

// The 21 equilibrium values of the non-conserved moments, in the order of m[5..25].
inline void equilibria(const Phys3& ph, double rho, const double u[3], double zeta, double p, double T, double* eq) {
  const double l2 = ph.lambda * ph.lambda, l4 = l2 * l2;
  const double s = zeta / rho;
  double Pi[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Pi[a][b] = rho * u[a] * u[b] + (a == b ? p : 0.0);
  const double tr = Pi[0][0] + Pi[1][1] + Pi[2][2];
  const double Qxy = Pi[0][0] * Pi[1][1] / rho, Qyz = Pi[1][1] * Pi[2][2] / rho, Qxz = Pi[0][0] * Pi[2][2] / rho;
  const double L = (rho * ph.cp * l2 / (ph.gamma * ph.beta)) * std::log(T / T_ref(ph));
  const double Exx = s * Pi[0][0] + L, Eyy = s * Pi[1][1] + L, Ezz = s * Pi[2][2] + L;
  const double trE = Exx + Eyy + Ezz;
  eq[0] = 19.0 * tr - 30.0 * l2 * rho;                                    // e
  eq[1] = 3.0 * Pi[0][0] - tr;                                            // pxx
  eq[2] = Pi[1][1] - Pi[2][2];                                            // pww
  eq[3] = Pi[0][1];                                                       // pxy
  eq[4] = Pi[1][2];                                                       // pyz
  eq[5] = Pi[0][2];                                                       // pxz
  for (int a = 0; a < 3; ++a) eq[6 + a] = -(2.0 / 3.0) * l2 * rho * u[a];  // q
  for (int a = 0; a < 3; ++a) eq[9 + a] = 0.0;                            // m
  eq[12] = 12.0 * l4 * rho - 16.0 * l2 * tr + 21.0 * (Qxy + Qyz + Qxz);   // eps
  eq[13] = 2.0 * l2 * (tr - 3.0 * Pi[0][0]) + 3.0 * (Qxy + Qxz) - 6.0 * Qyz;  // pixx
  eq[14] = -2.0 * l2 * (Pi[1][1] - Pi[2][2]) + 3.0 * (Qxy - Qxz);         // piww
  for (int a = 0; a < 3; ++a) eq[15 + a] = zeta * u[a];                   // psi
  eq[18] = 3.0 * trE - 6.0 * l2 * zeta;                                   // eps7
  eq[19] = 3.0 * Exx - trE;                                               // xixx
  eq[20] = Eyy - Ezz;                                                     // xiww
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
  std::vector<double> m, u, T;  // moments [N][Q], velocity [N][3], temperature [N]
};

void step(const Phys3& ph, const Matrices& mm, const Rates3& rt, int64_t Nx, int64_t Ny, int64_t Nz,
          const double* fd, double* out, Work& w, int nthreads) {
  const int64_t N = Nx * Ny * Nz;
  const double dt = ph.dx / ph.lambda;
  parallel_for(N, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t n = lo; n < hi; ++n) {
      double* m = &w.m[Q * n];
      matvec(mm.M, fd + Q * n, m);
      for (int a = 0; a < 3; ++a) w.u[3 * n + a] = m[1 + a] / m[0];
      double p;
      thermo(ph, m[0], m[4] / m[0], p, w.T[n]);
    }
  });
  const double sigma_e = 1.0 / rt.s_e - 0.5;
  const double nu = sigma_e * ph.lambda * ph.dx;
  double rate[21];
  for (int k = 0; k < 6; ++k) rate[k] = rt.s_e;
  for (int k = 6; k < 12; ++k) rate[k] = rt.s_q;
  for (int k = 12; k < 15; ++k) rate[k] = rt.s_h;
  for (int k = 15; k < 18; ++k) rate[k] = rt.s_psi;
  for (int k = 18; k < 21; ++k) rate[k] = rt.s_eps;
  parallel_for(N, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t n = lo; n < hi; ++n) {
      const int64_t x = n % Nx, y = (n / Nx) % Ny, z = n / (Nx * Ny);
      const double* m = &w.m[Q * n];
      const double rho = m[0], zeta = m[4], T = w.T[n];
      const double* u = &w.u[3 * n];
      double p, Tn;
      thermo(ph, rho, zeta / rho, p, Tn);  // T = Tn, stored by the first pass
      double eq[21];
      equilibria(ph, rho, u, zeta, p, T, eq);
      double ms[Q];
      for (int k = 0; k < 5; ++k) ms[k] = m[k];
      for (int k = 0; k < 21; ++k) ms[5 + k] = m[5 + k] + rate[k] * (eq[k] - m[5 + k]);
      if (ph.source_on) {
        // Neighbours along each axis: index of node (x, y, z) shifted by -1 and +1 along axis a.
        const int64_t nb[3][2] = {
            {(z * Ny + y) * Nx + (x == 0 ? Nx - 1 : x - 1), (z * Ny + y) * Nx + (x == Nx - 1 ? 0 : x + 1)},
            {(z * Ny + (y == 0 ? Ny - 1 : y - 1)) * Nx + x, (z * Ny + (y == Ny - 1 ? 0 : y + 1)) * Nx + x},
            {((z == 0 ? Nz - 1 : z - 1) * Ny + y) * Nx + x, ((z == Nz - 1 ? 0 : z + 1) * Ny + y) * Nx + x}};
        const double h2 = 2.0 * ph.dx;
        double G[3][3], dT[3];  // G[a][b] = d_a u_b
        for (int a = 0; a < 3; ++a) {
          for (int b = 0; b < 3; ++b) G[a][b] = (w.u[3 * nb[a][1] + b] - w.u[3 * nb[a][0] + b]) / h2;
          dT[a] = (w.T[nb[a][1]] - w.T[nb[a][0]]) / h2;
        }
        double DD = 0.0, div = 0.0, gT2 = 0.0;
        for (int a = 0; a < 3; ++a) {
          div = div + G[a][a];
          gT2 = gT2 + dT[a] * dT[a];
          for (int b = 0; b < 3; ++b) {
            const double D = 0.5 * (G[a][b] + G[b][a]);
            DD = DD + D * D;
          }
        }
        const double kappa = rho * nu * ph.cp / ph.Pr;
        const double S = rho * nu / (3.0 * T) * (2.0 * DD + div * div) + kappa / (T * T) * gT2;
        ms[4] = ms[4] + dt * S;
      }
      double fs[Q];
      matvec(mm.Minv, ms, fs);
      for (int i = 0; i < Q; ++i) {
        const int64_t xt = (x + CX[i] + Nx) % Nx, yt = (y + CY[i] + Ny) % Ny, zt = (z + CZ[i] + Nz) % Nz;
        out[Q * ((zt * Ny + yt) * Nx + xt) + i] = fs[i];
      }
    }
  });
}

bool valid(const Phys3* ph, int64_t Nx, int64_t Ny, int64_t Nz) {
  if (!ph || Nx < 3 || Ny < 3 || Nz < 3) return false;
  return ph->lambda > 0 && ph->dx > 0 && ph->gamma > 1 && ph->cp > 0 && ph->rho0 > 0 && ph->p0 > 0 && ph->Pr > 0 &&
         ph->beta > 0;
}

}  // namespace

extern "C" {

typedef Phys3 oracle3d_phys;
typedef Rates3 oracle3d_rates;

// M and M^{-1} as row-major 26 x 26 arrays.
int oracle3d_matrices(const oracle3d_phys* ph, double* M, double* Minv) {
  if (!ph) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) { M[Q * i + j] = mm.M[i][j]; Minv[Q * i + j] = mm.Minv[i][j]; }
  return 0;
}

// Equilibrium populations f_d = M^{-1} m_eq(rho, J = rho u, zeta = rho s), node-major [N][26].
int oracle3d_init(const oracle3d_phys* ph, int64_t Nx, int64_t Ny, int64_t Nz, const double* rho, const double* ux,
                  const double* uy, const double* uz, const double* s, double* fd) {
  if (!valid(ph, Nx, Ny, Nz)) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  for (int64_t n = 0; n < Nx * Ny * Nz; ++n) {
    double p, T;
    thermo(*ph, rho[n], s[n], p, T);
    const double u[3] = {ux[n], uy[n], uz[n]};
    double m[Q];
    m[0] = rho[n];
    for (int a = 0; a < 3; ++a) m[1 + a] = rho[n] * u[a];
    m[4] = rho[n] * s[n];
    equilibria(*ph, rho[n], u, m[4], p, T, m + 5);
    matvec(mm.Minv, m, fd + Q * n);
  }
  return 0;
}

// nsteps time steps in place.
int oracle3d_run(const oracle3d_phys* ph, const oracle3d_rates* rt, int64_t Nx, int64_t Ny, int64_t Nz,
                 int64_t nsteps, double* fd, int32_t nthreads) {
  if (!valid(ph, Nx, Ny, Nz) || !rt || nsteps < 0) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  const int64_t N = Nx * Ny * Nz;
  Work w;
  w.m.resize(Q * N);
  w.u.resize(3 * N);
  w.T.resize(N);
  std::vector<double> other(Q * N);
  double* a = fd;
  double* b = other.data();
  for (int64_t t = 0; t < nsteps; ++t) {
    step(*ph, mm, *rt, Nx, Ny, Nz, a, b, w, nthreads);
    std::swap(a, b);
  }
  if (a != fd) std::memcpy(fd, a, sizeof(double) * Q * N);
  return 0;
}

// Moments [N][26] in the order of the header.
int oracle3d_moments(const oracle3d_phys* ph, int64_t N, const double* fd, double* m) {
  if (!ph || N < 0) return -1;
  Matrices mm;
  build_matrices(*ph, mm);
  for (int64_t n = 0; n < N; ++n) matvec(mm.M, fd + Q * n, m + Q * n);
  return 0;
}

}  // extern "C"
