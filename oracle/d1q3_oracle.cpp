// CPU oracle of the two single-distribution D1Q3 schemes of Dubois, Graille and Lallemand,
// "Recovering the full Navier Stokes equations with lattice Boltzmann schemes":
//   section 2: the D1Q3 fluid scheme (moments rho, J, e; rho and J conserved, e relaxed toward
//              e_eq = 3 (rho u^2 + p) - 2 lambda^2 rho of eq. (energie-equilibre), isentropic
//              pressure p = p0 (rho / rho0)^gamma);
//   section 4: the D1Q3 advection-diffusion scheme (moments zeta, psi, eps; zeta conserved, psi and
//              eps relaxed toward psi_eq = u0 zeta and eps_eq = alpha lambda^2 zeta).
//
// TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously correct reference the CUDA kernels
// of these schemes are checked against. Only the tests load it. It shares no code, header, table or
// constant with the CUDA library or with the other oracles.
//
// FP64, no FMA contraction (compiled with -ffp-contract=off). One time step, in the paper's order:
//   m = M f with the 3x3 matrix of eq. (M-d1q3) (scale rho0, or zeta0 for section 4), applied as a
//   matrix-vector product; equilibria of the non-conserved moments; relaxation
//   m* = m + s (m_eq - m) with s_e (section 2) or s_psi, s_eps (section 4); f* = M^{-1} m*, M^{-1}
//   by Gauss-Jordan elimination; advection f0(x) = f0*(x), f+(x) = f+*(x - dx), f-(x) = f-*(x + dx)
//   on a periodic lattice.
// Reading where the paper is silent: section 2 names the isentropic Navier-Stokes equations but no
// pressure law; p = p0 (rho/rho0)^gamma (the polytropic law of eq. (gaz-parfait) at s = s0) is used.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct Params {
  int32_t scheme;  // 0: fluid (section 2), 1: advection-diffusion (section 4)
  int32_t pad;
  double lambda;   // lattice velocity dx / dt
  double scale;    // rho0 (section 2) or zeta0 (section 4): the factor of M, and rho0 of the EOS
  double s_e;      // section 2 relaxation rate of e
  double gamma;    // section 2 exponent of the isentropic pressure law
  double p0;       // section 2 reference pressure
  double u0;       // section 4 advection velocity: psi_eq = u0 zeta
  double alpha;    // section 4: eps_eq = alpha lambda^2 zeta
  double s_psi;    // section 4 relaxation rates
  double s_eps;
};

struct Mat {
  double M[3][3];
  double Minv[3][3];
};

// Eq. (M-d1q3), entry by entry, times the scale; the inverse by Gauss-Jordan with partial pivoting.
void build(const Params& p, Mat& mm) {
  const double l = p.lambda;
  const double A[3][3] = {{1, 1, 1}, {0, l, -l}, {-2 * l * l, l * l, l * l}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) mm.M[i][j] = p.scale * A[i][j];
  double a[3][6];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 6; ++j) a[i][j] = (j < 3) ? mm.M[i][j] : (j - 3 == i ? 1.0 : 0.0);
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int i = col + 1; i < 3; ++i)
      if (std::fabs(a[i][col]) > std::fabs(a[piv][col])) piv = i;
    if (piv != col)
      for (int j = 0; j < 6; ++j) { const double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t; }
    const double inv = 1.0 / a[col][col];
    for (int j = 0; j < 6; ++j) a[col][j] *= inv;
    for (int i = 0; i < 3; ++i) {
      if (i == col) continue;
      const double f = a[i][col];
      for (int j = 0; j < 6; ++j) a[i][j] -= f * a[col][j];
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) mm.Minv[i][j] = a[i][j + 3];
}

void matvec(const double A[3][3], const double* x, double* y) {
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += A[i][j] * x[j];
    y[i] = s;
  }
}

// Equilibrium values of the two non-conserved moments from the conserved one(s).
void equilibria(const Params& p, const double* m, double* eq) {
  if (p.scheme == 0) {
    const double rho = m[0], J = m[1];
    const double u = J / rho;
    const double pr = p.p0 * std::pow(rho / p.scale, p.gamma);
    eq[0] = rho;
    eq[1] = J;
    eq[2] = 3.0 * (rho * u * u + pr) - 2.0 * p.lambda * p.lambda * rho;  // eq. (energie-equilibre)
  } else {
    const double zeta = m[0];
    eq[0] = zeta;
    eq[1] = p.u0 * zeta;
    eq[2] = p.alpha * p.lambda * p.lambda * zeta;
  }
}

void relax(const Params& p, double* m) {
  double eq[3];
  equilibria(p, m, eq);
  if (p.scheme == 0) {
    m[2] = m[2] + p.s_e * (eq[2] - m[2]);
  } else {
    m[1] = m[1] + p.s_psi * (eq[1] - m[1]);
    m[2] = m[2] + p.s_eps * (eq[2] - m[2]);
  }
}

bool valid(const Params* p) {
  if (!p || !(p->lambda > 0) || !(p->scale > 0)) return false;
  if (p->scheme == 0) return p->s_e > 0 && p->s_e < 2 && p->gamma >= 1 && p->p0 > 0;
  if (p->scheme == 1) return p->s_psi > 0 && p->s_psi < 2 && p->s_eps > 0 && p->s_eps < 2;
  return false;
}

}  // namespace

extern "C" {

typedef Params d1q3_oracle_params;

// M and M^{-1} (row-major 3x3 each).
int d1q3_oracle_matrices(const d1q3_oracle_params* p, double* M, double* Minv) {
  if (!p || !(p->lambda > 0) || !(p->scale > 0)) return -1;
  Mat mm;
  build(*p, mm);
  std::memcpy(M, mm.M, sizeof(mm.M));
  std::memcpy(Minv, mm.Minv, sizeof(mm.Minv));
  return 0;
}

// Equilibrium populations, node-major f[N][3] = (f0, f+, f-): section 2 from (rho, J) = (m0, m1);
// section 4 from zeta = m0 (m1 unused).
int d1q3_oracle_init(const d1q3_oracle_params* p, int64_t N, const double* m0, const double* m1, double* f) {
  if (!valid(p) || N < 1) return -1;
  Mat mm;
  build(*p, mm);
  for (int64_t j = 0; j < N; ++j) {
    const double m[3] = {m0[j], p->scheme == 0 ? m1[j] : 0.0, 0.0};
    double eq[3];
    equilibria(*p, m, eq);
    matvec(mm.Minv, eq, f + 3 * j);
  }
  return 0;
}

// nsteps time steps in place on f[N][3], periodic.
int d1q3_oracle_run(const d1q3_oracle_params* p, int64_t N, int64_t nsteps, double* f) {
  if (!valid(p) || N < 1 || nsteps < 0) return -1;
  Mat mm;
  build(*p, mm);
  std::vector<double> post(3 * N);
  for (int64_t t = 0; t < nsteps; ++t) {
    for (int64_t j = 0; j < N; ++j) {
      double m[3];
      matvec(mm.M, f + 3 * j, m);
      relax(*p, m);
      matvec(mm.Minv, m, &post[3 * j]);
    }
    for (int64_t j = 0; j < N; ++j) {
      const int64_t l = (j == 0) ? N - 1 : j - 1, r = (j == N - 1) ? 0 : j + 1;
      f[3 * j + 0] = post[3 * j + 0];
      f[3 * j + 1] = post[3 * l + 1];
      f[3 * j + 2] = post[3 * r + 2];
    }
  }
  return 0;
}

// Moments m[N][3] = M f per node.
int d1q3_oracle_moments(const d1q3_oracle_params* p, int64_t N, const double* f, double* m) {
  if (!p || !(p->lambda > 0) || !(p->scale > 0) || N < 1) return -1;
  Mat mm;
  build(*p, mm);
  for (int64_t j = 0; j < N; ++j) matvec(mm.M, f + 3 * j, m + 3 * j);
  return 0;
}

}  // extern "C"
