// CPU oracle of the finite-difference comparison solver of section 9: the (rho, J, zeta)
// Navier-Stokes system of eq. (NS-rho-J-zeta) discretised with second-order centred differences in
// space and explicit first-order (forward Euler) time integration, on a periodic grid.
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct reference that the
// CUDA finite-difference kernel is checked against. Only the tests load it. It shares no code,
// header, table or constant with the CUDA library, nor with the lattice Boltzmann oracle.
//
// Everything is FP64 with no FMA contraction (compiled with -ffp-contract=off).
//
// The paper names the method (centred second-order differences, explicit first-order time steps)
// but not its stencil. The reading used here, in conservation form so that the discrete sums of
// rho and J are exactly conserved:
//   W = (rho, J, zeta),  u = J / rho,  s = zeta / rho,  p and T from eq. (gaz-parfait), p = rho r T,
//   convective flux F = (J, rho u^2 + p, zeta u), centred: (F_{j+1} - F_{j-1}) / (2 dx);
//   diffusive flux Phi = (0, rho nu d_x u, (kappa / T) d_x T), kappa = rho nu c_p / Pr, taken at the
//   faces j +- 1/2 as a_{j+1/2} (q_{j+1} - q_j) / dx with a_{j+1/2} the mean of the two nodal values,
//   and differenced: (Phi_{j+1/2} - Phi_{j-1/2}) / dx;
//   entropy production S = (rho nu / T) (d_x u)^2 + (kappa / T^2) (d_x T)^2 at the node, with the
//   centred d_x q = (q_{j+1} - q_{j-1}) / (2 dx) (the same differences as the lattice Boltzmann
//   source of section 8, step (vii));
//   W^{n+1} = W^n + dt (-d_x F + d_x Phi + (0, 0, S)).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct FdPhys {
  double gamma, Pr, cp, rho0, p0, s0, dx, nu;
  int32_t source_on, pad;
};

inline double gas_r(const FdPhys& ph) { return ph.cp * (1.0 - 1.0 / ph.gamma); }

// Eq. (gaz-parfait): p = p0 (rho/rho0)^gamma exp(gamma (s - s0)/c_p), T = p / (rho r).
inline void thermo(const FdPhys& ph, double rho, double s, double& p, double& T) {
  p = ph.p0 * std::pow(rho / ph.rho0, ph.gamma) * std::exp(ph.gamma * (s - ph.s0) / ph.cp);
  T = p / (rho * gas_r(ph));
}

bool valid(const FdPhys* ph, int64_t N, double dt) {
  if (!ph || N < 3 || !(dt > 0)) return false;
  return ph->gamma > 1 && ph->Pr > 0 && ph->cp > 0 && ph->rho0 > 0 && ph->p0 > 0 && ph->dx > 0 && ph->nu >= 0;
}

// One forward-Euler step, node-major arrays [N][3] = (rho, J, zeta).
void fd_step(const FdPhys& ph, int64_t N, double dt, const double* W, double* out, std::vector<double>& u,
             std::vector<double>& p, std::vector<double>& T) {
  for (int64_t j = 0; j < N; ++j) {
    const double rho = W[3 * j], J = W[3 * j + 1], zeta = W[3 * j + 2];
    u[j] = J / rho;
    thermo(ph, rho, zeta / rho, p[j], T[j]);
  }
  const double dx = ph.dx;
  for (int64_t j = 0; j < N; ++j) {
    const int64_t l = (j == 0) ? N - 1 : j - 1, r = (j == N - 1) ? 0 : j + 1;
    const double* Wl = W + 3 * l;
    const double* Wj = W + 3 * j;
    const double* Wr = W + 3 * r;
    // Convective fluxes at the neighbours.
    const double Fl[3] = {Wl[1], Wl[0] * u[l] * u[l] + p[l], Wl[2] * u[l]};
    const double Fr[3] = {Wr[1], Wr[0] * u[r] * u[r] + p[r], Wr[2] * u[r]};
    // Diffusion coefficients at the three nodes: a = rho nu, b = kappa / T.
    const double al = Wl[0] * ph.nu, aj = Wj[0] * ph.nu, ar = Wr[0] * ph.nu;
    const double kl = Wl[0] * ph.nu * ph.cp / ph.Pr, kj = Wj[0] * ph.nu * ph.cp / ph.Pr,
                 kr = Wr[0] * ph.nu * ph.cp / ph.Pr;
    const double bl = kl / T[l], bj = kj / T[j], br = kr / T[r];
    // Face fluxes Phi_{j+1/2} and Phi_{j-1/2}.
    const double phiJ_r = 0.5 * (aj + ar) * (u[r] - u[j]) / dx;
    const double phiJ_l = 0.5 * (al + aj) * (u[j] - u[l]) / dx;
    const double phiZ_r = 0.5 * (bj + br) * (T[r] - T[j]) / dx;
    const double phiZ_l = 0.5 * (bl + bj) * (T[j] - T[l]) / dx;
    // Entropy production at the node.
    double S = 0.0;
    if (ph.source_on) {
      const double dudx = (u[r] - u[l]) / (2.0 * dx);
      const double dTdx = (T[r] - T[l]) / (2.0 * dx);
      S = Wj[0] * ph.nu / T[j] * dudx * dudx + kj / (T[j] * T[j]) * dTdx * dTdx;
    }
    out[3 * j + 0] = Wj[0] - dt * (Fr[0] - Fl[0]) / (2.0 * dx);
    out[3 * j + 1] = Wj[1] - dt * (Fr[1] - Fl[1]) / (2.0 * dx) + dt * (phiJ_r - phiJ_l) / dx;
    out[3 * j + 2] = Wj[2] - dt * (Fr[2] - Fl[2]) / (2.0 * dx) + dt * (phiZ_r - phiZ_l) / dx + dt * S;
  }
}

void sums_of(const FdPhys& ph, int64_t N, const double* W, double* sums, int32_t* flags) {
  double a[4] = {0, 0, 0, 0};
  int32_t fl = 0;
  for (int64_t j = 0; j < N; ++j) {
    const double rho = W[3 * j], J = W[3 * j + 1], zeta = W[3 * j + 2];
    if (!std::isfinite(rho) || !std::isfinite(J) || !std::isfinite(zeta)) fl |= 1;
    if (!(rho > 0)) fl |= 2;
    double p, T;
    thermo(ph, rho, zeta / rho, p, T);
    if (!(T > 0) || !std::isfinite(T)) fl |= 4;
    const double u = J / rho;
    a[0] += rho;
    a[1] += J;
    a[2] += zeta;
    a[3] += p / (ph.gamma - 1.0) + 0.5 * rho * u * u;
  }
  for (int k = 0; k < 4; ++k) sums[k] = a[k];
  *flags = fl;
}

}  // namespace

extern "C" {

typedef FdPhys fd_oracle_phys;

// W[j] = (rho, rho u, rho s).
int fd_oracle_init(const fd_oracle_phys* ph, int64_t N, const double* rho, const double* u, const double* s,
                   double* W) {
  if (!ph || N < 1) return -1;
  for (int64_t j = 0; j < N; ++j) {
    W[3 * j] = rho[j];
    W[3 * j + 1] = rho[j] * u[j];
    W[3 * j + 2] = rho[j] * s[j];
  }
  return 0;
}

// nsteps forward-Euler steps of size dt, in place on W [N][3].
int fd_oracle_run(const fd_oracle_phys* ph, int64_t N, double dt, int64_t nsteps, double* W) {
  if (!valid(ph, N, dt) || nsteps < 0) return -1;
  std::vector<double> other(3 * N), u(N), p(N), T(N);
  double* a = W;
  double* b = other.data();
  for (int64_t t = 0; t < nsteps; ++t) {
    fd_step(*ph, N, dt, a, b, u, p, T);
    double* tmp = a; a = b; b = tmp;
  }
  if (a != W) std::memcpy(W, a, sizeof(double) * 3 * N);
  return 0;
}

// Sums of rho, J, zeta and the total energy p/(gamma-1) + rho u^2/2, and a flag word: bit 0 a
// non-finite field, bit 1 rho <= 0, bit 2 T <= 0 (or non-finite).
int fd_oracle_diagnostics(const fd_oracle_phys* ph, int64_t N, const double* W, double* sums, int32_t* flags) {
  if (!ph || N < 1) return -1;
  sums_of(*ph, N, W, sums, flags);
  return 0;
}

// Advances W by nsteps and records the diagnostics sums at steps 0, every, 2 every, ..., nsteps:
// out[(nsteps / every + 1)][4] (nsteps a multiple of every).
int fd_oracle_series(const fd_oracle_phys* ph, int64_t N, double dt, int64_t nsteps, int64_t every, double* W,
                     double* out) {
  if (!valid(ph, N, dt) || every <= 0 || nsteps < 0 || nsteps % every != 0) return -1;
  int32_t fl;
  for (int64_t r = 0; r <= nsteps / every; ++r) {
    if (r > 0 && fd_oracle_run(ph, N, dt, every, W) != 0) return -1;
    sums_of(*ph, N, W, out + 4 * r, &fl);
  }
  return 0;
}

}  // extern "C"
