// Host build of the three-dimensional kernel's node algebra (test infrastructure): reads states
// (rho, ux, uy, uz, s) from stdin and prints the equilibrium populations the kernel's equilibria and
// inverse give (unshifted, FP64), followed by the round-trip error of moments -> populations ->
// moments. The thermodynamic state is computed with the host's log1p / expm1 (the kernel's device
// versions are not callable here); everything else is the kernel's own __host__ __device__ code.
#include <cmath>
#include <cstdio>

#include "../paper_1802_02369_gb300/csrc/lbm3d.cu"

int main() {
  int M = 0;
  lbm3d_params in{};
  if (scanf("%d %lf %lf %lf %lf %lf %lf", &M, &in.gamma, &in.Pr, &in.cp, &in.rho0, &in.s0, &in.lambda) != 7) return 1;
  in.dx = 1.0;
  in.s_e = 1.2;
  in.source_on = 1;
  P3 p{};
  if (derive3(&in, p)) return 2;
  const P3T<double> q = lanes3<double>(p);
  for (int n = 0; n < M; ++n) {
    double rho, ux, uy, uz, s;
    if (scanf("%lf %lf %lf %lf %lf", &rho, &ux, &uy, &uz, &s) != 5) return 3;
    Cons3<double> c;
    c.r = rho / p.rho0 - 1.0;
    c.jx = rho * ux / (p.rho0 * p.lam);
    c.jy = rho * uy / (p.rho0 * p.lam);
    c.jz = rho * uz / (p.rho0 * p.lam);
    c.z = (rho * s - p.rho0 * p.s0) / (p.rho0 * p.cp);
    Thermo3<double> t;
    t.inv = 1.0 / (1.0 + c.r);
    t.ux = c.jx * t.inv;
    t.uy = c.jy * t.inv;
    t.uz = c.jz * t.inv;
    t.sig = (c.z - q.s0c * c.r) * t.inv;
    t.lr = std::log1p(c.r);
    t.dP = q.P0 * std::expm1(q.gamma * (t.lr + t.sig));
    double eq[21], f[kQ], m2[21];
    equilibria3(c, t, q, eq);
    populations3(c, eq, f);
    const Cons3<double> c2 = conserved3(f);
    nonconserved3(f, m2);
    double err = std::fabs(c2.r - c.r) + std::fabs(c2.jx - c.jx) + std::fabs(c2.jy - c.jy) +
                 std::fabs(c2.jz - c.jz) + std::fabs(c2.z - c.z);
    for (int k = 0; k < 21; ++k) err += std::fabs(m2[k] - eq[k]);
    for (int k = 0; k < kQ; ++k) printf("%.17g ", f[k] + p.w[k]);
    printf("%.17g\n", err);
  }
  return 0;
}
