// Host build of the three-dimensional kernel's node update (test infrastructure). Two modes:
//  - no argument: reads states (rho, ux, uy, uz, s) from stdin and prints the equilibrium populations
//    the kernel's equilibria and inverse give (unshifted, FP64), followed by the round-trip error of
//    moments -> populations -> moments;
//  - "step": reads nx ny nz nsteps, the physics and the fields, and runs nsteps time steps in FP64 with
//    the kernel's own node functions (conserved moments, thermodynamic state, temperature deviation,
//    collision with the production) and its neighbour and push-streaming rules, then prints the
//    populations node-major, unshifted.
// The thermodynamic state uses the host's log1p / expm1 and a division (the host branches of the
// kernel's math wrappers); everything else is the kernel's own __host__ __device__ code.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../paper_1802_02369_gb300/csrc/lbm3d.cu"

static int run_steps() {
  long long nx, ny, nz, T;
  lbm3d_params in{};
  if (scanf("%lld %lld %lld %lld %lf %lf %lf %lf %lf %lf %lf", &nx, &ny, &nz, &T, &in.gamma, &in.Pr, &in.cp,
            &in.rho0, &in.s0, &in.lambda, &in.s_e) != 11)
    return 1;
  in.dx = 1.0;
  in.source_on = 1;
  P3 p{};
  if (derive3(&in, p)) return 2;
  const P3T<double> q = lanes3<double>(p);
  const long long N = nx * ny * nz;
  std::vector<double> st(kQ * N), nx_st(kQ * N);
  for (long long n = 0; n < N; ++n) {
    double rho, ux, uy, uz, s;
    if (scanf("%lf %lf %lf %lf %lf", &rho, &ux, &uy, &uz, &s) != 5) return 3;
    Cons3<double> c;
    c.r = rho / p.rho0 - 1.0;
    c.jx = rho * ux / (p.rho0 * p.lam);
    c.jy = rho * uy / (p.rho0 * p.lam);
    c.jz = rho * uz / (p.rho0 * p.lam);
    c.z = (rho * s - p.rho0 * p.s0) / (p.rho0 * p.cp);
    const Thermo3<double> t = thermo3(c, q);
    double eq[21], f[kQ];
    equilibria3(c, t, q, eq);
    populations3(c, eq, f);
    for (int k = 0; k < kQ; ++k) st[k * N + n] = f[k];
  }
  std::vector<double> U(4 * N);  // ux, uy, uz, T' per node
  auto idx = [&](long long x, long long y, long long z) {
    return (wrap3(z, nz) * ny + wrap3(y, ny)) * nx + wrap3(x, nx);
  };
  for (long long step = 0; step < T; ++step) {
    for (long long n = 0; n < N; ++n) {
      double f[kQ];
      for (int k = 0; k < kQ; ++k) f[k] = st[k * N + n];
      const Cons3<double> c = conserved3(f);
      const Thermo3<double> t = thermo3(c, q);
      U[4 * n] = t.ux;
      U[4 * n + 1] = t.uy;
      U[4 * n + 2] = t.uz;
      U[4 * n + 3] = temp_dev3(c, t, q);
    }
    for (long long z = 0; z < nz; ++z)
      for (long long y = 0; y < ny; ++y)
        for (long long x = 0; x < nx; ++x) {
          const long long n = idx(x, y, z);
          const long long nb[3][2] = {{idx(x - 1, y, z), idx(x + 1, y, z)},
                                      {idx(x, y - 1, z), idx(x, y + 1, z)},
                                      {idx(x, y, z - 1), idx(x, y, z + 1)}};
          double du[3][3], dT[3];
          for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) du[a][b] = U[4 * nb[a][1] + b] - U[4 * nb[a][0] + b];
            dT[a] = U[4 * nb[a][1] + 3] - U[4 * nb[a][0] + 3];
          }
          double f[kQ];
          for (int k = 0; k < kQ; ++k) f[k] = st[k * N + n];
          collide3(f, q, du, dT, 1.0 + U[4 * n + 3]);
          for (int k = 0; k < kQ; ++k) nx_st[k * N + idx(x + cx3(k), y + cy3(k), z + cz3(k))] = f[k];
        }
    st.swap(nx_st);
  }
  for (long long n = 0; n < N; ++n) {
    for (int k = 0; k < kQ; ++k) printf("%.17g ", st[k * N + n] + p.w[k]);
    printf("\n");
  }
  return 0;
}

int main(int argc, char** argv) {
  if (argc > 1 && std::strcmp(argv[1], "step") == 0) return run_steps();
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
