"""The pins must catch plausible mistakes in the oracle: each case plants one mistake in a copy
of the oracle source (on the CPU), builds it, and requires the pin suite to fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "d1q3q3_oracle.cpp")

MUTANTS = {
    "e_eq pressure coefficient": ("3.0 * (rho * u * u + p)", "3.0 * (rho * u * u + 0.9 * p)"),
    "e_eq kinetic term dropped": ("3.0 * (rho * u * u + p)", "3.0 * (p)"),
    "psi_eq uses J": ("psi_eq = zeta * u;", "psi_eq = rho * u;"),
    "eps_eq drops e_eq s": ("log(T / T_ref(ph)) + e_eq * s;", "log(T / T_ref(ph));"),
    "eps_eq drops 1/gamma": ("(2.0 * rho * ph.cp * l2 / ph.gamma)", "(2.0 * rho * ph.cp * l2)"),
    "gradient missing factor 2": ("const R dudx = (ur - ul) / (2.0 * ph.dx);", "const R dudx = (ur - ul) / (ph.dx);"),
    "thermal term over T": ("kappa / (T * T) * dTdx * dTdx", "kappa / T * dTdx * dTdx"),
    "source sign": ("ms[2] = ms[2] + dt * S;", "ms[2] = ms[2] - dt * S;"),
    "nu drops lambda": ("const R nu = sigma_e * ph.lambda * ph.dx;", "const R nu = sigma_e * ph.dx;"),
    "psi relaxed with s_e": ("psi + rt.s_psi * (psi_eq - psi)", "psi + rt.s_e * (psi_eq - psi)"),
    "eps relaxed with s_psi": ("eps + rt.s_eps * (eps_eq - eps)", "eps + rt.s_psi * (eps_eq - eps)"),
    "M psi row sign": ("{0, 0, 0, 0, c * l, -c * l},", "{0, 0, 0, 0, -c * l, c * l},"),
    "M eps row weight": ("{0, 0, 0, -2 * c * l * l, c * l * l, c * l * l},", "{0, 0, 0, -c * l * l, c * l * l, c * l * l},"),
    "EOS exponent": ("exp(ph.gamma * (s - ph.s0) / ph.cp)", "exp((s - ph.s0) / ph.cp)"),
    "wall ghost velocity": ("if (j == 0) { ul = -u; Tl = T; }", "if (j == 0) { ul = u; Tl = T; }"),
    "stream wrap swapped": ("else if (ph.bc == 0) { out[1] = fs[1]; out[4] = fs[4]; }",
                            "else if (ph.bc == 0) { out[2] = fs[1]; out[5] = fs[4]; }"),
    "linear e_eq J coefficient": ("+ 6.0 * u0 * J + 3.0 * (u0 * u0 / cp) * zeta;",
                                  "+ 3.0 * u0 * J + 3.0 * (u0 * u0 / cp) * zeta;"),
    "linear psi_eq sign": ("psi_eq = -u0 * s0 * rho + s0 * J + u0 * zeta;",
                           "psi_eq = u0 * s0 * rho + s0 * J + u0 * zeta;"),
    "linear e_eq rho coefficient": ("(3.0 * (1.0 - s0 / cp) * c02 - 3.0 * u0 * u0 - 2.0 * l2) * rho",
                                    "(3.0 * (1.0 - s0 / cp) * c02 - 2.0 * l2) * rho"),
    "linear eps_eq rho constant": ("+ 3.0 * s0 * c02 + 2.0 - 2.0 * s0 - 2.0 / g) * rho",
                                   "+ 3.0 * s0 * c02 + 2.0 - 2.0 * s0) * rho"),
    "linear eps_eq zeta coefficient": ("3.0 * (cp * u0 * u0 + s0 * c02) * zeta;", "3.0 * (cp * u0 * u0) * zeta;"),
    "kappa drops Pr": ("const R kappa = rho * nu * ph.cp / ph.Pr;", "const R kappa = rho * nu * ph.cp;"),
    "coupled rate drops Pr": ("const double sigma_psi = 1.5 * (gamma / Pr) * sigma_e;",
                              "const double sigma_psi = 1.5 * gamma * sigma_e;"),
    "T0 drops rho0": ("return ph.p0 / (ph.rho0 * gas_r(ph));", "return ph.p0 / gas_r(ph);"),
    "EOS drops rho0": ("p = ph.p0 * pow(rho / ph.rho0, ph.gamma)", "p = ph.p0 * pow(rho, ph.gamma)"),
    "gas constant": ("return ph.cp * (1.0 - 1.0 / ph.gamma);", "return ph.cp / ph.gamma;"),
    "entropy from pressure drops 1/gamma": ("s[j] = ph->s0 + (ph->cp / ph->gamma) * std::log(",
                                            "s[j] = ph->s0 + ph->cp * std::log("),
    "total energy kinetic doubled": ("a[3] += p / (ph->gamma - 1.0) + 0.5 * rho * u * u;",
                                     "a[3] += p / (ph->gamma - 1.0) + rho * u * u;"),
    "total energy internal coefficient": ("a[3] += p / (ph->gamma - 1.0) + 0.5 * rho * u * u;",
                                          "a[3] += p / ph->gamma + 0.5 * rho * u * u;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not found exactly once"
    mut = tmp_path / "mutant.cpp"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                    "-o", str(lib), str(mut)], check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_linear.py"),
                        os.path.join(ROOT, "tests", "test_oracle_stability.py")],
                       env=env, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode != 0, f"pins did not catch the mutant {name!r}:\n{r.stdout[-2000:]}"


FD_SRC = os.path.join(ROOT, "oracle", "fd_oracle.cpp")

FD_MUTANTS = {
    "fd convective difference missing 2": ("out[3 * j + 0] = Wj[0] - dt * (Fr[0] - Fl[0]) / (2.0 * dx);",
                                           "out[3 * j + 0] = Wj[0] - dt * (Fr[0] - Fl[0]) / (dx);"),
    "fd momentum flux drops p": ("const double Fr[3] = {Wr[1], Wr[0] * u[r] * u[r] + p[r], Wr[2] * u[r]};",
                                 "const double Fr[3] = {Wr[1], Wr[0] * u[r] * u[r], Wr[2] * u[r]};"),
    "fd entropy flux uses J": ("const double Fl[3] = {Wl[1], Wl[0] * u[l] * u[l] + p[l], Wl[2] * u[l]};",
                               "const double Fl[3] = {Wl[1], Wl[0] * u[l] * u[l] + p[l], Wl[1] * u[l]};"),
    "fd viscosity face not averaged": ("const double phiJ_r = 0.5 * (aj + ar) * (u[r] - u[j]) / dx;",
                                       "const double phiJ_r = aj * (u[r] - u[j]) / dx;"),
    "fd kappa drops Pr": ("const double kl = Wl[0] * ph.nu * ph.cp / ph.Pr, kj = Wj[0] * ph.nu * ph.cp / ph.Pr,",
                          "const double kl = Wl[0] * ph.nu * ph.cp, kj = Wj[0] * ph.nu * ph.cp / ph.Pr,"),
    "fd heat flux over T squared": ("const double bl = kl / T[l], bj = kj / T[j], br = kr / T[r];",
                                    "const double bl = kl / T[l], bj = kj / (T[j] * T[j]), br = kr / T[r];"),
    "fd source thermal term over T": ("kj / (T[j] * T[j]) * dTdx * dTdx;", "kj / T[j] * dTdx * dTdx;"),
    "fd source halved": ("out[3 * j + 2] = Wj[2] - dt * (Fr[2] - Fl[2]) / (2.0 * dx) + dt * (phiZ_r - phiZ_l) / dx + dt * S;",
                         "out[3 * j + 2] = Wj[2] - dt * (Fr[2] - Fl[2]) / (2.0 * dx) + dt * (phiZ_r - phiZ_l) / dx + 0.5 * dt * S;"),
    "fd EOS exponent": ("std::exp(ph.gamma * (s - ph.s0) / ph.cp)", "std::exp((s - ph.s0) / ph.cp)"),
    "fd viscous term sign": ("+ dt * (phiJ_r - phiJ_l) / dx;", "- dt * (phiJ_r - phiJ_l) / dx;"),
}


@pytest.mark.parametrize("name", sorted(FD_MUTANTS))
def test_fd_pins_catch_planted_mistake(name, tmp_path):
    old, new = FD_MUTANTS[name]
    src = open(FD_SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not found exactly once"
    mut = tmp_path / "fd_mutant.cpp"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libfd_mutant.so"
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(lib), str(mut)], check=True)
    env = dict(os.environ, FD_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_fd.py")],
                       env=env, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode != 0, f"pins did not catch the mutant {name!r}:\n{r.stdout[-2000:]}"


D1Q3_SRC = os.path.join(ROOT, "oracle", "d1q3_oracle.cpp")

D1Q3_MUTANTS = {
    "d1q3 e_eq pressure coefficient": ("eq[2] = 3.0 * (rho * u * u + pr) - 2.0 * p.lambda * p.lambda * rho;",
                                       "eq[2] = 3.0 * (rho * u * u + 0.9 * pr) - 2.0 * p.lambda * p.lambda * rho;"),
    "d1q3 e_eq kinetic term dropped": ("eq[2] = 3.0 * (rho * u * u + pr) - 2.0 * p.lambda * p.lambda * rho;",
                                       "eq[2] = 3.0 * (pr) - 2.0 * p.lambda * p.lambda * rho;"),
    "d1q3 e_eq lattice term": ("eq[2] = 3.0 * (rho * u * u + pr) - 2.0 * p.lambda * p.lambda * rho;",
                               "eq[2] = 3.0 * (rho * u * u + pr) - 1.0 * p.lambda * p.lambda * rho;"),
    "d1q3 EOS exponent": ("std::pow(rho / p.scale, p.gamma)", "std::pow(rho / p.scale, p.gamma - 1.0)"),
    "d1q3 psi_eq sign": ("eq[1] = p.u0 * zeta;", "eq[1] = -p.u0 * zeta;"),
    "d1q3 eps_eq drops a lambda": ("eq[2] = p.alpha * p.lambda * p.lambda * zeta;",
                                   "eq[2] = p.alpha * p.lambda * zeta;"),
    "d1q3 psi relaxed with s_eps": ("m[1] = m[1] + p.s_psi * (eq[1] - m[1]);", "m[1] = m[1] + p.s_eps * (eq[1] - m[1]);"),
    "d1q3 e fully relaxed": ("m[2] = m[2] + p.s_e * (eq[2] - m[2]);", "m[2] = eq[2];"),
    "d1q3 M energy row": ("{-2 * l * l, l * l, l * l}", "{-l * l, l * l, l * l}"),
    "d1q3 M momentum row sign": ("{0, l, -l}", "{0, -l, l}"),
    "d1q3 stream direction": ("f[3 * j + 1] = post[3 * l + 1];", "f[3 * j + 1] = post[3 * r + 1];"),
}


@pytest.mark.parametrize("name", sorted(D1Q3_MUTANTS))
def test_d1q3_pins_catch_planted_mistake(name, tmp_path):
    old, new = D1Q3_MUTANTS[name]
    src = open(D1Q3_SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not found exactly once"
    mut = tmp_path / "d1q3_mutant.cpp"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libd1q3_mutant.so"
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(lib), str(mut)], check=True)
    env = dict(os.environ, D1Q3_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_d1q3.py")],
                       env=env, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode != 0, f"pins did not catch the mutant {name!r}:\n{r.stdout[-2000:]}"


D2_SRC = os.path.join(ROOT, "oracle", "d2q9q5_oracle.cpp")

D2_MUTANTS = {
    "2d q_eq coefficient": ("eq[3] = -l2 * Jx;", "eq[3] = -0.5 * l2 * Jx;"),
    "2d xi_eq sign": ("eq[9] = Exx - Eyy;", "eq[9] = Eyy - Exx;"),
    "2d shear term factor": ("+ 0.5 * shear * shear;", "+ shear * shear;"),
    "2d divergence term dropped": ("(2.0 * DD + div * div)", "(2.0 * DD)"),
    "2d log T term ignores beta": ("(rho * ph.cp * l2 / (ph.gamma * ph.beta))",
                                   "(2.0 * rho * ph.cp * l2 / (3.0 * ph.gamma))"),
    "2d e_eq lattice term": ("eq[0] = 3.0 * (Pxx + Pyy) - 4.0 * l2 * rho;", "eq[0] = 3.0 * (Pxx + Pyy) - 2.0 * l2 * rho;"),
    "2d h_eq drops 1/rho": ("9.0 * Pxx * Pyy / rho;", "9.0 * Pxx * Pyy;"),
    "2d streaming against c_x": ("const int64_t xt = (x + CX[i] + Nx) % Nx", "const int64_t xt = (x - CX[i] + Nx) % Nx"),
    "2d thermal term over T": ("kappa / (T * T) * (dxT * dxT + dyT * dyT)", "kappa / T * (dxT * dxT + dyT * dyT)"),
    "2d nu drops lambda": ("const double nu = sigma_e * ph.lambda * ph.dx;", "const double nu = sigma_e * ph.dx;"),
    "2d E_xx uses Pi_yy": ("const double Exx = s * Pxx + L, Eyy = s * Pyy + L;",
                           "const double Exx = s * Pyy + L, Eyy = s * Pyy + L;"),
    "2d psi_y uses u_x": ("eq[7] = zeta * uy;", "eq[7] = zeta * ux;"),
    "2d M xy row": ("mm.M[6][j] = vx * vy;", "mm.M[6][j] = vx * vy * 0.5;"),
    "2d q relaxed with s_h": ("{rt.s_e, rt.s_e, rt.s_e, rt.s_q, rt.s_q, rt.s_h,", "{rt.s_e, rt.s_e, rt.s_e, rt.s_h, rt.s_h, rt.s_h,"),
    "2d xi relaxed with s_psi": ("rt.s_psi, rt.s_psi, rt.s_eps, rt.s_eps};", "rt.s_psi, rt.s_psi, rt.s_eps, rt.s_psi};"),
}


@pytest.mark.parametrize("name", sorted(D2_MUTANTS))
def test_d2q9q5_pins_catch_planted_mistake(name, tmp_path):
    old, new = D2_MUTANTS[name]
    src = open(D2_SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not found exactly once"
    mut = tmp_path / "d2_mutant.cpp"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libd2_mutant.so"
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                    "-o", str(lib), str(mut)], check=True)
    env = dict(os.environ, D2Q9Q5_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_d2q9q5.py")],
                       env=env, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode != 0, f"pins did not catch the mutant {name!r}:\n{r.stdout[-2000:]}"


D3_SRC = os.path.join(ROOT, "oracle", "d3q19q7_oracle.cpp")

D3_MUTANTS = {
    "3d q_eq coefficient": ("eq[6 + a] = -(2.0 / 3.0) * l2 * rho * u[a];", "eq[6 + a] = -l2 * rho * u[a];"),
    "3d xiww sign": ("eq[20] = Eyy - Ezz;", "eq[20] = Ezz - Eyy;"),
    "3d divergence term dropped": ("(2.0 * DD + div * div)", "(2.0 * DD)"),
    "3d strain not symmetrised": ("const double D = 0.5 * (G[a][b] + G[b][a]);", "const double D = G[a][b];"),
    "3d log T term ignores beta": ("(rho * ph.cp * l2 / (ph.gamma * ph.beta))",
                                   "(2.0 * rho * ph.cp * l2 / (3.0 * ph.gamma))"),
    "3d e_eq lattice term": ("eq[0] = 19.0 * tr - 30.0 * l2 * rho;", "eq[0] = 19.0 * tr - 20.0 * l2 * rho;"),
    "3d Q4 drops 1/rho": ("const double Qxy = Pi[0][0] * Pi[1][1] / rho,", "const double Qxy = Pi[0][0] * Pi[1][1],"),
    "3d pixx Q4_yz coefficient": ("+ 3.0 * (Qxy + Qxz) - 6.0 * Qyz;", "+ 3.0 * (Qxy + Qxz) - 3.0 * Qyz;"),
    "3d streaming against c_z": ("zt = (z + CZ[i] + Nz) % Nz;", "zt = (z - CZ[i] + Nz) % Nz;"),
    "3d y neighbour not wrapped": ("(z * Ny + (y == 0 ? Ny - 1 : y - 1)) * Nx + x", "(z * Ny + (y == 0 ? 0 : y - 1)) * Nx + x"),
    "3d thermal term over T": ("kappa / (T * T) * gT2", "kappa / T * gT2"),
    "3d nu drops lambda": ("const double nu = sigma_e * ph.lambda * ph.dx;", "const double nu = sigma_e * ph.dx;"),
    "3d E_zz uses Pi_yy": ("Ezz = s * Pi[2][2] + L;", "Ezz = s * Pi[1][1] + L;"),
    "3d psi_eq uses J": ("eq[15 + a] = zeta * u[a];", "eq[15 + a] = rho * u[a];"),
    "3d M pyz row": ("mm.M[9][j] = l2 * cy * cz;", "mm.M[9][j] = l2 * cy * cz * 0.5;"),
    "3d eps7 row orthogonal": ("mm.M[23][j] = ph.cp * l2 * (3.0 * c2 - 6.0);", "mm.M[23][j] = ph.cp * l2 * (7.0 * c2 - 6.0);"),
    "3d psi relaxed with s_e": ("for (int k = 15; k < 18; ++k) rate[k] = rt.s_psi;",
                                "for (int k = 15; k < 18; ++k) rate[k] = rt.s_e;"),
    "3d entropy second moments relaxed with s_h": ("for (int k = 18; k < 21; ++k) rate[k] = rt.s_eps;",
                                                   "for (int k = 18; k < 21; ++k) rate[k] = rt.s_h;"),
    "3d pxx_eq coefficient": ("eq[1] = 3.0 * Pi[0][0] - tr;", "eq[1] = 2.0 * Pi[0][0] - tr;"),
    "3d pww_eq dropped": ("eq[2] = Pi[1][1] - Pi[2][2];", "eq[2] = 0.0;"),
    "3d m_eq not zero": ("for (int a = 0; a < 3; ++a) eq[9 + a] = 0.0;", "for (int a = 0; a < 3; ++a) eq[9 + a] = 0.1 * l2 * rho * u[a];"),
    "3d piww Q4 sign": ("+ 3.0 * (Qxy - Qxz);", "+ 3.0 * (Qxz - Qxy);"),
    "3d eps_eq Q4 coefficient": ("+ 21.0 * (Qxy + Qyz + Qxz);", "+ 20.0 * (Qxy + Qyz + Qxz);"),
    "3d z neighbour not wrapped": ("((z == Nz - 1 ? 0 : z + 1) * Ny + y) * Nx + x", "((z == Nz - 1 ? z : z + 1) * Ny + y) * Nx + x"),
    "3d q relaxed with s_h": ("for (int k = 6; k < 12; ++k) rate[k] = rt.s_q;", "for (int k = 6; k < 12; ++k) rate[k] = rt.s_h;"),
    "3d thermal gradient drops z": ("gT2 = gT2 + dT[a] * dT[a];", "gT2 = gT2 + (a < 2 ? dT[a] * dT[a] : 0.0);"),
}


@pytest.mark.parametrize("name", sorted(D3_MUTANTS))
def test_d3q19q7_pins_catch_planted_mistake(name, tmp_path):
    old, new = D3_MUTANTS[name]
    src = open(D3_SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not found exactly once"
    mut = tmp_path / "d3_mutant.cpp"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libd3_mutant.so"
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                    "-o", str(lib), str(mut)], check=True)
    env = dict(os.environ, D3Q19Q7_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_d3q19q7.py")],
                       env=env, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode != 0, f"pins did not catch the mutant {name!r}:\n{r.stdout[-2000:]}"
