"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: the matrices printed in the
paper, closed forms of the paper's Taylor-expansion analysis (sections 3, 7, 8), exact
invariants of the scheme, brute force on tiny lattices, or central finite differences.
"""
import numpy as np
import pytest

from conftest import read_params, read_symbolic_matrix
import _linear as L
from paper_1802_02369_gb300 import workloads as W


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _smooth_state(O, ph, N, seed, amp=0.02):
    """Random smooth periodic data (a few low Fourier modes) with varying entropy."""
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(N) / N
    def field(a):
        out = np.zeros(N)
        for k in range(1, 4):
            out += a * rng.uniform(-1, 1) * np.sin(k * x + rng.uniform(0, 2 * np.pi))
        return out
    rho = 1.0 + field(amp)
    u = field(amp)
    s = field(amp)
    return O.init(ph, rho, u, s=s), rho, u, s


# ---------------------------------------------------------------------------------------------
# Matrices: eq. (M-d1q3q3) and eq. (Lambda-d1q3q3).

@pytest.mark.parametrize("lam,cp,rho0", [(1.0, 1.0, 1.0), (2.0, 3.0, 1.5), (0.7, 2.5, 0.8)])
def test_moment_matrix_matches_paper(O, lam, cp, rho0):
    ph = O.default_phys(lam=lam, cp=cp, rho0=rho0)
    M, Minv = O.matrices(ph)
    expect = read_symbolic_matrix("M_d1q3q3.txt", l=lam, c=cp, rho0=rho0)
    np.testing.assert_allclose(M, expect, rtol=0, atol=1e-14)
    np.testing.assert_allclose(M @ Minv, np.eye(6), rtol=0, atol=1e-13)
    np.testing.assert_allclose(Minv @ M, np.eye(6), rtol=0, atol=1e-13)


@pytest.mark.parametrize("lam,cp", [(1.0, 1.0), (2.0, 3.0), (0.5, 0.25)])
def test_lambda_tensor_matches_paper(O, lam, cp):
    """Lambda = lambda M diag(v) M^{-1} (eq. Lambda-general) equals the printed eq. (Lambda-d1q3q3)."""
    ph = O.default_phys(lam=lam, cp=cp)
    M, Minv = O.matrices(ph)
    v = np.diag([0.0, 1.0, -1.0, 0.0, 1.0, -1.0])
    Lam = lam * M @ v @ Minv
    np.testing.assert_allclose(Lam, read_symbolic_matrix("Lambda_d1q3q3.txt", l=lam), rtol=0, atol=1e-12)


def test_paper_viscosity_value(O):
    """s_e = 1.9, dx = 1/40, lambda = 1 gives nu = sigma_e lambda dx = 6.579e-4 (sections 7, 9)."""
    p = read_params("paper_parameters.txt")
    sigma_e = 1.0 / p["s_e"] - 0.5
    assert abs(sigma_e * p["lambda"] * p["dx"] - p["nu"]) < 0.5e-7
    # The oracle's coupled rate: at G(0) the relaxed moments decay by 1 - s (checked below), and the
    # entropy diffusion is gamma nu / Pr at leading order (checked by the damping test).
    r = O.coupled_rates(p["s_e"], p["gamma"], p["Pr"])
    assert r[0] == p["s_e"] and r[2] == 1.5


# ---------------------------------------------------------------------------------------------
# Linear analysis around uniform states.

@pytest.mark.parametrize("s_e", [1.0, 1.2, 1.5, 1.9])
def test_symbol_at_zero_wavenumber(O, s_e):
    """At theta = 0 the step keeps (rho, J, zeta) and multiplies e, psi, eps by 1 - s."""
    ph = O.default_phys()
    r = O.coupled_rates(s_e)
    B = L.jacobian_blocks(ph, r, 1.0, 0.07, -0.05)
    w = np.sort(np.linalg.eigvals(L.symbol(B, 0.0)).real)
    expect = np.sort(np.r_[1.0, 1.0, 1.0, 1.0 - r])
    np.testing.assert_allclose(w, expect, atol=1e-12)


def test_full_jacobian_spectrum_is_union_of_symbols(O):
    """Brute force on N = 8: eig of the 48x48 Jacobian equals the union of eig G(2 pi k / N)."""
    ph = O.default_phys()
    r = O.coupled_rates(1.6)
    N = 8
    fd = L.uniform_state(ph, 1.1, 0.05, -0.03, N)
    full = np.linalg.eigvals(L.full_jacobian(ph, r, fd))
    B = L.jacobian_blocks(ph, r, 1.1, 0.05, -0.03, N=N)
    union = np.concatenate([np.linalg.eigvals(L.symbol(B, 2 * np.pi * k / N)) for k in range(N)])
    # Greedy matching (the spectra are well separated at this state).
    remaining = list(full)
    for z in union:
        i = int(np.argmin([abs(z - y) for y in remaining]))
        assert abs(z - remaining[i]) < 1e-8
        remaining.pop(i)
    assert not remaining


@pytest.mark.parametrize("rho,u0,s", [(1.0, 0.0, 0.0), (1.0, 0.05, 0.0), (0.8, -0.08, -0.1), (1.2, 0.1, 0.05)])
def test_phase_speeds_are_euler_characteristics(O, rho, u0, s):
    """First-order equivalent equations (eq. edp1-d1q3q3) with e_eq, psi_eq of eqs.
    (energie-equilibre, psi-equilibre) are the Euler equations: the conserved modes travel at
    u0 + c, u0 - c and u0 with c^2 = gamma p / rho (section 5)."""
    ph = O.default_phys()
    r = O.coupled_rates(1.2)
    B = L.jacobian_blocks(ph, r, rho, u0, s)
    th = 1e-3
    speeds = np.sort(-ph.lam * np.angle(L.conserved_modes(L.symbol(B, th))) / th)
    p = ph.p0 * (rho / ph.rho0) ** ph.gamma * np.exp(ph.gamma * (s - ph.s0) / ph.cp)
    c = np.sqrt(ph.gamma * p / rho)
    np.testing.assert_allclose(speeds, np.sort([u0 - c, u0, u0 + c]), rtol=0, atol=1e-5)


@pytest.mark.parametrize("s_e,lam,gamma,Pr", [(1.2, 1.0, 1.4, 1.0), (1.5, 1.0, 1.4, 1.0), (1.9, 1.0, 1.4, 1.0),
                                             (1.5, 2.0, 1.4, 1.0), (1.5, 1.0, 1.3, 0.71), (1.2, 2.0, 1.67, 2.0)])
def test_second_order_damping(O, s_e, lam, gamma, Pr):
    """Damping of the conserved modes at rest (u0 = 0, s = 0) against the second-order equivalent
    equations eq. (edp-ordre-2) with the defects eq. (thetas) and the tensor eq. (Lambda-d1q3q3).

    Linearising the equilibria at rest gives the diffusion matrix on (rho, J, zeta)
        D_JJ = sigma_e dt (lambda^2 - c0^2),
        D_zr = sigma_psi dt (2/3) lambda^2 (1 - 1/gamma) c_p,
        D_zz = sigma_psi dt (2 lambda^2/3 + c0^2/gamma),
    so an acoustic mode decays at (D_JJ + D_zr / c_p)/2 and the entropy mode at D_zz - D_zr / c_p
    (first-order perturbation of the Euler eigenvalues), with sigma = 1/s - 1/2 (eq. henon) and
    sigma_psi = (3/2)(gamma/Pr) sigma_e (eq. lien-sigma-sigma). Away from gamma/Pr = 1.4 the coupled
    rate s_psi changes D_zr and D_zz, which pins the Pr and gamma factors of the coupling."""
    ph = O.default_phys(lam=lam, gamma=gamma, Pr=Pr)
    r = O.coupled_rates(s_e, ph.gamma, ph.Pr)
    g, c0, dt, cp = ph.gamma, lam / 2, 1.0 / lam, ph.cp
    sig_e = 1 / s_e - 0.5
    sig_p = 1.5 * g / ph.Pr * sig_e
    D_JJ = sig_e * dt * (lam ** 2 - c0 ** 2)
    D_zr = sig_p * dt * (2 / 3) * lam ** 2 * (1 - 1 / g) * cp
    D_zz = sig_p * dt * (2 * lam ** 2 / 3 + c0 ** 2 / g)
    gam_ac = 0.5 * (D_JJ + D_zr / cp)
    gam_s = D_zz - D_zr / cp
    B = L.jacobian_blocks(ph, r, 1.0, 0.0, 0.0)
    th = 2e-3
    w = L.conserved_modes(L.symbol(B, th))
    # Re log(mu) = -Gamma k^2 dt with k = theta / dx (dx = 1).
    rates = np.sort(-np.log(np.abs(w)) / (th ** 2 * dt))
    np.testing.assert_allclose(rates, np.sort([gam_ac, gam_ac, gam_s]), rtol=2e-5)


@pytest.mark.parametrize("s_e", [1.0, 1.2, 1.5, 1.9])
def test_linearly_stable_at_rest(O, s_e):
    """Spectral radius <= 1 over all wavenumbers at the reference state of section 9 (u0 = 0,
    s0 = 0, c0 = lambda/2) and at a slow flow."""
    ph = O.default_phys()
    r = O.coupled_rates(s_e)
    for u0 in (0.0, 0.05):
        B = L.jacobian_blocks(ph, r, 1.0, u0, 0.0)
        rad = max(np.abs(np.linalg.eigvals(L.symbol(B, t))).max() for t in np.linspace(0, np.pi, 181))
        assert rad <= 1.0 + 1e-12


# ---------------------------------------------------------------------------------------------
# Invariants of the nonlinear step.

@pytest.mark.parametrize("bc", [0, 1])
def test_uniform_states_are_fixed_points(O, bc):
    rng = np.random.default_rng(3)
    for _ in range(3):
        ph = O.default_phys(bc=bc)
        rho, s = rng.uniform(0.7, 1.3), rng.uniform(-0.2, 0.1)
        u = 0.0 if bc else rng.uniform(-0.08, 0.08)
        fd = L.uniform_state(ph, rho, u, s, 17)
        out = O.run(ph, O.coupled_rates(1.7), fd, 50)
        np.testing.assert_allclose(out, fd, rtol=2e-14, atol=1e-15)


def test_mass_momentum_conserved_and_entropy_nondecreasing(O):
    ph = O.default_phys()
    r = O.coupled_rates(1.3)
    fd, *_ = _smooth_state(O, ph, 96, seed=11, amp=0.04)
    sums0, _ = O.diagnostics(ph, fd)
    prev = sums0[2]
    for _ in range(40):
        fd = O.run(ph, r, fd, 50)
        sums, flags = O.diagnostics(ph, fd)
        assert flags == 0
        assert abs(sums[0] - sums0[0]) <= 1e-13 * abs(sums0[0])
        assert abs(sums[1] - sums0[1]) <= 1e-13 * abs(sums0[0])
        assert sums[2] >= prev - 1e-15 * abs(sums0[0])
        prev = sums[2]
    assert prev > sums0[2]  # entropy is actually produced


def test_entropy_conserved_without_source(O):
    ph = O.default_phys(source_on=0)
    fd, *_ = _smooth_state(O, ph, 64, seed=5, amp=0.04)
    z0 = O.diagnostics(ph, fd)[0][2]
    z1 = O.diagnostics(ph, O.run(ph, O.coupled_rates(1.4), fd, 500))[0][2]
    assert abs(z1 - z0) <= 1e-14 * 64


def test_mirror_symmetry(O):
    """x -> -x with f+ <-> f-, g+ <-> g- maps solutions to solutions (J, psi change sign)."""
    ph = O.default_phys()
    r = O.coupled_rates(1.5)
    fd, *_ = _smooth_state(O, ph, 50, seed=7, amp=0.05)
    mir = fd[::-1][:, [0, 2, 1, 3, 5, 4]]
    a = O.run(ph, r, fd, 200)
    b = O.run(ph, r, mir, 200)
    np.testing.assert_allclose(b[::-1][:, [0, 2, 1, 3, 5, 4]], a, rtol=0, atol=2e-14)


def test_cp_covariance(O):
    """Scaling c_p by k with s/c_p fixed: rho, J unchanged, zeta, psi, eps scaled by k, so the g
    populations (zeta = rho0 c_p sum g) are unchanged."""
    r = O.coupled_rates(1.4)
    ph1 = O.default_phys(cp=1.0)
    ph2 = O.default_phys(cp=2.5)
    _, rho, u, s = _smooth_state(O, ph1, 40, seed=9, amp=0.05)
    a = O.run(ph1, r, O.init(ph1, rho, u, s=s), 300)
    b = O.run(ph2, r, O.init(ph2, rho, u, s=2.5 * s), 300)
    np.testing.assert_allclose(b, a, rtol=0, atol=5e-14)
    ma, mb = O.moments(ph1, a), O.moments(ph2, b)
    np.testing.assert_allclose(mb[:, :2], ma[:, :2], atol=5e-14)
    np.testing.assert_allclose(mb[:, 2:3], 2.5 * ma[:, 2:3], atol=5e-14)


def test_initial_pressure_round_trip(O):
    """Initialising from (rho, u = 0, p) inverts eq. (gaz-parfait) for the specific entropy; at rest the
    energy equilibrium of eq. (energie-equilibre) is 3 p - 2 lambda^2 rho, so it must return the given
    pressure (non-adiabatic data, so that the inversion is exercised away from s = s0)."""
    rng = np.random.default_rng(41)
    for lam, gamma, cp, rho0, s0 in ((1.0, 1.4, 1.0, 1.0, 0.0), (2.0, 1.3, 2.5, 1.3, -0.1)):
        ph = O.default_phys(lam=lam, gamma=gamma, cp=cp, rho0=rho0, s0=s0)
        N = 32
        rho = rho0 * rng.uniform(0.5, 1.5, N)
        p = ph.p0 * rng.uniform(0.4, 1.6, N)
        e_eq = O.equilibria(ph, O.init(ph, rho, np.zeros(N), p=p))[:, 0]
        np.testing.assert_allclose((e_eq + 2 * lam ** 2 * rho) / 3, p, rtol=1e-13)


def test_rho0_covariance(O):
    """Scaling the reference density and pressure (rho0, p0) -> (k rho0, k p0) together with the
    data rho -> k rho at fixed u and s scales p by k (eq. gaz-parfait) and leaves T = p/(rho r) and
    T0 = p0/(rho0 r) unchanged; every moment (rho, J, zeta = rho s, e_eq, psi_eq, eps_eq and the source,
    whose kappa = rho nu c_p / Pr is proportional to rho) then scales by k, as does M of
    eq. (M-d1q3q3), so the populations are identical at every step."""
    r = O.coupled_rates(1.4)
    ph1 = O.default_phys()
    _, rho, u, s = _smooth_state(O, ph1, 40, seed=19, amp=0.05)
    a = O.run(ph1, r, O.init(ph1, rho, u, s=s), 200)
    for k in (1.7, 0.6):
        phk = O.default_phys(rho0=k, p0=k * ph1.p0)
        b = O.run(phk, r, O.init(phk, k * rho, u, s=s), 200)
        np.testing.assert_allclose(b, a, rtol=0, atol=5e-14)


def test_total_energy_kinetic_part_is_galilean(O):
    """The total energy of the diagnostics, sum of rho E over the lattice, of a uniform state moving at
    u exceeds that of the same state at rest (same rho and s) by exactly the kinetic energy of a rigid
    translation, N rho u^2 / 2."""
    ph = O.default_phys()
    N = 16
    for rho, s, u in ((1.0, 0.0, 0.1), (0.7, -0.2, -0.25), (1.3, 0.1, 0.05)):
        e_rest = O.diagnostics(ph, L.uniform_state(ph, rho, 0.0, s, N))[0][3]
        e_move = O.diagnostics(ph, L.uniform_state(ph, rho, u, s, N))[0][3]
        assert abs((e_move - e_rest) - N * rho * u * u / 2) <= 1e-13 * N


def test_total_energy_internal_part_obeys_gibbs(O):
    """At rest the total energy is the internal energy, whose derivative in the specific entropy at
    fixed density is rho T (Gibbs relation de = T ds + p / rho^2 drho), with T from the gas law
    p = rho r T, r = c_p (1 - 1/gamma), and p from eq. (gaz-parfait)."""
    N, h = 8, 1e-5
    for gamma, cp, rho0 in ((1.4, 1.0, 1.0), (1.3, 2.5, 1.3)):
        ph = O.default_phys(gamma=gamma, cp=cp, rho0=rho0)
        for rho, s in ((1.0, 0.0), (0.6, -0.3), (1.4, 0.2)):
            rho = rho * rho0
            ep = O.diagnostics(ph, L.uniform_state(ph, rho, 0.0, s + h, N))[0][3]
            em = O.diagnostics(ph, L.uniform_state(ph, rho, 0.0, s - h, N))[0][3]
            p = ph.p0 * (rho / ph.rho0) ** gamma * np.exp(gamma * (s - ph.s0) / cp)
            T = p / (rho * cp * (1 - 1 / gamma))
            assert abs((ep - em) / (2 * h) / (N * rho * T) - 1) < 1e-8


def test_step_independent_of_dx(O):
    """With nu = sigma_e lambda dx (eq. nu-d1q3q3), dt = dx / lambda and centred differences, the
    step in lattice units does not depend on dx."""
    r = O.coupled_rates(1.9)
    ph1 = O.default_phys(dx=1.0)
    ph2 = O.default_phys(dx=1.0 / 40)
    fd, *_ = _smooth_state(O, ph1, 40, seed=13, amp=0.05)
    np.testing.assert_allclose(O.run(ph2, r, fd, 120), O.run(ph1, r, fd, 120), rtol=0, atol=1e-13)


@pytest.mark.parametrize("lam,dx,gamma,Pr,rho0", [(1.0, 1.0, 1.4, 1.0, 1.0), (2.0, 0.5, 1.4, 1.0, 1.0),
                                                  (0.5, 1.0 / 40, 1.4, 1.0, 1.0), (1.0, 1.0, 1.3, 0.71, 1.0),
                                                  (2.0, 0.5, 1.67, 0.71, 1.3)])
def test_entropy_production_closed_form(O, lam, dx, gamma, Pr, rho0):
    """One step of a small progressive wave u = c0 d sin(k x), rho = rho0 (1 + d sin(k x)),
    adiabatic: the collision keeps zeta and streaming permutes it, so the change of sum zeta is
    dt sum_j S_j with S of eq. (NS-rho-J-zeta). With T = T0 (rho/rho0)^(gamma-1), centred
    differences sin(k dx)/(k dx) times the exact gradients, and sum cos^2 = N/2 over a period:
        sum zeta(1) - sum zeta(0)
            = dt rho0 nu d^2 k^2 (N/2) (sin(k dx)/(k dx))^2 (c0^2 / T0 + c_p (gamma-1)^2 / Pr)
    up to O(d) relative corrections, with nu = sigma_e lambda dx (eq. nu-d1q3q3), dt = dx/lambda,
    kappa = rho nu c_p / Pr (the thermal term carries 1/Pr, the viscous one does not).
    T0 = c0^2 / (c_p (gamma - 1)) follows from p0 = rho0 c0^2 / gamma and the gas law p = rho r T with
    r = c_p (1 - 1/gamma), so the two terms stand in the ratio (gamma - 1) / Pr."""
    for s_e, N in ((1.9, 256), (1.2, 512), (1.5, 128)):
        ph = O.default_phys(lam=lam, dx=dx, gamma=gamma, Pr=Pr, rho0=rho0)
        g, c0, d = ph.gamma, ph.lam / 2, 1e-3
        T0 = c0 ** 2 / (ph.cp * (g - 1))
        rho, u, p = W.progressive_wave(N, d, c0, ph.p0, gamma=g, rho0=rho0)
        fd = O.init(ph, rho, u, p=p)
        dz = O.diagnostics(ph, O.run(ph, O.coupled_rates(s_e), fd, 1))[0][2] - O.diagnostics(ph, fd)[0][2]
        k = 2 * np.pi / (N * dx)
        nu = (1 / s_e - 0.5) * lam * dx
        corr = (np.sin(k * dx) / (k * dx)) ** 2
        pred = (dx / lam) * rho0 * nu * d * d * k * k * (N / 2) * corr * (c0 ** 2 / T0 + ph.cp * (g - 1) ** 2 / ph.Pr)
        assert abs(dz / pred - 1) < 2e-5


def test_source_reduces_total_energy_defect(O):
    """Section 9, figure 4 discussion: without the entropy source the total energy
    sum(p/(gamma-1) + rho u^2/2) is not conserved; with it the defect is much smaller."""
    N, d = 128, 0.01
    defects = {}
    for src in (1, 0):
        ph = O.default_phys(source_on=src)
        rho, u, p = W.progressive_wave(N, d, ph.lam / 2, ph.p0)
        fd = O.init(ph, rho, u, p=p)
        E0 = O.diagnostics(ph, fd)[0][3]
        E1 = O.diagnostics(ph, O.run(ph, O.coupled_rates(1.2), fd, 3000))[0][3]
        defects[src] = E1 - E0
    assert defects[0] < 0
    assert abs(defects[1]) < 0.3 * abs(defects[0])


def test_entropy_energy_equilibrium_two_forms(O):
    """eq. (eq-energie-entropie-d1q3q3) in its log(T/T0) form equals the printed polytropic form
    eps_eq = 2 lambda^2 [rho (s - s0) + (1 - 1/gamma) c_p rho log(rho/rho0)] + [3(rho u^2 + p) - 2 lambda^2 rho] s."""
    rng = np.random.default_rng(21)
    for lam, cp, s0, rho0 in ((1.0, 1.0, 0.0, 1.0), (2.0, 1.7, 0.3, 1.0), (1.5, 1.2, -0.1, 1.3)):
        ph = O.default_phys(lam=lam, cp=cp, s0=s0, rho0=rho0)
        N = 64
        rho = rho0 * rng.uniform(0.5, 1.5, N)
        u = rng.uniform(-0.3, 0.3, N)
        s = rng.uniform(-0.5, 0.5, N)
        eq = O.equilibria(ph, O.init(ph, rho, u, s=s))
        p = ph.p0 * (rho / ph.rho0) ** ph.gamma * np.exp(ph.gamma * (s - ph.s0) / cp)
        e_eq = 3 * (rho * u * u + p) - 2 * lam ** 2 * rho
        eps_poly = 2 * lam ** 2 * (rho * (s - s0) + (1 - 1 / ph.gamma) * cp * rho * np.log(rho / ph.rho0)) + e_eq * s
        np.testing.assert_allclose(eq[:, 2], eps_poly, rtol=1e-12, atol=1e-12)
        # First-order fluxes (eq. edp1-d1q3q3): 2 lambda^2 rho / 3 + e_eq / 3 = rho u^2 + p.
        np.testing.assert_allclose(2 * lam ** 2 * rho / 3 + eq[:, 0] / 3, rho * u * u + p, rtol=1e-12)
        np.testing.assert_allclose(eq[:, 1], rho * s * u, rtol=1e-12, atol=1e-14)


def test_bounce_back_equals_mirrored_periodic(O):
    """Halfway bounce-back with ghosts u_{-1} = -u_0, T_{-1} = T_0 is specular reflection: a
    bounce-back lattice of N nodes evolves like the first half of a periodic lattice of 2N nodes
    holding the data and its mirror image."""
    r = O.coupled_rates(1.3)
    N = 30
    rng = np.random.default_rng(17)
    rho = 1 + 0.05 * rng.uniform(-1, 1, N)
    u = 0.03 * rng.uniform(-1, 1, N)
    s = 0.05 * rng.uniform(-1, 1, N)
    phb = O.default_phys(bc=1)
    php = O.default_phys(bc=0)
    a = O.run(phb, r, O.init(phb, rho, u, s=s), 150)
    big = O.init(php, np.r_[rho, rho[::-1]], np.r_[u, -u[::-1]], s=np.r_[s, s[::-1]])
    b = O.run(php, r, big, 150)
    np.testing.assert_allclose(b[:N], a, rtol=0, atol=5e-14)
    sa, _ = O.diagnostics(phb, O.init(phb, rho, u, s=s))
    sb, _ = O.diagnostics(phb, a)
    assert abs(sb[0] - sa[0]) < 1e-13 * N   # mass conserved by the walls


def test_tangents_match_central_differences(O):
    """Forward-mode dual numbers (used to check gradients) against central differences, h = 1e-6."""
    ph = O.default_phys()
    N, T = 24, 40
    _, rho, u, s = _smooth_state(O, ph, N, seed=23, amp=0.05)
    rates = O.coupled_rates(1.4)
    rng = np.random.default_rng(29)
    drho = rng.standard_normal((3, N)) * 0.1
    du = rng.standard_normal((3, N)) * 0.1
    dr = np.array([[0.0, 0.0], [1.0, 0.0], [0.3, -0.7]])
    fd, dfd = O.run_tangent(ph, rates, dr, rho, u, s, drho, du, T)
    h = 1e-6
    for k in range(3):
        def F(eps):
            rr = rates.copy()
            rr[:2] += eps * dr[k]
            return O.run(ph, rr, O.init(ph, rho + eps * drho[k], u + eps * du[k], s=s), T)
        fd_c = (F(h) - F(-h)) / (2 * h)
        np.testing.assert_allclose(dfd[k], fd_c, rtol=0, atol=2e-8 * np.abs(fd_c).max() + 1e-10)
    np.testing.assert_allclose(fd, O.run(ph, rates, O.init(ph, rho, u, s=s), T), atol=1e-15)


# ---------------------------------------------------------------------------------------------
# Shapes of the section 9 experiments and of the Riemann data.

def test_strong_wave_forms_a_shock_with_localised_entropy(O):
    """Figure 3 (delta rho = 0.1 rho0, dx = 1/160, T_max = 3): the wave steepens into a shock and
    the entropy production is localised where the fields vary strongly."""
    ph = O.default_phys()
    N = 160
    rho, u, p = W.progressive_wave(N, 0.1, ph.lam / 2, ph.p0)
    fd = O.init(ph, rho, u, p=p)
    out = O.run(ph, O.coupled_rates(1.9), fd, 3 * N)   # T_max = 3 with dx = 1/N, lambda = 1
    sums, flags = O.diagnostics(ph, out)
    assert flags == 0
    m = O.moments(ph, out)
    grad = np.abs(np.diff(np.r_[m[:, 0], m[0, 0]]))
    assert grad.max() > 8 * np.abs(np.diff(np.r_[rho, rho[0]])).max()
    s = m[:, 2] / m[:, 0]
    jshock, jsmax = int(grad.argmax()), int(s.argmax())
    dist = min(abs(jshock - jsmax), N - abs(jshock - jsmax))
    assert dist <= 3


def test_riemann_sod_readings(O):
    """Sod data with pressures in units of p0 = rho0 c0^2 / gamma runs 500 steps at s_e = 1.2;
    at s_e = 1.5 the scheme goes unstable near step 130 (nonlinear instability at the
    discontinuities); the literal pressures (c^2 = 1.4 lambda^2) blow up within 10 steps."""
    ph = O.default_phys()
    rho, u, p = W.sod(256, ph.p0)
    fd = O.init(ph, rho, u, p=p)
    sums0, _ = O.diagnostics(ph, fd)
    sums, flags = O.diagnostics(ph, O.run(ph, O.coupled_rates(1.2), fd, 500))
    assert flags == 0 and abs(sums[0] - sums0[0]) < 1e-12 * sums0[0]
    assert O.diagnostics(ph, O.run(ph, O.coupled_rates(1.5), fd, 100))[1] == 0
    assert O.diagnostics(ph, O.run(ph, O.coupled_rates(1.5), fd, 500))[1] != 0
    rho, u, p = W.sod(256, 1.0)
    assert O.diagnostics(ph, O.run(ph, O.coupled_rates(1.5), O.init(ph, rho, u, p=p), 10))[1] != 0
