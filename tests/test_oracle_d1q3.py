"""Pins of the oracle of the single-distribution D1Q3 schemes (the fluid scheme of section 2 and the
advection-diffusion scheme of section 4), checked against what the paper and the mathematics fix:

- the printed matrix eq. (M-d1q3) and momentum-velocity tensor eq. (tenseur-Lambda);
- conservation of the conserved moments, fixed uniform states, mirror symmetry;
- an exact special case: with psi_eq = +-lambda zeta, eps_eq = lambda^2 zeta and full relaxation the
  advection-diffusion scheme shifts zeta by exactly one node per step;
- linear behaviour (von Neumann symbol built from the oracle's own one-step response): phase speeds
  and damping of the conserved modes equal the closed forms of the second-order equivalent
  equations, eq. (edp-d1q3) and eq. (edp-thermic-ordre-2) with the identification of kappa and
  s_psi, as the wavenumber goes to 0; the non-conserved modes relax at 1 - s;
- the stability range -2 < alpha < 1 the paper states for eps_eq = alpha lambda^2 zeta.
"""
import numpy as np
import pytest

import oracle.d1q3 as D
from conftest import read_symbolic_matrix


@pytest.fixture(scope="module", autouse=True)
def _built():
    D.build()


def _blocks(p, m0, m1, N=9, h=1e-6):
    """B_d of the one-step response of a uniform state to a perturbation of node 0 (central
    differences; the advection-diffusion scheme is linear, so there they are exact up to rounding)."""
    f0 = D.init(p, np.full(N, m0), np.full(N, m1))
    cols = []
    for k in range(3):
        fp, fm = f0.copy(), f0.copy()
        fp[0, k] += h
        fm[0, k] -= h
        cols.append((D.run(p, fp, 1) - D.run(p, fm, 1)) / (2 * h))
    B = {}
    for j in range(N):
        d = j if j <= N // 2 else j - N
        B[d] = np.stack([c[j] for c in cols], axis=1)
    return B


def _symbol(B, theta):
    return sum(Bd * np.exp(-1j * theta * d) for d, Bd in B.items())


def _smooth(N, seed, amp):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(N) / N
    k = np.arange(1, 5)
    c = rng.normal(size=(2, k.size)) * amp / k
    return (c[0][:, None] * np.sin(k[:, None] * x) + c[1][:, None] * np.cos(k[:, None] * x)).sum(0)


@pytest.mark.parametrize("lam,scale", [(1.0, 1.0), (2.0, 0.7), (0.5, 1.3)])
def test_matrix_and_lambda_tensor_are_the_printed_ones(lam, scale):
    for p in (D.fluid(1.2, lam=lam, rho0=scale), D.advection_diffusion(0.1, 0.0, 1.2, lam=lam, zeta0=scale)):
        M, Minv = D.matrices(p)
        assert np.allclose(M, read_symbolic_matrix("M_d1q3.txt", l=lam, r0=scale), rtol=0, atol=1e-14)
        assert np.allclose(M @ Minv, np.eye(3), atol=1e-14)
        Lam = lam * M @ np.diag([0.0, 1.0, -1.0]) @ Minv
        assert np.allclose(Lam, read_symbolic_matrix("Lambda_d1q3.txt", l=lam), atol=1e-13)


def test_fluid_conserves_mass_and_momentum_and_fixes_uniform_states():
    p = D.fluid(1.5)
    N = 120
    rho = 1 + _smooth(N, 1, 0.05)
    J = _smooth(N, 2, 0.02)
    f = D.init(p, rho, J)
    m0 = D.moments(p, f).sum(0)
    for _ in range(10):
        f = D.run(p, f, 200)
        m = D.moments(p, f).sum(0)
        assert abs(m[0] - m0[0]) <= 1e-13 * N
        assert abs(m[1] - m0[1]) <= 1e-13 * N
    fu = D.init(p, np.full(16, 1.3), np.full(16, 0.11))
    assert np.abs(D.run(p, fu, 300) - fu).max() <= 1e-15


def test_advection_diffusion_conserves_zeta_and_fixes_uniform_states():
    p = D.advection_diffusion(0.15, -0.5, 0.9)
    N = 96
    z = 1 + _smooth(N, 3, 0.1)
    f = D.init(p, z)
    s0 = D.moments(p, f)[:, 0].sum()
    f = D.run(p, f, 3000)
    assert abs(D.moments(p, f)[:, 0].sum() - s0) <= 1e-13 * N
    fu = D.init(p, np.full(12, 0.7))
    assert np.abs(D.run(p, fu, 500) - fu).max() <= 1e-15


def test_mirror_symmetry():
    """x -> -x (node j -> -j): f+ and f- trade places; J, psi and u0 change sign."""
    N = 40
    rho = 1 + _smooth(N, 4, 0.05)
    J = _smooth(N, 5, 0.02)
    mir = lambda a: np.roll(a[::-1], 1, axis=0)
    p = D.fluid(1.7)
    A = D.moments(p, D.run(p, D.init(p, rho, J), 250))
    B = D.moments(p, D.run(p, D.init(p, mir(rho), -mir(J)), 250))
    assert np.abs(mir(B) * np.array([1, -1, 1]) - A).max() <= 1e-13
    z = 1 + _smooth(N, 6, 0.1)
    pa, pb = D.advection_diffusion(0.2, 0.3, 1.1), D.advection_diffusion(-0.2, 0.3, 1.1)
    A = D.moments(pa, D.run(pa, D.init(pa, z), 250))
    B = D.moments(pb, D.run(pb, D.init(pb, mir(z)), 250))
    assert np.abs(mir(B) * np.array([1, -1, 1]) - A).max() <= 1e-13


@pytest.mark.parametrize("sign", [1, -1])
def test_advection_at_the_lattice_speed_is_an_exact_shift(sign):
    lam = 1.5
    p = D.advection_diffusion(sign * lam, 1.0, 1.0, lam=lam, s_eps=1.0)
    z = 1 + _smooth(50, 7, 0.3)
    m = D.moments(p, D.run(p, D.init(p, z), 7))
    assert np.abs(m[:, 0] - np.roll(z, sign * 7)).max() <= 1e-14


@pytest.mark.parametrize("alpha,s_psi,u0,lam", [(0.0, 1.2, 0.1, 1.0), (-1.0, 0.8, 0.2, 1.0), (0.5, 1.6, -0.15, 1.0),
                                                (0.0, 1.0, 0.3, 2.0)])
def test_advection_diffusion_modes_follow_the_equivalent_equation(alpha, s_psi, u0, lam):
    """Eq. (edp-thermic-ordre-2) with psi_eq = u0 zeta, eps_eq = alpha lambda^2 zeta: a Fourier mode of
    wavenumber k moves at u0 and decays at kappa k^2 with
    kappa = ((2 + alpha)/3 lambda^2 - u0^2) (1/s_psi - 1/2) dt (dx = 1, dt = 1/lambda)."""
    p = D.advection_diffusion(u0, alpha, s_psi, lam=lam)
    B = _blocks(p, 1.0, 0.0)
    dt = 1.0 / lam
    kappa = ((2 + alpha) / 3 * lam ** 2 - u0 ** 2) * (1 / s_psi - 0.5) * dt
    for theta, tol in ((0.02, 2e-4), (0.01, 5e-5)):
        w = np.linalg.eigvals(_symbol(B, theta))
        mu = w[np.argmin(np.abs(np.abs(w) - 1))]
        assert abs(-np.log(abs(mu)) / (kappa * theta ** 2 * dt) - 1) <= tol
        assert abs(-np.angle(mu) / (u0 * theta * dt) - 1) <= tol
    w0 = np.sort(np.linalg.eigvals(_symbol(B, 0.0)).real)
    assert np.allclose(w0, np.sort([1.0, 1 - s_psi, 1 - 1.5]), atol=1e-8)


@pytest.mark.parametrize("s_e,lam", [(1.2, 1.0), (1.5, 1.0), (1.9, 1.0), (1.4, 2.0)])
def test_fluid_acoustic_modes_follow_the_equivalent_equation(s_e, lam):
    """Eq. (edp-d1q3) linearised at rest: theta_e = d_t e_eq + lambda^2 d_x J = 3 (lambda^2 - c^2) d_x J
    with c^2 = gamma p0 / rho0 (the paper's 3 lambda^2 rho d_x u is its c << lambda limit), so the
    acoustic modes move at +-c and decay at (1/2) sigma_e dt (lambda^2 - c^2) k^2."""
    p = D.fluid(s_e, lam=lam)
    c = lam / 2
    B = _blocks(p, 1.0, 0.0)
    dt = 1.0 / lam
    gam = 0.5 * (1 / s_e - 0.5) * dt * (lam ** 2 - c ** 2)
    for theta, tol in ((0.02, 1e-4), (0.01, 1e-4)):
        w = np.linalg.eigvals(_symbol(B, theta))
        ac = w[np.argsort(np.abs(np.abs(w) - 1))[:2]]
        speeds = sorted(-np.angle(ac) / (theta * dt))
        assert abs(speeds[0] + c) <= tol * c and abs(speeds[1] - c) <= tol * c
        for mu in ac:
            assert abs(-np.log(abs(mu)) / (gam * theta ** 2 * dt) - 1) <= 5 * tol
    w0 = np.sort(np.linalg.eigvals(_symbol(B, 0.0)).real)
    assert np.allclose(w0, np.sort([1.0, 1.0, 1 - s_e]), atol=1e-8)


def test_fluid_moving_state_speeds_are_u_plus_minus_c():
    """At a uniform flow u the acoustic characteristics of the isentropic equations are u +- c(rho)."""
    rho, u = 1.1, 0.08
    p = D.fluid(1.3)
    c = np.sqrt(p.gamma * p.p0 * (rho / p.scale) ** (p.gamma - 1) / p.scale)
    B = _blocks(p, rho, rho * u)
    theta = 0.005
    w = np.linalg.eigvals(_symbol(B, theta))
    ac = w[np.argsort(np.abs(np.abs(w) - 1))[:2]]
    speeds = sorted(-np.angle(ac) / theta)
    assert abs(speeds[0] - (u - c)) <= 1e-4 and abs(speeds[1] - (u + c)) <= 1e-4


def test_stability_range_of_alpha():
    """Section 4: the scheme is stable for -2 < alpha < 1 (s_eps = 1.5, u0 = 0) and not outside."""
    def radius(alpha, s_psi):
        B = _blocks(D.advection_diffusion(0.0, alpha, s_psi), 1.0, 0.0)
        return max(np.abs(np.linalg.eigvals(_symbol(B, th))).max() for th in np.linspace(0, np.pi, 91))
    for s_psi in (0.5, 1.0, 1.9):
        for alpha in (-1.9, -1.0, 0.0, 0.9):
            assert radius(alpha, s_psi) <= 1 + 1e-8, (alpha, s_psi)
        for alpha in (-2.1, 1.1):
            assert radius(alpha, s_psi) >= 1.1, (alpha, s_psi)


def test_invalid_parameters_rejected():
    with pytest.raises(ValueError):
        D.run(D.fluid(2.0), np.zeros((4, 3)), 1)
    with pytest.raises(ValueError):
        D.run(D.advection_diffusion(0.0, 0.0, 0.0), np.zeros((4, 3)), 1)
