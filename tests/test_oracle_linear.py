"""Pins of the oracle's section 7 variant: the linear equilibria of eq. (equilibres-NS-linearise)
with sigma_psi from eq. (lien-sigma-sigma) and sigma_eps = 1.5 (no entropy source: the linearised
system has no production term). The printed coefficients are used in lattice units lambda = c_p = 1."""
import numpy as np
import pytest

import _linear as L


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _ph(O, u0, s0):
    return O.default_phys(eq_mode=1, u0_lin=u0, s0_lin=s0)


def test_linear_rates_follow_section_7(O):
    r = O.linear_rates(1.9)
    assert r[2] == 0.5                                   # sigma_eps = 1.5
    sig_e, sig_p = 1 / r[0] - 0.5, 1 / r[1] - 0.5
    assert abs(sig_p - 1.5 * 1.4 * sig_e) < 1e-15       # eq. (lien-sigma-sigma), gamma = 1.4, Pr = 1


def test_linear_variant_is_exactly_linear(O):
    """The step is a linear map of the populations (superposition to rounding)."""
    ph = _ph(O, 0.15, 0.2)
    r = O.linear_rates(1.9)
    rng = np.random.default_rng(1)
    f1, f2 = rng.normal(0, 0.1, (40, 6)), rng.normal(0, 0.1, (40, 6))
    a, b = 0.7, -1.3
    lhs = O.run(ph, r, a * f1 + b * f2, 25)
    rhs = a * O.run(ph, r, f1, 25) + b * O.run(ph, r, f2, 25)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-13)


@pytest.mark.parametrize("u0,s0", [(0.0, 0.0), (0.15, 0.2)])
@pytest.mark.parametrize("s_e", [1.9, 1.5, 1.2])
def test_linear_variant_stable_at_the_papers_parameter_sets(O, u0, s0, s_e):
    """Section 7 reports stability at s_e = 1.9, c0 = lambda/2, gamma = 1.4, Pr = 1 with
    (u0, s0) = (0, 0) and (0.15 lambda, 0.2 c_p): the spectral radius over all wavenumbers is <= 1."""
    ph = _ph(O, u0, s0)
    B = L.jacobian_blocks(ph, O.linear_rates(s_e), 1.0, u0, s0)
    rad = max(np.abs(np.linalg.eigvals(L.symbol(B, t))).max() for t in np.linspace(0, np.pi, 361))
    assert rad <= 1.0 + 1e-12


@pytest.mark.parametrize("u0,s0", [(0.0, 0.0), (0.15, 0.2), (-0.1, 0.1)])
def test_linear_variant_phase_speeds(O, u0, s0):
    """First-order equivalent equations, eq. (edp1-d1q3q3) with the Lambda tensor of
    eq. (Lambda-d1q3q3): the conserved modes travel at the eigenvalues of
    [[0, 1, 0], [2 lambda^2/3 + a/3, b/3, c/3], [p, q, r]] where (a, b, c) and (p, q, r) are the printed
    coefficients of e_eq and psi_eq on (rho, J, zeta); at u0 = s0 = 0 these are +-c0 and 0."""
    ph = _ph(O, u0, s0)
    c02 = 1.4 * ph.p0 / ph.rho0
    a = 3 * (1 - s0) * c02 - 3 * u0 ** 2 - 2
    A = np.array([[0, 1, 0], [2 / 3 + a / 3, 6 * u0 / 3, 3 * u0 ** 2 / 3], [-u0 * s0, s0, u0]])
    expect = np.sort(np.linalg.eigvals(A).real)
    if u0 == 0 and s0 == 0:
        np.testing.assert_allclose(expect, [-np.sqrt(c02), 0, np.sqrt(c02)], atol=1e-15)
    B = L.jacobian_blocks(ph, O.linear_rates(1.2), 1.0, u0, s0)
    th = 1e-3
    speeds = np.sort(-ph.lam * np.angle(L.conserved_modes(L.symbol(B, th))) / th)
    np.testing.assert_allclose(speeds, expect, atol=2e-5)


def test_linear_variant_symbol_at_zero(O):
    ph = _ph(O, 0.15, 0.2)
    r = O.linear_rates(1.9)
    B = L.jacobian_blocks(ph, r, 1.0, 0.15, 0.2)
    w = np.sort(np.linalg.eigvals(L.symbol(B, 0.0)).real)
    np.testing.assert_allclose(w, np.sort(np.r_[1.0, 1.0, 1.0, 1.0 - r]), atol=1e-12)


def test_linear_variant_requires_lattice_units(O):
    with pytest.raises(ValueError):
        ph = O.default_phys(eq_mode=1, lam=2.0)
        O.run(ph, O.linear_rates(1.5), np.zeros((8, 6)), 1)


def _printed_Q(u0, s0, c02, g=1.4):
    """Coefficients of eq. (equilibres-NS-linearise) on (rho, J, zeta) (lambda = c_p = 1)."""
    return np.array([
        [3 * (1 - s0) * c02 - 3 * u0 ** 2 - 2, 6 * u0, 3 * u0 ** 2],
        [-u0 * s0, s0, u0],
        [-3 * (s0 * s0 * c02) - 6 * s0 * u0 ** 2 + 3 * s0 * c02 + 2 - 2 * s0 - 2 / g, 6 * u0 * s0,
         3 * (u0 ** 2 + s0 * c02)]])


@pytest.mark.parametrize("u0,s0", [(0.0, 0.0), (0.15, 0.2), (0.1, -0.3), (-0.05, 0.4)])
def test_linear_variant_second_order_damping(O, u0, s0):
    """Second-order equivalent equations of a linear scheme, eq. (edp-ordre-2) with the defects of
    eq. (thetas): with m_eq = Q W on the non-conserved moments, A = Lam_WW + Lam_WN Q and
    D = dt Lam_WN diag(sigma) (Lam_NW + Lam_NN Q - Q A); a conserved mode (right/left eigenvectors
    r, l of A) decays at l D r / (l r). Lambda is the printed eq. (Lambda-d1q3q3) (tests/golden),
    Q the printed linear equilibria; the decay rates are compared with the oracle's exact Jacobian."""
    from conftest import read_symbolic_matrix

    ph = _ph(O, u0, s0)
    r = O.linear_rates(1.5)
    c02 = 1.4 * ph.p0 / ph.rho0
    Lam = read_symbolic_matrix("Lambda_d1q3q3.txt", l=1.0)   # order (rho, J, zeta, e, psi, eps)
    W, Nn = [0, 1, 2], [3, 4, 5]
    Q = _printed_Q(u0, s0, c02)
    A = Lam[np.ix_(W, W)] + Lam[np.ix_(W, Nn)] @ Q
    sig = np.diag(1 / r - 0.5)
    D = 1.0 * Lam[np.ix_(W, Nn)] @ sig @ (Lam[np.ix_(Nn, W)] + Lam[np.ix_(Nn, Nn)] @ Q - Q @ A)
    w, Rv = np.linalg.eig(A)
    Lv = np.linalg.inv(Rv)
    pred = {}
    for i in range(3):
        pred[np.real(w[i])] = np.real(Lv[i] @ D @ Rv[:, i])
    B = L.jacobian_blocks(ph, r, 1.0, u0, s0)
    th = 2e-3
    mu = L.conserved_modes(L.symbol(B, th))
    speeds = -np.angle(mu) / th
    damps = -np.log(np.abs(mu)) / th ** 2
    for sp, dm in zip(speeds, damps):
        key = min(pred, key=lambda v: abs(v - sp))
        assert abs(key - sp) < 1e-4
        assert abs(dm - pred[key]) <= 1e-3 * abs(pred[key]) + 1e-6, (sp, dm, pred[key])
