"""Linear stability of the nonlinear D1Q3Q3 scheme as read, pinned two ways (no GPU needed).

The amplification matrix of one time step around a uniform state (rho, u, s) is rebuilt here from the
paper alone, independently of the oracle's code:
    G(theta) = E(theta) M^{-1} C M,
with M typed from the printed eq. (M-d1q3q3) (tests/golden/M_d1q3q3.txt), E(theta) the streaming of
eq. (iteration-d1q3q3) on the Fourier mode exp(i theta j) (f+, g+ move one node to the right, so they
pick up exp(-i theta)), and C the linearised collision in moment space: (rho, J, zeta) kept, and
x* = x + s_x (x_eq - x) for x = e, psi, eps with the Jacobian of the equilibria
    e_eq = 3 (rho u^2 + p) - 2 lambda^2 rho                                  (eq. energie-equilibre)
    psi_eq = zeta u                                                          (eq. psi-equilibre)
    eps_eq = 2 lambda^2 [rho (s - s0) + (1 - 1/gamma) c_p rho log(rho/rho0)] + e_eq s
                                               (polytropic form of eq. eq-energie-entropie-d1q3q3)
with p from eq. (gaz-parfait), taken by the complex-step derivative. The entropy source is quadratic
in the gradients, so its Jacobian vanishes at a uniform state. Rates: s_psi from eq.
(lien-sigma-sigma), s_eps = 1.5 (step iii).

The restatement must agree with the oracle's exact (dual-number) Jacobian, and both show the
stability region of the scheme: stable at rest for -0.15 c_p <= s - s0 <= 0.05 c_p (densities
0.4-1.2 rho0; up to 0.1 c_p at rho <= rho0) and in slow flow, unstable once s - s0 reaches about 0.15 c_p or |u| about 0.15-0.2 lambda
(s_e-dependent), and weakly unstable below -0.17 c_p at s_e = 1.9. The ragged Riemann batch whose two
states both lie in -0.15 c_p <= s - s0 <= 0, and whose exact solution moves no faster than the stable
flow speed at its s_e, then stays stable.
"""
import numpy as np
import pytest

from conftest import read_symbolic_matrix
import _linear as L
from paper_1802_02369_gb300 import workloads as W

GAMMA, PR, CP, RHO0, LAM = 1.4, 1.0, 1.0, 1.0, 1.0
P0 = RHO0 * (LAM / 2) ** 2 / GAMMA
THETAS = np.linspace(0.0, np.pi, 91)


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def rates(s_e):
    sigma_psi = 1.5 * (GAMMA / PR) * (1.0 / s_e - 0.5)
    return np.array([s_e, 1.0 / (sigma_psi + 0.5), 1.5])


def equilibria(rho, J, zeta, s0=0.0):
    u = J / rho
    s = zeta / rho
    p = P0 * np.exp(GAMMA * np.log(rho / RHO0) + GAMMA * (s - s0) / CP)
    e_eq = 3.0 * (rho * u * u + p) - 2.0 * LAM ** 2 * rho
    psi_eq = zeta * u
    eps_eq = 2.0 * LAM ** 2 * (rho * (s - s0) + (1.0 - 1.0 / GAMMA) * CP * rho * np.log(rho / RHO0)) + e_eq * s
    return np.array([e_eq, psi_eq, eps_eq])


def symbol(rho, u, s, s_e):
    """G(theta) for every theta of THETAS, from the restatement above."""
    M = read_symbolic_matrix("M_d1q3q3.txt", l=LAM, c=CP, rho0=RHO0)
    Minv = np.linalg.inv(M)
    x0 = np.array([rho, rho * u, rho * s], dtype=complex)
    dq = np.zeros((3, 3))
    h = 1e-30
    for k in range(3):
        x = x0.copy()
        x[k] += 1j * h
        dq[:, k] = equilibria(*x).imag / h
    r = rates(s_e)
    C = np.eye(6)
    for i in range(3):
        C[3 + i, :3] = r[i] * dq[i]
        C[3 + i, 3 + i] = 1.0 - r[i]
    P = Minv @ C @ M
    out = []
    for th in THETAS:
        E = np.diag([1, np.exp(-1j * th), np.exp(1j * th), 1, np.exp(-1j * th), np.exp(1j * th)])
        out.append(E @ P)
    return out


def radius(rho, u, s, s_e):
    return max(np.abs(np.linalg.eigvals(G)).max() for G in symbol(rho, u, s, s_e))


@pytest.mark.parametrize("rho,u,s,s_e", [(1.0, 0.0, 0.0, 1.2), (1.0, 0.2, 0.0, 1.9), (0.8, -0.1, 0.2, 1.5),
                                         (1.3, 0.05, -0.3, 1.0)])
def test_restated_symbol_equals_oracle_jacobian(O, rho, u, s, s_e):
    """The paper's linearised step equals the oracle's dual-number Jacobian, entry by entry."""
    ph = O.default_phys()
    B = L.jacobian_blocks(ph, O.coupled_rates(s_e), rho, u, s)
    for th, G in zip(THETAS[::10], symbol(rho, u, s, s_e)[::10]):
        np.testing.assert_allclose(L.symbol(B, th), G, rtol=0, atol=1e-11)


@pytest.mark.parametrize("s_e", [1.0, 1.2, 1.5, 1.9])
def test_stability_region(O, s_e):
    """Stable (spectral radius <= 1) at rest for s in [-0.15, 0.05] c_p and densities 0.4-1.2 rho0 (up
    to 0.1 c_p at rho <= rho0; at rho = 1.2 rho0, s = 0.1 c_p the radius is 1.07), and in flow
    |u| <= 0.05 lambda; unstable at rest for s = 0.2 c_p (radius > 1.2) and in flow at
    |u| = 0.2 lambda (radius > 1.03). The radius at the extreme points is confirmed on the oracle's own
    Jacobian."""
    for rho in (0.4, 0.7, 1.0, 1.2):
        for s in (-0.15, -0.1, 0.0, 0.05) + ((0.1,) if rho <= 1.0 else ()):
            assert radius(rho, 0.0, s, s_e) <= 1.0 + 1e-12, (rho, s)
    assert radius(1.2, 0.0, 0.1, s_e) > 1.05
    for u in (-0.05, 0.02, 0.05):
        assert radius(1.0, u, 0.0, s_e) <= 1.0 + 1e-12, u
    assert radius(1.0, 0.0, 0.2, s_e) > 1.2
    assert radius(1.0, 0.2, 0.0, s_e) > 1.03
    assert radius(1.0, -0.2, 0.0, s_e) > 1.03
    ph = O.default_phys()
    for (u, s), bound in (((0.0, 0.2), 1.2), ((0.2, 0.0), 1.03)):
        B = L.jacobian_blocks(ph, O.coupled_rates(s_e), 1.0, u, s)
        rad = max(np.abs(np.linalg.eigvals(L.symbol(B, t))).max() for t in THETAS)
        assert rad > bound


def test_unstable_from_entropy_above_point_one_five(O):
    """The threshold in s at rest lies between 0.1 and 0.15 c_p for every s_e in [1, 1.9], and the
    steepening-wave amplitude 0.2 (|u| up to 0.2 lambda) is unstable for every s_e of that range,
    while amplitude 0.1 (|u| <= 0.1, the steepening wave of the benchmark) is stable for s_e <= 1.2
    (weakly unstable at s_e = 1.5: radius 1 + 2e-4 at rho = 1.1, u = 0.1). Below the band, at s_e = 1.9, the
    scheme turns weakly unstable (radius 1 + 4e-5 at s = -0.2 c_p, 1 + 5e-4 at rho = 1.2 rho0 and
    s = -0.17 c_p)."""
    for s_e in (1.0, 1.3, 1.6, 1.9):
        assert radius(1.0, 0.0, 0.10, s_e) <= 1.0 + 1e-12
        assert radius(1.0, 0.0, 0.15, s_e) > 1.05
        assert radius(1.0, 0.2, 0.0, s_e) > 1.03
    for s_e in (1.0, 1.2):
        for rho, u in ((1.1, 0.1), (0.9, -0.1), (1.0, 0.1)):
            s = 0.0   # the wave is adiabatic at s = s0 = 0
            assert radius(rho, u, s, s_e) <= 1.0 + 1e-12, (s_e, rho, u)
    assert 1.0 + 1e-5 < radius(1.1, 0.1, 0.0, 1.5) < 1.0 + 1e-3
    assert 1.0 + 1e-5 < radius(1.0, 0.0, -0.2, 1.9) < 1.0 + 1e-4
    assert radius(1.2, 0.0, -0.17, 1.9) > 1.0 + 1e-4


@pytest.mark.parametrize("i", range(len(W.STABLE_FLOW_SPEED)))
def test_stable_flow_speed_table(O, i):
    """The table of flow speeds the Riemann-data selection uses (W.STABLE_FLOW_SPEED) is the stability
    limit of the linearised step at the reference state (rho0, u, s0): radius <= 1 at the tabulated
    speed and > 1 beyond it by 0.002 lambda (the table is the limit rounded down to 0.001), on the restated symbol and on the oracle's Jacobian."""
    s_e, u = W.STABLE_FLOW_SPEED_S_E[i], W.STABLE_FLOW_SPEED[i]
    assert radius(1.0, u, 0.0, s_e) <= 1.0 + 1e-12
    assert radius(1.0, u + 0.002, 0.0, s_e) > 1.0 + 1e-9
    ph = O.default_phys()
    for uu, stable in ((u, True), (u + 0.002, False)):
        B = L.jacobian_blocks(ph, O.coupled_rates(s_e), 1.0, uu, 0.0)
        rad = max(np.abs(np.linalg.eigvals(L.symbol(B, t))).max() for t in THETAS)
        assert (rad <= 1.0 + 1e-12) == stable, (s_e, uu, rad)


def test_entropy_filtered_riemann_draws_stay_stable(O):
    """Riemann data drawn like the ragged batch but kept only when both states lie in the stable
    entropy band -0.15 c_p <= s - s0 <= 0 and the exact Riemann solution moves no faster than the
    stable flow speed of the lattice's s_e (W.ragged_batch(..., entropy_range=(-0.15, 0.0),
    stable_flow=True)): a seeded sample of such lattices (lengths capped for the oracle) runs 2000
    steps with no diagnostic flag."""
    ph = O.default_phys()
    bat = W.ragged_batch(10, 1802, ph.p0, n_min=512, n_max=1024, entropy_range=(-0.15, 0.0), stable_flow=True)
    sl = W.entropy_of_state(bat.states[:, 0], bat.states[:, 1])
    sr = W.entropy_of_state(bat.states[:, 2], bat.states[:, 3])
    assert np.all((sl >= -0.15) & (sl <= 0) & (sr >= -0.15) & (sr <= 0))
    _, us = W.riemann_star(bat.states[:, 0], bat.states[:, 1] * ph.p0, bat.states[:, 2], bat.states[:, 3] * ph.p0)
    assert np.all(np.abs(us) <= np.interp(bat.s_e, W.STABLE_FLOW_SPEED_S_E, W.STABLE_FLOW_SPEED))
    for b in range(bat.lengths.size):
        phb = O.default_phys(bc=int(bat.bc[b]))
        r, u, p = bat.lattice(b)
        fd = O.run(phb, O.coupled_rates(bat.s_e[b]), O.init(phb, r, u, p=p), 2000)
        assert O.diagnostics(phb, fd)[1] == 0, b
