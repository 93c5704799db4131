"""Pins of the finite-difference comparison solver's oracle (section 9): what the Navier-Stokes
system of eq. (NS-rho-J-zeta) and the stated discretisation fix, checked without calling the
oracle's own formulas again.

- Conservation form: the sums of rho and J are exactly conserved on a periodic grid; the sum of
  zeta is conserved without the source and grows by dt times the (non-negative) production with it.
- Uniform states are fixed points; the scheme commutes with the mirror x -> -x, u -> -u.
- Linear theory: a small-amplitude Fourier mode evolves by the amplification matrix I + dt A(k) of
  the linearised system, with A derived here from the equations (EOS derivatives from
  eq. (gaz-parfait)) and the centred stencils' symbols; at small k h its acoustic eigenvalues tend to
  the classical sound attenuation (nu + (gamma - 1) kappa / (rho c_p)) / 2.
- Energy: the continuous system conserves the total energy p/(gamma - 1) + rho u^2/2 because the
  entropy production returns the dissipated kinetic energy as heat; dropping the source loses it.
"""
import numpy as np
import pytest

import oracle.fd as F


def _wave(N, delta, c0=0.5):
    x = 2 * np.pi * np.arange(N) / N
    return 1 + delta * np.sin(x), c0 * delta * np.sin(x), np.zeros(N)


def _random_state(N, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    k = np.arange(1, 5)
    x = 2 * np.pi * np.arange(N) / N
    def f(a):
        c = rng.normal(size=(2, k.size)) * a / k
        return (c[0][:, None] * np.sin(k[:, None] * x) + c[1][:, None] * np.cos(k[:, None] * x)).sum(0)
    return 1 + f(amp), f(amp * 0.5), f(amp * 0.5)


def test_conservation_sums():
    ph = F.default_phys(0.08)
    rho, u, s = _random_state(96, 1)
    W = F.init(ph, rho, u, s)
    s0, _ = F.diagnostics(ph, W)
    prev = s0
    for _ in range(20):
        W = F.run(ph, W, 0.05, 50)
        sm, fl = F.diagnostics(ph, W)
        assert fl == 0
        assert abs(sm[0] - s0[0]) <= 1e-13 * abs(s0[0])
        assert abs(sm[1] - s0[1]) <= 1e-13 * np.abs(W[:, 1]).sum()
        assert sm[2] >= prev[2] - 1e-14 * np.abs(W[:, 2]).sum()   # production is non-negative
        prev = sm
    assert prev[2] > s0[2]
    # Without the source the entropy sum is conserved as well.
    ph0 = F.default_phys(0.08, source_on=0)
    W = F.run(ph0, F.init(ph0, rho, u, s), 0.05, 1000)
    sm, _ = F.diagnostics(ph0, W)
    assert abs(sm[2] - s0[2]) <= 1e-13 * np.abs(W[:, 2]).sum()


def test_uniform_state_fixed_and_mirror_symmetry():
    ph = F.default_phys(0.05)
    N = 40
    W = F.init(ph, np.full(N, 1.3), np.full(N, 0.07), np.full(N, 0.2))
    W2 = F.run(ph, W, 0.1, 200)
    assert np.abs(W2 - W).max() <= 1e-14
    rho, u, s = _random_state(N, 2)
    A = F.run(ph, F.init(ph, rho, u, s), 0.05, 300)
    B = F.run(ph, F.init(ph, np.roll(rho[::-1], 1), -np.roll(u[::-1], 1), np.roll(s[::-1], 1)), 0.05, 300)
    Bm = np.roll(B[::-1], 1, axis=0)
    assert np.abs(Bm[:, 0] - A[:, 0]).max() <= 1e-13
    assert np.abs(-Bm[:, 1] - A[:, 1]).max() <= 1e-13
    assert np.abs(Bm[:, 2] - A[:, 2]).max() <= 1e-13


def _linear_matrix(ph, k, h, rho0=1.0):
    """A(k) of the linearised discrete system about (rho0, u = 0, s = s0 = 0) in the conserved
    variables (rho', J', zeta'): centred first difference i sin(kh)/h, face-averaged second
    difference -4 sin^2(kh/2)/h^2 (coefficients are constant in the linear limit)."""
    D1 = 1j * np.sin(k * h) / h
    D2 = -4 * np.sin(k * h / 2) ** 2 / h ** 2
    g, cp, p0 = ph.gamma, ph.cp, ph.p0
    c2 = g * p0 / rho0                      # (dp/drho)_s
    dp_dzeta = g * p0 / (cp * rho0)         # (dp/ds)_rho / rho0
    kappa = rho0 * ph.nu * cp / ph.Pr
    # T' / T0 = p'/p0 - rho'/rho0; the entropy flux (kappa/T) d_x T linearises to kappa d_x (T'/T0).
    return np.array([[0, -D1, 0],
                     [-c2 * D1, ph.nu * D2, -dp_dzeta * D1],
                     [kappa * D2 * (c2 / p0 - 1 / rho0), 0, kappa * D2 * dp_dzeta / p0]], dtype=complex)


@pytest.mark.parametrize("kmode,Pr", [(1, 1.0), (3, 1.0), (2, 0.7)])
def test_small_amplitude_mode_follows_linear_theory(kmode, Pr):
    ph = F.default_phys(0.06, Pr=Pr)
    N, h, dt, n = 48, 1.0, 0.02, 2000
    k = 2 * np.pi * kmode / N
    x = np.arange(N) * h
    v = np.array([1.0 + 0.3j, 0.4 - 0.2j, -0.5 + 0.7j])
    delta = 1e-7
    mode = np.exp(1j * k * x)
    Wd = delta * np.real(v[:, None] * mode[None, :]).T          # [N, 3] deviations
    W0 = Wd + np.array([1.0, 0.0, 0.0])
    W = F.run(ph, W0, dt, n)
    got = np.fft.fft(W - np.array([1.0, 0.0, 0.0]), axis=0)[kmode] / (N / 2) / delta
    G = np.eye(3) + dt * _linear_matrix(ph, k, h)
    want = np.linalg.matrix_power(G, n) @ v
    assert np.abs(got - want).max() <= 2e-5 * np.abs(want).max(), (got, want)
    # The mode really moved and decayed (the test is not vacuous).
    assert np.abs(want - v).max() > 0.1


def test_linear_acoustic_attenuation_tends_to_classical():
    """Small k h, small dt: the acoustic eigenvalues of A(k) give damping k^2 (nu + (gamma-1) nu/Pr)/2
    and phase speed c0 (textbook sound attenuation for a viscous, heat-conducting gas)."""
    for Pr in (1.0, 0.71):
        ph = F.default_phys(0.01, Pr=Pr)
        k, h = 1e-3, 1.0
        ev = np.linalg.eigvals(_linear_matrix(ph, k, h))
        ac = ev[np.argsort(-np.abs(ev.imag))[:2]]
        c0 = np.sqrt(ph.gamma * ph.p0)
        gamma_classical = 0.5 * (ph.nu + (ph.gamma - 1) * ph.nu / Pr)
        for lam in ac:
            assert abs(abs(lam.imag) / k - c0) <= 1e-6 * c0
            assert abs(-lam.real / k ** 2 - gamma_classical) <= 1e-4 * gamma_classical


def test_energy_returned_by_entropy_production():
    """Paper-shaped strong wave (delta rho = 0.1 rho0, c0 = lambda/2), nu = 0.02 on N = 128 up to
    t = 200: with the source the total energy drifts far less than without it, where the dissipated
    kinetic energy is lost; what drift remains comes mostly from the explicit Euler step (it shrinks
    when dt is halved). The entropy grows only with the source."""
    N, t_end = 128, 200.0
    rho, u, s = _wave(N, 0.1)
    ratio = {}
    for dt in (0.01, 0.005):
        n = int(round(t_end / dt))
        res = {}
        for src in (1, 0):
            ph = F.default_phys(0.02, source_on=src)
            _, res[src] = F.series(ph, F.init(ph, rho, u, s), dt, n, n // 10)
        e_on = np.abs(res[1][:, 3] - res[1][0, 3]).max() / res[1][0, 3]
        e_off = np.abs(res[0][:, 3] - res[0][0, 3]).max() / res[0][0, 3]
        assert e_off > 1e-5                       # kinetic energy is dissipated
        ratio[dt] = e_on / e_off
        assert np.all(np.diff(res[1][:, 2]) > 0)
        assert np.abs(res[0][:, 2] - res[0][0, 2]).max() <= 1e-13 * N
    assert ratio[0.005] <= 0.03, ratio
    assert ratio[0.01] / ratio[0.005] >= 1.6, ratio    # shrinks with the time step


def test_invalid_arguments_rejected():
    ph = F.default_phys(0.01)
    W = F.init(ph, np.ones(8), np.zeros(8), np.zeros(8))
    with pytest.raises(ValueError):
        F.run(ph, W, -0.1, 1)
    with pytest.raises(ValueError):
        F.run(ph, W[:2], 0.1, 1)
    with pytest.raises(ValueError):
        F.series(ph, W, 0.1, 10, 3)
