"""Pins of the three-dimensional D3Q19-D3Q7 oracle against what the paper and the mathematics fix.

The paper's conclusion names the three-dimensional extension without specifying it, so the pins check
the readings through properties that do not depend on retyping them: exact reduction to the pinned
one-dimensional D1Q3Q3 oracle along each axis, textbook special cases, linear stability, decay rates
from the second-order analysis of section 8 carried to three dimensions, lattice symmetries and
conservation."""
import numpy as np
import pytest

import oracle as O1
import oracle.d3q19q7 as D

NT = 8  # oracle threads


def smooth_1d(N, seed):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(N) / N
    rho = 1.0 + 0.08 * np.sin(x + rng.uniform(0, 6)) + 0.03 * np.sin(2 * x + rng.uniform(0, 6))
    u = 0.08 * np.sin(x + rng.uniform(0, 6)) + 0.02 * np.cos(3 * x)
    s = 0.03 * np.cos(x + rng.uniform(0, 6))
    return rho, u, s


def smooth_3d(Nz, Ny, Nx, seed, amp=0.04):
    rng = np.random.default_rng(seed)
    zz, yy, xx = np.mgrid[0:Nz, 0:Ny, 0:Nx]
    X, Y, Z = 2 * np.pi * xx / Nx, 2 * np.pi * yy / Ny, 2 * np.pi * zz / Nz
    f = lambda: amp * (np.sin(X + rng.uniform(0, 6)) * np.cos(Y + rng.uniform(0, 6)) * np.cos(Z + rng.uniform(0, 6))
                       + 0.5 * np.sin(2 * Z + X + rng.uniform(0, 6)) + 0.3 * np.cos(Y - Z + rng.uniform(0, 6)))
    return 1.0 + f(), f(), f(), f(), 0.5 * f()


PHYS_CASES = [dict(), dict(gamma=1.3, Pr=0.71, cp=2.5, rho0=1.3, lam=2.0, s0=-0.1)]


def _reduce(line, C):
    """Sums of the 3-D populations of one node row over the velocities with the same component C."""
    idx = np.arange(26)
    return np.stack([line[:, (C == a) & (idx < 19)].sum(1) for a in (0, 1, -1)] +
                    [line[:, (C == a) & (idx >= 19)].sum(1) for a in (0, 1, -1)], axis=1)


@pytest.mark.parametrize("kw", PHYS_CASES)
def test_reduces_to_d1q3q3_on_one_dimensional_data(kw):
    """With the coupling of eq. (lien-sigma-sigma) (beta = 3/2), data that depend on one coordinate only,
    with the velocity along it, evolve exactly as the D1Q3Q3 scheme of sections 6 and 8 along that
    axis: the sums of the 3-D populations over the other two velocity components are the 1-D
    populations, source included; the transverse momenta stay zero and all rows stay equal."""
    ph1 = O1.default_phys(**kw)
    ph3 = D.default_phys(beta=1.5, **kw)
    N, steps, s_e = 40, 30, 1.25
    rho, u, s = smooth_1d(N, 5)
    u = u * ph1.lam
    s = s * ph1.cp + ph1.s0
    ref = O1.run(ph1, O1.coupled_rates(s_e, ph1.gamma, ph1.Pr), O1.init(ph1, rho, u, s=s), steps)
    rt = D.rates(s_e, ph1.gamma, ph1.Pr, beta=1.5, s_eps=1.5)  # the rate of eps of sections 4 and 8
    scale = max(1.0, np.abs(ref).max())
    for axis in range(3):
        shape = [3, 3, 3]
        shape[2 - axis] = N
        F = lambda a: np.broadcast_to(a.reshape([N if i == 2 - axis else 1 for i in range(3)]), shape).copy()
        vel = [F(0 * u), F(0 * u), F(0 * u)]
        vel[axis] = F(u)
        got = D.run(ph3, rt, D.init(ph3, F(rho), *vel, F(s)), steps, NT)
        line = np.moveaxis(got, 2 - axis, 0)
        assert np.abs(_reduce(line[:, 0, 0], (D.CX, D.CY, D.CZ)[axis]) - ref).max() <= 1e-13 * scale, axis
        assert np.array_equal(line[:, 0, 0], line[:, 1, 2]) and np.array_equal(line[:, 0, 0], line[:, 2, 1])
        m = D.moments(ph3, got)
        for b in range(3):
            if b != axis:
                assert np.abs(m[..., 1 + b]).max() <= 1e-13 * ph3.rho0 * ph3.lam  # rounding of M^-1 only


def test_isothermal_lattice_rest_state_has_the_textbook_weights():
    """At rest with p0 = rho0 lambda^2 / 3 (lattice temperature lambda^2/3) the D3Q19 equilibrium is the
    textbook one, weights 1/3, 1/18, 1/36 times rho; the D3Q7 rest state holds (1 - 3 a) zeta at rest
    and a zeta / 2 on each moving velocity, a the second moment per direction (a = p0 / rho0 at
    T = T0, where the log T term vanishes)."""
    z = np.zeros((3, 3, 3))
    for rho0 in (1.0, 1.2):  # populations are scaled by rho0 as in eq. (M-d1q3q3)
        ph = D.default_phys(rho0=rho0, p0=rho0 / 3.0)
        fd = D.init(ph, z + rho0, z, z, z, z)[1, 1, 1]
        w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
        assert np.abs(fd[:19] - w).max() <= 1e-15
    ph = D.default_phys(p0=0.25, s0=0.2)
    g = D.init(ph, z + 1.0, z, z, z, z + 0.2)[1, 1, 1][19:]
    a = 0.25
    assert abs(g[0] - 0.2 * (1 - 3 * a)) <= 1e-15 and np.abs(g[1:] - 0.2 * a / 2).max() <= 1e-15


def _jacobian(ph, rt, ux=0.0, uy=0.0, uz=0.0, s=0.0, eps=1e-7):
    """The collision Jacobian about a uniform state in uniform motion (streaming it is the identity)."""
    z = np.zeros((3, 3, 3))
    f0 = D.init(ph, z + ph.rho0, z + ux, z + uy, z + uz, z + s)
    base = D.run(ph, rt, f0, 1)[1, 1, 1]
    J = np.zeros((26, 26))
    for j in range(26):
        f = f0.copy()
        f[..., j] += eps
        J[:, j] = (D.run(ph, rt, f, 1)[1, 1, 1] - base) / eps
    return J


# Directions of the von Neumann scan: the axes, face and body diagonals and three generic directions
# (the symbol at -k is the conjugate of the one at k, so half the sphere suffices).
DIRS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (0, 1, 1), (1, 0, -1), (1, 1, 1), (1, -1, 1),
        (1, 2, 0), (1, 2, 3), (-2, 1, 1), (0.3, 0.7, 1)]


def _max_growth(J, nk=24):
    worst = 0.0
    for d in DIRS:
        d = np.asarray(d, float) / np.linalg.norm(d)
        for k in np.linspace(0.05, np.pi * np.sqrt(3), nk):
            ph_ = np.exp(-1j * k * (d[0] * D.CX + d[1] * D.CY + d[2] * D.CZ))
            worst = max(worst, np.abs(np.linalg.eigvals(ph_[:, None] * J)).max())
    return worst


def test_closure_of_section_8_is_unstable_on_d3q7_and_beta_9_is_stable():
    """Linear stability at rest (von Neumann symbol from the oracle's own collision Jacobian): with the
    1-D closure (beta = 3/2) the D3Q7 entropy block grows by more than 4 per step at the (pi, pi, pi)
    mode; with beta = 9 no mode grows, for s_e from 1 to 1.5 (the default rates)."""
    ph = D.default_phys(source_on=0, beta=1.5)
    J = _jacobian(ph, D.rates(1.2, beta=1.5))
    ph_ = np.exp(-1j * np.pi * (D.CX + D.CY + D.CZ))
    assert np.abs(np.linalg.eigvals((ph_[:, None] * J)[19:, 19:])).max() > 4.0  # the entropy block
    for s_e in (1.0, 1.2, 1.5):
        ph = D.default_phys(source_on=0)
        assert _max_growth(_jacobian(ph, D.rates(s_e))) <= 1.0 + 1e-6, s_e


def test_stability_region_in_flow_and_entropy():
    """Linear stability about uniform states with the default rates (beta = 9, s_q = 1.5, s_h = 1.2,
    s_eps = 1): stable in flow up to |u| = 0.15 lambda along an axis, a face diagonal and the body
    diagonal (s_e = 1.2 and 1.5); at rest for s - s0 from -0.2 to 0.05 c_p at s_e = 1.2 and at 0.1 c_p
    at s_e = 1.5. Growing, at the (pi, pi, pi) mode, for s - s0 = 0.1 c_p at s_e = 1.2, at rest for
    s_e = 1.9, and for s - s0 = 0.05 c_p when the fourth-order and entropy moments relax at 1.5."""
    ph = D.default_phys(source_on=0)
    for s_e in (1.2, 1.5):
        rt = D.rates(s_e)
        for u in ((0.15, 0, 0), (0, 0.15 / np.sqrt(2), 0.15 / np.sqrt(2)), (0.15 / np.sqrt(3),) * 3):
            assert _max_growth(_jacobian(ph, rt, *u), nk=12) <= 1.0 + 1e-6, (s_e, u)
    for s_e, s in ((1.2, -0.2), (1.2, 0.05), (1.5, 0.1)):
        assert _max_growth(_jacobian(ph, D.rates(s_e), s=s), nk=12) <= 1.0 + 1e-6, (s_e, s)
    pi3 = np.exp(-1j * np.pi * (D.CX + D.CY + D.CZ))
    growth = lambda J: np.abs(np.linalg.eigvals(pi3[:, None] * J)).max()
    assert growth(_jacobian(ph, D.rates(1.2), s=0.1)) > 1.1
    assert growth(_jacobian(ph, D.rates(1.9))) > 1.02
    assert growth(_jacobian(ph, D.rates(1.2, s_h=1.5, s_eps=1.5), s=0.05)) > 1.04


def test_transverse_wave_is_carried_by_the_mean_flow():
    """Galilean check of the nonlinear momentum flux rho u_a u_b: a transverse wave u_z = A sin(k x) in a
    uniform flow u_x = U translates at U (10 nodes in 200 steps at U = 0.05) to within 1 %."""
    ph, rt = D.default_phys(), D.rates(1.2)
    N, U, A, T = 64, 0.05, 1e-4, 200
    k = 2 * np.pi / N
    xx = np.arange(N)[None, None, :] * np.ones((3, 3, 1))
    one = np.ones((3, 3, N))
    f = D.init(ph, one, U * one, 0 * one, A * np.sin(k * xx), 0 * one)
    phase = lambda f: np.angle(np.sum(D.moments(ph, f)[0, 0, :, 3] * np.exp(-1j * k * np.arange(N))))
    d = phase(D.run(ph, rt, f, T, NT)) - phase(f)
    shift = -((d + np.pi) % (2 * np.pi) - np.pi) / k
    assert abs(shift - U * T) <= 0.01 * U * T


def _one_step_production(ph, G, g_s, n=7):
    """zeta after one step with the source minus without it, at the centre node, for the linear fields
    u = G x and s = g_s . x (centred differences are exact on linear fields)."""
    c = n // 2
    zz, yy, xx = np.mgrid[0:n, 0:n, 0:n].astype(float)
    X = np.stack([xx - c, yy - c, zz - c])
    u = np.einsum("ab,b...->a...", G, X)
    s = np.einsum("b,b...->...", np.asarray(g_s, float), X)
    rho = np.ones((n, n, n)) * ph.rho0
    off = D.default_phys(source_on=0)
    rt = D.rates(1.2)
    fd = D.init(ph, rho, u[0], u[1], u[2], s)
    return D.moments(ph, D.run(ph, rt, fd, 1))[c, c, c, 4] - D.moments(off, D.run(off, rt, fd, 1))[c, c, c, 4]


def _rotation(axis, th):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


def test_entropy_production_is_rotation_invariant_and_has_the_shear_to_dilatation_ratio():
    """The production rho nu (2 D:D + (div u)^2) / (3 T) + kappa |grad T|^2 / T^2 depends on the velocity
    gradient only through rotation invariants: rotating a uniform gradient (not by a lattice symmetry)
    leaves it unchanged; the thermal part alone is invariant too; a pure shear d_y u_x = g gives
    2 D:D + (div u)^2 = g^2 and a dilatation d_z u_z = g gives 3 g^2."""
    ph = D.default_phys()
    R = _rotation((0.3, -0.5, 0.8), 0.7)
    G = 0.004 * np.array([[0.3, -0.7, 0.1], [0.2, 0.5, -0.4], [0.6, 0.0, -0.2]])
    a, b = _one_step_production(ph, G, (0, 0, 0)), _one_step_production(ph, R @ G @ R.T, (0, 0, 0))
    assert a > 0 and abs(a - b) <= 1e-10 * a
    gs = 2e-3 * np.array([0.6, -0.3, 0.4])
    a, b = _one_step_production(ph, 0 * G, gs), _one_step_production(ph, 0 * G, R @ gs)
    assert a > 0 and abs(a - b) <= 1e-3 * a  # T is not exactly linear in s: centred differences of T
    shear = _one_step_production(ph, 0.004 * np.array([[0, 1.0, 0], [0, 0, 0], [0, 0, 0]]), (0, 0, 0))
    dil = _one_step_production(ph, 0.004 * np.array([[0, 0, 0], [0, 0, 0], [0, 0, 1.0]]), (0, 0, 0))
    assert abs(shear / dil - 1.0 / 3.0) <= 1e-6  # (2 * 1/2) / (2 + 1)
    # The viscous part at the default state: rho nu g^2 / (3 T) with T = T0, dt = dx / lambda.
    nu = (1.0 / 1.2 - 0.5) * ph.lam * ph.dx
    T0 = ph.p0 / (ph.rho0 * ph.cp * (1 - 1 / ph.gamma))
    assert abs(shear / (ph.dx / ph.lam * ph.rho0 * nu * 0.004 ** 2 / (3 * T0)) - 1) <= 1e-9


def _velocity_permutation(perm_axes):
    """Population index j of the velocity whose components are those of velocity i permuted by
    perm_axes (component a of the image is component perm_axes[a] of c_i), within each block."""
    C = np.stack([D.CX, D.CY, D.CZ], 1)
    out = np.empty(26, dtype=int)
    for i in range(26):
        img = C[i][list(perm_axes)]
        block = range(19) if i < 19 else range(19, 26)
        out[i] = [j for j in block if np.array_equal(C[j], img)][0]
    return out


def test_axis_permutation_covariance():
    """Swapping x and y, and the cyclic permutation (x, y, z) -> (y, z, x), are symmetries of both
    lattices: they commute with the step, population by population."""
    ph, rt = D.default_phys(), D.rates(1.2)
    rho, ux, uy, uz, s = smooth_3d(6, 8, 10, 3)
    a = D.run(ph, rt, D.init(ph, rho, ux, uy, uz, s), 10, NT)
    # Swap x <-> y: arrays [z, y, x] -> [z, x, y]; new u = (uy, ux, uz).
    T = lambda f: f.transpose(0, 2, 1)
    b = D.run(ph, rt, D.init(ph, T(rho), T(uy), T(ux), T(uz), T(s)), 10, NT)
    j = _velocity_permutation((1, 0, 2))
    assert np.abs(b.transpose(0, 2, 1, 3)[..., j] - a).max() <= 1e-13
    # Cyclic: new coordinates (x', y', z') = (y, z, x); new u' = (uy, uz, ux); arrays [z', y', x'] = [x, z, y].
    C = lambda f: f.transpose(2, 0, 1)
    b = D.run(ph, rt, D.init(ph, C(rho), C(uy), C(uz), C(ux), C(s)), 10, NT)
    j = _velocity_permutation((1, 2, 0))
    assert np.abs(b.transpose(1, 2, 0, 3)[..., j] - a).max() <= 1e-13


def test_conservation_and_uniform_state():
    """Mass and momentum are conserved exactly (periodic lattice); without the source so is sum zeta,
    with it sum zeta grows; a uniform state in uniform motion is a fixed point of the collision and
    is only translated."""
    ph, rt = D.default_phys(), D.rates(1.2)
    off = D.default_phys(source_on=0)
    rho, ux, uy, uz, s = smooth_3d(6, 7, 8, 7, amp=0.06)
    f0 = D.init(ph, rho, ux, uy, uz, s)
    m0 = D.moments(ph, f0).sum((0, 1, 2))
    m1 = D.moments(ph, D.run(ph, rt, f0, 20, NT)).sum((0, 1, 2))
    m2 = D.moments(off, D.run(off, rt, f0, 20, NT)).sum((0, 1, 2))
    assert np.abs(m1[:4] - m0[:4]).max() <= 1e-12 * np.abs(m0[0])
    assert abs(m2[4] - m0[4]) <= 1e-12 * np.abs(m0[0]) and m1[4] > m0[4] + 1e-9
    one = np.ones((3, 4, 5))
    f = D.init(ph, 1.1 * one, 0.05 * one, -0.03 * one, 0.02 * one, 0.02 * one)
    assert np.abs(D.run(ph, rt, f, 3) - f).max() <= 1e-14


def _sound_speed(ph, rt, shape, kvec, N, t1, t2):
    """Phase speed of a right-going isentropic acoustic wave of wave vector 2 pi kvec / N, from the phase of
    its density mode between steps t1 and t2."""
    zz, yy, xx = np.mgrid[0:shape[0], 0:shape[1], 0:shape[2]].astype(float)
    k = [2 * np.pi * a / N for a in kvec]
    kk = np.sqrt(sum(a * a for a in k))
    phase = k[0] * xx + k[1] * yy + k[2] * zz
    c0 = np.sqrt(ph.gamma * ph.p0 / ph.rho0)
    A = 1e-5
    rho = ph.rho0 * (1 + A * np.cos(phase))
    un = c0 * A * np.cos(phase)
    f = D.init(ph, rho, *(un * a / kk for a in k), np.zeros_like(rho) + ph.s0)
    a = D.run(ph, rt, f, t1, NT)
    b = D.run(ph, rt, a, t2 - t1, NT)
    ang = lambda f: np.angle(np.sum((D.moments(ph, f)[..., 0] - ph.rho0) * np.exp(-1j * phase)))
    d = -((ang(b) - ang(a) + np.pi) % (2 * np.pi) - np.pi)
    return d / kk / (t2 - t1), kk


def test_sound_speed_is_isotropic():
    """Acoustic waves travel at the same speed along an axis, a face diagonal and the body diagonal at
    (nearly) the same |k| (0.3 %, 1 %), and near c0 = sqrt(gamma p0 / rho0) (the scheme's own offset,
    the same in the one-dimensional oracle, is 3 % at these wavelengths and s_e = 1.2)."""
    ph, rt = D.default_phys(source_on=0), D.rates(1.2)
    c0 = np.sqrt(ph.gamma * ph.p0 / ph.rho0)
    ax, k_ax = _sound_speed(ph, rt, (3, 3, 45), (1, 0, 0), 45, 10, 30)
    fd, k_fd = _sound_speed(ph, rt, (3, 64, 64), (1, 1, 0), 64, 10, 30)
    assert abs(k_fd / k_ax - 1) < 0.01 and abs(fd / ax - 1) <= 0.003
    assert abs(ax / c0 - 1) <= 0.04
    ax, k_ax = _sound_speed(ph, rt, (3, 3, 14), (1, 0, 0), 14, 4, 8)
    bd, k_bd = _sound_speed(ph, rt, (24, 24, 24), (1, 1, 1), 24, 4, 8)
    assert abs(k_bd / k_ax - 1) < 0.015 and abs(bd / ax - 1) <= 0.01


def test_relaxation_spectrum_at_rest():
    """At a uniform state at rest the equilibria depend on the conserved moments only and the production
    vanishes, so the one-step Jacobian is block-triangular in moment space: its eigenvalues are 1 for
    the five conserved moments and 1 - s for each relaxed family, with the family's size: s_e for e and
    the five deviators (6), s_q for q and m (6), s_h for the fourth-order moments (3), s_psi (3) and s_eps
    (3). Distinct rates make every assignment of a family to its rate visible."""
    ph = D.default_phys(s0=0.05)
    rt = D.rates(1.3, s_q=1.55, s_h=1.1, s_eps=0.9)
    rt.s_psi = 0.7
    J = _jacobian(ph, rt, s=0.05)
    got = np.sort(np.linalg.eigvals(J).real)
    want = np.sort(np.array([1.0] * 5 + [1 - rt.s_e] * 6 + [1 - rt.s_q] * 6 + [1 - rt.s_h] * 3 +
                            [1 - rt.s_psi] * 3 + [1 - rt.s_eps] * 3))
    assert np.abs(np.linalg.eigvals(J).imag).max() <= 1e-6
    assert np.abs(got - want).max() <= 1e-6


def _decay_rate(ph, rt, fd, proj, t1, t2):
    a = D.run(ph, rt, fd, t1, NT)
    b = D.run(ph, rt, a, t2 - t1, NT)
    return -np.log(proj(D.moments(ph, b)) / proj(D.moments(ph, a))) / (t2 - t1)


def test_shear_waves_decay_at_nu_over_3_along_axes_and_diagonals():
    """Section 8 with theta_e ~ lambda^2 d J gives the viscous stress sigma_e dt theta; q_eq = -(2/3)
    lambda^2 J makes it isotropic in three dimensions with shear viscosity nu/3 (nu of eq. nu-d1q3q3):
    a shear wave of wave vector k decays at (nu/3)|k|^2 along an axis, a face diagonal (velocity in
    the plane and normal to it) and the body diagonal, to within the O(k^2) dispersion."""
    ph, s_e = D.default_phys(), 1.2
    rt = D.rates(s_e)
    nu = (1.0 / s_e - 0.5) * ph.lam * ph.dx
    A = 1e-5
    N = 32
    k = 2 * np.pi / N
    zz, yy, xx = np.mgrid[0:3, 0:N, 0:3].astype(float)
    one, zero = np.ones_like(xx), np.zeros_like(xx)
    w = np.sin(k * yy)
    r = _decay_rate(ph, rt, D.init(ph, one, A * w, zero, zero, zero), lambda m: np.sum(m[..., 1] * w), 50, 250)
    assert abs(r / (nu / 3 * k * k) - 1) <= 0.006
    zz, yy, xx = np.mgrid[0:3, 0:N, 0:N].astype(float)
    one, zero = np.ones_like(xx), np.zeros_like(xx)
    w = np.sin(k * (xx + yy))
    fd = D.init(ph, one, -A * w / np.sqrt(2), A * w / np.sqrt(2), zero, zero)
    r = _decay_rate(ph, rt, fd, lambda m: np.sum((m[..., 2] - m[..., 1]) * w), 50, 250)
    assert abs(r / (nu / 3 * 2 * k * k) - 1) <= 0.005
    r = _decay_rate(ph, rt, D.init(ph, one, zero, zero, A * w, zero), lambda m: np.sum(m[..., 3] * w), 50, 250)
    assert abs(r / (nu / 3 * 2 * k * k) - 1) <= 0.005
    N = 24
    k = 2 * np.pi / N
    zz, yy, xx = np.mgrid[0:N, 0:N, 0:N].astype(float)
    one, zero = np.ones_like(xx), np.zeros_like(xx)
    w = np.sin(k * (xx + yy + zz))
    fd = D.init(ph, one, A * w / np.sqrt(2), -A * w / np.sqrt(2), zero, zero)
    r = _decay_rate(ph, rt, fd, lambda m: np.sum((m[..., 1] - m[..., 2]) * w), 30, 130)
    assert abs(r / (nu / 3 * 3 * k * k) - 1) <= 0.03


@pytest.mark.parametrize("beta", [1.5, 9.0])
def test_entropy_mode_diffusivity(beta):
    """An entropy mode at rest and uniform pressure diffuses at kappa/(rho0 c_p) + sigma_psi dt p0/rho0:
    the section 8 flux kappa d log T plus the p d s term that section 8 neglects. Along z (the axis on
    which both xi rows of the D3Q7 block carry the flux), for both couplings; a long wave (N = 192)
    keeps the O(k^2) correction, which grows with sigma_psi, below the bound."""
    ph, s_e = D.default_phys(beta=beta), 1.2
    rt = D.rates(s_e, beta=beta)
    sigma_e = 1.0 / s_e - 0.5
    pred = sigma_e * ph.lam * ph.dx / ph.Pr + beta * ph.gamma / ph.Pr * sigma_e * (ph.dx / ph.lam) * ph.p0 / ph.rho0
    N, B = 192, 1e-4
    k = 2 * np.pi / N
    zz = np.mgrid[0:N, 0:3, 0:3][0].astype(float)
    s = B * np.sin(k * zz)
    rho = ph.rho0 * np.exp(-s / ph.cp)  # uniform pressure
    z = 0 * s
    r = _decay_rate(ph, rt, D.init(ph, rho, z, z, z, s), lambda m: np.sum(m[..., 4] / m[..., 0] * np.sin(k * zz)),
                    200, 800)
    assert abs(r / (pred * k * k) - 1) <= 0.01, (beta, r / (k * k), pred)
