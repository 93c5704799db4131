"""The synthetic input generators: seeded, deterministic, and the exact Riemann solver they use to
select Riemann problems (no GPU needed)."""
import numpy as np

from paper_1802_02369_gb300 import workloads as W


def test_riemann_star_sod_values():
    """Sod's problem (rho, u, p) = (1, 0, 1) | (0.125, 0, 0.1), gamma = 1.4: the star state of the
    exact solution is p* = 0.30313, u* = 0.92745 (Toro, Riemann Solvers and Numerical Methods for Fluid
    Dynamics, test 1 of chapter 4)."""
    p, u = W.riemann_star(1.0, 1.0, 0.125, 0.1)
    assert abs(p - 0.30313) < 5e-6 and abs(u - 0.92745) < 5e-6


def test_riemann_star_special_cases():
    """Equal states: no wave, u* = 0, p* = p. Mirror image: u* changes sign, p* is kept. A pure
    two-rarefaction problem (gas receding on both sides at |u| small) has p* below both pressures,
    and a two-shock problem (colliding streams) above."""
    p, u = W.riemann_star(0.7, 0.3, 0.7, 0.3)
    assert abs(p - 0.3) < 1e-14 and abs(u) < 1e-14
    p1, u1 = W.riemann_star(1.0, 1.0, 0.5, 0.4)
    p2, u2 = W.riemann_star(0.5, 0.4, 1.0, 1.0)
    assert abs(p1 - p2) < 1e-12 and abs(u1 + u2) < 1e-12
    p, u = W.riemann_star(1.0, 0.4, 1.0, 0.4, u_l=-0.2, u_r=0.2)
    assert p < 0.4 and abs(u) < 1e-12
    p, u = W.riemann_star(1.0, 0.4, 1.0, 0.4, u_l=0.2, u_r=-0.2)
    assert p > 0.4 and abs(u) < 1e-12


def test_ragged_batch_deterministic_and_filtered():
    a = W.ragged_batch(64, 7, 0.25 / 1.4, n_min=33, n_max=300)
    b = W.ragged_batch(64, 7, 0.25 / 1.4, n_min=33, n_max=300)
    assert np.array_equal(a.rho, b.rho) and np.array_equal(a.s_e, b.s_e) and np.array_equal(a.bc, b.bc)
    assert a.offsets[-1] == a.lengths.sum() and a.lengths.min() >= 33 and a.lengths.max() <= 300
    f = W.ragged_batch(64, 7, 0.25 / 1.4, n_min=33, n_max=300, entropy_range=(-0.15, 0.0), stable_flow=True)
    sl = W.entropy_of_state(f.states[:, 0], f.states[:, 1])
    sr = W.entropy_of_state(f.states[:, 2], f.states[:, 3])
    assert np.all((sl >= -0.15) & (sl <= 0.0) & (sr >= -0.15) & (sr <= 0.0))
    assert f.s_e.min() >= 1.0 and f.s_e.max() <= 1.9
    g = W.ragged_batch(64, 7, 0.25 / 1.4, n_min=33, n_max=300, entropy_range=(-0.15, 0.0), stable_flow=True)
    assert np.array_equal(f.rho, g.rho)


def test_waves_windows_regenerate_the_full_lattice():
    """A window generated alone with ``period`` equals the same window of the full periodic lattice,
    including windows that wrap past the edges (the full-size parity tests rely on this), in two and
    three dimensions; the entropy stays within the three-dimensional scheme's stable range."""
    full = W.waves_2d(40, 24, 23, amp=0.05)
    win = W.waves_2d(9, 7, 23, amp=0.05, x0=35, y0=-3, period=(40, 24))
    ys, xs = (np.arange(-3, 4) % 24)[:, None], (np.arange(35, 44) % 40)[None, :]
    for a, b in zip(full, win):
        assert np.array_equal(a[ys, xs], b)
    full = W.waves_3d(20, 12, 10, 23, amp=0.05)
    win = W.waves_3d(6, 5, 4, 23, amp=0.05, x0=17, y0=-2, z0=8, period=(20, 12, 10))
    zs = (np.arange(8, 12) % 10)[:, None, None]
    ys = (np.arange(-2, 3) % 12)[None, :, None]
    xs = (np.arange(17, 23) % 20)[None, None, :]
    for a, b in zip(full, win):
        assert np.array_equal(a[zs, ys, xs], b)
    assert np.abs(full[4]).max() <= 0.05
