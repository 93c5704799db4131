"""Parity of the CUDA single-distribution D1Q3 schemes (section 2 fluid, section 4 advection-diffusion;
lbm_d1q3_* of the C-ABI) with their FP64 CPU oracle.

Tolerances: a moment a (GPU) and b (oracle) agree when |a - b| <= tol * max(|b|, S) with S the
natural scale of the moment (scale, scale lambda, scale lambda^2); tol = 1e-12 in FP64 and 1e-5 in
FP32 on smooth states.
"""
import numpy as np
import pytest

import oracle.d1q3 as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_02369_gb300 import build, lbm as L

    build.build()
    D.build()
    return L


def _smooth(N, seed, amp, kmax=6):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(N) / N
    k = np.arange(1, kmax + 1)
    c = rng.normal(size=(2, k.size)) * amp / k
    return (c[0][:, None] * np.sin(k[:, None] * x) + c[1][:, None] * np.cos(k[:, None] * x)).sum(0)


def _fluid_state(N, seed):
    rho = 1 + _smooth(N, seed, 0.05)
    return rho, rho * _smooth(N, seed + 1, 0.03)


def _err(gpu, ref, p):
    sc = p.scale * np.array([1.0, p.lam, p.lam ** 2])
    g = np.stack(gpu, axis=1)
    return (np.abs(g - ref) / np.maximum(np.abs(ref), sc)).max(axis=0)


def _gpu_fluid(L, p, rho, J, n, precision="f64", config=None):
    lat = L.D1q3Lattice(rho.size, "fluid", lam=p.lam, precision=precision, s_e=p.s_e, gamma=p.gamma, p0=p.p0,
                        scale=p.scale)
    if config:
        lat.set_config(*config)
    lat.set_state(rho, J)
    lat.step(n)
    m = lat.moments()
    lat.close()
    return m


def _gpu_ad(L, p, z, n, precision="f64", config=None):
    lat = L.D1q3Lattice(z.size, "advection_diffusion", lam=p.lam, precision=precision, u0=p.u0, alpha=p.alpha,
                        s_psi=p.s_psi, s_eps=p.s_eps, scale=p.scale)
    if config:
        lat.set_config(*config)
    lat.set_state(z)
    lat.step(n)
    m = lat.moments()
    lat.close()
    return m


CONFIGS = [(1, 128, 1), (8, 256, 4), (16, 128, 8), (3, 512, 2), (64, 256, 8), (5, 128, 1)]


@pytest.mark.parametrize("config", CONFIGS)
def test_fluid_fp64_parity_ragged(lbm, config):
    p = D.fluid(1.3)
    rho, J = _fluid_state(1999, 1)
    ref = D.moments(p, D.run(p, D.init(p, rho, J), 301))
    assert _err(_gpu_fluid(lbm, p, rho, J, 301, config=config), ref, p).max() <= 1e-12


@pytest.mark.parametrize("config", CONFIGS)
def test_advection_diffusion_fp64_parity_ragged(lbm, config):
    p = D.advection_diffusion(0.17, -0.4, 0.9, lam=1.0, zeta0=1.0)
    z = 1 + _smooth(1999, 3, 0.1)
    ref = D.moments(p, D.run(p, D.init(p, z), 301))
    assert _err(_gpu_ad(lbm, p, z, 301, config=config), ref, p).max() <= 1e-12


@pytest.mark.parametrize("lam,scale", [(2.0, 0.8), (0.5, 1.7)])
def test_other_lattice_speeds_and_scales(lbm, lam, scale):
    p = D.fluid(1.7, lam=lam, rho0=scale, gamma=1.3)
    rho, J = _fluid_state(777, 4)
    rho, J = scale * rho, scale * lam * J
    ref = D.moments(p, D.run(p, D.init(p, rho, J), 120))
    assert _err(_gpu_fluid(lbm, p, rho, J, 120), ref, p).max() <= 1e-12
    q = D.advection_diffusion(-0.3 * lam, 0.5, 1.4, lam=lam, zeta0=scale, s_eps=1.2)
    z = scale * (1 + _smooth(777, 5, 0.1))
    ref = D.moments(q, D.run(q, D.init(q, z), 120))
    assert _err(_gpu_ad(lbm, q, z, 120), ref, q).max() <= 1e-12


@pytest.mark.parametrize("N", [3, 4, 31, 33, 126, 127, 480, 481, 1008])
def test_small_and_edge_sizes(lbm, N):
    """The minimum N = 3, lattices shorter than one tile (the halo wraps around several times), one
    tile interior exactly (126 = 128 - 2 at K = 1; 480 = 512 - 32 at K = 16; 1008 = 1024 - 16 at
    K = 8, 256 x 4) and one node more."""
    p = D.fluid(1.5)
    rho, J = _fluid_state(N, 10 + N)
    ref = D.moments(p, D.run(p, D.init(p, rho, J), 50))
    q = D.advection_diffusion(0.2, 0.0, 1.1)
    z = 1 + _smooth(N, 20 + N, 0.1, kmax=1)
    refq = D.moments(q, D.run(q, D.init(q, z), 50))
    for config in ((1, 128, 1), (16, 128, 4), (8, 256, 4)):
        assert _err(_gpu_fluid(lbm, p, rho, J, 50, config=config), ref, p).max() <= 1e-12, config
        assert _err(_gpu_ad(lbm, q, z, 50, config=config), refq, q).max() <= 1e-12, config


def test_fp32_parity_smooth(lbm):
    p = D.fluid(1.2)
    rho, J = _fluid_state(4001, 6)
    ref = D.moments(p, D.run(p, D.init(p, rho, J), 500))
    q = D.advection_diffusion(0.1, 0.0, 1.2)
    z = 1 + _smooth(4001, 7, 0.1)
    refq = D.moments(q, D.run(q, D.init(q, z), 500))
    for config in ((8, 256, 4), (16, 128, 8), (4, 128, 1)):
        assert _err(_gpu_fluid(lbm, p, rho, J, 500, "f32", config), ref, p).max() <= 1e-5, config
        assert _err(_gpu_ad(lbm, q, z, 500, "f32", config), refq, q).max() <= 1e-5, config


def test_kappa_identification_sets_s_psi(lbm):
    """Section 4: ((2 + alpha)/3 lambda^2 - u0^2)(1/s_psi - 1/2) dt = kappa, dt = 1/lambda."""
    lam, u0, alpha, kappa = 1.5, 0.2, 0.4, 0.05
    lat = lbm.D1q3Lattice(64, "advection_diffusion", lam=lam, u0=u0, alpha=alpha, kappa=kappa)
    s_psi, s_eps = lat.rates()
    lat.close()
    assert abs(((2 + alpha) / 3 * lam ** 2 - u0 ** 2) * (1 / s_psi - 0.5) / lam - kappa) <= 1e-15
    assert s_eps == 1.5
    with pytest.raises(lbm.LbmError):  # no s_psi in (0, 2) gives a negative diffusivity
        lbm.D1q3Lattice(64, "advection_diffusion", lam=lam, u0=u0, alpha=alpha, kappa=-0.01)


def test_exact_shift_at_the_lattice_speed(lbm):
    z = 1 + _smooth(1000, 8, 0.3)
    for sign in (1, -1):
        lat = lbm.D1q3Lattice(1000, "advection_diffusion", u0=float(sign), alpha=1.0, s_psi=1.0, s_eps=1.0)
        lat.set_state(z)
        lat.step(37)
        m = lat.moments()[0]
        lat.close()
        assert np.abs(m - np.roll(z, sign * 37)).max() <= 1e-14


def test_conservation_on_gpu(lbm):
    rho, J = _fluid_state(10000, 9)
    z = 1 + _smooth(10000, 10, 0.1)
    for precision, tol in (("f64", 1e-13), ("f32", 1e-6)):
        for lat, m0 in ((lbm.D1q3Lattice(10000, "fluid", s_e=1.4, precision=precision), (rho, J)),
                        (lbm.D1q3Lattice(10000, "advection_diffusion", u0=0.1, alpha=-0.5, s_psi=1.3,
                                         precision=precision), (z,))):
            lat.set_state(*m0)
            s0, fl, rc = lat.sums()
            for _ in range(5):
                lat.step(400)
                s, fl, rc = lat.sums()
                assert rc == lbm.LBM_OK and fl == 0
                assert abs(s[0] - s0[0]) <= tol * abs(s0[0])
                if lat.scheme == "fluid":
                    assert abs(s[1] - s0[1]) <= tol * abs(s0[0])
            lat.close()


def test_populations_roundtrip_and_autotune(lbm):
    p = D.fluid(1.6)
    rho, J = _fluid_state(30000, 11)
    f0 = D.init(p, rho, J)
    ref = D.moments(p, D.run(p, f0, 64))
    lat = lbm.D1q3Lattice(30000, "fluid", s_e=1.6)
    lat.set_populations(f0.T.copy())
    assert np.abs(lat.populations() - f0.T).max() <= 1e-15
    k, nt, v = lat.autotune(1)
    assert nt in (128, 256, 512) and v in (1, 2, 4, 8) and 1 <= k <= 64
    assert np.abs(lat.populations() - f0.T).max() <= 1e-15   # the trials leave the state alone
    lat.step(64)
    assert _err(lat.moments(), ref, p).max() <= 1e-12
    assert lat.steps_done == 64
    lat.close()


def test_invalid_arguments(lbm):
    with pytest.raises(lbm.LbmError):
        lbm.D1q3Lattice(2, "fluid")
    with pytest.raises(lbm.LbmError):
        lbm.D1q3Lattice(64, "fluid", s_e=2.0)
    with pytest.raises(lbm.LbmError):
        lbm.D1q3Lattice(64, "advection_diffusion", s_psi=1.0, s_eps=2.5)
    lat = lbm.D1q3Lattice(64, "fluid")
    with pytest.raises(lbm.LbmError):
        lat.step(1)
    with pytest.raises(lbm.LbmError):
        lat.set_config(0, 64, 0)
    with pytest.raises(lbm.LbmError):
        lat.set_config(65, 512, 8)
    lat.close()


@pytest.mark.parametrize("scheme", ["fluid", "advection_diffusion"])
def test_full_size_sampled_windows(lbm, scheme):
    """N = 2^26 in the benchmark's launch configuration: windows around sampled nodes (both ends of
    the periodic lattice included) against the oracle on an extended periodic window, exact on its
    central 2m + 1 nodes after T steps (advection reaches one node per step)."""
    import torch

    N, T, m = 1 << 26, 64, 8
    x = 2 * np.pi * np.arange(N) / N
    rng = np.random.default_rng(12)
    idx = rng.integers(0, N, size=4096)
    noise = np.zeros(N)
    noise[idx] = rng.normal(size=idx.size) * 1e-3
    if scheme == "fluid":
        p = D.fluid(1.2)
        m0 = 1 + 0.1 * np.sin(x) + noise
        m1 = m0 * (0.1 * np.sin(x) + np.roll(noise, 5))
        lat = lbm.D1q3Lattice(N, "fluid", s_e=1.2)
        lat.set_config(16, 128, 8)
        lat.set_state(torch.tensor(m0, device="cuda"), torch.tensor(m1, device="cuda"))
    else:
        p = D.advection_diffusion(0.1, 0.0, 1.2)
        m0 = 1 + 0.1 * np.sin(x) + noise
        m1 = None
        lat = lbm.D1q3Lattice(N, "advection_diffusion", u0=0.1, alpha=0.0, s_psi=1.2)
        lat.set_config(32, 256, 8)
        lat.set_state(torch.tensor(m0, device="cuda"))
    lat.step(T)
    g = lat.moments(device=True)
    half = T + m
    for c in [0, 1, N - 1, N // 2, int(idx[0]), int(idx[1]) + 1, N - 9]:
        win = (c + np.arange(-half, half + 1)) % N
        f = D.init(p, m0[win], None if m1 is None else m1[win])
        ref = D.moments(p, D.run(p, f, T))[half - m:half + m + 1]
        sel = torch.tensor(win[half - m:half + m + 1], device="cuda")
        got = [t[sel].cpu().numpy() for t in g]
        assert _err(got, ref, p).max() <= 1e-12, c
    lat.close()
