"""Parity of the CUDA finite-difference comparison solver (section 9, lbm_fd_* of the C-ABI) with
its FP64 CPU oracle, and the figure 4 comparison of the lattice Boltzmann scheme with it.

Tolerances: a field value a (GPU) and b (oracle) agree when |a - b| <= tol * max(|b|, S) with S = 1
(rho0 = c_p = 1; J and zeta are of order 0.1 here); tol = 1e-12 in FP64 and 1e-5 in FP32 on smooth
states. The diagnostics sums are compared with tol * sum |.| (fixed-order GPU reduction vs the
oracle's sequential sum).
"""
import numpy as np
import pytest

import oracle.fd as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_02369_gb300 import build, lbm as L

    build.build()
    F.build()
    return L


def _random_state(N, seed, amp=0.05, kmax=6):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(N) / N
    k = np.arange(1, kmax + 1)

    def f(a):
        c = rng.normal(size=(2, k.size)) * a / k
        return (c[0][:, None] * np.sin(k[:, None] * x) + c[1][:, None] * np.cos(k[:, None] * x)).sum(0)

    return 1 + f(amp), f(amp * 0.5), f(amp * 0.5)


def _phys_dict(ph):
    return dict(gamma=ph.gamma, Pr=ph.Pr, cp=ph.cp, rho0=ph.rho0, p0=ph.p0, s0=ph.s0, source_on=ph.source_on)


def _gpu(L, ph, rho, u, s, dt, nsteps, precision="f64", config=None):
    g = L.FdGrid(rho.size, ph.dx, dt, ph.nu, precision=precision, phys=_phys_dict(ph))
    if config:
        g.set_config(*config)
    g.set_state(rho, u, s)
    g.step(nsteps)
    out = np.stack(g.fields(), axis=1)
    sums, flags, rc = g.diagnostics()
    g.close()
    return out, sums, flags, rc


def _err(a, b):
    return (np.abs(a - b) / np.maximum(np.abs(b), 1.0)).max(axis=0)


@pytest.mark.parametrize("config", [(1, 128, 1), (4, 256, 2), (8, 512, 4), (16, 128, 4), (3, 256, 1), (5, 512, 2)])
def test_fp64_parity_multi_tile_ragged(lbm, config):
    """N = 1999 spans several tiles with a ragged tail for every configuration; 203 steps leave a
    remainder after the K-step launches."""
    ph = F.default_phys(0.08)
    rho, u, s = _random_state(1999, 11)
    ref = F.run(ph, F.init(ph, rho, u, s), 0.05, 203)
    out, _, flags, rc = _gpu(lbm, ph, rho, u, s, 0.05, 203, config=config)
    assert rc == lbm.LBM_OK and flags == 0
    assert _err(out, ref).max() <= 1e-12, _err(out, ref)


@pytest.mark.parametrize("N", [3, 4, 31, 32, 33, 126, 127, 255, 480, 504, 505])
def test_fp64_small_and_edge_sizes(lbm, N):
    """The minimum N = 3, grids shorter than one tile (the halo wraps around several times), and grids
    of exactly one tile interior (126 = 128 - 2 for K = 1, 480 = 512 - 32 for K = 16 and 504 = 512 - 8
    for K = 4 at 256 x 2) or one node more."""
    ph = F.default_phys(0.1, Pr=0.71)
    rho, u, s = _random_state(N, 100 + N, amp=0.03, kmax=1)
    ref = F.run(ph, F.init(ph, rho, u, s), 0.05, 60)
    for config in ((4, 256, 2), (1, 128, 1), (16, 256, 2)):
        out, _, flags, rc = _gpu(lbm, ph, rho, u, s, 0.05, 60, config=config)
        assert rc == lbm.LBM_OK and flags == 0
        assert _err(out, ref).max() <= 1e-12, (config, _err(out, ref))


def test_fp32_parity_smooth(lbm):
    ph = F.default_phys(0.08)
    rho, u, s = _random_state(3001, 12)
    ref = F.run(ph, F.init(ph, rho, u, s), 0.05, 400)
    for config in ((4, 256, 2), (8, 128, 4)):
        out, _, flags, rc = _gpu(lbm, ph, rho, u, s, 0.05, 400, precision="f32", config=config)
        assert rc == lbm.LBM_OK and flags == 0
        assert _err(out, ref).max() <= 1e-5, _err(out, ref)


def test_paper_wave_shock_section9(lbm):
    """The strong wave of figure 3 (delta rho = 0.1 rho0, progressive, one wavelength) on the paper's
    coarsest mesh dx = 1/40 with nu = 6.579e-4, to T_max = 3: FP64 parity with the oracle."""
    N, dx, nu, delta, c0 = 40, 1.0 / 40, 6.579e-4, 0.1, 0.5
    ph = F.default_phys(nu, dx=dx)
    x = 2 * np.pi * np.arange(N) / N
    rho, u, s = 1 + delta * np.sin(x), c0 * delta * np.sin(x), np.zeros(N)
    dt = 0.004
    ref = F.run(ph, F.init(ph, rho, u, s), dt, 750)
    out, sums, flags, rc = _gpu(lbm, ph, rho, u, s, dt, 750, config=(8, 128, 1))
    assert rc == lbm.LBM_OK and flags == 0
    assert _err(out, ref).max() <= 1e-12, _err(out, ref)
    rs, _ = F.diagnostics(ph, ref)
    scale = np.r_[np.abs(ref).sum(axis=0), abs(rs[3])]
    assert np.all(np.abs(sums - rs) <= 1e-12 * scale), (sums, rs)


def test_conservation_and_entropy_production_on_gpu(lbm):
    """Sums of rho and J are conserved by the conservation form, zeta grows by the non-negative
    production (and is conserved without the source), in both precisions."""
    rho, u, s = _random_state(5000, 13)
    for precision, tol in (("f64", 1e-13), ("f32", 2e-6)):
        for src in (1, 0):
            ph = F.default_phys(0.08, source_on=src)
            g = lbm.FdGrid(5000, 1.0, 0.05, 0.08, precision=precision, phys=_phys_dict(ph))
            g.set_state(rho, u, s)
            s0, fl, _ = g.diagnostics()
            prev = s0
            for _ in range(10):
                g.step(100)
                sm, fl, rc = g.diagnostics()
                assert rc == lbm.LBM_OK and fl == 0
                assert abs(sm[0] - s0[0]) <= tol * abs(s0[0])
                assert abs(sm[1] - s0[1]) <= tol * abs(s0[0])
                if src:
                    assert sm[2] >= prev[2] - tol * abs(s0[0])
                else:
                    assert abs(sm[2] - s0[2]) <= tol * abs(s0[0])
                prev = sm
            if src:
                assert prev[2] - s0[2] > 1e-6
            g.close()


def test_host_and_device_buffers_and_raw_fields(lbm):
    import torch

    ph = F.default_phys(0.08)
    rho, u, s = _random_state(700, 14)
    W0 = F.init(ph, rho, u, s)
    ref = F.run(ph, W0, 0.05, 37)
    g = lbm.FdGrid(700, 1.0, 0.05, 0.08, phys=_phys_dict(ph))
    g.set_fields(torch.tensor(W0.T.copy(), device="cuda"))
    g.step(37)
    r, J, z = g.fields(device=True)
    torch.cuda.synchronize()
    out = np.stack([r.cpu().numpy(), J.cpu().numpy(), z.cpu().numpy()], axis=1)
    assert _err(out, ref).max() <= 1e-12
    assert g.steps_done == 37
    g.close()


def test_invalid_arguments(lbm):
    with pytest.raises(lbm.LbmError):
        lbm.FdGrid(2, 1.0, 0.1, 0.1)
    with pytest.raises(lbm.LbmError):
        lbm.FdGrid(64, 1.0, 0.0, 0.1)
    with pytest.raises(lbm.LbmError):
        lbm.FdGrid(64, 1.0, 0.1, 0.1, phys=dict(equilibria=1))
    g = lbm.FdGrid(64, 1.0, 0.1, 0.1)
    with pytest.raises(lbm.LbmError):
        g.step(1)  # no state yet
    with pytest.raises(lbm.LbmError):
        g.set_config(17, 256, 2)
    with pytest.raises(lbm.LbmError):
        g.set_config(0, 1024, 0)
    with pytest.raises(lbm.LbmError):
        g.set_config(0, 128, 3)
    g.close()


def test_full_size_sampled_windows(lbm):
    """N = 2^26 with the benchmark's launch configuration: windows around sampled nodes (both ends of
    the periodic grid included) against the oracle on an extended window. After T steps a periodic
    window of 2T + 2m + 1 nodes is exact on its central 2m + 1 nodes (the stencil reaches one node per
    step)."""
    import torch

    N, T, m = 1 << 26, 48, 8
    nu, dt = 1.0 / 3.0, 1.0
    ph = F.default_phys(nu)
    j = np.arange(N, dtype=np.float64)
    x = 2 * np.pi * j / N
    rng = np.random.default_rng(7)
    noise = np.zeros(N)
    idx = rng.integers(0, N, size=4096)
    noise[idx] = rng.normal(size=idx.size) * 1e-3
    rho = 1 + 0.1 * np.sin(x) + noise
    u = 0.1 * np.sin(x) + np.roll(noise, 3)
    s = np.zeros(N)
    g = lbm.FdGrid(N, 1.0, dt, nu, phys=_phys_dict(ph))
    g.set_config(8, 256, 2)
    g.set_state(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"), torch.tensor(s, device="cuda"))
    g.step(T)
    r, J, z = g.fields(device=True)
    centres = [0, 1, N - 1, N // 2, int(idx[0]), int(idx[1]), int(idx[2]) + 1, N - 17]
    half = T + m
    for c in centres:
        win = (c + np.arange(-half, half + 1)) % N
        Wr = F.run(ph, F.init(ph, rho[win], u[win], s[win]), dt, T)[half - m:half + m + 1]
        sel = torch.tensor(win[half - m:half + m + 1], device="cuda")
        out = np.stack([r[sel].cpu().numpy(), J[sel].cpu().numpy(), z[sel].cpu().numpy()], axis=1)
        assert _err(out, Wr).max() <= 1e-12, (c, _err(out, Wr))
    g.close()


def test_figure4_lattice_boltzmann_against_finite_differences(lbm):
    """Figure 4 of section 9 on the GPU: the strong wave (delta rho = 0.1 rho0) on 40 nodes with the
    paper's nu (s_e = 1.9 at dx = 1/40, lattice units) to T_max = 3 (120 lattice steps), with and
    without the entropy source, beside the finite-difference solver on the same grid (dt = 0.05
    lattice units). Every series matches its oracle, and the paper's statements hold:
    - without the source the total entropy stays constant and the total energy drifts;
    - with it the energy defect is much smaller;
    - the lattice Boltzmann entropy production is close to the finite-difference one."""
    import oracle as O

    O.build()
    N, delta, c0, s_e = 40, 0.1, 0.5, 1.9
    x = 2 * np.pi * np.arange(N) / N
    rho, u, s = 1 + delta * np.sin(x), c0 * delta * np.sin(x), np.zeros(N)
    sigma_e = 1 / s_e - 0.5
    series = {}
    for src in (1, 0):
        ph = O.default_phys(source_on=src)
        fd = O.init(ph, rho, u, s=s)
        ref = [O.diagnostics(ph, fd)[0]]
        lat = lbm.Lattice(N, s_e=s_e, phys=dict(source_on=src))
        lat.set_state_entropy(rho, u, s)
        got = [lat.diagnostics()[0][0]]
        for _ in range(12):
            fd = O.run(ph, O.coupled_rates(s_e), fd, 10)
            ref.append(O.diagnostics(ph, fd)[0])
            lat.step(10)
            got.append(lat.diagnostics()[0][0])
        lat.close()
        ref, got = np.array(ref), np.array(got)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), np.abs(got - ref).max()
        series[("lbm", src)] = got
        phf = F.default_phys(sigma_e, source_on=src)
        _, fref = F.series(phf, F.init(phf, rho, u, s), 0.05, 2400, 200)
        g = lbm.FdGrid(N, 1.0, 0.05, sigma_e, phys=_phys_dict(phf))
        g.set_state(rho, u, s)
        fgot = [g.diagnostics()[0]]
        for _ in range(12):
            g.step(200)
            fgot.append(g.diagnostics()[0])
        g.close()
        fgot = np.array(fgot)
        assert np.abs(fgot - fref).max() <= 1e-12 * np.abs(fref).max(), np.abs(fgot - fref).max()
        series[("fd", src)] = fgot
    l1, l0, f1 = series[("lbm", 1)], series[("lbm", 0)], series[("fd", 1)]
    assert np.abs(l0[:, 2] - l0[0, 2]).max() <= 1e-13            # entropy constant without the source
    e_defect_on = np.abs(l1[:, 3] - l1[0, 3]).max()
    e_defect_off = np.abs(l0[:, 3] - l0[0, 3]).max()
    assert e_defect_on < 0.1 * e_defect_off, (e_defect_on, e_defect_off)
    prod_lbm, prod_fd = l1[-1, 2] - l1[0, 2], f1[-1, 2] - f1[0, 2]
    assert prod_lbm > 0 and prod_fd > 0
    assert 0.8 < prod_lbm / prod_fd < 1.1, (prod_lbm, prod_fd)


def test_autotune_keeps_state_and_result(lbm):
    """lbm_fd_autotune leaves the state unchanged and picks a valid configuration whose result is the
    oracle's."""
    ph = F.default_phys(0.08)
    rho, u, s = _random_state(20000, 15)
    ref = F.run(ph, F.init(ph, rho, u, s), 0.05, 40)
    g = lbm.FdGrid(20000, 1.0, 0.05, 0.08, phys=_phys_dict(ph))
    g.set_state(rho, u, s)
    k, nt, v = g.autotune(1)
    assert nt in (128, 256, 512) and v in (1, 2, 4) and 1 <= k <= 16 and nt * v - 2 * k >= 32
    g.step(40)
    out = np.stack(g.fields(), axis=1)
    g.close()
    assert _err(out, ref).max() <= 1e-12
