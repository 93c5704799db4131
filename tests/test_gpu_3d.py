"""Parity of the three-dimensional D3Q19-D3Q7 kernel (through the C-ABI) with the FP64 CPU oracle.

Populations are compared element by element in units of rho0: FP64 and double-float within 1e-12
(absolute; the populations are of order 0.01 to 0.5), FP32 within 1e-5 of the fields' scales (rho0,
lambda, c_p) on rho, u, s and within 1e-5 on the populations."""
import numpy as np
import pytest

from paper_1802_02369_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import oracle.d3q19q7 as D

    return D


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_02369_gb300 import build, lbm as L

    build.build()
    return L


PHYS = [dict(), dict(gamma=1.3, Pr=0.71, cp=2.5, rho0=1.3, lam=2.0, s0=-0.1)]


def run_both(D, lbm, nx, ny, nz, steps, precision, kw, s_e=1.2, beta=9.0, seed=11, amp=0.04, fields=None,
             config=None):
    ph = D.default_phys(beta=beta, **kw)
    if fields is None:
        fields = W.waves_3d(nx, ny, nz, seed, amp=amp, lam=ph.lam, rho0=ph.rho0, cp=ph.cp, s0=ph.s0)
    ref = D.run(ph, D.rates(s_e, ph.gamma, ph.Pr, beta=beta), D.init(ph, *fields), steps, nthreads=8)
    lat = lbm.Lattice3D(nx, ny, nz, precision=precision, s_e=s_e, beta=beta, **kw)
    if config:
        lat.set_config(**config)
    lat.set_state(*fields)
    lat.step(steps)
    pops, got_fields = lat.populations(), lat.fields()
    lat.close()
    return ph, ref, pops, got_fields


@pytest.mark.parametrize("precision", ["f64", "f64df"])
@pytest.mark.parametrize("kw", PHYS)
@pytest.mark.parametrize("shape", [(37, 11, 7), (3, 3, 3), (5, 19, 4), (33, 4, 9)])
def test_fp64_populations_match_the_oracle(D, lbm, kw, shape, precision):
    """Ragged tile edges (37 x 11 on 32 x 4 tiles), lattices smaller than the tile and its ring (the
    periodic wrap taken several times along every axis), non-default physics; FP64 and double-float
    arithmetic."""
    _, ref, pops, _ = run_both(D, lbm, *shape, 20, precision, kw)
    assert np.abs(pops - ref).max() <= 1e-12


@pytest.mark.parametrize("precision", ["f64", "f64df", "f32"])
def test_kernel_configurations_agree_bit_for_bit(D, lbm, precision):
    """Tile rows, planes per CTA (one plane, a ragged last chunk, all planes) and where a plane's
    populations wait across the barrier (re-read, registers, shared buffer) change the schedule only:
    the populations are identical."""
    fields = W.waves_3d(40, 21, 13, 3, amp=0.05)
    outs = []
    configs = [dict(ty=4, zc=1, keep=0), dict(ty=8, zc=5, keep=1), dict(ty=4, zc=13, keep=1), dict(ty=8, zc=4, keep=0),
               dict(ty=4, zc=6, keep=0)]
    if precision == "f32":
        configs += [dict(ty=16, zc=3, keep=0), dict(ty=16, zc=2, keep=1), dict(ty=4, zc=1, keep=2),
                    dict(ty=4, zc=5, keep=2), dict(ty=4, zc=13, keep=2)]
    for cfg in configs:
        lat = lbm.Lattice3D(40, 21, 13, precision=precision, s_e=1.3)
        lat.set_config(**cfg)
        assert lat.get_config() == (cfg["ty"], cfg["zc"], cfg["keep"])
        lat.set_state(*fields)
        lat.step(7)
        outs.append(lat.populations())
        lat.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("kw", PHYS)
def test_fp32_matches_the_oracle(D, lbm, kw):
    ph, ref, pops, (rho, ux, uy, uz, s) = run_both(D, lbm, 37, 11, 7, 20, "f32", kw)
    m = D.moments(ph, ref)
    r_ref = m[..., 0]
    assert np.abs(rho - r_ref).max() <= 1e-5 * ph.rho0
    for a, u in enumerate((ux, uy, uz)):
        assert np.abs(u - m[..., 1 + a] / r_ref).max() <= 1e-5 * ph.lam
    assert np.abs(s - m[..., 4] / r_ref).max() <= 1e-5 * ph.cp
    assert np.abs(pops - ref).max() <= 1e-5


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_one_dimensional_data_with_the_1d_closure(D, lbm, axis):
    """beta = 3/2 on data that depend on one coordinate only: the kernel follows the oracle, which is
    exactly the D1Q3Q3 scheme there (the pin of the oracle), and all rows stay equal."""
    N = 40
    x = 2 * np.pi * np.arange(N) / N
    prof = [1 + 0.08 * np.sin(x), 0.08 * np.cos(x), 0.02 * np.sin(2 * x)]
    shape = [4, 4, 4]
    shape[2 - axis] = N
    F = lambda a: np.broadcast_to(a.reshape([N if i == 2 - axis else 1 for i in range(3)]), shape).copy()
    vel = [F(0 * x), F(0 * x), F(0 * x)]
    vel[axis] = F(prof[1])
    fields = (F(prof[0]), *vel, F(prof[2]))
    _, ref, pops, _ = run_both(D, lbm, shape[2], shape[1], shape[0], 40, "f64", {}, beta=1.5, fields=fields)
    assert np.abs(pops - ref).max() <= 1e-12
    line = np.moveaxis(pops, 2 - axis, 0)
    assert np.array_equal(line[:, 0, 0], line[:, 3, 1])


def test_source_off_and_rates(D, lbm):
    """Without the production term, and with explicit rates of the non-hydrodynamic moments."""
    ph = D.default_phys(source_on=0)
    fields = W.waves_3d(20, 12, 9, 5, amp=0.05)
    rt = D.rates(1.4, s_q=1.1, s_h=1.3, s_eps=1.2)
    ref = D.run(ph, rt, D.init(ph, *fields), 20, nthreads=8)
    lat = lbm.Lattice3D(20, 12, 9, precision="f64", s_e=1.4, s_q=1.1, s_h=1.3, s_eps=1.2, source_on=0)
    assert np.allclose(lat.rates(), (rt.s_e, rt.s_psi, rt.s_eps, rt.s_q, rt.s_h), rtol=1e-15, atol=0)
    lat.set_state(*fields)
    lat.step(20)
    assert np.abs(lat.populations() - ref).max() <= 1e-12
    lat.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f64df", 1e-12), ("f32", 1e-5)])
def test_long_horizon(D, lbm, precision, tol):
    """300 steps on a 24 x 20 x 16 lattice: the errors stay within the same bounds."""
    _, ref, pops, _ = run_both(D, lbm, 24, 20, 16, 300, precision, {}, seed=13)
    assert np.abs(pops - ref).max() <= tol


@pytest.mark.parametrize("precision", ["f64", "f64df", "f32"])
def test_full_size_sampled_windows(D, lbm, precision):
    """A 256 x 256 x 256 lattice after 6 steps, compared on 8 x 8 x 8 windows: the oracle runs each
    window with a halo of 2 nodes per step (the dependency radius of a step: streaming plus the centred
    differences of the production), and only the inner window is compared."""
    import torch

    N, T, w = 256, 6, 8
    fields = W.waves_3d(N, N, N, 23, amp=0.05)
    lat = lbm.Lattice3D(N, N, N, precision=precision, s_e=1.2)
    lat.set_state(*(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields))
    del fields
    lat.step(T)
    pops = lat.populations(device=True)
    torch.cuda.synchronize()
    ph = D.default_phys()
    rt = D.rates(1.2)
    h = 2 * T
    tol = 1e-5 if precision == "f32" else 1e-12
    for (x0, y0, z0) in [(0, 0, 0), (N - 4, 100, N - 3), (129, N - 5, 77), (31, 200, 128)]:
        win = W.waves_3d(w + 2 * h, w + 2 * h, w + 2 * h, 23, amp=0.05, x0=x0 - h, y0=y0 - h, z0=z0 - h,
                         period=(N, N, N))
        ref = D.run(ph, rt, D.init(ph, *win), T, nthreads=8)[h:h + w, h:h + w, h:h + w]
        idx = lambda o: torch.from_numpy((o + np.arange(w)) % N).cuda()
        got = pops[idx(z0)][:, idx(y0)][:, :, idx(x0)].cpu().numpy()
        assert np.abs(got - ref).max() <= tol, (x0, y0, z0)
    del pops
    lat.close()
