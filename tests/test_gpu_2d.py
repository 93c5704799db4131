"""Parity of the two-dimensional D2Q9-D2Q5 kernel (through the C-ABI) with the FP64 CPU oracle.

Populations are compared element by element in units of rho0: FP64 and double-float within 1e-12
(absolute; the populations are of order 0.1 to 1), FP32 within 1e-5 of the fields' scales (rho0, lambda, c_p) on
rho, u, s and within 1e-5 on the populations."""
import numpy as np
import pytest

from paper_1802_02369_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import oracle.d2q9q5 as D

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


def run_both(D, lbm, nx, ny, steps, precision, kw, s_e=1.2, beta=4.5, seed=11, amp=0.04, fields=None):
    ph = D.default_phys(beta=beta, **kw)
    if fields is None:
        fields = W.waves_2d(nx, ny, seed, amp=amp, lam=ph.lam, rho0=ph.rho0, cp=ph.cp, s0=ph.s0)
    ref = D.run(ph, D.rates(s_e, ph.gamma, ph.Pr, beta=beta), D.init(ph, *fields), steps, nthreads=8)
    lat = lbm.Lattice2D(nx, ny, precision=precision, s_e=s_e, beta=beta, **kw)
    lat.set_state(*fields)
    lat.step(steps)
    pops, got_fields = lat.populations(), lat.fields()
    lat.close()
    return ph, ref, pops, got_fields


@pytest.mark.parametrize("precision", ["f64", "f64df"])
@pytest.mark.parametrize("kw", PHYS)
@pytest.mark.parametrize("shape", [(45, 37), (3, 3), (5, 70), (33, 4)])
def test_fp64_populations_match_the_oracle(D, lbm, kw, shape, precision):
    """Ragged tile edges (45 x 37 on 32 x 4 tiles), lattices smaller than the tile and its halo (the
    periodic wrap taken several times), non-default physics; FP64 and double-float arithmetic."""
    nx, ny = shape
    _, ref, pops, _ = run_both(D, lbm, nx, ny, 40, precision, kw)
    assert np.abs(pops - ref).max() <= 1e-12


@pytest.mark.parametrize("kw", PHYS)
def test_fp32_matches_the_oracle(D, lbm, kw):
    ph, ref, pops, (rho, ux, uy, s) = run_both(D, lbm, 45, 37, 40, "f32", kw)
    m = D.moments(ph, ref)
    r_ref = m[..., 0]
    assert np.abs(rho - r_ref).max() <= 1e-5 * ph.rho0
    assert np.abs(ux - m[..., 1] / r_ref).max() <= 1e-5 * ph.lam
    assert np.abs(uy - m[..., 2] / r_ref).max() <= 1e-5 * ph.lam
    assert np.abs(s - m[..., 3] / r_ref).max() <= 1e-5 * ph.cp
    assert np.abs(pops - ref).max() <= 1e-5


def test_one_dimensional_data_with_the_1d_closure(D, lbm):
    """beta = 3/2 on data that do not depend on y: the kernel follows the oracle, which is exactly the
    D1Q3Q3 scheme there (the pin of the oracle)."""
    ph = D.default_phys(beta=1.5)
    rho1, u1, s1 = (np.tile(a, (4, 1)) for a in (1 + 0.08 * np.sin(2 * np.pi * np.arange(64) / 64),
                                                 0.08 * np.cos(2 * np.pi * np.arange(64) / 64),
                                                 0.02 * np.sin(4 * np.pi * np.arange(64) / 64)))
    _, ref, pops, _ = run_both(D, lbm, 64, 4, 60, "f64", {}, beta=1.5, fields=(rho1, u1, 0 * u1, s1))
    assert np.abs(pops - ref).max() <= 1e-12
    assert np.array_equal(pops[0], pops[3])


def test_source_off_and_rates(D, lbm):
    """Without the production term, and with explicit rates of the non-hydrodynamic moments."""
    kw = dict(source_on=0)
    ph = D.default_phys(beta=4.5, source_on=0)
    fields = W.waves_2d(40, 24, 5, amp=0.05)
    rt = D.rates(1.6, beta=4.5, s_q=1.1, s_h=1.3, s_eps=1.2)
    ref = D.run(ph, rt, D.init(ph, *fields), 30)
    lat = lbm.Lattice2D(40, 24, precision="f64", s_e=1.6, s_q=1.1, s_h=1.3, s_eps=1.2, **kw)
    assert np.allclose(lat.rates(), (rt.s_e, rt.s_psi, rt.s_eps, rt.s_q, rt.s_h), rtol=1e-15, atol=0)
    lat.set_state(*fields)
    lat.step(30)
    assert np.abs(lat.populations() - ref).max() <= 1e-12
    lat.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f64df", 1e-12), ("f32", 1e-5)])
def test_long_horizon(D, lbm, precision, tol):
    """500 steps on a 48 x 40 lattice: the errors stay within the same bounds."""
    _, ref, pops, _ = run_both(D, lbm, 48, 40, 500, precision, {}, seed=13)
    assert np.abs(pops - ref).max() <= tol


@pytest.mark.parametrize("precision", ["f64", "f64df", "f32"])
def test_full_size_sampled_windows(D, lbm, precision):
    """A 4096 x 4096 lattice after 12 steps, compared on 16 x 16 windows: the oracle runs each window
    with a halo of 2 nodes per step (the dependency radius of a step: streaming plus the centred
    differences of the production), and only the inner window is compared."""
    import torch

    N, T, w = 4096, 12, 16
    fields = W.waves_2d(N, N, 23, amp=0.05)
    lat = lbm.Lattice2D(N, N, precision=precision, s_e=1.2)
    lat.set_state(*(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields))
    lat.step(T)
    pops = lat.populations(device=True)
    torch.cuda.synchronize()
    ph = D.default_phys()
    rt = D.rates(1.2)
    h = 2 * T
    tol = 1e-5 if precision == "f32" else 1e-12
    for (x0, y0) in [(0, 0), (N - 8, 1000), (2049, N - 9), (777, 3333)]:
        win = W.waves_2d(w + 2 * h, w + 2 * h, 23, amp=0.05, x0=x0 - h, y0=y0 - h, period=(N, N))
        ref = D.run(ph, rt, D.init(ph, *win), T)[h:h + w, h:h + w]
        ys = (y0 + np.arange(w)) % N
        xs = (x0 + np.arange(w)) % N
        got = pops[torch.from_numpy(ys).cuda()][:, torch.from_numpy(xs).cuda()].cpu().numpy()
        assert np.abs(got - ref).max() <= tol, (x0, y0)
    lat.close()
