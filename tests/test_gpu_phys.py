"""Parity of the CUDA path with the FP64 oracle away from the paper's default physics.

The experiments of section 9 fix gamma = 1.4, Pr = 1, c_p = 1, rho0 = 1, s0 = 0 and lambda = 1; the
scheme itself (sections 6 and 8) is defined for any polytropic gas, Prandtl number, moment scale and
lattice velocity. Here every one of those parameters is moved at once (gamma = 1.3, Pr = 0.71,
c_p = 2.5, rho0 = 1.3, s0 = -0.1) at lambda = 0.5 and 2, so that the Pr factors of the coupled rate
(eq. lien-sigma-sigma) and of kappa, the rho0 of the equation of state (eq. gaz-parfait) and of M
(eq. M-d1q3q3), the c_p scalings and the host-rounded FP32 constants are all exercised; and a batch
gives each lattice its own reference entropy s0 (lbm_create_batch's per-lattice s0).

Tolerances as in the other parity tests: |a - b| <= tol * max(|b|, S) with S the field's lattice scale
(rho0, rho0 lambda, rho0 c_p, rho0 lambda^2, rho0 c_p lambda, rho0 c_p lambda^2), tol = 1e-12 for FP64
storage (native and double-float) and 1e-5 for FP32; beside it the pure relative error of rho and e,
which are of order rho0 and rho0 lambda^2 everywhere, is held to the same tol.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(16, os.cpu_count() or 1))
PHYS = dict(gamma=1.3, Pr=0.71, cp=2.5, rho0=1.3, s0=-0.1)
TOL = {"f64": 1e-12, "f64df": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_02369_gb300 import build, lbm as L

    build.build()
    return L


def scales(lam, cp, rho0):
    return np.array([rho0, rho0 * lam, rho0 * cp, rho0 * lam ** 2, rho0 * cp * lam, rho0 * cp * lam ** 2])


def errors(gpu_m, ora_m, sc):
    """(max scale-floored error per field, max pure relative error of rho and e)."""
    g = np.stack([np.asarray(x) for x in gpu_m], axis=1)
    floored = (np.abs(g - ora_m) / np.maximum(np.abs(ora_m), sc[None, :])).max(axis=0)
    pure = (np.abs(g[:, [0, 3]] - ora_m[:, [0, 3]]) / np.abs(ora_m[:, [0, 3]])).max()
    return floored, pure


def fields(N, seed, lam, ph, bc=0, amp=0.03):
    """Smooth data around (rho0, u = 0, s = s0): a few Fourier modes, velocities in units of lambda,
    entropies in units of c_p (inside the scheme's stable band), and the pressure of that state."""
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(N) / N
    rho = ph.rho0 * (1.0 + sum(amp * rng.uniform(-1, 1) * np.sin(k * x + rng.uniform(0, 6.3)) for k in (1, 2, 3)))
    u = lam * sum(amp * rng.uniform(-1, 1) * np.sin(k * x + rng.uniform(0, 6.3)) for k in (1, 2))
    if bc:
        u = u * np.sin(np.pi * (np.arange(N) + 0.5) / N)
    s = ph.s0 + ph.cp * sum(amp * rng.uniform(-1, 1) * np.cos(k * x + rng.uniform(0, 6.3)) for k in (1, 2))
    p = ph.p0 * (rho / ph.rho0) ** ph.gamma * np.exp(ph.gamma * (s - ph.s0) / ph.cp)
    return rho, u, s, p


@pytest.mark.parametrize("lam", [0.5, 2.0])
@pytest.mark.parametrize("precision", ["f64", "f32", "f64df"])
def test_nondefault_physics_against_oracle(O, lbm, lam, precision):
    """Two lattices (3001 nodes periodic, 1234 bounce-back; several tiles and a ragged tail), one set
    from pressures and one from entropies, 300 steps, s_e = 1.3 and 1.7, every parameter of lbm_phys
    away from its default: GPU against the oracle at the same parameters, and the FP64 diagnostics
    (sums of rho, J, zeta and the total energy p/(gamma-1) + rho u^2/2) against the oracle's."""
    lengths, bcs, s_e = np.array([3001, 1234]), np.array([0, 1]), np.array([1.3, 1.7])
    T = 300
    phs = [O.default_phys(lam=lam, bc=int(b), **PHYS) for b in bcs]
    data = [fields(int(n), 11 + b, lam, phs[b], bc=int(bcs[b])) for b, n in enumerate(lengths)]
    refs, osums = [], []
    for b in range(2):
        ph = phs[b]
        rho, u, s, p = data[b]
        fd = O.run(ph, O.coupled_rates(s_e[b], ph.gamma, ph.Pr), O.init(ph, rho, u, s=s), T, NTHREADS)
        refs.append(O.moments(ph, fd))
        sums, flags = O.diagnostics(ph, fd)
        assert flags == 0
        osums.append(sums)
    sc = scales(lam, PHYS["cp"], PHYS["rho0"])
    for how in ("pressure", "entropy"):
        lat = lbm.Lattice(lengths, lam=lam, s_e=s_e, bc=bcs, precision=precision, phys=PHYS)
        cat = [np.concatenate([d[k] for d in data]) for k in range(4)]
        if how == "pressure":
            lat.set_state(cat[0], cat[1], cat[3])
        else:
            lat.set_state_entropy(cat[0], cat[1], cat[2])
        lat.step(T)
        g = np.stack(lat.moments(device=False), axis=1)
        sums, flags, rc = lat.diagnostics()
        lat.close()
        assert rc == lbm.LBM_OK and np.all(flags == 0)
        off = np.r_[0, np.cumsum(lengths)]
        for b in range(2):
            floored, pure = errors(list(g[off[b]:off[b + 1]].T), refs[b], sc)
            assert floored.max() <= TOL[precision], (how, b, floored)
            assert pure <= TOL[precision], (how, b, pure)
            tol_sum = 1e-12 if precision != "f32" else 1e-6
            np.testing.assert_allclose(sums[b], osums[b], rtol=tol_sum, atol=tol_sum * lengths[b] * sc[:4].max())


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_per_lattice_reference_entropy(O, lbm, precision):
    """lbm_create_batch with one reference entropy s0 per lattice (eq. gaz-parfait's s0; the stored
    populations are shifted by each lattice's own rest state): every lattice against the oracle run
    with its s0, at the non-default gas and lambda = 2, periodic and bounce-back lattices."""
    lam = 2.0
    s0s = np.array([-0.1, 0.0, -0.25, 0.05])
    lengths = np.array([777, 2050, 129, 1500])
    bcs = np.array([0, 1, 1, 0])
    s_e = np.array([1.2, 1.4, 1.6, 1.9])
    T = 200
    phs = [O.default_phys(lam=lam, bc=int(bcs[b]), **dict(PHYS, s0=float(s0s[b]))) for b in range(4)]
    data = [fields(int(n), 60 + b, lam, phs[b], bc=int(bcs[b])) for b, n in enumerate(lengths)]
    lat = lbm.Lattice(lengths, lam=lam, s_e=s_e, bc=bcs, precision=precision, phys=PHYS, s0=s0s)
    lat.set_state_entropy(*[np.concatenate([d[k] for d in data]) for k in range(3)])
    lat.step(T)
    g = np.stack(lat.moments(device=False), axis=1)
    lat.close()
    off = np.r_[0, np.cumsum(lengths)]
    sc = scales(lam, PHYS["cp"], PHYS["rho0"])
    for b in range(4):
        ph = phs[b]
        rho, u, s, _ = data[b]
        ref = O.moments(ph, O.run(ph, O.coupled_rates(s_e[b], ph.gamma, ph.Pr), O.init(ph, rho, u, s=s), T))
        floored, pure = errors(list(g[off[b]:off[b + 1]].T), ref, sc)
        assert floored.max() <= TOL[precision], (b, floored)
        assert pure <= TOL[precision], (b, pure)


def test_adjoint_nondefault_physics_against_dual_numbers(O, lbm):
    """The FP64 adjoint at the non-default gas and lambda = 0.5: directional derivatives of
    loss = sum (rho_T - rho*)^2 along random directions in (rho(0), u(0), s_e, s_psi) against the
    oracle's forward-mode dual numbers at the same parameters, within 1e-6 relative."""
    lam, T = 0.5, 50
    lengths, bcs, s_e = np.array([41, 66]), np.array([0, 1]), np.array([1.25, 1.6])
    phs = [O.default_phys(lam=lam, bc=int(b), **PHYS) for b in bcs]
    data = [fields(int(n), 90 + b, lam, phs[b], bc=int(bcs[b])) for b, n in enumerate(lengths)]
    targets = [fields(int(n), 95 + b, lam, phs[b], amp=0.02)[0] for b, n in enumerate(lengths)]
    lat = lbm.Lattice(lengths, lam=lam, s_e=s_e, bc=bcs, precision="f64", phys=PHYS)
    lat.set_state_entropy(*[np.concatenate([d[k] for d in data]) for k in range(3)])
    loss, drho, du, drates = lat.adjoint(T, np.concatenate(targets))
    lat.close()
    off = np.r_[0, np.cumsum(lengths)]
    rng = np.random.default_rng(3)
    oracle_loss = 0.0
    for b, n in enumerate(lengths):
        ph = phs[b]
        rates = O.coupled_rates(s_e[b], ph.gamma, ph.Pr)
        rho, u, s, _ = data[b]
        vr, vu, vs = rng.standard_normal((3, n)), rng.standard_normal((3, n)), rng.standard_normal((3, 2))
        vr[0] = 0.0
        vu[0] = 0.0
        vs[1] = 0.0
        fd, dfd = O.run_tangent(ph, rates, vs, rho, u, s, vr, vu, T)
        rho_T = O.moments(ph, fd)[:, 0]
        oracle_loss += np.sum((rho_T - targets[b]) ** 2)
        for k in range(3):
            drho_T = ph.rho0 * dfd[k][:, :3].sum(axis=1)
            d_oracle = np.sum(2 * (rho_T - targets[b]) * drho_T)
            d_gpu = (np.dot(drho[off[b]:off[b + 1]], vr[k]) + np.dot(du[off[b]:off[b + 1]], vu[k])
                     + np.dot(drates[b], vs[k]))
            assert abs(d_gpu - d_oracle) <= 1e-6 * abs(d_oracle) + 1e-14, (b, k, d_gpu, d_oracle)
    assert abs(loss - oracle_loss) <= 1e-12 * oracle_loss
