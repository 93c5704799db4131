"""The GPU adjoint (reverse mode through the C-ABI) against the oracle's forward-mode dual numbers
and against central differences of the GPU forward run."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_02369_gb300 import build, lbm as L

    build.build()
    return L


def _fields(N, seed, amp=0.03, bc=0):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(N) / N
    rho = 1.0 + sum(amp * rng.uniform(-1, 1) * np.sin(k * x + rng.uniform(0, 6.3)) for k in (1, 2, 3))
    u = sum(amp * rng.uniform(-1, 1) * np.sin(k * x + rng.uniform(0, 6.3)) for k in (1, 2))
    if bc:
        u = u * np.sin(np.pi * (np.arange(N) + 0.5) / N)
    s = -0.05 + sum(amp * rng.uniform(-1, 1) * np.cos(k * x + rng.uniform(0, 6.3)) for k in (1, 2))
    return rho, u, s


def _case():
    lengths = np.array([40, 67, 33])
    bc = np.array([0, 1, 0])
    s_e = np.array([1.2, 1.5, 1.35])
    data = [_fields(int(n), 31 + b, bc=int(bc[b])) for b, n in enumerate(lengths)]
    targets = [_fields(int(n), 77 + b, amp=0.02)[0] for b, n in enumerate(lengths)]
    return lengths, bc, s_e, data, targets


def _gpu_adjoint(lbm, lengths, bc, s_e, data, targets, T, precision="f64"):
    lat = lbm.Lattice(lengths, s_e=s_e, bc=bc, precision=precision)
    lat.set_state_entropy(*[np.concatenate([d[k] for d in data]) for k in range(3)])
    loss, drho, du, drates = lat.adjoint(T, np.concatenate(targets))
    s_psi = None
    lat.close()
    return loss, drho, du, drates


def test_adjoint_matches_oracle_dual_numbers(O, lbm):
    """Directional derivatives of loss = sum (rho_T - rho*)^2 along random directions in
    (rho0, u0, s_e, s_psi), per lattice (the loss is separable), FP64, within 1e-6 relative."""
    T = 60
    lengths, bc, s_e, data, targets = _case()
    loss, drho, du, drates = _gpu_adjoint(lbm, lengths, bc, s_e, data, targets, T)
    off = np.r_[0, np.cumsum(lengths)]
    rng = np.random.default_rng(5)
    oracle_loss = 0.0
    for b, n in enumerate(lengths):
        ph = O.default_phys(bc=int(bc[b]))
        rates = O.coupled_rates(s_e[b])
        rho, u, s = data[b]
        ndir = 4
        vr = rng.standard_normal((ndir, n))
        vu = rng.standard_normal((ndir, n))
        vs = rng.standard_normal((ndir, 2))
        vr[0] = 0.0; vu[0] = 0.0           # direction 0: rates only
        vs[1] = 0.0                        # direction 1: fields only
        fd, dfd = O.run_tangent(ph, rates, vs, rho, u, s, vr, vu, T, NTHREADS)
        rho_T = O.moments(ph, fd)[:, 0]
        oracle_loss += np.sum((rho_T - targets[b]) ** 2)
        for k in range(ndir):
            drho_T = ph.rho0 * dfd[k][:, :3].sum(axis=1)
            d_oracle = np.sum(2 * (rho_T - targets[b]) * drho_T)
            d_gpu = (np.dot(drho[off[b]:off[b + 1]], vr[k]) + np.dot(du[off[b]:off[b + 1]], vu[k])
                     + np.dot(drates[b], vs[k]))
            assert abs(d_gpu - d_oracle) <= 1e-6 * abs(d_oracle) + 1e-14, (b, k, d_gpu, d_oracle)
    assert abs(loss - oracle_loss) <= 1e-12 * oracle_loss


def test_adjoint_matches_central_differences_of_gpu_forward(lbm):
    """Central differences (h = 1e-6) of the GPU's own forward loss along 3 probe directions."""
    import torch

    T = 45
    lengths, bc, s_e, data, targets = _case()
    rho0, u0, s0 = [np.concatenate([d[k] for d in data]) for k in range(3)]
    tgt = np.concatenate(targets)
    loss, drho, du, drates = _gpu_adjoint(lbm, lengths, bc, s_e, data, targets, T)
    rng = np.random.default_rng(8)

    def L(r, v):
        lat = lbm.Lattice(lengths, s_e=s_e, bc=bc)
        lat.set_state_entropy(r, v, s0)
        lat.step(T)
        rt = lat.moments(device=False)[0]
        lat.close()
        return float(np.sum((rt - tgt) ** 2))

    h = 1e-6
    for _ in range(3):
        vr, vu = rng.standard_normal(rho0.size), rng.standard_normal(rho0.size)
        fdiff = (L(rho0 + h * vr, u0 + h * vu) - L(rho0 - h * vr, u0 - h * vu)) / (2 * h)
        grad = np.dot(drho, vr) + np.dot(du, vu)
        assert abs(grad - fdiff) <= 1e-6 * abs(grad) + 1e-12, (grad, fdiff)
    torch.cuda.synchronize()


def test_adjoint_fp32_close_to_fp64(lbm):
    """The FP32 adjoint against the FP64 one, element by element: every component of dL/drho(0) and
    dL/du(0) within 1e-3 of the largest component of its field (FP32 rounding over the 60 forward and 60
    reverse steps, amplified by the cancellation in the misfit rho_T - rho*), the rate gradients within
    1e-3 relative, and the loss within 1e-4."""
    T = 60
    lengths, bc, s_e, data, targets = _case()
    l64, r64, u64, s64 = _gpu_adjoint(lbm, lengths, bc, s_e, data, targets, T, "f64")
    l32, r32, u32, s32 = _gpu_adjoint(lbm, lengths, bc, s_e, data, targets, T, "f32")
    assert abs(l32 - l64) <= 1e-4 * l64
    for name, a, b in (("drho", r32, r64), ("du", u32, u64)):
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err <= 1e-3, (name, err)
    assert np.all(np.abs(s32 - s64) <= 1e-3 * np.abs(s64)), (s32, s64)


def test_autograd_function_matches_adjoint(lbm):
    """torch.autograd.Function around the adjoint: gradients of sum((rho_T - rho*)^2)."""
    import torch

    from paper_1802_02369_gb300.autograd import lattice_run

    T = 50
    lengths, bc, s_e, data, targets = _case()
    rho0, u0, s0 = [torch.from_numpy(np.concatenate([d[k] for d in data])).cuda() for k in range(3)]
    rho0.requires_grad_(True)
    u0.requires_grad_(True)
    se_t = torch.tensor(s_e, dtype=torch.float64, requires_grad=True)
    from oracle import coupled_rates
    sp_t = torch.tensor([coupled_rates(x)[1] for x in s_e], dtype=torch.float64, requires_grad=True)
    rho_T = lattice_run(rho0, u0, s0, se_t, sp_t, lengths, T, bc=bc)
    tgt = torch.from_numpy(np.concatenate(targets)).cuda()
    loss = ((rho_T - tgt) ** 2).sum()
    loss.backward()
    l2, drho, du, drates = _gpu_adjoint(lbm, lengths, bc, s_e, data, targets, T)
    assert abs(loss.item() - l2) <= 1e-12 * l2
    np.testing.assert_allclose(rho0.grad.cpu().numpy(), drho, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(u0.grad.cpu().numpy(), du, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(se_t.grad.cpu().numpy(), drates[:, 0], rtol=1e-10)
    np.testing.assert_allclose(sp_t.grad.cpu().numpy(), drates[:, 1], rtol=1e-10)


def test_adjoint_bump_batch_probe_directions(lbm):
    """The differentiation workload's shape (Gaussian density bumps, seed 2369, target from seed
    2370, lattices of 65536 nodes), reduced to 4 lattices and T = 400 for test time: the FP64
    adjoint gradient against central differences (h = 1e-6) of the GPU forward on 8 random probe
    directions in (rho0, u0), within 1e-6 relative."""
    from paper_1802_02369_gb300 import workloads as W

    B, N, T = 4, 65536, 400
    p_ref = W.reference_pressure()
    rho, u, p = W.gaussian_bumps(B, N, 2369, p_ref)
    rt, ut, pt = W.gaussian_bumps(B, N, 2370, p_ref)
    s_e = 1.5
    ref = lbm.Lattice(np.full(B, N), s_e=s_e)
    ref.set_state(rt.ravel(), ut.ravel(), pt.ravel())
    ref.step(T)
    target = ref.moments(device=False)[0]
    ref.close()
    lat = lbm.Lattice(np.full(B, N), s_e=s_e)
    lat.set_state(rho.ravel(), u.ravel(), p.ravel())
    s0 = np.asarray(lat.moments(device=False)[2]) / rho.ravel()   # initial specific entropy
    loss, drho, du, drates = lat.adjoint(T, target)
    lat.close()

    def L(r, v):
        x = lbm.Lattice(np.full(B, N), s_e=s_e)
        x.set_state_entropy(r, v, s0)
        x.step(T)
        out = float(np.sum((np.asarray(x.moments(device=False)[0]) - target) ** 2))
        x.close()
        return out

    rng = np.random.default_rng(2369)
    h = 1e-6
    r0, u0 = rho.ravel(), u.ravel()
    for _ in range(8):
        vr = rng.standard_normal(r0.size)
        vu = rng.standard_normal(r0.size)
        fdiff = (L(r0 + h * vr, u0 + h * vu) - L(r0 - h * vr, u0 - h * vu)) / (2 * h)
        grad = np.dot(drho, vr) + np.dot(du, vu)
        assert abs(grad - fdiff) <= 1e-6 * abs(grad), (grad, fdiff)


def test_adjoint_full_batch_consistency_and_probes(lbm):
    """The differentiation workload at full size (256 lattices of 65536 nodes, Gaussian bumps with
    seeds 2369 / 2370, T = 4000, sqrt(T) checkpointing, FP32): the gradients of sampled lattices
    are bitwise those of a 2-lattice run of the same lattices (the loss is separable and every
    lattice is computed alike), and for those two lattices the FP64 gradient at T = 4000 matches
    central differences (h = 1e-6) on 8 probe directions within 1e-6."""
    from paper_1802_02369_gb300 import workloads as W

    B, N, T = 256, 65536, 4000
    p_ref = W.reference_pressure()
    rho, u, p = W.gaussian_bumps(B, N, 2369, p_ref)
    rt, ut, pt = W.gaussian_bumps(B, N, 2370, p_ref)
    pick = [0, 137]

    def target(prec, idx):
        t = lbm.Lattice(np.full(len(idx), N), s_e=1.5, precision=prec)
        t.set_state(rt[idx].ravel(), ut[idx].ravel(), pt[idx].ravel())
        t.step(T)
        out = np.asarray(t.moments(device=False)[0])
        t.close()
        return out

    def adjoint(prec, idx, tgt):
        a = lbm.Lattice(np.full(len(idx), N), s_e=1.5, precision=prec)
        a.set_state(rho[idx].ravel(), u[idx].ravel(), p[idx].ravel())
        res = a.adjoint(T, tgt)
        a.close()
        return res

    full_tgt = target("f32", list(range(B)))
    _, d_rho, d_u, d_rates = adjoint("f32", list(range(B)), full_tgt)
    sub_tgt = np.concatenate([full_tgt[b * N:(b + 1) * N] for b in pick])
    _, s_rho, s_u, s_rates = adjoint("f32", pick, sub_tgt)
    for j, b in enumerate(pick):
        assert np.array_equal(d_rho[b * N:(b + 1) * N], s_rho[j * N:(j + 1) * N])
        assert np.array_equal(d_u[b * N:(b + 1) * N], s_u[j * N:(j + 1) * N])
        assert np.array_equal(d_rates[b], s_rates[j])

    tgt64 = target("f64", pick)
    _, g_rho, g_u, _ = adjoint("f64", pick, tgt64)
    lat = lbm.Lattice(np.full(2, N), s_e=1.5)
    lat.set_state(rho[pick].ravel(), u[pick].ravel(), p[pick].ravel())
    s0 = np.asarray(lat.moments(device=False)[2]) / rho[pick].ravel()
    lat.close()

    def L(r, v):
        x = lbm.Lattice(np.full(2, N), s_e=1.5)
        x.set_state_entropy(r, v, s0)
        x.step(T)
        out = float(np.sum((np.asarray(x.moments(device=False)[0]) - tgt64) ** 2))
        x.close()
        return out

    rng = np.random.default_rng(2370)
    r0, u0 = rho[pick].ravel(), u[pick].ravel()
    h = 1e-6
    for _ in range(8):
        vr, vu = rng.standard_normal(r0.size), rng.standard_normal(r0.size)
        fdiff = (L(r0 + h * vr, u0 + h * vu) - L(r0 - h * vr, u0 - h * vu)) / (2 * h)
        grad = np.dot(g_rho, vr) + np.dot(g_u, vu)
        assert abs(grad - fdiff) <= 1e-6 * abs(grad), (grad, fdiff)


@pytest.mark.parametrize("T", [37, 50, 64])
def test_adjoint_depths_agree(lbm, T):
    """The backward sweep gives the same gradients for 1, 2, 4 or 8 reverse steps per launch. In FP64
    the forward recomputation on chip is bitwise that of the step kernel, so dL/drho0 and dL/du0 are
    bitwise equal and only the summation order of the rate gradients differs. The segment lengths
    round(sqrt(T)) = 6, 7, 8 leave blocks of every length from 1 to 8."""
    lengths, bc, s_e, data, targets = _case()
    init = [np.concatenate([d[k] for d in data]) for k in range(3)]
    res = {}
    for prec in ("f64", "f32"):
        for K in (1, 2, 4, 8):
            lat = lbm.Lattice(lengths, s_e=s_e, bc=bc, precision=prec)
            lat.set_adjoint_config(K)
            assert lat.get_adjoint_config() == K
            lat.set_state_entropy(*init)
            res[prec, K] = lat.adjoint(T, np.concatenate(targets))
            lat.close()
    for K in (2, 4, 8):
        a, b = res["f64", K], res["f64", 1]
        assert a[0] == b[0]
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
        assert np.abs(a[3] - b[3]).max() <= 1e-13 * np.abs(b[3]).max()
        for i in (1, 2, 3):  # FP32: the inner states are recomputed in scalar lanes
            c, d = res["f32", K][i], res["f64", 1][i]
            assert np.abs(c - d).max() <= 2e-4 * np.abs(d).max(), (K, i)


def test_double_float_adjoint_matches_fp64(lbm):
    """A double-float context (LBM_F64_DF) runs its forward steps and the adjoint's recomputation and
    reverse steps in double-float: the gradients agree with the native FP64 adjoint to FP64-class
    accuracy, for every depth."""
    lengths, bc, s_e, data, targets = _case()
    init = [np.concatenate([d[k] for d in data]) for k in range(3)]
    res = {}
    for prec, K in (("f64", 1), ("f64df", 1), ("f64df", 4), ("f64df", 8)):
        lat = lbm.Lattice(lengths, s_e=s_e, bc=bc, precision=prec)
        lat.set_adjoint_config(K)
        lat.set_state_entropy(*init)
        res[prec, K] = lat.adjoint(50, np.concatenate(targets))
        lat.close()
    ref = res["f64", 1]
    for key in (("f64df", 1), ("f64df", 4), ("f64df", 8)):
        got = res[key]
        assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])
        for i in (1, 2, 3):
            assert np.abs(got[i] - ref[i]).max() <= 1e-10 * np.abs(ref[i]).max(), (key, i)
