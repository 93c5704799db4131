"""The double-float precision mode (LBM_F64_DF: FP64 storage, the time step in double-float on the
FP32 pipes): its arithmetic against FP64, and the step against the FP64 oracle at the FP64 tolerance.

The double-float operations are checked on inputs x' = hi + lo (the input split into two floats),
against numpy's FP64 evaluation of the same function at x'. The step is checked like the FP64 path:
|a - b| <= 1e-12 max(|b|, S) per moment with S its natural scale."""
import os

import numpy as np
import pytest

from paper_1802_02369_gb300 import workloads as W

pytestmark = pytest.mark.gpu
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_02369_gb300 import build, lbm as L

    build.build()
    return L


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _split(x):
    hi = x.astype(np.float32).astype(np.float64)
    return hi + (x - hi).astype(np.float32).astype(np.float64)


def _eval(lbm, fn, x, x2=None):
    import torch

    lib = lbm.load_library()
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    x2d = None if x2 is None else torch.from_numpy(np.ascontiguousarray(x2)).cuda()
    yd = torch.empty_like(xd)
    rc = lib.lbm_debug_eval_df(xd.data_ptr(), None if x2d is None else x2d.data_ptr(), yd.data_ptr(), x.size, fn,
                               None)
    assert rc == 0
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("fn,ref,lim", [(0, np.log1p, 0.3), (1, np.expm1, 0.35)])
def test_series_accuracy(lbm, fn, ref, lim):
    rng = np.random.default_rng(5)
    x = np.concatenate([np.linspace(-lim, lim, 100001), rng.uniform(-lim, lim, 100000),
                        [0.0, 1e-30, -1e-20, 1e-9, lim, -lim]])
    xs = _split(x)
    exact = ref(xs)
    got = _eval(lbm, fn, x)
    rel = np.abs(got - exact) / np.maximum(np.abs(exact), 1e-300)
    assert rel.max() <= 2.0 ** -45, rel.max()
    # Outside the series range: FP64 evaluation, rounded to double-float.
    wide = rng.uniform(0.31, 5.0, 1000) * rng.choice([-1.0, 1.0], 1000)
    wide = wide[wide > -0.95] if fn == 0 else wide
    got = _eval(lbm, fn, wide)
    exact = ref(_split(wide))
    assert (np.abs(got - exact) / np.abs(exact)).max() <= 2.0 ** -46


def test_fp64_lane_functions(lbm):
    """The FP64 lanes of the LBM_F64 node update: log1p and expm1 evaluated in double-float from the FP64
    argument (its split into hi + lo loses under 2^-48 of it) against numpy's FP64 functions of the
    argument itself, and the reciprocal (an FP32 estimate and two FP64 Newton steps) against 1/x, over
    the node update's ranges (densities and temperatures of order one) and across the series limits."""
    rng = np.random.default_rng(9)
    for fn, ref, lim in ((6, np.log1p, 0.3), (7, np.expm1, 0.35)):
        x = np.concatenate([np.linspace(-lim, lim, 100001), rng.uniform(-lim, lim, 100000),
                            rng.uniform(0.3, 3.0, 20000) * rng.choice([-1.0, 1.0], 20000),
                            [0.0, 1e-30, -1e-20, 1e-9, lim, -lim]])
        if fn == 6:
            x = x[x > -0.9]
        got = _eval(lbm, fn, x)
        exact = ref(x)
        rel = np.abs(got - exact) / np.maximum(np.abs(exact), 1e-300)
        assert rel.max() <= 2.0 ** -44, (fn, rel.max())
    x = np.concatenate([np.linspace(0.05, 5.0, 200001), 10.0 ** rng.uniform(-3, 3, 100000), [1.0, 2.0, 0.75]])
    got = _eval(lbm, 8, x)
    assert (np.abs(got - 1.0 / x) / (1.0 / x)).max() <= 2.0 ** -51


def test_basic_operations_accuracy(lbm):
    rng = np.random.default_rng(6)
    n = 200000
    x = rng.uniform(-2, 2, n) * 10.0 ** rng.uniform(-3, 0, n)
    y = rng.uniform(-2, 2, n) * 10.0 ** rng.uniform(-3, 0, n)
    xs, ys = _split(x), _split(y)
    r = _eval(lbm, 2, 1.0 + np.abs(x))
    ex = 1.0 / _split(1.0 + np.abs(x))
    assert (np.abs(r - ex) / ex).max() <= 2.0 ** -45
    r = _eval(lbm, 3, x, y)
    assert (np.abs(r - xs * ys) / np.abs(xs * ys)).max() <= 2.0 ** -46
    r = _eval(lbm, 4, x, y)
    assert (np.abs(r - (xs + ys)) / (np.abs(xs) + np.abs(ys))).max() <= 2.0 ** -46
    r = _eval(lbm, 5, x, y)
    ex = xs * ys + np.roll(ys, -1)
    # One normalisation after the exact product and the sum: a few units of 2^-48.
    assert (np.abs(r - ex) / (np.abs(xs * ys) + np.abs(np.roll(ys, -1)))).max() <= 2.0 ** -45


def _scales():
    return np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1.0])


def _err(g, ref):
    g = np.stack([np.asarray(v) for v in g], axis=1)
    return (np.abs(g - ref) / np.maximum(np.abs(ref), _scales()[None, :])).max()


def _run(lbm, rho, u, p, T, s_e, precision, config=None, bc=0):
    lat = lbm.Lattice(rho.size, s_e=s_e, bc=bc, precision=precision)
    if config:
        lat.set_config(*config)
    lat.set_state(rho, u, p)
    lat.step(T)
    m = lat.moments(device=False)
    fd = lat.populations()
    lat.close()
    return m, fd


@pytest.mark.parametrize("config", [(1, 128, 1), (2, 256, 1), (4, 256, 2), (8, 512, 2), (8, 128, 1), (4, 256, 4),
                                    (8, 128, 4)])
def test_steepening_wave_1000_steps_against_oracle(O, lbm, config):
    ph = O.default_phys()
    N = (1 << 14) + 77
    rho, u, p = W.steepening_wave(N, 0.1, ph.p0)
    ref = O.moments(ph, O.run(ph, O.coupled_rates(1.2), O.init(ph, rho, u, p=p), 1000, NTHREADS))
    m, _ = _run(lbm, rho, u, p, 1000, 1.2, "f64df", config)
    assert _err(m, ref) <= 1e-12


def test_configurations_agree(lbm):
    """Every double-float operation is an explicit round-to-nearest FP32 instruction, so tiles of any
    shape give bitwise the same state for the same steps per launch. Between launches the state is
    stored as hi + lo in FP64 and split again on the next load: the value is kept exactly, but a pair
    with |lo| = ulp(hi)/2 may come back as the other pair of the same sum, so different depths agree to
    rounding only."""
    rho, u, p = W.steepening_wave(5000, 0.1, W.reference_pressure())
    same_k = [_run(lbm, rho, u, p, 64, 1.3, "f64df", cfg)[1]
              for cfg in ((4, 128, 1), (4, 256, 2), (4, 512, 1), (4, 128, 4), (4, 512, 4))]
    for st in same_k[1:]:
        assert np.array_equal(same_k[0], st)
    other_k = [_run(lbm, rho, u, p, 64, 1.3, "f64df", cfg)[1] for cfg in ((1, 128, 1), (8, 256, 2))]
    for st in other_k:
        assert np.abs(st - same_k[0]).max() <= 1e-14


def test_paired_lanes_equal_scalar_lanes_with_walls_and_fallbacks(lbm):
    """Two and four nodes per thread run on paired df2 lanes, one node per thread on scalar df lanes:
    the same FP32 operations lane by lane, so the states are bitwise equal, also at bounce-back walls,
    at lattice joints of a ragged batch, and where only one node of a pair takes the FP64 fallback of
    log1p / expm1 (|rho/rho0 - 1| > 0.3 on alternate nodes)."""
    bat = W.ragged_batch(13, 5, W.reference_pressure(), n_min=33, n_max=900)
    rng = np.random.default_rng(21)
    n = int(np.sum(bat.lengths))
    rho = 1 + 0.02 * rng.standard_normal(n)
    rho[::2] += 0.45  # every other node outside the series ranges
    u = 0.02 * rng.standard_normal(n)
    p = W.reference_pressure() * rho ** 1.4
    out = []
    for cfg in ((2, 128, 1), (2, 128, 2), (2, 256, 4)):
        lat = lbm.Lattice(bat.lengths, s_e=bat.s_e, bc=bat.bc, precision="f64df")
        lat.set_config(*cfg)
        lat.set_state(rho, u, p)
        lat.step(6)
        out.append(lat.populations())
        lat.close()
    assert np.all(np.isfinite(out[0]))
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


@pytest.mark.parametrize("s_e,T", [(1.5, 100), (1.2, 500), (1.0, 500)])
def test_sod_against_oracle(O, lbm, s_e, T):
    ph = O.default_phys()
    rho, u, p = W.sod(256, ph.p0)
    ref = O.moments(ph, O.run(ph, O.coupled_rates(s_e), O.init(ph, rho, u, p=p), T))
    m, _ = _run(lbm, rho, u, p, T, s_e, "f64df", (2, 128, 1))
    assert _err(m, ref) <= 1e-12


def test_ragged_bounce_back_batch_against_native_fp64(lbm):
    """Ragged lattices with both boundary kinds, double-float against the native FP64 kernel: smooth
    random data over 300 steps, and the Riemann data of the batched workload (|rho/rho0 - 1| up to 0.7:
    the FP64 fallback of log1p and expm1) over 5 steps, before its discontinuities blow up (which they
    do in both precisions alike within 30 steps at these rates)."""
    bat = W.ragged_batch(24, 99, W.reference_pressure(), n_min=40, n_max=3000)
    rng = np.random.default_rng(8)
    smooth = []
    for n, b in zip(bat.lengths, bat.bc):
        x = 2 * np.pi * (np.arange(n) + 0.5) / n
        a = rng.uniform(0.01, 0.05, 3)
        rho = 1 + a[0] * np.sin(x + rng.uniform(0, 6))
        u = a[1] * (np.sin(x / 2) if b else np.sin(x + rng.uniform(0, 6)))
        p = W.reference_pressure() * rho ** 1.4 * (1 + a[2] * np.cos(x))
        smooth.append((rho, u, p))
    cases = [([np.concatenate([c[k] for c in smooth]) for k in range(3)], 300),
             ([bat.rho, bat.u, bat.p], 5)]
    for fields, T in cases:
        out = {}
        for prec in ("f64", "f64df"):
            lat = lbm.Lattice(bat.lengths, s_e=bat.s_e, bc=bat.bc, precision=prec)
            lat.set_state(*fields)
            lat.step(T)
            out[prec] = np.stack(lat.moments(device=False), axis=1)
            _, flags, _ = lat.diagnostics()
            assert np.all(flags == 0)
            lat.close()
        err = (np.abs(out["f64df"] - out["f64"]) / np.maximum(np.abs(out["f64"]), 1.0)).max()
        assert err <= 1e-12, (T, err)


def test_full_size_sampled_windows(O, lbm):
    """N = 2^26, 1000 steps, autotuned: sampled windows against the oracle (a node after T steps
    depends on the initial data within 2T nodes)."""
    import torch

    ph = O.default_phys()
    N, T = 1 << 26, 1000
    rho, u, p = W.steepening_wave(N, 0.1, ph.p0)
    lat = lbm.Lattice(N, s_e=1.2, precision="f64df")
    lat.set_state(rho, u, p)
    lat.autotune(1)
    lat.set_state(rho, u, p)
    lat.step(T)
    g = [x.cpu().numpy() for x in lat.moments(device=True)]
    lat.close()
    torch.cuda.empty_cache()
    r = O.coupled_rates(1.2)
    for c in (0, N // 2 + 5, N - 33):
        idx = (np.arange(c - 2 * T - 32, c + 2 * T + 32)) % N
        ref = O.moments(ph, O.run(ph, r, O.init(ph, rho[idx], u[idx], p=p[idx]), T, NTHREADS))[2 * T:2 * T + 64]
        assert _err([x[idx[2 * T:2 * T + 64]] for x in g], ref) <= 1e-12, c


def test_modes_and_configs(lbm):
    lat = lbm.Lattice(1000, precision="f64df")
    with pytest.raises(lbm.LbmError):
        lat.set_mode("persistent")
    with pytest.raises(lbm.LbmError):
        lat.set_config(4, 256, 8)
    lat.set_state(np.ones(1000), np.zeros(1000), np.full(1000, W.reference_pressure()))
    k, nt, v = lat.autotune(1)
    assert k in (1, 2, 4, 8) and nt in (128, 256, 512) and v in (1, 2, 4)
    lat.close()
