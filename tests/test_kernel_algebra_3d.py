"""The three-dimensional kernel's node update, built for the host and checked against the oracle without
a GPU: its equilibria and D3Q19 / D3Q7 inverses give the oracle's equilibrium populations (within
1e-15) at random states, default and non-default physics, and moments -> populations -> moments is the
identity to rounding; and full time steps run with the kernel's own node functions, neighbour
differences and push streaming follow the oracle within 1e-13 on a small periodic lattice."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle.d3q19q7 as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    from paper_1802_02369_gb300 import build

    lib = build.build()
    exe = str(tmp_path_factory.mktemp("alg") / "host_algebra_3d")
    libdir = os.path.dirname(lib)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17",
                    "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(ROOT, "tests", "host_algebra_3d.cu"), "-L", libdir, "-llbm",
                    f"-Xlinker=-rpath={libdir}"], check=True, capture_output=True)
    return exe


@pytest.mark.parametrize("kw", [dict(), dict(gamma=1.3, Pr=0.71, cp=2.5, rho0=1.3, lam=2.0, s0=-0.1)])
def test_equilibrium_populations_and_round_trip(harness, kw):
    rng = np.random.default_rng(3)
    ph = D.default_phys(**kw)
    M = 64
    rho = ph.rho0 * (1 + 0.1 * rng.standard_normal(M))
    u = 0.1 * ph.lam * rng.standard_normal((3, M))
    s = ph.s0 + 0.05 * ph.cp * rng.standard_normal(M)
    lines = [f"{M} {ph.gamma!r} {ph.Pr!r} {ph.cp!r} {ph.rho0!r} {ph.s0!r} {ph.lam!r}"]
    lines += [" ".join(repr(float(v)) for v in (rho[i], u[0, i], u[1, i], u[2, i], s[i])) for i in range(M)]
    out = subprocess.run([harness], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    vals = np.array([[float(x) for x in line.split()] for line in out.stdout.strip().split("\n")])
    B = lambda a: np.broadcast_to(a.reshape(1, 1, -1), (3, 3, M)).copy()
    ref = D.init(ph, B(rho), B(u[0]), B(u[1]), B(u[2]), B(s))[0, 0]
    assert np.abs(vals[:, :26] - ref).max() <= 1e-15 * max(1.0, ph.rho0)
    assert vals[:, 26].max() <= 1e-13


@pytest.mark.parametrize("kw", [dict(), dict(gamma=1.3, Pr=0.71, cp=2.5, rho0=1.3, lam=2.0, s0=-0.1)])
def test_host_steps_follow_the_oracle(harness, kw):
    from paper_1802_02369_gb300 import workloads as W

    ph = D.default_phys(**kw)
    nx, ny, nz, T, s_e = 7, 5, 4, 6, 1.3
    fields = W.waves_3d(nx, ny, nz, 9, amp=0.05, lam=ph.lam, rho0=ph.rho0, cp=ph.cp, s0=ph.s0)
    head = f"{nx} {ny} {nz} {T} {ph.gamma!r} {ph.Pr!r} {ph.cp!r} {ph.rho0!r} {ph.s0!r} {ph.lam!r} {s_e!r}"
    flat = [a.reshape(-1) for a in fields]
    lines = [head] + [" ".join(repr(float(a[i])) for a in flat) for i in range(nx * ny * nz)]
    out = subprocess.run([harness, "step"], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True)
    got = np.array([[float(x) for x in line.split()] for line in out.stdout.strip().split("\n")])
    ref = D.run(ph, D.rates(s_e, ph.gamma, ph.Pr), D.init(ph, *fields), T).reshape(-1, 26)
    assert np.abs(got - ref).max() <= 1e-13 * max(1.0, ph.rho0)
