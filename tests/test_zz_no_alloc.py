"""lbm_diagnostics_noalloc, the diagnostics entry point for callers that cannot allocate device
memory (it keeps its scratch in a fixed __device__ array), must give the same sums and flags as
lbm_diagnostics. Checked through the C-ABI on two calls in a row with different states, so that a
leftover from the first call would show in the second; at non-default physical parameters and lattice
velocity; and on states with a non-finite or a negative-density node, whose flag bits and status must
match. This file is collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_diagnostics_match_lbm_diagnostics():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_02369_gb300 import build, lbm
    from paper_1802_02369_gb300 import workloads as W

    build.build()
    N = 300_001                     # 37 scratch chunks, ragged last chunk
    rho, u, p = W.steepening_wave(N, 0.1, W.reference_pressure())
    lat = lbm.Lattice(N, s_e=1.3)
    lat.set_state(rho, u, p)
    for call, nsteps in enumerate((0, 120)):
        lat.step(nsteps)
        ref_sums, ref_flags, ref_rc = lat.diagnostics()
        fd = lat.populations(device=True).contiguous()
        sums = np.full(4, np.nan)
        flags = np.full(1, -1, dtype=np.int32)
        rc = lbm.diagnostics_noalloc(fd, N, 1.0, sums=sums, flags=flags, stream=lat.stream)
        assert rc == ref_rc == lbm.LBM_OK, (call, rc)
        np.testing.assert_allclose(sums, ref_sums[0], rtol=1e-12, atol=1e-12)
        assert flags[0] == ref_flags[0] == 0
        # Device outputs: same values, no host synchronisation inside the call.
        d_sums = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        d_flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rc = lbm.diagnostics_noalloc(fd, N, 1.0, sums=d_sums, flags=d_flags, stream=lat.stream)
        torch.cuda.synchronize()
        assert rc == lbm.LBM_OK
        np.testing.assert_allclose(d_sums.cpu().numpy(), ref_sums[0], rtol=1e-12, atol=1e-12)
        assert int(d_flags.item()) == 0
    lat.close()
    # Sizes beyond the fixed scratch are refused before any work is enqueued.
    big = torch.empty(6, dtype=torch.float64, device="cuda")
    rc = lbm.load_library().lbm_diagnostics_noalloc(big.data_ptr(), (1 << 26) + 1, 1.0, None,
                                                    np.zeros(4).ctypes.data, np.zeros(1, np.int32).ctypes.data, None)
    assert rc == lbm.LBM_ERR_TOO_LARGE


PHYS = dict(gamma=1.3, Pr=0.71, cp=2.5, rho0=1.3, p0=0.21, s0=-0.1)


def test_noalloc_diagnostics_nondefault_physics():
    """A context created with non-default lbm_phys (s0 != 0 so the stored populations are shifted by a
    non-zero g rest state; explicit p0; rho0, c_p, gamma away from 1, 1, 1.4) at lambda = 2: the entry
    point, given the same parameters, returns lbm_diagnostics' sums (absolute zeta summed directly,
    against the library's rest-state zeta plus the shifted sum) on two calls in a row."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_02369_gb300 import build, lbm

    build.build()
    N, lam = 50_003, 2.0
    x = 2 * np.pi * np.arange(N) / N
    rho = PHYS["rho0"] * (1 + 0.02 * np.sin(x))
    u = lam * 0.02 * np.cos(x)
    s = PHYS["s0"] + PHYS["cp"] * 0.02 * np.sin(2 * x)
    lat = lbm.Lattice(N, lam=lam, s_e=1.4, phys=PHYS)
    lat.set_state_entropy(rho, u, s)
    ph = lbm._phys_struct(PHYS)
    for call, nsteps in enumerate((0, 75)):
        lat.step(nsteps)
        ref_sums, ref_flags, ref_rc = lat.diagnostics()
        fd = lat.populations(device=True).contiguous()
        sums = np.full(4, np.nan)
        flags = np.full(1, -1, dtype=np.int32)
        rc = lbm.diagnostics_noalloc(fd, N, lam, phys=ph, sums=sums, flags=flags, stream=lat.stream)
        assert rc == ref_rc == lbm.LBM_OK, (call, rc)
        np.testing.assert_allclose(sums, ref_sums[0], rtol=1e-12, atol=1e-12 * N)
        assert flags[0] == ref_flags[0] == 0
    lat.close()


def test_noalloc_diagnostics_flags_match():
    """A population made non-finite, then a node with negative density, written from the host with
    lbm_set_populations: the entry point sets the same flag bits as lbm_diagnostics and, with host
    outputs, returns LBM_ERR_UNSTABLE like it; with device outputs it only enqueues and the flags appear
    in device memory."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_02369_gb300 import build, lbm
    from paper_1802_02369_gb300 import workloads as W

    build.build()
    N = 20_000
    rho, u, p = W.steepening_wave(N, 0.05, W.reference_pressure())
    lat = lbm.Lattice(N, s_e=1.3)
    lat.set_state(rho, u, p)
    good = lat.populations()
    for bad_node, make_bad in ((123, lambda f: f.__setitem__((1, 123), np.nan)),
                               (19_999, lambda f: f[:3, 19_999].__imul__(-1.0))):
        f = good.copy()
        make_bad(f)
        lat.set_populations(np.ascontiguousarray(f))
        ref_sums, ref_flags, ref_rc = lat.diagnostics()
        assert ref_rc == lbm.LBM_ERR_UNSTABLE and ref_flags[0] != 0
        fd = lat.populations(device=True).contiguous()
        sums = np.zeros(4)
        flags = np.zeros(1, dtype=np.int32)
        rc = lbm.diagnostics_noalloc(fd, N, 1.0, sums=sums, flags=flags, stream=lat.stream)
        assert rc == lbm.LBM_ERR_UNSTABLE, (bad_node, rc)
        assert flags[0] == ref_flags[0], (bad_node, flags[0], ref_flags[0])
        d_sums = torch.zeros(4, dtype=torch.float64, device="cuda")
        d_flags = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc = lbm.diagnostics_noalloc(fd, N, 1.0, sums=d_sums, flags=d_flags, stream=lat.stream)
        torch.cuda.synchronize()
        assert rc == lbm.LBM_OK and int(d_flags.item()) == int(ref_flags[0])
    lat.close()
