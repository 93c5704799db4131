"""lbm_diagnostics_noalloc, the diagnostics entry point for callers that cannot allocate device
memory (it keeps its scratch in a fixed __device__ array), must give the same sums and flags as
lbm_diagnostics. Checked through the C-ABI on two calls in a row with different states, so that a
leftover from the first call would show in the second. This file is collected last."""
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
