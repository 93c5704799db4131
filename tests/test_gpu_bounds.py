"""The bounds-checked debug build: the library compiled with -DLBM_DEBUG_BOUNDS checks every global and
shared-memory index of the step, persistent, double-float, adjoint, two- and three-dimensional kernels before
the access, and counts instead of faulting. The edge-size parity tests (lattices of 3 to 4099 nodes on
every tile shape and depth, ragged periodic and bounce-back batches, paired FP32 lanes at walls and
joints, the vector and per-node memory paths, the persistent and graph modes with their bounded waits,
the linear variant, the double-float kernels, the adjoint at every depth, the two- and three-dimensional
kernels on ragged and tiny lattices and every configuration of the latter) run again in a child process on that build, and every one must leave the
record empty."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SELECTION = [
    ("tests/test_gpu_parity.py", "small_and_ragged or paired_lane or batched_ragged or persistent_and_graph "
                                 "or wait_timeout or linear_variant or sod_fp64 or vector_and_per_node"),
    ("tests/test_gpu_df.py", "configurations_agree or paired_lanes or ragged_bounce or sod_against or modes_and"),
    ("tests/test_gpu_adjoint.py", "dual_numbers or depths_agree or double_float or fp32_close"),
    ("tests/test_gpu_phys.py", "per_lattice"),
    ("tests/test_gpu_2d.py", "fp64_populations or fp32_matches or one_dimensional or source_off"),
    ("tests/test_gpu_3d.py", "fp64_populations or configurations_agree or fp32_matches or one_dimensional"),
]


def test_debug_bounds_build_edge_cases_have_no_violations():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_02369_gb300 import build

    lib = build.build(debug_bounds=True)
    env = dict(os.environ, LBM_LIBRARY=lib, LBM_BOUNDS_CHECK="1")
    # The debug build reports a count (0), not the -1 of a build without checks.
    probe = ("from paper_1802_02369_gb300 import lbm; import torch; torch.zeros(1, device='cuda'); "
             "print(lbm.debug_bounds()[0])")
    r = subprocess.run([sys.executable, "-c", probe], env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().splitlines()[-1] == "0", r.stdout + r.stderr
    for path, expr in SELECTION:
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                            os.path.join(ROOT, path), "-k", expr], env=env, cwd=ROOT, capture_output=True,
                           text=True, timeout=1500)
        assert r.returncode == 0, f"{path}:\n{r.stdout[-3000:]}\n{r.stderr[-2000:]}"
        assert " passed" in r.stdout, r.stdout[-2000:]
