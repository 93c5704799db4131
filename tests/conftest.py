import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for p in (ROOT, os.path.join(ROOT, "tests")):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built liblbm.so")


GOLDEN = os.path.join(ROOT, "tests", "golden")


def read_symbolic_matrix(name: str, **symbols):
    """Parses a golden matrix file (comment lines start with '#'; an optional 'prefactor X' line)."""
    import numpy as np

    rows, pref = [], 1.0
    env = {"__builtins__": {}}
    env.update(symbols)
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("prefactor"):
                pref = float(eval(line.split()[1], env))  # noqa: S307 - fixed local fixture
                continue
            rows.append([float(eval(tok, env)) for tok in line.split()])  # noqa: S307
    return pref * np.array(rows)


def read_params(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [float(v) for v in vals] if len(vals) > 1 else float(vals[0])
    return out


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(autouse=True)
def _bounds_record(request):
    """Under the bounds-checked debug build (LBM_BOUNDS_CHECK=1, the library chosen by LBM_LIBRARY), every
    GPU test must leave the library's record of out-of-range indices empty, and the build must have the
    checks compiled in."""
    yield
    if os.environ.get("LBM_BOUNDS_CHECK") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    from paper_1802_02369_gb300 import lbm

    violations, index, extent = lbm.debug_bounds()
    assert violations == 0, f"{violations} out-of-range accesses (first index {index}, extent {extent})"
