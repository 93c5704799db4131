"""The C-ABI library builds for sm_103a, loads, and exports every function include/*.h declares.
No compute call is made (no GPU here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1802_02369_gb300 import build

    return build.build()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(lbm(?:[23]d)?_[a-z_0-9]+)\s*\(", txt))
    return sorted(names - {"lbm_alloc_fn", "lbm_free_fn"})


def test_library_exports_every_declared_function(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_declares_the_same_functions(lib_path):
    from paper_1802_02369_gb300 import lbm

    lib = lbm.load_library(lib_path)
    assert lbm.header_functions() == _declared()
    for n in _declared():
        assert getattr(lib, n).argtypes is not None or n in ("lbm_destroy",)
    assert any(n.startswith("lbm2d_") for n in _declared())
    assert any(n.startswith("lbm3d_") for n in _declared())


def test_invalid_arguments_are_rejected_without_gpu(lib_path):
    """Argument validation happens before any CUDA call."""
    from paper_1802_02369_gb300 import lbm

    lib = lbm.load_library(lib_path)
    ctx = ctypes.c_void_p()
    r = lbm.lbm_rates(1.5, 0.0, 0.0)
    assert lib.lbm_create(ctypes.byref(ctx), 2, 1.0, ctypes.byref(r), 0, 0, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_create(ctypes.byref(ctx), 64, 0.0, ctypes.byref(r), 0, 0, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_create(ctypes.byref(ctx), 64, 1.0, ctypes.byref(r), 7, 0, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_create(ctypes.byref(ctx), 64, 1.0, ctypes.byref(r), 0, 5, None, None) == lbm.LBM_ERR_INVALID_ARG
    bad = lbm.lbm_rates(2.0, 0.0, 0.0)
    assert lib.lbm_create(ctypes.byref(ctx), 64, 1.0, ctypes.byref(bad), 0, 0, None, None) == lbm.LBM_ERR_INVALID_ARG
    bad = lbm.lbm_rates(1.5, 2.5, 0.0)
    assert lib.lbm_create(ctypes.byref(ctx), 64, 1.0, ctypes.byref(bad), 0, 0, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_step(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_total_nodes(None) == -1
    # The two-dimensional scheme.
    ok2 = dict(gamma=1.4, Pr=1.0, cp=1.0, rho0=1.0, p0=0.0, s0=0.0, lam=1.0, dx=1.0, beta=0.0, s_e=1.2,
               s_psi=0.0, s_eps=0.0, s_q=0.0, s_h=0.0, source_on=1, pad=0)
    for change in (dict(s_e=2.0), dict(gamma=1.0), dict(lam=0.0), dict(s_q=2.5), dict(rho0=-1.0), dict(Pr=0.0)):
        p2 = lbm.lbm2d_params(**{**ok2, **change})
        assert lib.lbm2d_create(ctypes.byref(ctx), 16, 16, ctypes.byref(p2), 0, None) == lbm.LBM_ERR_INVALID_ARG, change
    p2 = lbm.lbm2d_params(**ok2)
    assert lib.lbm2d_create(ctypes.byref(ctx), 2, 16, ctypes.byref(p2), 0, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm2d_create(ctypes.byref(ctx), 16, 16, ctypes.byref(p2), 3, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm2d_create(ctypes.byref(ctx), 16, 4 * 65535 + 1, ctypes.byref(p2), 0, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm2d_step(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm2d_steps_done(None) == -1
    # The three-dimensional scheme: same parameter checks, sizes and precisions.
    for change in (dict(s_e=2.0), dict(gamma=1.0), dict(lam=0.0), dict(s_h=2.5), dict(rho0=-1.0), dict(Pr=0.0),
                   dict(s_eps=-0.0 + 2.0), dict(cp=0.0)):
        p3 = lbm.lbm3d_params(**{**ok2, **change})
        assert lib.lbm3d_create(ctypes.byref(ctx), 16, 16, 16, ctypes.byref(p3), 0, None) == lbm.LBM_ERR_INVALID_ARG, change
    p3 = lbm.lbm3d_params(**ok2)
    for dims in ((2, 16, 16), (16, 2, 16), (16, 16, 2), (16, 4 * 65535 + 1, 16), (1 << 20, 1 << 10, 1 << 4)):
        assert lib.lbm3d_create(ctypes.byref(ctx), *dims, ctypes.byref(p3), 0, None) == lbm.LBM_ERR_INVALID_ARG, dims
    for precision in (3, -1):
        assert lib.lbm3d_create(ctypes.byref(ctx), 16, 16, 16, ctypes.byref(p3), precision, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm3d_create(None, 16, 16, 16, ctypes.byref(p3), 0, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm3d_create(ctypes.byref(ctx), 16, 16, 16, None, 0, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm3d_step(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm3d_steps_done(None) == -1
    assert lib.lbm3d_set_config(None, 8, 0, 0) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm3d_rates(None, None) == lbm.LBM_ERR_INVALID_ARG


def test_noalloc_pointer_placement_rule(lib_path):
    """lbm_diagnostics_noalloc accepts populations in device memory of the current device (or managed
    memory) and outputs both on the host or both on the current device; memory of another GPU, a host
    fd and mixed outputs are refused. The rule is evaluated by its test hook, with no CUDA call."""
    from paper_1802_02369_gb300 import lbm

    lib = lbm.load_library(lib_path)
    ok, bad = lbm.LBM_OK, lbm.LBM_ERR_INVALID_ARG
    H, D, M = 0, 1, 2
    cases = [
        ((0, D, 0, H, -1, H, -1), ok),      # device fd, host outputs
        ((0, D, 0, D, 0, D, 0), ok),        # everything on the current device
        ((1, D, 1, D, 1, M, 0), ok),        # device 1 current; managed flags
        ((0, M, 1, H, -1, H, -1), ok),      # managed fd allocated on another device
        ((0, H, -1, H, -1, H, -1), bad),    # host fd
        ((0, D, 1, H, -1, H, -1), bad),     # fd on another GPU
        ((1, D, 1, D, 0, D, 1), bad),       # sums on another GPU
        ((1, D, 1, D, 1, D, 0), bad),       # flags on another GPU
        ((0, D, 0, D, 0, H, -1), bad),      # mixed outputs
        ((0, D, 0, H, -1, M, 0), bad),
    ]
    for args, want in cases:
        assert lib.lbm_debug_noalloc_placement(*args) == want, args
