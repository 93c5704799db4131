"""The FP32 series used on paired lanes (log1p by the atanh series, expm1 by its Taylor series)
against FP64 and against CUDA's log1pf / expm1f, on their whole ranges and across the switch to
CUDA's functions; the FP32 reciprocal against FP64."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _eval(x, fn):
    import torch
    from paper_1802_02369_gb300 import build, lbm

    build.build()
    lib = lbm.load_library()
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    yd = torch.empty_like(xd)
    assert lib.lbm_debug_eval_f32(xd.data_ptr(), yd.data_ptr(), xd.numel(), fn, None) == 0
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("fn_pair,fn_cuda,ref,lim", [(0, 1, np.log1p, 0.3), (2, 3, np.expm1, 0.35)])
def test_paired_series_accuracy(fn_pair, fn_cuda, ref, lim):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(3)
    wide = rng.uniform(-0.95, 3.0, 200000) if fn_pair == 0 else rng.uniform(-6.0, 6.0, 200000)
    x = np.concatenate([np.linspace(-lim, lim, 200001), wide,
                        [-lim, lim, 0.0, 1e-30, -1e-20, 1e-7, 0.30001, -0.30001, 0.35001, -0.35001]]).astype(np.float32)
    x32 = x.astype(np.float64)
    exact = ref(x32)
    pair, cuda = _eval(x, fn_pair), _eval(x, fn_cuda)
    ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
    err_pair = np.abs(pair - exact) / ulp
    err_cuda = np.abs(cuda - exact) / ulp
    assert err_pair.max() <= 4.0, err_pair.max()
    assert err_cuda.max() <= 4.0
    # On the series range the paired result stays within 4 ulp of CUDA's function.
    inr = np.abs(x32) <= lim
    assert (np.abs(pair - cuda)[inr] / ulp[inr]).max() <= 4.0


def test_reciprocal_accuracy():
    """The FP32 reciprocal of the node update (densities 1 + r, 2 + t, temperatures theta: positive and
    of order one, here over 1e-6 .. 1e6) within 2 ulp of the exact reciprocal of its FP32 input."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(5)
    x = np.concatenate([np.linspace(0.05, 4.0, 300001), 10.0 ** rng.uniform(-6, 6, 200000),
                        [1.0, 2.0, 0.5, 1.5, np.nextafter(np.float32(1), np.float32(2))]]).astype(np.float32)
    exact = 1.0 / x.astype(np.float64)
    got = _eval(x, 4)
    ulp = np.spacing(exact.astype(np.float32)).astype(np.float64)
    assert (np.abs(got - exact) / ulp).max() <= 2.0
