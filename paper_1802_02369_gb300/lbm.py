"""Python binding of the C-ABI in include/lbm.h (argument marshalling only).

Every step of the method runs in the CUDA library ``_build/liblbm.so``; this module loads it with
ctypes, installs PyTorch's caching allocator as the library's device allocator, and passes torch
streams and tensor pointers through. There is no fallback: if the library is missing or CUDA is
unavailable, the calls raise.

Function names follow the C-ABI (``lbm_create`` ...); :class:`Lattice` wraps a context.
Arrays may be numpy arrays (host memory, staged by the library) or torch tensors (device or host).
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the same library (the bounds-checked debug build of the tests).
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(HERE, "_build", "liblbm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "lbm.h")

LBM_OK = 0
LBM_ERR_INVALID_ARG = -1
LBM_ERR_CUDA = -2
LBM_ERR_OOM = -3
LBM_ERR_UNSTABLE = -4
LBM_ERR_TIMEOUT = -5
LBM_ERR_IO = -6
LBM_ERR_TOO_LARGE = -7
LBM_BC_PERIODIC = 0
LBM_BC_BOUNCEBACK = 1
LBM_F64 = 0
LBM_F32_SHIFTED = 1
LBM_F64_DF = 2
LBM_MODE_LAUNCH = 0
LBM_MODE_PERSISTENT = 1
LBM_MODE_PERSISTENT_GRAPH = 2
MODES = {"launch": LBM_MODE_LAUNCH, "persistent": LBM_MODE_PERSISTENT, "graph": LBM_MODE_PERSISTENT_GRAPH}
PRECISIONS = {"f64": LBM_F64, "f32": LBM_F32_SHIFTED, "f64df": LBM_F64_DF}


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class lbm_rates(ctypes.Structure):
    _fields_ = [("s_e", ctypes.c_double), ("s_psi", ctypes.c_double), ("s_eps", ctypes.c_double)]


class lbm_phys(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("cp", ctypes.c_double),
                ("rho0", ctypes.c_double), ("p0", ctypes.c_double), ("s0", ctypes.c_double),
                ("source_on", ctypes.c_int32), ("equilibria", ctypes.c_int32),
                ("u0_lin", ctypes.c_double), ("s0_lin", ctypes.c_double)]


LBM_D1Q3_FLUID = 0
LBM_D1Q3_ADVECTION_DIFFUSION = 1
D1Q3_SCHEMES = {"fluid": LBM_D1Q3_FLUID, "advection_diffusion": LBM_D1Q3_ADVECTION_DIFFUSION}


class lbm_d1q3_params(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("pad", ctypes.c_int32), ("lam", ctypes.c_double),
                ("scale", ctypes.c_double), ("s_e", ctypes.c_double), ("gamma", ctypes.c_double),
                ("p0", ctypes.c_double), ("u0", ctypes.c_double), ("alpha", ctypes.c_double),
                ("kappa", ctypes.c_double), ("s_psi", ctypes.c_double), ("s_eps", ctypes.c_double)]


class lbm2d_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("cp", ctypes.c_double),
                ("rho0", ctypes.c_double), ("p0", ctypes.c_double), ("s0", ctypes.c_double),
                ("lam", ctypes.c_double), ("dx", ctypes.c_double), ("beta", ctypes.c_double),
                ("s_e", ctypes.c_double), ("s_psi", ctypes.c_double), ("s_eps", ctypes.c_double),
                ("s_q", ctypes.c_double), ("s_h", ctypes.c_double),
                ("source_on", ctypes.c_int32), ("pad", ctypes.c_int32)]


class lbm3d_params(ctypes.Structure):
    _fields_ = lbm2d_params._fields_


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_lock = threading.Lock()
_callbacks = []


def header_functions() -> list[str]:
    """Names of the functions declared in include/lbm.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm(?:[23]d)?_[a-z_0-9]+)\s*\(", txt)) - {"lbm_alloc_fn", "lbm_free_fn"})


def load_library(path: str = LIB_PATH):
    """Loads liblbm.so and declares the signatures (no CUDA call is made)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"liblbm.so not built ({path}); run paper_1802_02369_gb300.build.build()")
        lib = ctypes.CDLL(path)
        i32, i64, d, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        P = ctypes.POINTER
        sig = {
            "lbm_set_allocator": (i32, [ALLOC_FN, FREE_FN, vp]),
            "lbm_create": (i32, [P(vp), i64, d, P(lbm_rates), i32, i32, P(lbm_phys), vp]),
            "lbm_create_batch": (i32, [P(vp), i32, P(i64), d, P(lbm_rates), P(i32), P(d), i32, P(lbm_phys), vp]),
            "lbm_destroy": (None, [vp]),
            "lbm_last_error": (ctypes.c_char_p, [vp]),
            "lbm_total_nodes": (i64, [vp]),
            "lbm_steps_done": (i64, [vp]),
            "lbm_set_state": (i32, [vp, vp, vp, vp]),
            "lbm_set_state_entropy": (i32, [vp, vp, vp, vp]),
            "lbm_step": (i32, [vp, i64]),
            "lbm_moments": (i32, [vp, vp, vp, vp, vp, vp, vp]),
            "lbm_get_populations": (i32, [vp, vp]),
            "lbm_set_populations": (i32, [vp, vp]),
            "lbm_diagnostics": (i32, [vp, P(d), P(i32)]),
            "lbm_set_config": (i32, [vp, i32, i32, i32]),
            "lbm_get_config": (i32, [vp, P(i32), P(i32), P(i32)]),
            "lbm_autotune": (i32, [vp, i32]),
            "lbm_save": (i32, [vp, ctypes.c_char_p]),
            "lbm_load": (i32, [vp, ctypes.c_char_p]),
            "lbm_diagnostics_noalloc": (i32, [vp, i64, d, P(lbm_phys), vp, vp, vp]),
            "lbm_debug_noalloc_placement": (i32, [i32] * 7),
            "lbm_set_mode": (i32, [vp, i32]),
            "lbm_debug_eval_f32": (i32, [vp, vp, i64, i32, vp]),
            "lbm_debug_eval_df": (i32, [vp, vp, vp, i64, i32, vp]),
            "lbm_adjoint_forward": (i32, [vp, i64]),
            "lbm_adjoint_backward": (i32, [vp, vp, vp, vp, vp, vp]),
            "lbm_adjoint": (i32, [vp, i64, vp, vp, vp, vp, vp]),
            "lbm_adjoint_release": (i32, [vp]),
            "lbm_adjoint_set_config": (i32, [vp, i32]),
            "lbm_adjoint_get_config": (i32, [vp, P(i32)]),
            "lbm_status": (i32, [vp]),
            "lbm_debug_persistent": (i32, [vp, i64, i64]),
            "lbm_debug_bounds": (i32, [P(i64), P(i64), P(i64)]),
            "lbm_fd_create": (i32, [P(vp), i64, d, d, d, i32, P(lbm_phys), vp]),
            "lbm_fd_destroy": (None, [vp]),
            "lbm_fd_last_error": (ctypes.c_char_p, [vp]),
            "lbm_fd_steps_done": (i64, [vp]),
            "lbm_fd_set_state": (i32, [vp, vp, vp, vp]),
            "lbm_fd_set_fields": (i32, [vp, vp]),
            "lbm_fd_step": (i32, [vp, i64]),
            "lbm_fd_fields": (i32, [vp, vp, vp, vp]),
            "lbm_fd_diagnostics": (i32, [vp, P(d), P(i32)]),
            "lbm_fd_set_config": (i32, [vp, i32, i32, i32]),
            "lbm_fd_get_config": (i32, [vp, P(i32), P(i32), P(i32)]),
            "lbm_fd_autotune": (i32, [vp, i32]),
            "lbm_d1q3_create": (i32, [P(vp), i64, P(lbm_d1q3_params), i32, vp]),
            "lbm_d1q3_destroy": (None, [vp]),
            "lbm_d1q3_last_error": (ctypes.c_char_p, [vp]),
            "lbm_d1q3_steps_done": (i64, [vp]),
            "lbm_d1q3_rates": (i32, [vp, P(d), P(d)]),
            "lbm_d1q3_set_state": (i32, [vp, vp, vp]),
            "lbm_d1q3_step": (i32, [vp, i64]),
            "lbm_d1q3_moments": (i32, [vp, vp, vp, vp]),
            "lbm_d1q3_get_populations": (i32, [vp, vp]),
            "lbm_d1q3_set_populations": (i32, [vp, vp]),
            "lbm_d1q3_sums": (i32, [vp, P(d), P(i32)]),
            "lbm_d1q3_set_config": (i32, [vp, i32, i32, i32]),
            "lbm_d1q3_get_config": (i32, [vp, P(i32), P(i32), P(i32)]),
            "lbm_d1q3_autotune": (i32, [vp, i32]),
            "lbm2d_create": (i32, [P(vp), i64, i64, P(lbm2d_params), i32, vp]),
            "lbm2d_destroy": (None, [vp]),
            "lbm2d_last_error": (ctypes.c_char_p, [vp]),
            "lbm2d_steps_done": (i64, [vp]),
            "lbm2d_rates": (i32, [vp, P(d)]),
            "lbm2d_set_state": (i32, [vp, vp, vp, vp, vp]),
            "lbm2d_step": (i32, [vp, i64]),
            "lbm2d_get_populations": (i32, [vp, vp]),
            "lbm2d_fields": (i32, [vp, vp, vp, vp, vp]),
            "lbm3d_create": (i32, [P(vp), i64, i64, i64, P(lbm3d_params), i32, vp]),
            "lbm3d_destroy": (None, [vp]),
            "lbm3d_last_error": (ctypes.c_char_p, [vp]),
            "lbm3d_steps_done": (i64, [vp]),
            "lbm3d_rates": (i32, [vp, P(d)]),
            "lbm3d_set_state": (i32, [vp, vp, vp, vp, vp, vp]),
            "lbm3d_step": (i32, [vp, i64]),
            "lbm3d_get_populations": (i32, [vp, vp]),
            "lbm3d_fields": (i32, [vp, vp, vp, vp, vp, vp]),
            "lbm3d_set_config": (i32, [vp, i32, i32, i32]),
            "lbm3d_get_config": (i32, [vp, P(i32), P(i32), P(i32)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("CUDA is not available: the D1Q3Q3 library runs on the GPU only")
    return torch


def install_torch_allocator():
    """Routes the library's device allocations through torch's caching allocator."""
    torch = _torch()
    lib = load_library()
    if _callbacks:
        return

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        except Exception:  # out of memory: the library reports LBM_ERR_OOM
            return None

    def _free(ptr, user):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _callbacks.extend([a, f])
    rc = lib.lbm_set_allocator(a, f, None)
    if rc != LBM_OK:
        raise LbmError(rc, "lbm_set_allocator failed")


def debug_bounds():
    """(violations, first index, its extent) of the bounds-checked debug build since the last call;
    violations = -1 for a build without the checks (lbm_debug_bounds)."""
    lib = load_library()
    v, i, n = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = lib.lbm_debug_bounds(ctypes.byref(v), ctypes.byref(i), ctypes.byref(n))
    if rc != LBM_OK:
        raise LbmError(rc, "lbm_debug_bounds failed")
    return v.value, i.value, n.value


def diagnostics_noalloc(fd, N: int, lam: float = 1.0, phys=None, sums=None, flags=None, stream=None) -> int:
    """lbm_diagnostics_noalloc: FP64 sums of one lattice from device populations fd ([6, N] float64
    torch tensor on the GPU) without any device allocation. sums/flags: numpy (host) or torch
    (device) outputs of 4 float64 / 1 int32. Returns the status code."""
    lib = load_library()
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    ph = None if phys is None else ctypes.byref(phys)

    def ptr(x):
        return x.data_ptr() if isinstance(x, torch.Tensor) else x.ctypes.data

    return lib.lbm_diagnostics_noalloc(ptr(fd), int(N), float(lam), ph, ptr(sums), ptr(flags),
                                       ctypes.c_void_p(st.cuda_stream))


class _Arr:
    """A host or device float64 array passed by pointer; keeps the owner alive."""

    def __init__(self, x, n: int, writable: bool = False):
        torch = None
        try:
            import torch as _t
            torch = _t
        except ImportError:
            pass
        if torch is not None and isinstance(x, torch.Tensor):
            if x.dtype != torch.float64 or not x.is_contiguous() or x.numel() != n:
                raise ValueError(f"expected a contiguous float64 tensor of {n} elements")
            self.obj, self.ptr = x, x.data_ptr()
        else:
            a = np.asarray(x)
            if writable:
                if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n:
                    raise ValueError(f"expected a contiguous float64 array of {n} elements")
            else:
                a = np.ascontiguousarray(a, dtype=np.float64)
                if a.size != n:
                    raise ValueError(f"expected {n} elements, got {a.size}")
            self.obj, self.ptr = a, a.ctypes.data


class Lattice:
    """One context: B >= 1 independent lattices advanced by the CUDA library.

    lengths: int or sequence of ints (>= 3). s_e: the free rate (scalar or per lattice).
    s_psi / s_eps: <= 0 selects the paper's coupling / 1.5. bc: 0 periodic, 1 bounce-back
    (scalar or per lattice). precision: "f64" or "f32" (FP32 shifted populations).
    s0: per-lattice reference entropy (None: phys["s0"]). phys: dict of lbm_phys fields
    (e.g. dict(equilibria=1, u0_lin=0.15, s0_lin=0.2, source_on=0) for the section 7 linear scheme).
    """

    def __init__(self, lengths, lam: float = 1.0, s_e=1.5, s_psi=0.0, s_eps=0.0, bc=0,
                 precision: str = "f64", phys: dict | None = None, s0=None, stream=None):
        torch = _torch()
        self.lib = load_library()
        install_torch_allocator()
        lengths = np.atleast_1d(np.asarray(lengths, dtype=np.int64))
        B = lengths.size
        s_e = np.broadcast_to(np.asarray(s_e, dtype=np.float64), (B,))
        s_psi = np.broadcast_to(np.asarray(s_psi, dtype=np.float64), (B,))
        s_eps = np.broadcast_to(np.asarray(s_eps, dtype=np.float64), (B,))
        bcs = np.ascontiguousarray(np.broadcast_to(np.asarray(bc, dtype=np.int32), (B,)))
        rates = (lbm_rates * B)(*[lbm_rates(float(a), float(b), float(c)) for a, b, c in zip(s_e, s_psi, s_eps)])
        ph = None
        if phys is not None:
            base = dict(gamma=1.4, Pr=1.0, cp=1.0, rho0=1.0, p0=0.0, s0=0.0, source_on=1, equilibria=0,
                        u0_lin=0.0, s0_lin=0.0)
            base.update(phys)
            ph = lbm_phys(**base)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.precision = PRECISIONS[precision]
        self.lengths = lengths
        self.B = B
        ctx = ctypes.c_void_p()
        s0_arr = None if s0 is None else np.ascontiguousarray(np.broadcast_to(np.asarray(s0, dtype=np.float64), (B,)))
        rc = self.lib.lbm_create_batch(
            ctypes.byref(ctx), B, lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), float(lam), rates,
            bcs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            None if s0_arr is None else s0_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            self.precision, None if ph is None else ctypes.byref(ph), ctypes.c_void_p(self.stream.cuda_stream))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_create_batch failed")
        self.ctx = ctx
        self.N = int(self.lib.lbm_total_nodes(ctx))
        self.offsets = np.r_[0, np.cumsum(lengths)]

    # -- helpers ---------------------------------------------------------------------------------
    def _check(self, rc: int, what: str):
        if rc != LBM_OK:
            raise LbmError(rc, f"{what}: {self.lib.lbm_last_error(self.ctx).decode()}")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C-ABI mirrors ---------------------------------------------------------------------------
    def set_state(self, rho, u, p):
        a, b, c = (_Arr(x, self.N) for x in (rho, u, p))
        self._check(self.lib.lbm_set_state(self.ctx, a.ptr, b.ptr, c.ptr), "lbm_set_state")

    def set_state_entropy(self, rho, u, s):
        a, b, c = (_Arr(x, self.N) for x in (rho, u, s))
        self._check(self.lib.lbm_set_state_entropy(self.ctx, a.ptr, b.ptr, c.ptr), "lbm_set_state_entropy")

    def step(self, nsteps: int):
        self._check(self.lib.lbm_step(self.ctx, int(nsteps)), "lbm_step")

    def moments(self, out=None, device: bool = True):
        """(rho, J, zeta, e, psi, eps) as six float64 arrays: torch tensors on the GPU (device=True)
        or numpy arrays (device=False). ``out`` may give six preallocated arrays (or None)."""
        torch = _torch()
        if out is None:
            if device:
                out = [torch.empty(self.N, dtype=torch.float64, device="cuda") for _ in range(6)]
            else:
                out = [np.empty(self.N) for _ in range(6)]
        arrs = [None if o is None else _Arr(o, self.N, writable=True) for o in out]
        ptrs = [None if a is None else a.ptr for a in arrs]
        self._check(self.lib.lbm_moments(self.ctx, *ptrs), "lbm_moments")
        return out

    def populations(self, device: bool = False):
        torch = _torch()
        out = torch.empty(6 * self.N, dtype=torch.float64, device="cuda") if device else np.empty(6 * self.N)
        a = _Arr(out, 6 * self.N, writable=True)
        self._check(self.lib.lbm_get_populations(self.ctx, a.ptr), "lbm_get_populations")
        return out.reshape(6, self.N)

    def set_populations(self, fd):
        a = _Arr(fd.reshape(-1) if hasattr(fd, "reshape") else fd, 6 * self.N)
        self._check(self.lib.lbm_set_populations(self.ctx, a.ptr), "lbm_set_populations")

    def diagnostics(self, raise_unstable: bool = False):
        """(sums [B, 4] = (sum rho, sum J, sum zeta, sum rho E), flags [B], status)."""
        sums = np.zeros((self.B, 4))
        flags = np.zeros(self.B, dtype=np.int32)
        rc = self.lib.lbm_diagnostics(self.ctx, sums.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      flags.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if rc not in (LBM_OK, LBM_ERR_UNSTABLE) or (raise_unstable and rc != LBM_OK):
            self._check(rc, "lbm_diagnostics")
        return sums, flags, rc

    def set_config(self, steps_per_launch: int = 0, block_threads: int = 0, nodes_per_thread: int = 0):
        self._check(self.lib.lbm_set_config(self.ctx, int(steps_per_launch), int(block_threads),
                                            int(nodes_per_thread)), "lbm_set_config")

    def get_config(self):
        """(steps_per_launch, block_threads, nodes_per_thread)."""
        k, nt, v = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.lbm_get_config(self.ctx, ctypes.byref(k), ctypes.byref(nt), ctypes.byref(v)),
                    "lbm_get_config")
        return k.value, nt.value, v.value

    # -- adjoint ---------------------------------------------------------------------------------
    def adjoint_forward(self, T: int):
        self._check(self.lib.lbm_adjoint_forward(self.ctx, int(T)), "lbm_adjoint_forward")

    def adjoint_backward(self, dL_drho_T, want_fd0: bool = False, device: bool = False):
        """Returns (dL/drho0 [N], dL/du0 [N], dL/drates [B, 2], dL/df0 [6, N] or None)."""
        torch = _torch()
        seed = _Arr(dL_drho_T, self.N)
        if device:
            out = [torch.empty(self.N, dtype=torch.float64, device="cuda") for _ in range(2)]
            fd0 = torch.empty(6 * self.N, dtype=torch.float64, device="cuda") if want_fd0 else None
        else:
            out = [np.empty(self.N) for _ in range(2)]
            fd0 = np.empty(6 * self.N) if want_fd0 else None
        rates = np.empty(2 * self.B)
        a = [_Arr(x, self.N, writable=True) for x in out]
        f = None if fd0 is None else _Arr(fd0, 6 * self.N, writable=True)
        self._check(self.lib.lbm_adjoint_backward(self.ctx, seed.ptr, a[0].ptr, a[1].ptr, rates.ctypes.data,
                                                  None if f is None else f.ptr), "lbm_adjoint_backward")
        return out[0], out[1], rates.reshape(self.B, 2), (None if fd0 is None else fd0.reshape(6, self.N))

    def adjoint(self, T: int, rho_target):
        """loss = sum (rho(T) - rho_target)^2 and its gradients: (loss, dL/drho0, dL/du0, dL/drates [B, 2])."""
        tgt = _Arr(rho_target, self.N)
        loss = np.zeros(1)
        drho, du = np.empty(self.N), np.empty(self.N)
        rates = np.empty(2 * self.B)
        self._check(self.lib.lbm_adjoint(self.ctx, int(T), tgt.ptr, loss.ctypes.data, drho.ctypes.data,
                                         du.ctypes.data, rates.ctypes.data), "lbm_adjoint")
        return float(loss[0]), drho, du, rates.reshape(self.B, 2)

    def adjoint_release(self):
        self._check(self.lib.lbm_adjoint_release(self.ctx), "lbm_adjoint_release")

    def set_adjoint_config(self, steps_per_launch: int = 0):
        """Reverse steps per launch of the backward sweep (1, 2, 4, 8; 0 = the default: 1 in FP64, else 4)."""
        self._check(self.lib.lbm_adjoint_set_config(self.ctx, int(steps_per_launch)), "lbm_adjoint_set_config")

    def get_adjoint_config(self) -> int:
        k = ctypes.c_int32()
        self._check(self.lib.lbm_adjoint_get_config(self.ctx, ctypes.byref(k)), "lbm_adjoint_get_config")
        return k.value

    def set_mode(self, mode: str):
        """"launch" (one kernel per k steps), "persistent" or "graph" (persistent, CUDA graph)."""
        self._check(self.lib.lbm_set_mode(self.ctx, MODES[mode]), "lbm_set_mode")

    def status(self) -> int:
        """Synchronises; LBM_OK or LBM_ERR_TIMEOUT if a bounded wait of a persistent launch expired."""
        return int(self.lib.lbm_status(self.ctx))

    def debug_persistent(self, spin_limit: int = 20000000, withhold_tile: int = -1):
        self._check(self.lib.lbm_debug_persistent(self.ctx, int(spin_limit), int(withhold_tile)),
                    "lbm_debug_persistent")

    def autotune(self, trials: int = 3):
        self._check(self.lib.lbm_autotune(self.ctx, int(trials)), "lbm_autotune")
        return self.get_config()

    def save(self, path: str):
        self._check(self.lib.lbm_save(self.ctx, path.encode()), "lbm_save")

    def load(self, path: str):
        self._check(self.lib.lbm_load(self.ctx, path.encode()), "lbm_load")

    @property
    def steps_done(self) -> int:
        return int(self.lib.lbm_steps_done(self.ctx))


def _phys_struct(phys: dict | None):
    if phys is None:
        return None
    base = dict(gamma=1.4, Pr=1.0, cp=1.0, rho0=1.0, p0=0.0, s0=0.0, source_on=1, equilibria=0,
                u0_lin=0.0, s0_lin=0.0)
    base.update(phys)
    return lbm_phys(**base)


class FdGrid:
    """Finite-difference comparison solver of section 9 (lbm_fd_* of the C-ABI): one periodic grid of
    N >= 3 nodes, spacing dx, time step dt, kinematic viscosity nu; precision "f64" or "f32".
    phys: dict of lbm_phys fields (gamma, Pr, cp, rho0, p0, s0, source_on); None = section 9 values."""

    def __init__(self, N: int, dx: float, dt: float, nu: float, precision: str = "f64",
                 phys: dict | None = None, stream=None):
        torch = _torch()
        self.lib = load_library()
        install_torch_allocator()
        ph = _phys_struct(phys)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.N = int(N)
        ctx = ctypes.c_void_p()
        rc = self.lib.lbm_fd_create(ctypes.byref(ctx), self.N, float(dx), float(dt), float(nu),
                                    PRECISIONS[precision], None if ph is None else ctypes.byref(ph),
                                    ctypes.c_void_p(self.stream.cuda_stream))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_fd_create failed")
        self.ctx = ctx

    def _check(self, rc: int, what: str):
        if rc != LBM_OK:
            raise LbmError(rc, f"{what}: {self.lib.lbm_fd_last_error(self.ctx).decode()}")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbm_fd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, rho, u, s):
        a, b, c = (_Arr(x, self.N) for x in (rho, u, s))
        self._check(self.lib.lbm_fd_set_state(self.ctx, a.ptr, b.ptr, c.ptr), "lbm_fd_set_state")

    def set_fields(self, W):
        """W: plane-major [3, N] (rho, J, zeta)."""
        a = _Arr(W.reshape(-1) if hasattr(W, "reshape") else W, 3 * self.N)
        self._check(self.lib.lbm_fd_set_fields(self.ctx, a.ptr), "lbm_fd_set_fields")

    def step(self, nsteps: int):
        self._check(self.lib.lbm_fd_step(self.ctx, int(nsteps)), "lbm_fd_step")

    def fields(self, device: bool = False):
        """(rho, J, zeta): torch tensors on the GPU (device=True) or numpy arrays."""
        torch = _torch()
        if device:
            out = [torch.empty(self.N, dtype=torch.float64, device="cuda") for _ in range(3)]
        else:
            out = [np.empty(self.N) for _ in range(3)]
        a = [_Arr(o, self.N, writable=True) for o in out]
        self._check(self.lib.lbm_fd_fields(self.ctx, a[0].ptr, a[1].ptr, a[2].ptr), "lbm_fd_fields")
        return out

    def diagnostics(self):
        """(sums [4] = (sum rho, sum J, sum zeta, sum rho E), flags, status)."""
        sums = np.zeros(4)
        flags = np.zeros(1, dtype=np.int32)
        rc = self.lib.lbm_fd_diagnostics(self.ctx, sums.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         flags.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if rc not in (LBM_OK, LBM_ERR_UNSTABLE):
            self._check(rc, "lbm_fd_diagnostics")
        return sums, int(flags[0]), rc

    def set_config(self, steps_per_launch: int = 0, block_threads: int = 0, nodes_per_thread: int = 0):
        self._check(self.lib.lbm_fd_set_config(self.ctx, int(steps_per_launch), int(block_threads),
                                               int(nodes_per_thread)), "lbm_fd_set_config")

    def get_config(self):
        k, nt, v = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.lbm_fd_get_config(self.ctx, ctypes.byref(k), ctypes.byref(nt), ctypes.byref(v)),
                    "lbm_fd_get_config")
        return k.value, nt.value, v.value

    def autotune(self, trials: int = 3):
        self._check(self.lib.lbm_fd_autotune(self.ctx, int(trials)), "lbm_fd_autotune")
        return self.get_config()

    @property
    def steps_done(self) -> int:
        return int(self.lib.lbm_fd_steps_done(self.ctx))


class D1q3Lattice:
    """Single-distribution D1Q3 scheme of section 2 (scheme="fluid": s_e, gamma, p0, scale = rho0) or
    section 4 (scheme="advection_diffusion": u0, alpha, kappa or s_psi, s_eps, scale = zeta0) on one
    periodic lattice of N >= 3 nodes (lbm_d1q3_* of the C-ABI); precision "f64" or "f32"."""

    def __init__(self, N: int, scheme: str = "fluid", lam: float = 1.0, precision: str = "f64", stream=None,
                 **params):
        torch = _torch()
        self.lib = load_library()
        install_torch_allocator()
        base = dict(scheme=D1Q3_SCHEMES[scheme], pad=0, lam=lam, scale=0.0, s_e=1.5, gamma=0.0, p0=0.0, u0=0.0,
                    alpha=0.0, kappa=0.0, s_psi=0.0, s_eps=0.0)
        unknown = set(params) - set(base)
        if unknown:
            raise TypeError(f"unknown D1Q3 parameters {sorted(unknown)}")
        base.update(params)
        self.params = lbm_d1q3_params(**base)
        self.scheme = scheme
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.N = int(N)
        ctx = ctypes.c_void_p()
        rc = self.lib.lbm_d1q3_create(ctypes.byref(ctx), self.N, ctypes.byref(self.params), PRECISIONS[precision],
                                      ctypes.c_void_p(self.stream.cuda_stream))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_d1q3_create failed")
        self.ctx = ctx

    def _check(self, rc: int, what: str):
        if rc != LBM_OK:
            raise LbmError(rc, f"{what}: {self.lib.lbm_d1q3_last_error(self.ctx).decode()}")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbm_d1q3_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rates(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.lbm_d1q3_rates(self.ctx, ctypes.byref(a), ctypes.byref(b)), "lbm_d1q3_rates")
        return a.value, b.value

    def set_state(self, m0, m1=None):
        a = _Arr(m0, self.N)
        b = None if m1 is None else _Arr(m1, self.N)
        self._check(self.lib.lbm_d1q3_set_state(self.ctx, a.ptr, None if b is None else b.ptr), "lbm_d1q3_set_state")

    def step(self, nsteps: int):
        self._check(self.lib.lbm_d1q3_step(self.ctx, int(nsteps)), "lbm_d1q3_step")

    def moments(self, device: bool = False):
        torch = _torch()
        if device:
            out = [torch.empty(self.N, dtype=torch.float64, device="cuda") for _ in range(3)]
        else:
            out = [np.empty(self.N) for _ in range(3)]
        a = [_Arr(o, self.N, writable=True) for o in out]
        self._check(self.lib.lbm_d1q3_moments(self.ctx, a[0].ptr, a[1].ptr, a[2].ptr), "lbm_d1q3_moments")
        return out

    def populations(self):
        out = np.empty(3 * self.N)
        self._check(self.lib.lbm_d1q3_get_populations(self.ctx, out.ctypes.data), "lbm_d1q3_get_populations")
        return out.reshape(3, self.N)

    def set_populations(self, f):
        a = _Arr(f.reshape(-1) if hasattr(f, "reshape") else f, 3 * self.N)
        self._check(self.lib.lbm_d1q3_set_populations(self.ctx, a.ptr), "lbm_d1q3_set_populations")

    def sums(self):
        """(sums [3] of the three moments, flags, status)."""
        sums = np.zeros(3)
        flags = np.zeros(1, dtype=np.int32)
        rc = self.lib.lbm_d1q3_sums(self.ctx, sums.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    flags.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if rc not in (LBM_OK, LBM_ERR_UNSTABLE):
            self._check(rc, "lbm_d1q3_sums")
        return sums, int(flags[0]), rc

    def set_config(self, steps_per_launch: int = 0, block_threads: int = 0, nodes_per_thread: int = 0):
        self._check(self.lib.lbm_d1q3_set_config(self.ctx, int(steps_per_launch), int(block_threads),
                                                 int(nodes_per_thread)), "lbm_d1q3_set_config")

    def get_config(self):
        k, nt, v = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.lbm_d1q3_get_config(self.ctx, ctypes.byref(k), ctypes.byref(nt), ctypes.byref(v)),
                    "lbm_d1q3_get_config")
        return k.value, nt.value, v.value

    def autotune(self, trials: int = 3):
        self._check(self.lib.lbm_d1q3_autotune(self.ctx, int(trials)), "lbm_d1q3_autotune")
        return self.get_config()

    @property
    def steps_done(self) -> int:
        return int(self.lib.lbm_d1q3_steps_done(self.ctx))


class Lattice2D:
    """Two-dimensional coupled D2Q9-D2Q5 scheme (lbm2d_* of the C-ABI) on a periodic nx x ny lattice;
    precision "f64" or "f32". Fields are [ny, nx] arrays (x fastest); populations [ny, nx, 14] in the
    order (f0..f8, g0..g4). Keyword parameters are the lbm2d_params fields (gamma, Pr, cp, rho0, p0,
    s0, lam, dx, beta, s_e, s_psi, s_eps, s_q, s_h, source_on); the defaults are the section 9 values
    with beta = 9/2."""

    def __init__(self, nx: int, ny: int, precision: str = "f64", stream=None, **params):
        torch = _torch()
        self.lib = load_library()
        install_torch_allocator()
        base = dict(gamma=1.4, Pr=1.0, cp=1.0, rho0=1.0, p0=0.0, s0=0.0, lam=1.0, dx=1.0, beta=0.0, s_e=1.2,
                    s_psi=0.0, s_eps=0.0, s_q=0.0, s_h=0.0, source_on=1, pad=0)
        unknown = set(params) - set(base)
        if unknown:
            raise TypeError(f"unknown lbm2d parameters {sorted(unknown)}")
        base.update(params)
        self.params = lbm2d_params(**base)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.nx, self.ny = int(nx), int(ny)
        self.N = self.nx * self.ny
        ctx = ctypes.c_void_p()
        rc = self.lib.lbm2d_create(ctypes.byref(ctx), self.nx, self.ny, ctypes.byref(self.params),
                                   PRECISIONS[precision], ctypes.c_void_p(self.stream.cuda_stream))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm2d_create failed")
        self.ctx = ctx

    def _check(self, rc: int, what: str):
        if rc != LBM_OK:
            raise LbmError(rc, f"{what}: {self.lib.lbm2d_last_error(self.ctx).decode()}")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbm2d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rates(self):
        r = (ctypes.c_double * 5)()
        self._check(self.lib.lbm2d_rates(self.ctx, r), "lbm2d_rates")
        return tuple(r)

    def set_state(self, rho, ux, uy, s):
        a = [_Arr(x, self.N) for x in (rho, ux, uy, s)]
        self._check(self.lib.lbm2d_set_state(self.ctx, *(x.ptr for x in a)), "lbm2d_set_state")

    def step(self, nsteps: int):
        self._check(self.lib.lbm2d_step(self.ctx, int(nsteps)), "lbm2d_step")

    def populations(self, device: bool = False):
        torch = _torch()
        n = 14 * self.N
        out = torch.empty(n, dtype=torch.float64, device="cuda") if device else np.empty(n)
        a = _Arr(out, n, writable=True)
        self._check(self.lib.lbm2d_get_populations(self.ctx, a.ptr), "lbm2d_get_populations")
        return out.reshape(self.ny, self.nx, 14)

    def fields(self, device: bool = False):
        """(rho, ux, uy, s), each [ny, nx]."""
        torch = _torch()
        if device:
            out = [torch.empty(self.N, dtype=torch.float64, device="cuda") for _ in range(4)]
        else:
            out = [np.empty(self.N) for _ in range(4)]
        a = [_Arr(x, self.N, writable=True) for x in out]
        self._check(self.lib.lbm2d_fields(self.ctx, *(x.ptr for x in a)), "lbm2d_fields")
        return tuple(x.reshape(self.ny, self.nx) for x in out)

    @property
    def steps_done(self) -> int:
        return int(self.lib.lbm2d_steps_done(self.ctx))


class Lattice3D:
    """Three-dimensional coupled D3Q19-D3Q7 scheme (lbm3d_* of the C-ABI) on a periodic nx x ny x nz
    lattice; precision "f64", "f64df" or "f32". Fields are [nz, ny, nx] arrays (x fastest); populations
    [nz, ny, nx, 26] in the order (f0..f18, g0..g6). Keyword parameters are the lbm3d_params fields
    (gamma, Pr, cp, rho0, p0, s0, lam, dx, beta, s_e, s_psi, s_eps, s_q, s_h, source_on); the defaults
    are the section 9 values with beta = 9, s_q = 1.5, s_h = 1.2, s_eps = 1."""

    def __init__(self, nx: int, ny: int, nz: int, precision: str = "f64", stream=None, **params):
        torch = _torch()
        self.lib = load_library()
        install_torch_allocator()
        base = dict(gamma=1.4, Pr=1.0, cp=1.0, rho0=1.0, p0=0.0, s0=0.0, lam=1.0, dx=1.0, beta=0.0, s_e=1.2,
                    s_psi=0.0, s_eps=0.0, s_q=0.0, s_h=0.0, source_on=1, pad=0)
        unknown = set(params) - set(base)
        if unknown:
            raise TypeError(f"unknown lbm3d parameters {sorted(unknown)}")
        base.update(params)
        self.params = lbm3d_params(**base)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        ctx = ctypes.c_void_p()
        rc = self.lib.lbm3d_create(ctypes.byref(ctx), self.nx, self.ny, self.nz, ctypes.byref(self.params),
                                   PRECISIONS[precision], ctypes.c_void_p(self.stream.cuda_stream))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm3d_create failed")
        self.ctx = ctx

    def _check(self, rc: int, what: str):
        if rc != LBM_OK:
            raise LbmError(rc, f"{what}: {self.lib.lbm3d_last_error(self.ctx).decode()}")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbm3d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rates(self):
        r = (ctypes.c_double * 5)()
        self._check(self.lib.lbm3d_rates(self.ctx, r), "lbm3d_rates")
        return tuple(r)

    def set_config(self, ty: int = 0, zc: int = 0, keep: int = -1):
        self._check(self.lib.lbm3d_set_config(self.ctx, int(ty), int(zc), int(keep)), "lbm3d_set_config")

    def get_config(self):
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.lbm3d_get_config(self.ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
                    "lbm3d_get_config")
        return a.value, b.value, c.value

    def set_state(self, rho, ux, uy, uz, s):
        a = [_Arr(x, self.N) for x in (rho, ux, uy, uz, s)]
        self._check(self.lib.lbm3d_set_state(self.ctx, *(x.ptr for x in a)), "lbm3d_set_state")

    def step(self, nsteps: int):
        self._check(self.lib.lbm3d_step(self.ctx, int(nsteps)), "lbm3d_step")

    def populations(self, device: bool = False):
        torch = _torch()
        n = 26 * self.N
        out = torch.empty(n, dtype=torch.float64, device="cuda") if device else np.empty(n)
        a = _Arr(out, n, writable=True)
        self._check(self.lib.lbm3d_get_populations(self.ctx, a.ptr), "lbm3d_get_populations")
        return out.reshape(self.nz, self.ny, self.nx, 26)

    def fields(self, device: bool = False):
        """(rho, ux, uy, uz, s), each [nz, ny, nx]."""
        torch = _torch()
        if device:
            out = [torch.empty(self.N, dtype=torch.float64, device="cuda") for _ in range(5)]
        else:
            out = [np.empty(self.N) for _ in range(5)]
        a = [_Arr(x, self.N, writable=True) for x in out]
        self._check(self.lib.lbm3d_fields(self.ctx, *(x.ptr for x in a)), "lbm3d_fields")
        return tuple(x.reshape(self.nz, self.ny, self.nx) for x in out)

    @property
    def steps_done(self) -> int:
        return int(self.lib.lbm3d_steps_done(self.ctx))
