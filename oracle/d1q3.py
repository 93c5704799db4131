"""CPU oracle of the single-distribution D1Q3 schemes: the fluid scheme of section 2 and the
advection-diffusion scheme of section 4.

TEST INFRASTRUCTURE ONLY: the tests use this module; the library in ``paper_1802_02369_gb300``
never imports it and shares no code with it. The arithmetic lives in ``d1q3_oracle.cpp`` (plain
FP64 C++, no FMA contraction); this file builds it with g++ and marshals numpy arrays.

Arrays are node-major: populations ``[N, 3]`` in the order (f0, f+, f-), moments ``[N, 3]`` in the
order (rho, J, e) for section 2 and (zeta, psi, eps) for section 4.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "d1q3_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libd1q3_oracle.so")
_lock = threading.Lock()
_lib = None

FLUID = 0
ADVECTION_DIFFUSION = 1


def build(force: bool = False) -> str:
    """Compiles the D1Q3 oracle with g++ (FP64, -ffp-contract=off) if missing or stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("pad", ctypes.c_int32), ("lam", ctypes.c_double),
                ("scale", ctypes.c_double), ("s_e", ctypes.c_double), ("gamma", ctypes.c_double),
                ("p0", ctypes.c_double), ("u0", ctypes.c_double), ("alpha", ctypes.c_double),
                ("s_psi", ctypes.c_double), ("s_eps", ctypes.c_double)]


def fluid(s_e: float, lam: float = 1.0, rho0: float = 1.0, gamma: float = 1.4, p0: float | None = None) -> Params:
    """Section 2 fluid scheme; p0 defaults to rho0 c0^2 / gamma with c0 = lam / 2 (so that the sound
    speed at rest is lam / 2, as in the experiments of section 9)."""
    if p0 is None:
        p0 = rho0 * (lam / 2.0) ** 2 / gamma
    return Params(scheme=FLUID, pad=0, lam=lam, scale=rho0, s_e=s_e, gamma=gamma, p0=p0, u0=0.0, alpha=0.0,
                  s_psi=1.0, s_eps=1.5)


def advection_diffusion(u0: float, alpha: float, s_psi: float, lam: float = 1.0, zeta0: float = 1.0,
                        s_eps: float = 1.5) -> Params:
    """Section 4 advection-diffusion scheme: psi_eq = u0 zeta, eps_eq = alpha lam^2 zeta."""
    return Params(scheme=ADVECTION_DIFFUSION, pad=0, lam=lam, scale=zeta0, s_e=1.0, gamma=1.0, p0=1.0, u0=u0,
                  alpha=alpha, s_psi=s_psi, s_eps=s_eps)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # D1Q3_ORACLE_LIB points at a deliberately mutated build (mutation tests of the pins only).
            lib = ctypes.CDLL(os.environ.get("D1Q3_ORACLE_LIB") or build())
            i64 = ctypes.c_int64
            P = ctypes.POINTER(ctypes.c_double)
            PP = ctypes.POINTER(Params)
            lib.d1q3_oracle_matrices.argtypes = [PP, P, P]
            lib.d1q3_oracle_init.argtypes = [PP, i64, P, P, P]
            lib.d1q3_oracle_run.argtypes = [PP, i64, i64, P]
            lib.d1q3_oracle_moments.argtypes = [PP, i64, P, P]
            for n in ("d1q3_oracle_matrices", "d1q3_oracle_init", "d1q3_oracle_run", "d1q3_oracle_moments"):
                getattr(lib, n).restype = ctypes.c_int32
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"D1Q3 oracle {what} rejected its arguments (rc={rc})")


def matrices(p: Params):
    M, Minv = np.zeros(9), np.zeros(9)
    _check(_load().d1q3_oracle_matrices(ctypes.byref(p), _p(M), _p(Minv)), "matrices")
    return M.reshape(3, 3), Minv.reshape(3, 3)


def init(p: Params, m0, m1=None) -> np.ndarray:
    m0 = _f64(m0)
    m1 = _f64(np.zeros_like(m0) if m1 is None else m1)
    f = np.zeros((m0.size, 3))
    _check(_load().d1q3_oracle_init(ctypes.byref(p), m0.size, _p(m0), _p(m1), _p(f)), "init")
    return f


def run(p: Params, f, nsteps: int) -> np.ndarray:
    f = _f64(f).copy()
    _check(_load().d1q3_oracle_run(ctypes.byref(p), f.shape[0], int(nsteps), _p(f)), "run")
    return f


def moments(p: Params, f) -> np.ndarray:
    f = _f64(f)
    m = np.zeros_like(f)
    _check(_load().d1q3_oracle_moments(ctypes.byref(p), f.shape[0], _p(f), _p(m)), "moments")
    return m
