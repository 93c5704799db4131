"""CPU oracle of the finite-difference comparison solver of section 9 (the (rho, J, zeta)
Navier-Stokes system of eq. (NS-rho-J-zeta), centred second-order differences, forward Euler).

TEST INFRASTRUCTURE ONLY: the tests use this module; the library in ``paper_1802_02369_gb300``
never imports it and shares no code with it. The arithmetic lives in ``fd_oracle.cpp`` (plain
FP64 C++, no FMA contraction); this file builds it with g++ and marshals numpy arrays.

State arrays are node-major ``[N, 3]`` float64 with the order (rho, J, zeta). Units: the grid
spacing dx and the time step dt are given explicitly; nu is the kinematic viscosity of the
momentum equation and kappa = rho nu c_p / Pr.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fd_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libfd_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the finite-difference oracle with g++ (FP64, -ffp-contract=off) if missing or stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class FdPhys(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("cp", ctypes.c_double),
                ("rho0", ctypes.c_double), ("p0", ctypes.c_double), ("s0", ctypes.c_double),
                ("dx", ctypes.c_double), ("nu", ctypes.c_double),
                ("source_on", ctypes.c_int32), ("pad", ctypes.c_int32)]


def default_phys(nu: float, **kw) -> FdPhys:
    """Section 9 parameters (gamma = 1.4, Pr = 1, rho0 = 1, c_p = 1, s0 = 0, p0 = rho0 c0^2/gamma
    with c0 = lam/2); keyword overrides: gamma, Pr, cp, rho0, p0, s0, lam, dx, source_on."""
    lam = kw.get("lam", 1.0)
    gamma = kw.get("gamma", 1.4)
    rho0 = kw.get("rho0", 1.0)
    c0 = lam / 2.0
    return FdPhys(gamma=gamma, Pr=kw.get("Pr", 1.0), cp=kw.get("cp", 1.0), rho0=rho0,
                  p0=kw.get("p0", rho0 * c0 * c0 / gamma), s0=kw.get("s0", 0.0), dx=kw.get("dx", 1.0),
                  nu=nu, source_on=int(kw.get("source_on", 1)), pad=0)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # FD_ORACLE_LIB points at a deliberately mutated build (mutation tests of the pins only).
            lib = ctypes.CDLL(os.environ.get("FD_ORACLE_LIB") or build())
            d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
            P = ctypes.POINTER(d)
            PP = ctypes.POINTER(FdPhys)
            lib.fd_oracle_init.argtypes = [PP, i64, P, P, P, P]
            lib.fd_oracle_run.argtypes = [PP, i64, d, i64, P]
            lib.fd_oracle_diagnostics.argtypes = [PP, i64, P, P, ctypes.POINTER(i32)]
            lib.fd_oracle_series.argtypes = [PP, i64, d, i64, i64, P, P]
            for name in ("fd_oracle_init", "fd_oracle_run", "fd_oracle_diagnostics", "fd_oracle_series"):
                getattr(lib, name).restype = i32
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"finite-difference oracle {what} rejected its arguments (rc={rc})")


def init(ph: FdPhys, rho, u, s) -> np.ndarray:
    rho, u, s = _f64(rho), _f64(u), _f64(s)
    W = np.zeros((rho.size, 3))
    _check(_load().fd_oracle_init(ctypes.byref(ph), rho.size, _p(rho), _p(u), _p(s), _p(W)), "init")
    return W


def run(ph: FdPhys, W, dt: float, nsteps: int) -> np.ndarray:
    W = _f64(W).copy()
    _check(_load().fd_oracle_run(ctypes.byref(ph), W.shape[0], dt, nsteps, _p(W)), "run")
    return W


def diagnostics(ph: FdPhys, W):
    W = _f64(W)
    sums = np.zeros(4)
    fl = ctypes.c_int32(0)
    _check(_load().fd_oracle_diagnostics(ctypes.byref(ph), W.shape[0], _p(W), _p(sums), ctypes.byref(fl)),
           "diagnostics")
    return sums, fl.value


def series(ph: FdPhys, W, dt: float, nsteps: int, every: int):
    """(W after nsteps, sums at steps 0, every, ..., nsteps as an array [nsteps/every + 1, 4])."""
    W = _f64(W).copy()
    out = np.zeros((nsteps // every + 1, 4))
    _check(_load().fd_oracle_series(ctypes.byref(ph), W.shape[0], dt, nsteps, every, _p(W), _p(out)), "series")
    return W, out


def primitives(ph: FdPhys, W):
    """(u, s, p, T) of a state, from eq. (gaz-parfait) written out in numpy (test helper)."""
    W = _f64(W)
    rho, J, zeta = W[:, 0], W[:, 1], W[:, 2]
    u, s = J / rho, zeta / rho
    p = ph.p0 * (rho / ph.rho0) ** ph.gamma * np.exp(ph.gamma * (s - ph.s0) / ph.cp)
    T = p / (rho * ph.cp * (1.0 - 1.0 / ph.gamma))
    return u, s, p, T
