"""CPU oracle of the two-dimensional coupled D2Q9-D2Q5 scheme for (rho, J, zeta): the extension to two
space dimensions that the paper's conclusion names as the next step (it specifies nothing more; the
readings are stated in ``d2q9q5_oracle.cpp``; with the coupling beta = 3/2 of eq. (lien-sigma-sigma)
the scheme reduces exactly to the D1Q3Q3 scheme of sections 6 and 8 on one-dimensional data, and the
two-dimensional scheme takes beta = 9/2 for the stability of its D2Q5 part).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module; the library in ``paper_1802_02369_gb300`` never imports it and shares
no code with it. The arithmetic lives in ``d2q9q5_oracle.cpp`` (plain FP64 C++, no FMA contraction);
this file builds it with g++ and marshals numpy arrays.

Arrays: fields are ``[Ny, Nx]`` (x fastest, periodic in both directions); populations and moments
are node-major ``[Ny, Nx, 14]`` with the population order (f0..f8, g0..g4) for the velocities
c = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1) and (0,0) (1,0) (0,1) (-1,0) (0,-1),
and the moment order (rho, Jx, Jy, zeta, e, xx, xy, qx, qy, h, psi_x, psi_y, eps, xi).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "d2q9q5_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libd2q9q5_oracle.so")
_lock = threading.Lock()
_lib = None

# Coupling sigma_psi = BETA (gamma / Pr) sigma_e of the two-dimensional scheme: 9/2, three times the
# 3/2 of eq. (lien-sigma-sigma), so that the D2Q5 entropy equilibrium keeps a non-negative rest
# population (with 3/2 the scheme equals D1Q3Q3 on one-dimensional data but is linearly unstable at
# the diagonal modes).
BETA = 4.5
MOMENTS = ("rho", "Jx", "Jy", "zeta", "e", "xx", "xy", "qx", "qy", "h", "psi_x", "psi_y", "eps", "xi")
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1, 0, 1, 0, -1, 0])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1, 0, 0, 1, 0, -1])


def build(force: bool = False) -> str:
    """Compiles the oracle with g++ (FP64, -ffp-contract=off) if it is missing or stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                        "-pthread", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Phys2(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("cp", ctypes.c_double),
                ("rho0", ctypes.c_double), ("p0", ctypes.c_double), ("s0", ctypes.c_double),
                ("lam", ctypes.c_double), ("dx", ctypes.c_double), ("beta", ctypes.c_double),
                ("source_on", ctypes.c_int32), ("pad", ctypes.c_int32)]


class Rates2(ctypes.Structure):
    _fields_ = [("s_e", ctypes.c_double), ("s_psi", ctypes.c_double), ("s_eps", ctypes.c_double),
                ("s_q", ctypes.c_double), ("s_h", ctypes.c_double)]


def default_phys(**kw) -> Phys2:
    """The parameters of the one-dimensional experiments of section 9 (gamma = 1.4, Pr = 1,
    c0 = lambda / 2, s0 = 0, rho0 = c_p = 1, p0 = rho0 c0^2 / gamma); keyword overrides: gamma, Pr,
    cp, rho0, p0, s0, lam, dx, beta (default BETA), source_on."""
    lam = kw.get("lam", 1.0)
    gamma = kw.get("gamma", 1.4)
    rho0 = kw.get("rho0", 1.0)
    c0 = lam / 2.0
    return Phys2(gamma=gamma, Pr=kw.get("Pr", 1.0), cp=kw.get("cp", 1.0), rho0=rho0,
                 p0=kw.get("p0", rho0 * c0 * c0 / gamma), s0=kw.get("s0", 0.0), lam=lam, dx=kw.get("dx", 1.0),
                 beta=kw.get("beta", BETA), source_on=int(kw.get("source_on", 1)), pad=0)


def rates(s_e: float, gamma: float = 1.4, Pr: float = 1.0, s_eps: float = 1.5, s_q: float = 1.5,
          s_h: float = 1.5, beta: float | None = None) -> Rates2:
    """sigma_psi = beta (gamma / Pr) sigma_e (beta = 3/2 is eq. lien-sigma-sigma; default BETA); s_eps =
    1.5 as in section 9; the rates of the third- and fourth-order fluid moments (which the paper does
    not have) 1.5."""
    sigma_e = 1.0 / s_e - 0.5
    s_psi = 1.0 / ((BETA if beta is None else beta) * (gamma / Pr) * sigma_e + 0.5)
    return Rates2(s_e=s_e, s_psi=s_psi, s_eps=s_eps, s_q=s_q, s_h=s_h)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # D2Q9Q5_ORACLE_LIB points at a deliberately mutated build (mutation tests of the pins only).
            lib = ctypes.CDLL(os.environ.get("D2Q9Q5_ORACLE_LIB") or build())
            P = ctypes.c_void_p
            PP = ctypes.POINTER(Phys2)
            i64 = ctypes.c_int64
            lib.oracle2d_matrices.argtypes = [PP, P, P]
            lib.oracle2d_init.argtypes = [PP, i64, i64, P, P, P, P, P]
            lib.oracle2d_run.argtypes = [PP, ctypes.POINTER(Rates2), i64, i64, i64, P, ctypes.c_int32]
            lib.oracle2d_moments.argtypes = [PP, i64, P, P]
            lib.oracle2d_equilibria.argtypes = [PP, i64, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"{what} rejected its arguments")


def matrices(ph: Phys2):
    M = np.empty((14, 14))
    Minv = np.empty((14, 14))
    _check(_load().oracle2d_matrices(ctypes.byref(ph), _p(M), _p(Minv)), "oracle2d_matrices")
    return M, Minv


def init(ph: Phys2, rho, ux, uy, s) -> np.ndarray:
    """Equilibrium populations [Ny, Nx, 14] of the fields rho, u = (ux, uy), s (each [Ny, Nx])."""
    rho, ux, uy, s = (_f64(a) for a in (rho, ux, uy, s))
    Ny, Nx = rho.shape
    fd = np.empty((Ny, Nx, 14))
    _check(_load().oracle2d_init(ctypes.byref(ph), Nx, Ny, _p(rho), _p(ux), _p(uy), _p(s), _p(fd)), "oracle2d_init")
    return fd


def run(ph: Phys2, rt: Rates2, fd, nsteps: int, nthreads: int = 1) -> np.ndarray:
    """nsteps time steps from fd [Ny, Nx, 14]; returns the new populations."""
    out = _f64(fd).copy()
    Ny, Nx, _ = out.shape
    _check(_load().oracle2d_run(ctypes.byref(ph), ctypes.byref(rt), Nx, Ny, int(nsteps), _p(out), int(nthreads)),
           "oracle2d_run")
    return out


def moments(ph: Phys2, fd) -> np.ndarray:
    fd = _f64(fd)
    m = np.empty_like(fd)
    _check(_load().oracle2d_moments(ctypes.byref(ph), fd.size // 14, _p(fd), _p(m)), "oracle2d_moments")
    return m


def equilibria(ph: Phys2, fd) -> np.ndarray:
    fd = _f64(fd)
    eq = np.empty(fd.shape[:-1] + (10,))
    _check(_load().oracle2d_equilibria(ctypes.byref(ph), fd.size // 14, _p(fd), _p(eq)), "oracle2d_equilibria")
    return eq
