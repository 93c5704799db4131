"""CPU oracle of the three-dimensional coupled D3Q19-D3Q7 scheme for (rho, J, zeta): the second extension
that the paper's conclusion names (it specifies nothing more; the readings are stated in
``d3q19q7_oracle.cpp``: with the coupling beta = 3/2 of eq. (lien-sigma-sigma) the scheme reduces
exactly to the D1Q3Q3 scheme of sections 6 and 8 on one-dimensional data, and the three-dimensional
scheme takes beta = 9 for the stability of its D3Q7 part).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module; the library in ``paper_1802_02369_gb300`` never imports it and shares
no code with it. The arithmetic lives in ``d3q19q7_oracle.cpp`` (plain FP64 C++, no FMA contraction);
this file builds it with g++ and marshals numpy arrays.

Arrays: fields are ``[Nz, Ny, Nx]`` (x fastest, periodic in all directions); populations and moments
are node-major ``[Nz, Ny, Nx, 26]`` with the population order (f0..f18, g0..g6) of the velocities CX,
CY, CZ below and the moment order MOMENTS.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "d3q19q7_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libd3q19q7_oracle.so")
_lock = threading.Lock()
_lib = None

# Coupling sigma_psi = BETA (gamma / Pr) sigma_e of the three-dimensional scheme: 9, six times the 3/2
# of eq. (lien-sigma-sigma), so that the D3Q7 entropy equilibrium keeps a non-negative rest population.
BETA = 9.0
MOMENTS = ("rho", "Jx", "Jy", "Jz", "zeta", "e", "pxx", "pww", "pxy", "pyz", "pxz", "qx", "qy", "qz", "mx",
           "my", "mz", "eps", "pixx", "piww", "psi_x", "psi_y", "psi_z", "eps7", "xixx", "xiww")
CX = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0])
CY = np.array([0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 1, -1, 0, 0])
CZ = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 0, 0, 0, 0, 0, 1, -1])
NF = 19  # fluid populations first


def build(force: bool = False) -> str:
    """Compiles the oracle with g++ (FP64, -ffp-contract=off) if it is missing or stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                        "-pthread", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Phys3(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("cp", ctypes.c_double),
                ("rho0", ctypes.c_double), ("p0", ctypes.c_double), ("s0", ctypes.c_double),
                ("lam", ctypes.c_double), ("dx", ctypes.c_double), ("beta", ctypes.c_double),
                ("source_on", ctypes.c_int32), ("pad", ctypes.c_int32)]


class Rates3(ctypes.Structure):
    _fields_ = [("s_e", ctypes.c_double), ("s_psi", ctypes.c_double), ("s_eps", ctypes.c_double),
                ("s_q", ctypes.c_double), ("s_h", ctypes.c_double)]


def default_phys(**kw) -> Phys3:
    """The parameters of the one-dimensional experiments of section 9 (gamma = 1.4, Pr = 1,
    c0 = lambda / 2, s0 = 0, rho0 = c_p = 1, p0 = rho0 c0^2 / gamma); keyword overrides: gamma, Pr,
    cp, rho0, p0, s0, lam, dx, beta (default BETA), source_on."""
    lam = kw.get("lam", 1.0)
    gamma = kw.get("gamma", 1.4)
    rho0 = kw.get("rho0", 1.0)
    c0 = lam / 2.0
    return Phys3(gamma=gamma, Pr=kw.get("Pr", 1.0), cp=kw.get("cp", 1.0), rho0=rho0,
                 p0=kw.get("p0", rho0 * c0 * c0 / gamma), s0=kw.get("s0", 0.0), lam=lam, dx=kw.get("dx", 1.0),
                 beta=kw.get("beta", BETA), source_on=int(kw.get("source_on", 1)), pad=0)


def rates(s_e: float, gamma: float = 1.4, Pr: float = 1.0, s_eps: float = 1.0, s_q: float = 1.5,
          s_h: float = 1.2, beta: float | None = None) -> Rates3:
    """sigma_psi = beta (gamma / Pr) sigma_e (beta = 3/2 is eq. lien-sigma-sigma; default BETA). The paper
    fixes none of the other rates in three dimensions: s_q = 1.5 (third-order fluid moments), s_h = 1.2
    (fourth-order) and s_eps = 1.0 (second-order entropy moments) are the defaults because they keep
    the scheme linearly stable at rest for s_e up to 1.5 and for s - s0 up to 0.05 c_p (with s_h =
    s_eps = 1.5 it grows at the (pi, pi, pi) mode from s - s0 = 0.03 c_p on)."""
    sigma_e = 1.0 / s_e - 0.5
    s_psi = 1.0 / ((BETA if beta is None else beta) * (gamma / Pr) * sigma_e + 0.5)
    return Rates3(s_e=s_e, s_psi=s_psi, s_eps=s_eps, s_q=s_q, s_h=s_h)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # D3Q19Q7_ORACLE_LIB points at a deliberately mutated build (mutation tests of the pins only).
            lib = ctypes.CDLL(os.environ.get("D3Q19Q7_ORACLE_LIB") or build())
            P = ctypes.c_void_p
            PP = ctypes.POINTER(Phys3)
            i64 = ctypes.c_int64
            lib.oracle3d_matrices.argtypes = [PP, P, P]
            lib.oracle3d_init.argtypes = [PP, i64, i64, i64, P, P, P, P, P, P]
            lib.oracle3d_run.argtypes = [PP, ctypes.POINTER(Rates3), i64, i64, i64, i64, P, ctypes.c_int32]
            lib.oracle3d_moments.argtypes = [PP, i64, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"{what} rejected its arguments")


def matrices(ph: Phys3):
    M = np.empty((26, 26))
    Minv = np.empty((26, 26))
    _check(_load().oracle3d_matrices(ctypes.byref(ph), _p(M), _p(Minv)), "oracle3d_matrices")
    return M, Minv


def init(ph: Phys3, rho, ux, uy, uz, s) -> np.ndarray:
    """Equilibrium populations [Nz, Ny, Nx, 26] of the fields rho, u, s (each [Nz, Ny, Nx])."""
    rho, ux, uy, uz, s = (_f64(a) for a in (rho, ux, uy, uz, s))
    Nz, Ny, Nx = rho.shape
    fd = np.empty((Nz, Ny, Nx, 26))
    _check(_load().oracle3d_init(ctypes.byref(ph), Nx, Ny, Nz, _p(rho), _p(ux), _p(uy), _p(uz), _p(s), _p(fd)),
           "oracle3d_init")
    return fd


def run(ph: Phys3, rt: Rates3, fd, nsteps: int, nthreads: int = 1) -> np.ndarray:
    """nsteps time steps from fd [Nz, Ny, Nx, 26]; returns the new populations."""
    out = _f64(fd).copy()
    Nz, Ny, Nx, _ = out.shape
    _check(_load().oracle3d_run(ctypes.byref(ph), ctypes.byref(rt), Nx, Ny, Nz, int(nsteps), _p(out),
                                int(nthreads)), "oracle3d_run")
    return out


def moments(ph: Phys3, fd) -> np.ndarray:
    fd = _f64(fd)
    m = np.empty_like(fd)
    _check(_load().oracle3d_moments(ctypes.byref(ph), fd.size // 26, _p(fd), _p(m)), "oracle3d_moments")
    return m
