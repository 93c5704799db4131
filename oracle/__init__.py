"""CPU oracle for the D1Q3Q3 entropy lattice Boltzmann scheme (sections 6 and 8 of Dubois,
Graille and Lallemand, "Recovering the full Navier Stokes equations with lattice Boltzmann
schemes").

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module; the library in ``paper_1802_02369_gb300`` never imports it and
shares no code with it. The arithmetic lives in ``d1q3q3_oracle.cpp`` (plain FP64 C++, no FMA
contraction); this file only builds it with g++ and marshals numpy arrays through ctypes.

Array conventions here: populations and moments are node-major ``[N, 6]`` float64 arrays with the
population order ``(f0, f+, f-, g0, g+, g-)`` and the moment order ``(rho, J, zeta, e, psi, eps)``
of eq. (M-d1q3q3).

Parameter defaults follow the experiments of section 9: gamma = 1.4, Pr = 1, c0 = lambda/2,
s0 = 0; rho0 = 1 and c_p = 1 where the paper leaves them free, and the reference pressure
p0 = rho0 c0^2 / gamma (definition of c0 in section 7).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "d1q3q3_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with g++ (FP64, -ffp-contract=off) if it is missing or stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Phys(ctypes.Structure):
    """Physical and lattice constants (mirrors the oracle's own struct)."""

    _fields_ = [("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("cp", ctypes.c_double),
                ("rho0", ctypes.c_double), ("p0", ctypes.c_double), ("s0", ctypes.c_double),
                ("lam", ctypes.c_double), ("dx", ctypes.c_double),
                ("source_on", ctypes.c_int32), ("bc", ctypes.c_int32),
                ("eq_mode", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("u0_lin", ctypes.c_double), ("s0_lin", ctypes.c_double)]


def default_phys(**kw) -> Phys:
    """Section 9 parameters; keyword overrides: gamma, Pr, cp, rho0, p0, s0, lam, dx, source_on, bc,
    eq_mode (1: the linear equilibria of section 7 around u0_lin, s0_lin; the source is then off by
    default since the linearised system has no production term)."""
    lam = kw.get("lam", 1.0)
    gamma = kw.get("gamma", 1.4)
    rho0 = kw.get("rho0", 1.0)
    c0 = lam / 2.0
    ph = Phys(gamma=gamma, Pr=kw.get("Pr", 1.0), cp=kw.get("cp", 1.0), rho0=rho0,
              p0=kw.get("p0", rho0 * c0 * c0 / gamma), s0=kw.get("s0", 0.0), lam=lam,
              dx=kw.get("dx", 1.0), source_on=int(kw.get("source_on", 0 if kw.get("eq_mode", 0) else 1)),
              bc=int(kw.get("bc", 0)), eq_mode=int(kw.get("eq_mode", 0)), pad=0,
              u0_lin=kw.get("u0_lin", 0.0), s0_lin=kw.get("s0_lin", 0.0))
    return ph


def linear_rates(s_e: float, gamma: float = 1.4, Pr: float = 1.0) -> np.ndarray:
    """Rates of the section 7 linear scheme: s_psi from eq. (lien-sigma-sigma), sigma_eps = 1.5
    (so s_eps = 1/(1.5 + 1/2) = 0.5), as section 7 states."""
    r = coupled_rates(s_e, gamma, Pr)
    r[2] = 1.0 / (1.5 + 0.5)
    return r


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB points at a deliberately mutated build (mutation tests of the pins only).
            lib = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
            d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
            P = ctypes.POINTER(d)
            PP = ctypes.POINTER(Phys)
            lib.oracle_coupled_s_psi.restype = d
            lib.oracle_coupled_s_psi.argtypes = [d, d, d]
            lib.oracle_matrices.argtypes = [PP, P, P]
            lib.oracle_entropy_from_pressure.argtypes = [PP, i64, P, P, P]
            lib.oracle_init.argtypes = [PP, i64, P, P, P, P]
            lib.oracle_equilibria.argtypes = [PP, i64, P, P]
            lib.oracle_run.argtypes = [PP, P, i64, i64, P, i32]
            lib.oracle_moments.argtypes = [PP, i64, P, P]
            lib.oracle_diagnostics.argtypes = [PP, i64, P, P, ctypes.POINTER(i32)]
            lib.oracle_run_tangent.argtypes = [PP, P, P, i32, i64, i64, P, P, P, P, P, P, P, i32]
            lib.oracle_step_jvp.argtypes = [PP, P, i32, i64, i64, P, P, P, P]
            for name in ("oracle_matrices", "oracle_entropy_from_pressure", "oracle_init",
                         "oracle_equilibria", "oracle_run", "oracle_moments", "oracle_diagnostics",
                         "oracle_run_tangent", "oracle_step_jvp"):
                getattr(lib, name).restype = i32
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def coupled_rates(s_e: float, gamma: float = 1.4, Pr: float = 1.0) -> np.ndarray:
    """(s_e, s_psi, s_eps): s_psi from eq. (lien-sigma-sigma), s_eps = 1.5 (sections 4 and 8)."""
    return np.array([s_e, _load().oracle_coupled_s_psi(s_e, gamma, Pr), 1.5])


def matrices(ph: Phys):
    M = np.zeros((6, 6))
    Minv = np.zeros((6, 6))
    _check(_load().oracle_matrices(ctypes.byref(ph), _p(M), _p(Minv)), "matrices")
    return M, Minv


def entropy_from_pressure(ph: Phys, rho, p) -> np.ndarray:
    rho, p = _f64(rho), _f64(p)
    s = np.empty_like(rho)
    _check(_load().oracle_entropy_from_pressure(ctypes.byref(ph), rho.size, _p(rho), _p(p), _p(s)), "entropy")
    return s


def init(ph: Phys, rho, u, s=None, p=None) -> np.ndarray:
    """Equilibrium populations [N, 6] from rho, u and either s (specific entropy) or p."""
    rho, u = _f64(rho), _f64(u)
    if s is None:
        s = entropy_from_pressure(ph, rho, p)
    s = _f64(s)
    fd = np.empty((rho.size, 6))
    _check(_load().oracle_init(ctypes.byref(ph), rho.size, _p(rho), _p(u), _p(s), _p(fd)), "init")
    return fd


def equilibria(ph: Phys, fd) -> np.ndarray:
    fd = _f64(fd)
    out = np.empty((fd.shape[0], 3))
    _check(_load().oracle_equilibria(ctypes.byref(ph), fd.shape[0], _p(fd), _p(out)), "equilibria")
    return out


def run(ph: Phys, rates, fd, nsteps: int, nthreads: int = 1) -> np.ndarray:
    """Returns the populations after nsteps time steps (input left unchanged)."""
    out = np.array(fd, dtype=np.float64, copy=True, order="C")
    r = _f64(rates)
    _check(_load().oracle_run(ctypes.byref(ph), _p(r), out.shape[0], int(nsteps), _p(out), int(nthreads)), "run")
    return out


def moments(ph: Phys, fd) -> np.ndarray:
    fd = _f64(fd)
    m = np.empty_like(fd)
    _check(_load().oracle_moments(ctypes.byref(ph), fd.shape[0], _p(fd), _p(m)), "moments")
    return m


def diagnostics(ph: Phys, fd):
    """(sums[rho, J, zeta, rho E], flags): flags bit 0 non-finite, bit 1 rho <= 0, bit 2 T <= 0."""
    fd = _f64(fd)
    sums = np.empty(4)
    flags = ctypes.c_int32(0)
    _check(_load().oracle_diagnostics(ctypes.byref(ph), fd.shape[0], _p(fd), _p(sums), ctypes.byref(flags)), "diagnostics")
    return sums, int(flags.value)


def run_tangent(ph: Phys, rates, drates, rho, u, s, drho, du, nsteps: int, nthreads: int = 1):
    """Forward-mode run: returns (fd [N,6], dfd [ndir,N,6]) for tangents of the initial rho, u
    (at fixed s) and of the rates (s_e, s_psi); ndir <= 8."""
    rho, u, s = _f64(rho), _f64(u), _f64(s)
    drho, du, drates = _f64(np.atleast_2d(drho)), _f64(np.atleast_2d(du)), _f64(np.atleast_2d(drates))
    ndir, N = drho.shape
    assert du.shape == (ndir, N) and drates.shape == (ndir, 2) and ndir <= 8
    fd = np.empty((N, 6))
    dfd = np.empty((ndir, N, 6))
    r = _f64(rates)
    _check(_load().oracle_run_tangent(ctypes.byref(ph), _p(r), _p(drates), ndir, N, int(nsteps), _p(rho), _p(u), _p(s),
                                      _p(drho), _p(du), _p(fd), _p(dfd), int(nthreads)), "run_tangent")
    return fd, dfd


def step_jvp(ph: Phys, rates, fd0, dfd0, nsteps: int = 1):
    """Jacobian-vector products of nsteps steps with respect to the populations (ndir <= 8)."""
    fd0 = _f64(fd0)
    dfd0 = _f64(dfd0)
    if dfd0.ndim == 2:
        dfd0 = dfd0[None]
    ndir, N = dfd0.shape[0], fd0.shape[0]
    assert ndir <= 8 and dfd0.shape[1:] == fd0.shape
    fd = np.empty_like(fd0)
    dfd = np.empty_like(dfd0)
    r = _f64(rates)
    _check(_load().oracle_step_jvp(ctypes.byref(ph), _p(r), ndir, N, int(nsteps), _p(fd0), _p(dfd0), _p(fd), _p(dfd)), "step_jvp")
    return fd, dfd
