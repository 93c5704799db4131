"""Seeded synthetic initial data shaped like the experiments of section 9 (periodic acoustic
waves of growing amplitude) and the Riemann problems used to exercise shocks.

This module holds no arithmetic of the lattice Boltzmann method: it only produces the
macroscopic fields (rho, u, p) and per-lattice parameters that both the CUDA library and the CPU
oracle take as inputs. Every generator is deterministic in its arguments
(``numpy.random.default_rng(PCG64(seed))`` where randomness is drawn).

Pressures are given in physical units. ``p_ref`` is the reference pressure the caller uses for
its equation of state (section 9 takes c0 = lambda/2, so p_ref = rho0 c0^2 / gamma); "adiabatic"
pressure means the isentrope through (rho0, p_ref): p = p_ref (rho/rho0)^gamma.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def reference_pressure(lam: float = 1.0, gamma: float = 1.4, rho0: float = 1.0) -> float:
    """p_ref = rho0 c0^2 / gamma with c0 = lambda / 2 (section 9 parameters)."""
    c0 = lam / 2.0
    return rho0 * c0 * c0 / gamma


def sod(N: int, p_unit: float, rho_l: float = 1.0, p_l: float = 1.0, rho_r: float = 0.5,
        p_r: float = 0.5):
    """Riemann data split at N/2: x < N/2 has (rho_l, 0, p_l * p_unit), x >= N/2 has
    (rho_r, 0, p_r * p_unit)."""
    j = np.arange(N)
    left = j < N // 2
    rho = np.where(left, rho_l, rho_r).astype(np.float64)
    u = np.zeros(N)
    p = np.where(left, p_l, p_r) * p_unit
    return rho, u, p.astype(np.float64)


def steepening_wave(N: int, amp: float, p_ref: float, gamma: float = 1.4, rho0: float = 1.0):
    """One wavelength over the lattice: rho = rho0 (1 + amp sin(2 pi j / N)),
    u = amp sin(2 pi j / N), adiabatic pressure."""
    j = np.arange(N, dtype=np.float64)
    w = np.sin(2.0 * np.pi * j / N)
    rho = rho0 * (1.0 + amp * w)
    u = amp * w
    p = p_ref * (rho / rho0) ** gamma
    return rho, u, p


def progressive_wave(N: int, delta: float, c0: float, p_ref: float, gamma: float = 1.4, rho0: float = 1.0):
    """Linear progressive acoustic wave of relative amplitude delta (figures 1-3 of section 9):
    rho = rho0 (1 + delta sin), u = c0 delta sin, adiabatic pressure."""
    j = np.arange(N, dtype=np.float64)
    w = np.sin(2.0 * np.pi * j / N)
    rho = rho0 * (1.0 + delta * w)
    u = c0 * delta * w
    p = p_ref * (rho / rho0) ** gamma
    return rho, u, p


def gaussian_bumps(B: int, N: int, seed: int, p_ref: float, amp: float = 0.05, width: float = 64.0,
                   nbumps: int = 8, gamma: float = 1.4, rho0: float = 1.0):
    """B periodic lattices of N nodes: rho = rho0 (1 + sum of nbumps Gaussian bumps of amplitude
    amp * U[0.5, 1] and 1/e half-width width * U[0.5, 1.5] at uniform centres), u = 0,
    adiabatic pressure. Returns arrays of shape [B, N]."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    j = np.arange(N, dtype=np.float64)
    rho = np.full((B, N), rho0)
    for b in range(B):
        centres = rng.uniform(0, N, nbumps)
        amps = amp * rng.uniform(0.5, 1.0, nbumps)
        widths = width * rng.uniform(0.5, 1.5, nbumps)
        for c, a, w in zip(centres, amps, widths):
            d = np.abs(j - c)
            d = np.minimum(d, N - d)
            rho[b] += rho0 * a * np.exp(-(d / w) ** 2)
    u = np.zeros((B, N))
    p = p_ref * (rho / rho0) ** gamma
    return rho, u, p


@dataclass
class RaggedBatch:
    """Independent lattices concatenated back to back (CSR layout)."""

    lengths: np.ndarray   # int64 [B]
    offsets: np.ndarray   # int64 [B + 1]
    s_e: np.ndarray       # float64 [B], the free relaxation rate of each lattice
    bc: np.ndarray        # int32 [B], 0 periodic, 1 bounce-back
    rho: np.ndarray       # float64 [sum lengths]
    u: np.ndarray
    p: np.ndarray
    states: np.ndarray    # float64 [B, 4] = (rho_L, p_L, rho_R, p_R), pressures in units of p_unit

    def lattice(self, b: int):
        lo, hi = self.offsets[b], self.offsets[b + 1]
        return self.rho[lo:hi], self.u[lo:hi], self.p[lo:hi]


def waves_2d(nx: int, ny: int, seed: int, amp: float = 0.04, lam: float = 1.0, rho0: float = 1.0,
             cp: float = 1.0, s0: float = 0.0, x0: int = 0, y0: int = 0, period=None):
    """Smooth periodic two-dimensional fields (rho, ux, uy, s), each [ny, nx] with x fastest: a few
    seeded Fourier modes of relative amplitude amp in density, velocity (units of lam) and entropy
    (units of c_p, about s0). ``period`` = (Px, Py) evaluates the fields of a Px x Py periodic domain
    on the window of nx x ny nodes starting at (x0, y0) (coordinates taken modulo the period), so that
    a window of a large lattice can be regenerated alone."""
    Px, Py = (nx, ny) if period is None else period
    rng = np.random.default_rng(seed)
    xs = (x0 + np.arange(nx)) % Px
    ys = (y0 + np.arange(ny)) % Py
    X = 2 * np.pi * xs[None, :] / Px
    Y = 2 * np.pi * ys[:, None] / Py
    modes = [(1, 0), (0, 1), (1, 1), (2, -1), (1, 2)]

    def field():
        out = np.zeros((ny, nx))
        for kx, ky in modes:
            a, ph = rng.uniform(-1, 1), rng.uniform(0, 2 * np.pi)
            out = out + a * np.sin(kx * X + ky * Y + ph)
        return amp * out / len(modes) ** 0.5

    rho = rho0 * (1.0 + field())
    ux, uy = lam * field(), lam * field()
    s = s0 + cp * 0.5 * field()
    return rho, ux, uy, s


def waves_3d(nx: int, ny: int, nz: int, seed: int, amp: float = 0.04, lam: float = 1.0, rho0: float = 1.0,
             cp: float = 1.0, s0: float = 0.0, x0: int = 0, y0: int = 0, z0: int = 0, period=None):
    """Smooth periodic three-dimensional fields (rho, ux, uy, uz, s), each [nz, ny, nx] with x fastest:
    a few seeded Fourier modes of relative amplitude amp in density, velocity (units of lam) and
    entropy (units of c_p, about s0, at a quarter of amp: the three-dimensional scheme is linearly
    stable for s - s0 up to about 0.05 c_p). ``period`` = (Px, Py, Pz) evaluates the fields of a
    periodic domain on the window of nx x ny x nz nodes starting at (x0, y0, z0), so that a window of a
    large lattice can be regenerated alone."""
    Px, Py, Pz = (nx, ny, nz) if period is None else period
    rng = np.random.default_rng(seed)
    X = 2 * np.pi * ((x0 + np.arange(nx)) % Px)[None, None, :] / Px
    Y = 2 * np.pi * ((y0 + np.arange(ny)) % Py)[None, :, None] / Py
    Z = 2 * np.pi * ((z0 + np.arange(nz)) % Pz)[:, None, None] / Pz
    modes = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, -1), (1, -2, 1)]

    def field():
        out = np.zeros((nz, ny, nx))
        for kx, ky, kz in modes:
            a, ph = rng.uniform(-1, 1), rng.uniform(0, 2 * np.pi)
            out += a * np.sin(kx * X + ky * Y + kz * Z + ph)
        out *= amp / len(modes) ** 0.5
        return out

    rho = rho0 * (1.0 + field())
    ux, uy, uz = lam * field(), lam * field(), lam * field()
    s = s0 + cp * 0.25 * field()
    return rho, ux, uy, uz, s


def entropy_of_state(rho, p_rel, gamma: float = 1.4, cp: float = 1.0, rho0: float = 1.0):
    """Specific entropy s - s0 of an ideal-gas state of density rho and pressure p_rel * p_unit,
    measured from the isentrope through (rho0, p_unit): (c_p / gamma) log(p_rel (rho0 / rho)^gamma).
    Used only to select Riemann data (a property of the drawn inputs)."""
    return (cp / gamma) * (np.log(p_rel) - gamma * np.log(np.asarray(rho) / rho0))


def riemann_star(rho_l, p_l, rho_r, p_r, gamma: float = 1.4, u_l=0.0, u_r=0.0):
    """Pressure and velocity (p*, u*) of the star region of the exact solution of the ideal-gas Riemann
    problem with states (rho, u, p) left and right: the root of the pressure function
    f_L(p) + f_R(p) + u_r - u_l = 0, where f_K is the shock (Rankine-Hugoniot) branch for p > p_K and
    the rarefaction (isentropic) branch for p <= p_K, found by Newton's method from the mean pressure;
    u* = (u_l + u_r)/2 + (f_R(p*) - f_L(p*))/2 (Toro, "Riemann Solvers and Numerical Methods for Fluid
    Dynamics", chapter 4). Vectorised over numpy arrays. A property of the input data (gas dynamics),
    used to select Riemann problems."""
    rho_l, p_l, rho_r, p_r = (np.asarray(x, dtype=np.float64) for x in (rho_l, p_l, rho_r, p_r))
    g = gamma

    def f_and_df(p, rho, pk):
        ck = np.sqrt(g * pk / rho)
        a, b = 2.0 / ((g + 1.0) * rho), (g - 1.0) / (g + 1.0) * pk
        q = np.sqrt(a / (p + b))
        f_sh = (p - pk) * q
        df_sh = q * (1.0 - 0.5 * (p - pk) / (p + b))
        r = (p / pk) ** ((g - 1.0) / (2.0 * g))
        f_ra = 2.0 * ck / (g - 1.0) * (r - 1.0)
        df_ra = r / (rho * ck) * (pk / p)
        shock = p > pk
        return np.where(shock, f_sh, f_ra), np.where(shock, df_sh, df_ra)

    p = 0.5 * (p_l + p_r)
    for _ in range(50):
        fl, dl = f_and_df(p, rho_l, p_l)
        fr, dr = f_and_df(p, rho_r, p_r)
        step = (fl + fr + (u_r - u_l)) / (dl + dr)
        p = np.maximum(p - step, 1e-12 * np.maximum(p_l, p_r))
        if np.all(np.abs(step) <= 1e-14 * p):
            break
    fl, _ = f_and_df(p, rho_l, p_l)
    fr, _ = f_and_df(p, rho_r, p_r)
    return p, 0.5 * (u_l + u_r) + 0.5 * (fr - fl)


# Flow speed |u| / lambda below which the linearised D1Q3Q3 step around the reference state (rho0, u,
# s0) of the paper's gas (gamma = 1.4, Pr = 1, c0 = lambda / 2) has spectral radius <= 1, for the free
# rate s_e = 1.0, 1.1, ..., 1.9 (s_psi coupled, s_eps = 1.5). Values of the stability analysis of the
# scheme, rounded down to 0.001; the stability tests check each against the oracle's exact Jacobian.
# Used only to select Riemann data whose flow stays in the stable region.
STABLE_FLOW_SPEED_S_E = (1.0, 1.1, 1.2, 1.3, 1.4, 1.5, 1.6, 1.7, 1.8, 1.9)
STABLE_FLOW_SPEED = (0.155, 0.150, 0.144, 0.138, 0.131, 0.123, 0.114, 0.102, 0.087, 0.064)


def ragged_batch(B: int, seed: int, p_unit: float, n_min: int = 512, n_max: int = 65536,
                 s_range=(1.0, 1.9), left=(0.8, 1.2), right=(0.3, 0.7), p_bounce: float = 0.5,
                 entropy_range=None, gamma: float = 1.4, stable_flow: bool = False) -> RaggedBatch:
    """B Riemann problems of uneven lengths: N_b uniform in [n_min, n_max], s_e uniform in
    s_range, left state (rho, p) uniform in ``left``, right state uniform in ``right`` (pressures
    times p_unit), u = 0, split at N_b / 2; boundary periodic or bounce-back with probability
    p_bounce each.

    entropy_range = (lo, hi): keep only the draws whose left and right states both have a specific
    entropy (``entropy_of_state``, c_p = 1) in [lo, hi]. stable_flow: keep only the draws whose exact
    Riemann solution moves no faster than STABLE_FLOW_SPEED at their s_e (|u*| from ``riemann_star``,
    the table interpolated linearly in s_e). Candidates are drawn from the same distribution in chunks
    from the same generator and the first B accepted ones are kept, so the result is the conditional
    distribution of the unfiltered draw."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    if entropy_range is None and not stable_flow:
        lengths = rng.integers(n_min, n_max + 1, B).astype(np.int64)
        s_e = rng.uniform(s_range[0], s_range[1], B)
        states = np.stack([rng.uniform(*left, B), rng.uniform(*left, B),
                           rng.uniform(*right, B), rng.uniform(*right, B)], axis=1)
        bc = (rng.uniform(0, 1, B) < p_bounce).astype(np.int32)
    else:
        lo, hi = entropy_range if entropy_range is not None else (-np.inf, np.inf)
        keep = [[], [], [], []]
        got = 0
        while got < B:
            C = 8192
            ln = rng.integers(n_min, n_max + 1, C).astype(np.int64)
            se = rng.uniform(s_range[0], s_range[1], C)
            st = np.stack([rng.uniform(*left, C), rng.uniform(*left, C),
                           rng.uniform(*right, C), rng.uniform(*right, C)], axis=1)
            bb = (rng.uniform(0, 1, C) < p_bounce).astype(np.int32)
            sl = entropy_of_state(st[:, 0], st[:, 1], gamma)
            sr = entropy_of_state(st[:, 2], st[:, 3], gamma)
            ok = (sl >= lo) & (sl <= hi) & (sr >= lo) & (sr <= hi)
            if stable_flow:
                _, us = riemann_star(st[:, 0], st[:, 1] * p_unit, st[:, 2], st[:, 3] * p_unit, gamma)
                ok &= np.abs(us) <= np.interp(se, STABLE_FLOW_SPEED_S_E, STABLE_FLOW_SPEED)
            for lst, arr in zip(keep, (ln, se, st, bb)):
                lst.append(arr[ok])
            got += int(ok.sum())
        lengths, s_e, states, bc = (np.concatenate(lst)[:B] for lst in keep)
    offsets = np.zeros(B + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    tot = int(offsets[-1])
    rho = np.empty(tot)
    u = np.zeros(tot)
    p = np.empty(tot)
    for b in range(B):
        n = int(lengths[b])
        r, _, pp = sod(n, p_unit, states[b, 0], states[b, 1], states[b, 2], states[b, 3])
        rho[offsets[b]:offsets[b + 1]] = r
        p[offsets[b]:offsets[b + 1]] = pp
    return RaggedBatch(lengths, offsets, s_e, bc, rho, u, p, states)
