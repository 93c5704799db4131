"""Linear (von Neumann) analysis of one time step around a uniform state, used to pin the oracle
against closed forms of the paper's Taylor-expansion analysis (sections 3, 7 and 8).

At a uniform state the step is translation invariant, so its Jacobian is block circulant:
J_{j,i} = B_{j-i} (6x6 blocks). The blocks are read off the oracle's exact forward-mode
derivative (dual numbers) of one step with respect to the six populations of node 0, and the
amplification matrix of the Fourier mode exp(i theta j) is G(theta) = sum_d B_d exp(-i theta d).
"""
from __future__ import annotations

import numpy as np

import oracle as O


def uniform_state(ph, rho: float, u: float, s: float, N: int) -> np.ndarray:
    return O.init(ph, np.full(N, rho), np.full(N, u), s=np.full(N, s))


def jacobian_blocks(ph, rates, rho: float, u: float, s: float, N: int = 9) -> dict:
    """B_d for d = -(N//2) .. N//2 from one JVP sweep seeded at node 0."""
    fd = uniform_state(ph, rho, u, s, N)
    seeds = np.zeros((6, N, 6))
    for k in range(6):
        seeds[k, 0, k] = 1.0
    _, dfd = O.step_jvp(ph, rates, fd, seeds, 1)
    blocks = {}
    for j in range(N):
        d = j if j <= N // 2 else j - N
        blocks[d] = dfd[:, j, :].T.copy()  # column k = response to seed k
    return blocks


def symbol(blocks: dict, theta: float) -> np.ndarray:
    G = np.zeros((6, 6), dtype=complex)
    for d, B in blocks.items():
        G += B * np.exp(-1j * theta * d)
    return G


def full_jacobian(ph, rates, fd: np.ndarray) -> np.ndarray:
    """Dense 6N x 6N Jacobian of one step at state fd (columns by 8-direction JVP sweeps)."""
    N = fd.shape[0]
    n = 6 * N
    Jm = np.zeros((n, n))
    for c0 in range(0, n, 8):
        cols = list(range(c0, min(n, c0 + 8)))
        seeds = np.zeros((len(cols), N, 6))
        for a, c in enumerate(cols):
            seeds[a].flat[c] = 1.0
        _, dfd = O.step_jvp(ph, rates, fd, seeds, 1)
        for a, c in enumerate(cols):
            Jm[:, c] = dfd[a].ravel()
    return Jm


def conserved_modes(G: np.ndarray, k: int = 3):
    """The k eigenvalues of G closest to the unit circle near theta -> 0 (conserved modes)."""
    w = np.linalg.eigvals(G)
    order = np.argsort(np.abs(np.abs(w) - 1.0))
    return w[order[:k]]
