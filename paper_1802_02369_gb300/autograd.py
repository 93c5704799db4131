"""torch.autograd bridge to the adjoint of the D1Q3Q3 time stepping.

``lattice_run(rho0, u0, s0, s_e, s_psi, lengths, T)`` advances the equilibrium state built from
(rho0, u0, s0) by T time steps in the CUDA library and returns rho(T). Its backward pass runs the
library's reverse-mode sweep (sqrt(T) checkpointing) and returns gradients with respect to rho0,
u0 (at fixed specific entropy s0) and the per-lattice rates s_e, s_psi (taken as independent).
All arithmetic runs in the library; this module only moves tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm


class LatticeRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, u0, s_e, s_psi, s0, lengths, T, precision, lam, bc):
        lat = lbm.Lattice(lengths, lam=lam, s_e=s_e.detach().cpu().numpy(), s_psi=s_psi.detach().cpu().numpy(),
                          bc=bc, precision=precision)
        lat.set_state_entropy(rho0.detach().contiguous(), u0.detach().contiguous(), s0.detach().contiguous())
        lat.adjoint_forward(int(T))
        rho_T = lat.moments(device=True)[0]
        ctx.lat = lat
        ctx.rate_device = s_e.device
        return rho_T

    @staticmethod
    def backward(ctx, g):
        lat = ctx.lat
        drho, du, drates, _ = lat.adjoint_backward(g.detach().contiguous(), device=True)
        lat.close()
        ctx.lat = None
        dr = torch.from_numpy(np.ascontiguousarray(drates)).to(ctx.rate_device)
        return drho, du, dr[:, 0], dr[:, 1], None, None, None, None, None, None


def lattice_run(rho0, u0, s0, s_e, s_psi, lengths, T: int, precision: str = "f64", lam: float = 1.0, bc=0):
    """rho(T) of the batch of lattices (float64 device tensors of the concatenated nodes)."""
    return LatticeRun.apply(rho0, u0, s_e, s_psi, s0, lengths, T, precision, lam, bc)
