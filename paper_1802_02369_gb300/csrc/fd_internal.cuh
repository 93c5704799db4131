// Internal declarations of the finite-difference comparison solver of section 9: the (rho, J, zeta)
// Navier-Stokes system of eq. (NS-rho-J-zeta), second-order centred differences in space, explicit
// first-order (forward Euler) time integration, periodic grid. Used by fd_step.cu and fd_api.cu only.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// Constants of the finite-difference update in the arithmetic type R. The state is stored shifted
// like the lattice Boltzmann populations: w = (rho - rho0, J, zeta - rho0 s0), so that small
// deviations from the reference state keep their relative precision in FP32.
template <typename R>
struct FdConsts {
  R rho0, inv_rho0;  // reference density of eq. (gaz-parfait)
  R s0, rho0s0;      // reference entropy s0 and rho0 s0
  R gamma, inv_cp;   // gamma, 1 / c_p
  R p0, inv_r, T0;   // p0, 1 / r with r = c_p (1 - 1/gamma), T0 = p0 / (rho0 r)
  R nu, nu_k;        // kinematic viscosity nu and nu c_p / Pr (kappa = rho nu c_p / Pr)
  R c_adv;           // dt / (2 dx): centred convective difference
  R c_dif;           // dt / (2 dx^2): face-averaged diffusion coefficient times the face difference
  R c_src;           // dt / (4 dx^2): source with the centred derivatives squared
  int source_on;
};

// One launch: K forward-Euler steps of the whole periodic grid of N nodes, from `in` to `out`
// (plane-major [3][N]). Tiles of NT*V nodes, NT threads, V nodes per thread, K halo nodes per side.
// max_tiles > 0 computes only the first max_tiles tiles (timing trials of the autotuner).
template <typename R>
cudaError_t launch_fd_step(const R* in, R* out, long long N, int K, int NT, int V, const FdConsts<R>& c,
                           cudaStream_t st, long long max_tiles = 0);

bool valid_fd_config(int K, int NT, int V);

}  // namespace lbm
