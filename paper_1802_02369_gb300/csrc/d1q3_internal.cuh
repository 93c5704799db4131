// Internal declarations of the single-distribution D1Q3 schemes: the fluid scheme of section 2 and
// the advection-diffusion scheme of section 4. Used by d1q3_step.cu and d1q3_api.cu only.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

enum { kD1q3Fluid = 0, kD1q3AdvDiff = 1 };

// Constants of the node update in the lane type X (double, float, or float2 holding one value twice).
// The update works on dimensionless moments of the populations shifted by the rest state:
// r = sum f, j = f+ - f-, q = f+ + f- - 2 f0 (the moments of eq. (M-d1q3) over scale, scale lambda
// and scale lambda^2).
template <typename X>
struct D1q3Consts {
  X one, two, three, half, m_half, third, sixth, m_two;
  X s1, s2;     // fluid: s_e (s1); advection-diffusion: s_psi (s1), s_eps (s2)
  X kp, gamma;  // fluid: p0 / (rho0 lambda^2) and the isentropic exponent
  X ul, alpha;  // advection-diffusion: u0 / lambda and alpha of eps_eq = alpha lambda^2 zeta
};

// Both lane forms for FP32 (scalar lanes for one node per thread, paired lanes otherwise).
template <typename R>
struct D1q3ConstSet;
template <>
struct D1q3ConstSet<double> {
  D1q3Consts<double> s;
};
template <>
struct D1q3ConstSet<float> {
  D1q3Consts<float> s;
  D1q3Consts<float2> p;
};

// One launch: K time steps of the periodic lattice of N nodes, from `in` to `out` (shifted populations,
// plane-major [3][N] in the order f0, f+, f-). Tiles of NT*V nodes (NT threads, V nodes per thread),
// K halo nodes per side. max_tiles > 0 computes only the first max_tiles tiles (autotuner trials).
template <typename R>
cudaError_t launch_d1q3_step(const R* in, R* out, long long N, int scheme, int K, int NT, int V,
                             const D1q3ConstSet<R>& c, cudaStream_t st, long long max_tiles = 0);

bool valid_d1q3_config(int K, int NT, int V);

}  // namespace lbm
