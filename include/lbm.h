/*
 * C-ABI of the GB300 library for the coupled D1Q3Q3 entropy lattice Boltzmann scheme of
 * Dubois, Graille and Lallemand, "Recovering the full Navier Stokes equations with lattice
 * Boltzmann schemes" (sections 6 and 8). One "step" is the time iteration of section 8,
 * steps (i)-(viii): moments m = M f_d (eq. M-d1q3q3), equilibria (eqs. energie-equilibre,
 * psi-equilibre, eq-energie-entropie-d1q3q3) with the polytropic equation of state
 * (eq. gaz-parfait), relaxation (eq. relaxation-d1q3q3) with the rates of step (iii), the
 * entropy-production source of eq. (NS-rho-J-zeta), f_d* = M^{-1} m*, and streaming
 * (eq. iteration-d1q3q3).
 *
 * Conventions
 *  - Lattice units: dx = 1, dt = 1/lambda. A step does not depend on dx once nu = sigma_e lambda dx
 *    (eq. nu-d1q3q3) and centred differences are used, so no dx is taken.
 *  - A context holds B >= 1 independent lattices of lengths N[b], concatenated back to back
 *    (lattice b occupies nodes offset[b] .. offset[b] + N[b] - 1, offset[0] = 0). Per-node arrays
 *    passed to or returned from the library are float64 and indexed by that global node number.
 *  - Pointers to per-node arrays may be host or device pointers (told apart with
 *    cudaPointerGetAttributes). Host arrays are staged through a device buffer and the call
 *    synchronises the stream before returning; device arrays are used in place and the call only
 *    enqueues work on the context's stream (except where stated). lbm_set_state,
 *    lbm_set_state_entropy and lbm_moments read or write page-locked (pinned) host arrays in place
 *    from their kernels, over the CPU-GPU link, without the staging copy; they still synchronise.
 *  - All GPU work is enqueued on the stream given at creation (NULL = legacy default stream).
 *  - Ownership: the library owns the context and its device state; the caller owns every array
 *    it passes. Device memory is obtained through the allocator installed with
 *    lbm_set_allocator (cudaMalloc/cudaFree if none).
 *  - Every function returns LBM_OK (0) or a negative status; lbm_last_error(ctx) then describes it.
 *    A failed call leaves the context usable unless the status is LBM_ERR_CUDA.
 */
#ifndef LBM_D1Q3Q3_H
#define LBM_D1Q3Q3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define LBM_OK 0
#define LBM_ERR_INVALID_ARG (-1) /* N < 3, lambda <= 0, a rate outside (0, 2), unknown bc ... */
#define LBM_ERR_CUDA (-2)        /* a CUDA runtime call or kernel launch failed */
#define LBM_ERR_OOM (-3)         /* the allocator returned NULL */
#define LBM_ERR_UNSTABLE (-4)    /* diagnostics found a non-finite value, rho <= 0 or T <= 0 */
#define LBM_ERR_TIMEOUT (-5)     /* a bounded device-side wait expired */
#define LBM_ERR_IO (-6)          /* checkpoint file could not be written or read, or mismatched */
#define LBM_ERR_TOO_LARGE (-7)   /* input larger than a fixed-size scratch area allows */

/* Boundary conditions (per lattice). Periodic is the paper's (section 9). Bounce-back is not in
 * the paper: halfway bounce-back at both ends, f+(0) <- f-*(0), f-(N-1) <- f+*(N-1) (same for g),
 * with source ghosts u_{-1} = -u_0, T_{-1} = T_0 (an adiabatic no-slip wall), mirrored at the
 * right end. */
enum { LBM_BC_PERIODIC = 0, LBM_BC_BOUNCEBACK = 1 };

/* Storage/arithmetic precision of the populations.
 * LBM_F64: FP64 storage and arithmetic.
 * LBM_F32_SHIFTED: FP32 storage and arithmetic of the shifted populations f - w, where w are the
 *   populations of the rest state (rho0, u = 0, s = s0) (the same shift is used in FP64).
 * LBM_F64_DF: FP64 storage of the shifted populations; the time step computes in double-float (each
 *   value an unevaluated sum of two FP32 numbers, about 48 significant bits) on the FP32 pipes, which
 *   GB300 runs far faster than its FP64 pipe. Results agree with LBM_F64 and the FP64 reference within
 *   the FP64 tolerance (1e-12 relative after 1000 steps; about 1e-14 per step); initialisation,
 *   moments and diagnostics run in FP64 as for LBM_F64, the adjoint in double-float.
 *   Only LBM_MODE_LAUNCH; kernel configurations: steps_per_launch in {1, 2, 4, 8}, block_threads in
 *   {128, 256, 512}, nodes_per_thread in {1, 2, 4} (2 and 4 on paired FP32 lanes, bitwise equal to 1).
 *   The two- and three-dimensional schemes, one step per launch, store the (hi, lo) pairs themselves
 *   (8 bytes a population, as FP64) so that their steps convert nothing on the FP64 pipe. */
enum { LBM_F64 = 0, LBM_F32_SHIFTED = 1, LBM_F64_DF = 2 };

/* Relaxation rates of step (iii). s_e is the free rate (eq. henon-d1q3q3, nu = sigma_e lambda dx).
 * s_psi <= 0 selects the coupling of eq. (lien-sigma-sigma), sigma_psi = (3/2)(gamma/Pr) sigma_e.
 * s_eps <= 0 selects s_eps = 1.5 (sections 4 and 8). Every rate used must lie in (0, 2). */
typedef struct {
  double s_e, s_psi, s_eps;
} lbm_rates;

/* Physical constants shared by all lattices of a context. A NULL lbm_phys selects the section 9
 * values: gamma = 1.4, Pr = 1, c_p = 1, rho0 = 1, s0 = 0, p0 = rho0 c0^2 / gamma with
 * c0 = lambda / 2, source on, nonlinear equilibria. p0 <= 0 selects that p0 as well. rho0 is both
 * the scale of M (eq. M-d1q3q3) and the reference density of eq. (gaz-parfait); s0 its reference
 * entropy.
 * equilibria = 0: the nonlinear equilibria of section 8. equilibria = 1: the linear equilibria of
 *   eq. (equilibres-NS-linearise) (section 7) around the state (rho0, u0_lin, s0_lin) with
 *   c0^2 = gamma p0 / rho0, as printed; their units hold only for lambda = c_p = 1, which is
 *   required, and the linearised system has no entropy production, so source_on must be 0. */
typedef struct {
  double gamma, Pr, cp, rho0, p0, s0;
  int32_t source_on;  /* 1: entropy-production source of eq. (NS-rho-J-zeta); 0: off */
  int32_t equilibria; /* 0 nonlinear (section 8), 1 linear (section 7) */
  double u0_lin, s0_lin;
} lbm_phys;

/* Device allocator used for all device memory of contexts created afterwards.
 * alloc(bytes, stream, user) returns a device pointer or NULL; free(ptr, user) releases it.
 * Passing NULL for both restores cudaMalloc/cudaFree. Not thread-safe with concurrent creates. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*lbm_free_fn)(void *ptr, void *user);
int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void *user);

typedef struct lbm_ctx lbm_ctx;

/* One periodic or bounce-back lattice of N >= 3 nodes. rates: one lbm_rates. precision: LBM_F64 or
 * LBM_F32_SHIFTED. phys: NULL for the section 9 defaults. stream: a cudaStream_t or NULL.
 * The state is undefined until lbm_set_state (or lbm_load / lbm_set_populations). */
int lbm_create(lbm_ctx **out, int64_t N, double lambda, const lbm_rates *rates, int32_t bc,
               int32_t precision, const lbm_phys *phys, void *stream);

/* B >= 1 independent lattices in one context (host arrays): N[B] lengths (each >= 3), rates[B],
 * bc[B], s0[B] per-lattice reference entropy of eq. (gaz-parfait) (NULL: phys->s0 for all).
 * Lattices advance together in one kernel per launch (ragged tiles, no inter-lattice coupling). */
int lbm_create_batch(lbm_ctx **out, int32_t B, const int64_t *N, double lambda, const lbm_rates *rates,
                     const int32_t *bc, const double *s0, int32_t precision, const lbm_phys *phys,
                     void *stream);

void lbm_destroy(lbm_ctx *ctx);
const char *lbm_last_error(const lbm_ctx *ctx);
int64_t lbm_total_nodes(const lbm_ctx *ctx);  /* sum of N[b] */
int64_t lbm_steps_done(const lbm_ctx *ctx);   /* time steps taken since the last state set/load */

/* Equilibrium initial state f_d = M^{-1} m_eq(rho, J = rho u, zeta = rho s) from per-node rho, u
 * and pressure p (the specific entropy s follows from eq. (gaz-parfait)). Arrays of
 * lbm_total_nodes() float64, host or device. Resets the step counter. Computed in FP64 and rounded
 * once to the storage type; for LBM_F32_SHIFTED the logarithms and the exponential are evaluated in
 * double-float (about 48 bits), so the stored floats are the FP64 ones but for rare one-ulp ties. */
int lbm_set_state(lbm_ctx *ctx, const double *rho, const double *u, const double *p);
/* Same from rho, u and the specific entropy s. */
int lbm_set_state_entropy(lbm_ctx *ctx, const double *rho, const double *u, const double *s);

/* Advances every lattice by nsteps >= 0 time steps (enqueued; no synchronisation). */
int lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* Moments m = (rho, J, zeta, e, psi, eps) per node (eq. M-d1q3q3) of the current state, each into a
 * caller array of lbm_total_nodes() float64 (host or device); any pointer may be NULL. */
int lbm_moments(lbm_ctx *ctx, double *rho, double *J, double *zeta, double *e, double *psi,
                double *eps);

/* Raw populations as float64, plane-major [6][lbm_total_nodes()] in the order
 * (f0, f+, f-, g0, g+, g-) (the shift of LBM_F32_SHIFTED removed), host or device. */
int lbm_get_populations(lbm_ctx *ctx, double *fd);
/* Sets the populations from the same layout (rounded to FP32 for LBM_F32_SHIFTED after shifting). */
int lbm_set_populations(lbm_ctx *ctx, const double *fd);

/* Per-lattice FP64 sums, deterministic (fixed reduction order): sums[4 b + k] for k = 0..3 is
 * sum rho, sum J, sum zeta and sum of the total energy p/(gamma-1) + rho u^2/2 over lattice b;
 * flags[b] has bit 0 for a non-finite population, bit 1 for rho <= 0, bit 2 for T <= 0.
 * Host arrays (B * 4 and B entries); synchronises. Returns LBM_ERR_UNSTABLE if any flag is set
 * (the arrays are still filled). */
int lbm_diagnostics(lbm_ctx *ctx, double *sums, int32_t *flags);

/* Kernel configuration: steps_per_launch k in {1, 2, 4, 8} (temporal blocking: k steps per HBM
 * round trip, 2k halo nodes recomputed on each tile side), block_threads in {128, 256, 512, 1024}
 * and nodes_per_thread in {1, 2, 4} (tile width block_threads * nodes_per_thread; 1024 x 4 is not
 * supported; the tile must keep at least 32 interior nodes). 0 keeps the current value. */
int lbm_set_config(lbm_ctx *ctx, int32_t steps_per_launch, int32_t block_threads, int32_t nodes_per_thread);
int lbm_get_config(const lbm_ctx *ctx, int32_t *steps_per_launch, int32_t *block_threads,
                   int32_t *nodes_per_thread);

/* Execution mode of lbm_step.
 * LBM_MODE_LAUNCH: one kernel launch per k steps (default).
 * LBM_MODE_PERSISTENT: all whole blocks of k steps in ONE persistent launch; CTAs claim work units
 *   (a block of k steps on 16 consecutive tiles) in order, and a unit waits only for the units holding
 *   its tiles' lattice neighbours to finish the previous block (bounded spin; see lbm_status).
 *   Results are bitwise equal to LBM_MODE_LAUNCH.
 * LBM_MODE_PERSISTENT_GRAPH: the same launch (with its counter resets) captured once in a CUDA graph
 *   per (number of blocks, buffer parity, configuration) and replayed.
 * A remainder of nsteps not divisible by k runs as ordinary launches. */
enum { LBM_MODE_LAUNCH = 0, LBM_MODE_PERSISTENT = 1, LBM_MODE_PERSISTENT_GRAPH = 2 };
int lbm_set_mode(lbm_ctx *ctx, int32_t mode);

/* Synchronises the stream and reports whether a bounded device-side wait of a persistent launch
 * expired since the last call: LBM_ERR_TIMEOUT (the state is then not a valid time step; set it
 * again) or LBM_OK. Clears the status word. */
int lbm_status(lbm_ctx *ctx);

/* Failure-detection test hook for persistent launches: spin_limit >= 1 polls (about 100 ns apart)
 * before a wait gives up (default 2e7), and withhold_tile >= 0 names a work unit (16 consecutive tiles)
 * whose first time block is never computed nor released, so that its neighbours' waits must expire
 * (-1: none). */
int lbm_debug_persistent(lbm_ctx *ctx, int64_t spin_limit, int64_t withhold_tile);

/* Bounds-checked debug build (the library compiled with -DLBM_DEBUG_BOUNDS, a stand-in for a memory
 * checker): the step, persistent, double-float and adjoint kernels check every global and shared-memory
 * index against the extent it must lie in, count and skip an access outside it instead of faulting.
 * Synchronises the device, then returns in *violations the number of skipped accesses since the last
 * call (and clears it), with the first bad index and its extent (-1 when none); a build without the
 * checks returns *violations = -1. LBM_ERR_INVALID_ARG on a null pointer, LBM_ERR_CUDA on a CUDA error. */
int lbm_debug_bounds(int64_t *violations, int64_t *first_index, int64_t *first_extent);

/* Test hook: applies one of the FP32 functions of the node update elementwise to n floats
 * (device pointers x -> y, enqueued on stream): fn 0 = log(1+x) as evaluated on paired lanes,
 * 1 = log(1+x) on single lanes (CUDA's log1pf), 2 = exp(x)-1 on paired lanes, 3 = exp(x)-1 on
 * single lanes (CUDA's expm1f), 4 = the FP32 reciprocal. */
int lbm_debug_eval_f32(const float *x, float *y, int64_t n, int32_t fn, void *stream);

/* Test hook: the double-float operations of the LBM_F64_DF step, elementwise on n doubles (device
 * pointers, enqueued on stream), each input split into hi + lo floats and the result summed back to
 * FP64: fn 0 = log(1+x), 1 = exp(x)-1, 2 = 1/x, 3 = x*x2, 4 = x+x2, 5 = x*x2[i] + x2[(i+1) mod n];
 * fn 6, 7, 8 = the FP64-lane log(1+x), exp(x)-1 and 1/x of the LBM_F64 node update (double-float series
 * and FP64 Newton steps), on the FP64 input (x2 unused and may be NULL for fn 0-2 and 6-8). */
int lbm_debug_eval_df(const double *x, const double *x2, double *y, int64_t n, int32_t fn, void *stream);

/* Times every valid (k, block_threads, nodes_per_thread) on the current state (which is left
 * unchanged; each trial writes only the second buffer, over at most 16384 tiles) and keeps the
 * fastest per node-update. trials >= 1 timed launches per candidate. Synchronises. Needs a state. */
int lbm_autotune(lbm_ctx *ctx, int32_t trials);

/* Checkpoint: writes / reads the populations, step counter and parameters to a host file. A load
 * must match the context's lattice lengths, precision and parameters exactly; the resumed run is
 * bitwise identical to an uninterrupted one. Synchronises. */
int lbm_save(lbm_ctx *ctx, const char *path);
int lbm_load(lbm_ctx *ctx, const char *path);

/* Reverse mode (adjoint) of T time steps, with sqrt(T) checkpointing: the forward run keeps
 * ceil(T / S) checkpoints (S = round(sqrt(T))) and the backward sweep recomputes each segment's S
 * states before stepping the adjoint back through them. Device memory: about ceil(T/S) + S + 1
 * copies of the state, released by lbm_adjoint_release (or lbm_destroy).
 *
 * lbm_adjoint_forward: runs T >= 1 steps from the current state (which must have been set by
 *   lbm_set_state or lbm_set_state_entropy for the rho/u gradients below to be meaningful; the
 *   population gradient is exact for any state) and leaves the state at time T.
 * lbm_adjoint_backward: given dL/drho(T) per node (float64, host or device), returns
 *   dL/drho(0) and dL/du(0) per node at fixed initial specific entropy (through the equilibrium
 *   initialisation), dL/ds_e and dL/ds_psi per lattice in dL_drates[2 b + 0/1] (s_e and s_psi
 *   taken as independent; nu and kappa of the source follow s_e as in eq. (nu-d1q3q3)), and
 *   optionally dL/df(0) as float64 plane-major [6][N]. Outputs may be NULL, host or device.
 *   Rate gradients are accumulated in FP64 in a fixed order. Synchronises.
 * lbm_adjoint: forward T steps, loss = sum over all nodes of (rho(T) - rho_target)^2 (FP64,
 *   fixed-order reduction) into *loss, then the backward sweep. */
int lbm_adjoint_forward(lbm_ctx *ctx, int64_t T);
int lbm_adjoint_backward(lbm_ctx *ctx, const double *dL_drho_T, double *dL_drho0, double *dL_du0,
                         double *dL_drates, double *dL_dfd0);
int lbm_adjoint(lbm_ctx *ctx, int64_t T, const double *rho_target, double *loss, double *dL_drho0,
                double *dL_du0, double *dL_drates);
int lbm_adjoint_release(lbm_ctx *ctx);
/* Reverse steps per launch of the backward sweep: 1, 2, 4 or 8 (0 selects the default: 4 for
 * LBM_F32_SHIFTED and LBM_F64_DF, where it halves the backward time against 1, and 1 for LBM_F64,
 * whose arithmetic bound makes the on-chip recomputation of inner states a net cost). A LBM_F64_DF
 * context runs its forward steps, the recomputation and the reverse steps in double-float. Each
 * segment is split into blocks of that many steps; the states at the block starts are recomputed
 * with launches of the step kernel, and one launch per block recomputes the block's inner states on
 * chip and runs its reverse steps (HBM traffic per node-step falls with the depth; the tile halo,
 * 4k - 2 nodes per side of 256, grows with it). The gradients do not depend on it beyond rounding
 * (FP64: the forward recomputation is bitwise that of the step kernel). */
int lbm_adjoint_set_config(lbm_ctx *ctx, int32_t steps_per_launch);
int lbm_adjoint_get_config(const lbm_ctx *ctx, int32_t *steps_per_launch);

/* Diagnostics that allocate no device memory. The paper has no counterpart: this exists for callers
 * that cannot call cudaMalloc (code inside host callbacks or another framework's memory pool, or a
 * process whose device memory is all handed to its own allocator). It computes, for ONE lattice,
 * the same FP64 sums as lbm_diagnostics (sum rho, sum J, sum zeta, sum of p/(gamma-1) + rho u^2/2)
 * and the same flag bits, from populations the caller holds.
 *  fd: DEVICE pointer to float64 populations, plane-major [6][N] in the order (f0, f+, f-, g0, g+, g-)
 *      (the layout lbm_get_populations writes). N >= 1 and N <= 2^26 (else LBM_ERR_TOO_LARGE).
 *  lambda, phys: as for lbm_create (phys NULL = the lbm_phys defaults, see lbm_phys; phys->s0 is the
 *      entropy reference).
 *  sums[4], flags[1]: both host or both device pointers. Host outputs: the call synchronises `stream`
 *      and returns LBM_ERR_UNSTABLE if a flag is set. Device outputs: the call only enqueues work.
 *  stream: cudaStream_t or NULL.
 * fd, and sums/flags when they are device pointers, must be memory of the current device (or managed
 * memory): memory of another GPU returns LBM_ERR_INVALID_ARG, as does a host fd. A CUDA error already
 * pending on the calling thread (from the caller's earlier work) returns LBM_ERR_CUDA and is left in
 * place; only this call's own failures are cleared.
 * The reduction scratch is a file-scope __device__ array of about 300 KB that every GPU loading the
 * library holds until exit; its address is looked up once per device on the first call with that
 * device current, so make the first call on each device before any stream capture. Every call
 * shares the array: calls whose kernels overlap on the GPU race (issue them on one stream). */
int lbm_diagnostics_noalloc(const double *fd, int64_t N, double lambda, const lbm_phys *phys, double *sums,
                            int32_t *flags, void *stream);
/* Test hook of the pointer-placement rule of lbm_diagnostics_noalloc, evaluated without any CUDA call:
 * each pointer is described by its kind (0 host, 1 device memory, 2 managed memory) and, for device
 * memory, its device ordinal; returns LBM_OK when the call would accept that placement on
 * current_device, else LBM_ERR_INVALID_ARG. */
int lbm_debug_noalloc_placement(int32_t current_device, int32_t fd_kind, int32_t fd_device, int32_t sums_kind,
                                int32_t sums_device, int32_t flags_kind, int32_t flags_device);

/* ------------------------------------------------------------------------------------------------
 * Finite-difference comparison solver (section 9). The paper checks its lattice Boltzmann results
 * against a finite-difference program for the (rho, J, zeta) system of eq. (NS-rho-J-zeta) with
 * second-order centred differences in space and explicit first-order time steps. The stencil is not
 * printed; the one built here is in conservation form on a periodic grid of N nodes:
 *   W = (rho, J, zeta), u = J/rho, s = zeta/rho, p and T from eq. (gaz-parfait);
 *   W_j(t + dt) = W_j - dt/(2 dx) (F_{j+1} - F_{j-1}) + dt/dx (Phi_{j+1/2} - Phi_{j-1/2}) + dt (0, 0, S_j),
 *   F = (J, rho u^2 + p, zeta u), Phi_{j+1/2} = (0, a (u_{j+1} - u_j)/dx, b (T_{j+1} - T_j)/dx) with
 *   a, b the means over nodes j, j+1 of rho nu and kappa/T, kappa = rho nu c_p / Pr, and the entropy
 *   production S = (rho nu/T)(d_x u)^2 + (kappa/T^2)(d_x T)^2 from centred derivatives (the
 *   differences of step (vii) of section 8); S is dropped when phys->source_on = 0.
 * The sums of rho and J are conserved exactly (up to rounding); the sum of zeta grows by dt sum S.
 * Explicit centred differences are stable only for dt <= 2 nu / (|u| + c)^2 and dt <= dx^2 / (2 nu)
 * (roughly); the caller chooses dt. Same status codes, pointer and stream conventions as above. */
typedef struct lbm_fd_ctx lbm_fd_ctx;

/* N >= 3 periodic nodes of spacing dx > 0, time step dt > 0, kinematic viscosity nu >= 0.
 * precision: LBM_F64, or LBM_F32_SHIFTED (FP32 storage and arithmetic of (rho - rho0, J, zeta - rho0 s0)).
 * phys: gamma, Pr, c_p, rho0, p0, s0 and source_on of eq. (gaz-parfait) and eq. (NS-rho-J-zeta);
 * NULL selects the section 9 values (gamma = 1.4, Pr = 1, c_p = 1, rho0 = 1, s0 = 0, source on) with
 * p0 = rho0 c0^2 / gamma, c0 = 1/2; p0 <= 0 selects that p0 too. phys->equilibria must be 0. */
int lbm_fd_create(lbm_fd_ctx **out, int64_t N, double dx, double dt, double nu, int32_t precision,
                  const lbm_phys *phys, void *stream);
void lbm_fd_destroy(lbm_fd_ctx *ctx);
const char *lbm_fd_last_error(const lbm_fd_ctx *ctx);
int64_t lbm_fd_steps_done(const lbm_fd_ctx *ctx);
/* State from per-node rho, u and specific entropy s (N float64 each, host or device); resets the
 * step counter. */
int lbm_fd_set_state(lbm_fd_ctx *ctx, const double *rho, const double *u, const double *s);
/* State from the conserved fields W, plane-major [3][N] float64 (rho, J, zeta), host or device. */
int lbm_fd_set_fields(lbm_fd_ctx *ctx, const double *W);
/* Advances nsteps >= 0 time steps of size dt (enqueued; no synchronisation). */
int lbm_fd_step(lbm_fd_ctx *ctx, int64_t nsteps);
/* rho, J, zeta per node into caller arrays of N float64 (host or device; any may be NULL). */
int lbm_fd_fields(lbm_fd_ctx *ctx, double *rho, double *J, double *zeta);
/* FP64 sums (host sums[4]: sum rho, sum J, sum zeta, sum of p/(gamma-1) + rho u^2/2) and flag bits
 * (host flags[1]: bit 0 non-finite field, bit 1 rho <= 0, bit 2 T <= 0) in a fixed reduction order;
 * synchronises; LBM_ERR_UNSTABLE if a flag is set (outputs still filled). */
int lbm_fd_diagnostics(lbm_fd_ctx *ctx, double *sums, int32_t *flags);
/* Kernel configuration: steps_per_launch k in 1..16 (temporal blocking, k halo nodes per tile side),
 * block_threads in {128, 256, 512}, nodes_per_thread in {1, 2, 4}, with block_threads *
 * nodes_per_thread - 2k >= 32. 0 keeps the current value. Results do not depend on it beyond
 * rounding of contracted multiply-adds. Default 4, 256, 2. */
int lbm_fd_set_config(lbm_fd_ctx *ctx, int32_t steps_per_launch, int32_t block_threads, int32_t nodes_per_thread);
int lbm_fd_get_config(const lbm_fd_ctx *ctx, int32_t *steps_per_launch, int32_t *block_threads,
                      int32_t *nodes_per_thread);
/* Times every valid configuration on the current state (left unchanged; each trial writes only the
 * spare buffer, over at most 16384 tiles) and keeps the fastest per node-update. trials >= 1 timed
 * launches per candidate. Synchronises. Needs a state. */
int lbm_fd_autotune(lbm_fd_ctx *ctx, int32_t trials);

/* ------------------------------------------------------------------------------------------------
 * Single-distribution D1Q3 schemes (sections 2 and 4), the building blocks the coupled scheme is made
 * of. One periodic lattice of N nodes, dx = 1, dt = 1/lambda, three populations (f0, f+, f-) with the
 * moments of eq. (M-d1q3), m = scale (sum f, lambda (f+ - f-), lambda^2 (f+ + f- - 2 f0)).
 *  LBM_D1Q3_FLUID (section 2): m = (rho, J, e); rho, J conserved; e relaxed with s_e toward
 *    e_eq = 3 (rho u^2 + p) - 2 lambda^2 rho (eq. energie-equilibre), with the isentropic pressure
 *    p = p0 (rho / rho0)^gamma (rho0 = scale). The paper names the isentropic Navier-Stokes equations
 *    but no pressure law; this polytropic one is eq. (gaz-parfait) at s = s0.
 *  LBM_D1Q3_ADVECTION_DIFFUSION (section 4): m = (zeta, psi, eps); zeta conserved; psi relaxed with
 *    s_psi toward psi_eq = u0 zeta, eps with s_eps toward eps_eq = alpha lambda^2 zeta. Section 4
 *    identifies the diffusivity: ((2 + alpha)/3 lambda^2 - u0^2)(1/s_psi - 1/2) dt = kappa; it states
 *    stability for -2 < alpha < 1.
 * Then f* = M^{-1} m* and advection: f0 stays, f+ moves to x + dx, f- to x - dx.
 * Same status codes, pointer and stream conventions as the coupled scheme. */
enum { LBM_D1Q3_FLUID = 0, LBM_D1Q3_ADVECTION_DIFFUSION = 1 };

typedef struct {
  int32_t scheme; /* LBM_D1Q3_FLUID or LBM_D1Q3_ADVECTION_DIFFUSION */
  int32_t pad;
  double lambda;  /* > 0 */
  double scale;   /* rho0 (fluid) or zeta0 (advection-diffusion) of eq. (M-d1q3); <= 0 selects 1 */
  double s_e;     /* fluid: relaxation rate of e, in (0, 2) */
  double gamma;   /* fluid: isentropic exponent >= 1; <= 0 selects 1.4 */
  double p0;      /* fluid: pressure at rho0; <= 0 selects rho0 c0^2 / gamma with c0 = lambda / 2 */
  double u0;      /* advection-diffusion: advection velocity */
  double alpha;   /* advection-diffusion: eps_eq = alpha lambda^2 zeta */
  double kappa;   /* advection-diffusion: diffusivity, used when s_psi <= 0 (identification above) */
  double s_psi;   /* advection-diffusion: rate of psi in (0, 2); <= 0: from kappa */
  double s_eps;   /* advection-diffusion: rate of eps in (0, 2); <= 0 selects 1.5 (section 4) */
} lbm_d1q3_params;

typedef struct lbm_d1q3_ctx lbm_d1q3_ctx;

/* N >= 3 periodic nodes; precision LBM_F64 or LBM_F32_SHIFTED (FP32 populations shifted by those of
 * the rest state rho0, J = 0 or zeta0). LBM_ERR_INVALID_ARG for a rate outside (0, 2), lambda <= 0,
 * or a kappa that no s_psi in (0, 2) reproduces. */
int lbm_d1q3_create(lbm_d1q3_ctx **out, int64_t N, const lbm_d1q3_params *params, int32_t precision,
                    void *stream);
void lbm_d1q3_destroy(lbm_d1q3_ctx *ctx);
const char *lbm_d1q3_last_error(const lbm_d1q3_ctx *ctx);
int64_t lbm_d1q3_steps_done(const lbm_d1q3_ctx *ctx);
/* The rates in use: fluid (s_e, 0); advection-diffusion (s_psi, s_eps). Host outputs, may be NULL. */
int lbm_d1q3_rates(const lbm_d1q3_ctx *ctx, double *s1, double *s2);
/* Equilibrium state from per-node conserved moments (N float64, host or device): fluid m0 = rho,
 * m1 = J; advection-diffusion m0 = zeta (m1 unused, may be NULL). Resets the step counter. */
int lbm_d1q3_set_state(lbm_d1q3_ctx *ctx, const double *m0, const double *m1);
/* Advances nsteps >= 0 time steps (enqueued; no synchronisation). */
int lbm_d1q3_step(lbm_d1q3_ctx *ctx, int64_t nsteps);
/* Moments m = M f per node: (rho, J, e) or (zeta, psi, eps), N float64 each, host or device, any NULL. */
int lbm_d1q3_moments(lbm_d1q3_ctx *ctx, double *m0, double *m1, double *m2);
/* Populations (f0, f+, f-) as float64, plane-major [3][N], host or device (shift removed / applied). */
int lbm_d1q3_get_populations(lbm_d1q3_ctx *ctx, double *f);
int lbm_d1q3_set_populations(lbm_d1q3_ctx *ctx, const double *f);
/* FP64 sums of the three moments over the lattice in a fixed order (host sums[3]) and flag bits
 * (host flags[1]: bit 0 non-finite population, bit 1 rho <= 0 for the fluid scheme); synchronises;
 * LBM_ERR_UNSTABLE if a flag is set (outputs still filled). */
int lbm_d1q3_sums(lbm_d1q3_ctx *ctx, double *sums, int32_t *flags);
/* Kernel configuration: steps_per_launch k in 1..64 (k halo nodes per tile side), block_threads in
 * {128, 256, 512}, nodes_per_thread in {1, 2, 4, 8}, block_threads * nodes_per_thread - 2k >= 32;
 * 0 keeps the current value. Default 8, 256, 4. */
int lbm_d1q3_set_config(lbm_d1q3_ctx *ctx, int32_t steps_per_launch, int32_t block_threads,
                        int32_t nodes_per_thread);
int lbm_d1q3_get_config(const lbm_d1q3_ctx *ctx, int32_t *steps_per_launch, int32_t *block_threads,
                        int32_t *nodes_per_thread);
/* Times every valid configuration on the current state (left unchanged; trials write only the spare
 * buffer, over at most 16384 tiles) and keeps the fastest per node-update. Synchronises. */
int lbm_d1q3_autotune(lbm_d1q3_ctx *ctx, int32_t trials);

/* ---------------------------------------------------------------------------------------------
 * Two-dimensional coupled D2Q9-D2Q5 scheme for (rho, J, zeta). The paper's conclusion names this
 * coupling as the next step and specifies nothing more; the scheme here carries section 8 to two
 * dimensions (the readings of the CPU reference): D2Q9 populations f0..f8 for the velocities
 * lambda c, c = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1), D2Q5 populations g0..g4
 * for c = (0,0) (1,0) (0,1) (-1,0) (0,-1), periodic in x and y.
 *  - Moments (rows scaled by rho0, the entropy rows also by c_p, as in eq. M-d1q3q3): rho, J,
 *    e = sum (3|v|^2 - 4 lambda^2) f, xx = sum (vx^2 - vy^2) f, xy = sum vx vy f,
 *    q = sum (3|v|^2 - 5 lambda^2) v f, h = sum (4 lambda^4 - 21/2 lambda^2 |v|^2 + 9/2 |v|^4) f;
 *    zeta, psi = c_p sum v g, eps = c_p sum (3|v|^2 - 4 lambda^2) g, xi = c_p sum (vx^2 - vy^2) g.
 *  - Equilibria, with p(rho, s) of eq. (gaz-parfait), Pi = rho u u + p I and
 *    E = s Pi + (rho c_p lambda^2 / (gamma beta)) log(T/T0) I: e_eq = 3 tr Pi - 4 lambda^2 rho,
 *    xx_eq = Pi_xx - Pi_yy, xy_eq = Pi_xy, q_eq = -lambda^2 J, h_eq = 4 lambda^4 rho
 *    - 6 lambda^2 tr Pi + 9 Pi_xx Pi_yy / rho, psi_eq = zeta u, eps_eq = 3 tr E - 4 lambda^2 zeta,
 *    xi_eq = E_xx - E_yy.
 *  - Rates: s_e (e, xx, xy), s_q, s_h, s_psi, s_eps (eps, xi); sigma_psi = beta (gamma/Pr) sigma_e.
 *    beta = 3/2 (eq. lien-sigma-sigma) makes the scheme the D1Q3Q3 one on one-dimensional data but
 *    leaves its D2Q5 part linearly unstable at the diagonal modes; the default is beta = 9/2.
 *  - Production added to zeta after relaxation: dt [rho nu (2 D:D + (div u)^2) / (3T)
 *    + kappa |grad T|^2 / T^2], nu = sigma_e lambda dx, kappa = rho nu c_p / Pr, centred
 *    differences of u and T at time t; then streaming f_i(x + c_i dx) = f_i*(x).
 * Storage: 14 planes of nx * ny values (x fastest), LBM_F64 / LBM_F64_DF or LBM_F32_SHIFTED (populations less
 * those of the rest state rho0, u = 0, s0, in units of rho0). Same status codes and pointer
 * conventions as the other schemes: arrays may be host or device memory. */
typedef struct {
  double gamma;   /* > 1 */
  double Pr;      /* > 0 */
  double cp;      /* > 0 */
  double rho0;    /* > 0 */
  double p0;      /* pressure at rho0, s0; <= 0 selects rho0 c0^2 / gamma with c0 = lambda / 2 */
  double s0;      /* reference entropy */
  double lambda;  /* > 0 */
  double dx;      /* > 0 */
  double beta;    /* coupling of sigma_psi; <= 0 selects 9/2 */
  double s_e;     /* rate of e, xx, xy in (0, 2) */
  double s_psi;   /* <= 0: from beta */
  double s_eps;   /* <= 0 selects 1.5 */
  double s_q;     /* <= 0 selects 1.5 */
  double s_h;     /* <= 0 selects 1.5 */
  int32_t source_on;
  int32_t pad;
} lbm2d_params;

typedef struct lbm2d_ctx lbm2d_ctx;

/* nx, ny >= 3 nodes, precision LBM_F64, LBM_F32_SHIFTED or LBM_F64_DF (planes of 8-byte (hi, lo) FP32 pairs,
 * the node update in double-float on the FP32 pipes; FP64 accuracy). LBM_ERR_INVALID_ARG for a rate outside
 * (0, 2) or a non-positive constant; LBM_ERR_OOM if the two 14-plane state buffers cannot be had. */
int lbm2d_create(lbm2d_ctx **out, int64_t nx, int64_t ny, const lbm2d_params *params, int32_t precision,
                 void *stream);
void lbm2d_destroy(lbm2d_ctx *ctx);
const char *lbm2d_last_error(const lbm2d_ctx *ctx);
int64_t lbm2d_steps_done(const lbm2d_ctx *ctx);
/* The rates in use (s_e, s_psi, s_eps, s_q, s_h): host rates[5]. */
int lbm2d_rates(const lbm2d_ctx *ctx, double *rates);
/* Equilibrium state from the fields rho, ux, uy, s (float64 [ny][nx] each, host or device, all of
 * one kind), computed in FP64 and stored rounded to the storage type. Resets the step counter. */
int lbm2d_set_state(lbm2d_ctx *ctx, const double *rho, const double *ux, const double *uy, const double *s);
/* Advances nsteps >= 0 time steps, one launch each (enqueued; no synchronisation). */
int lbm2d_step(lbm2d_ctx *ctx, int64_t nsteps);
/* Populations as float64, node-major [ny][nx][14] in the order (f0..f8, g0..g4), shift removed, in
 * units of rho0 (the layout of the CPU reference); host or device. */
int lbm2d_get_populations(lbm2d_ctx *ctx, double *f);
/* The fields rho, ux, uy, s (float64 [ny][nx], host or device, any NULL). */
int lbm2d_fields(lbm2d_ctx *ctx, double *rho, double *ux, double *uy, double *s);

/* ---------------------------------------------------------------------------------------------
 * Three-dimensional coupled D3Q19-D3Q7 scheme for (rho, J, zeta): the second extension the paper's
 * conclusion names, specified nowhere in it; the readings are those of the two-dimensional scheme
 * carried to three dimensions. D3Q19 populations f0..f18 for the velocities lambda c,
 * c = 0; (+-1,0,0) (0,+-1,0) (0,0,+-1) in that order; (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0)
 * (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1); D3Q7 populations g0..g6
 * for c = 0; (+-1,0,0) (0,+-1,0) (0,0,+-1); periodic in x, y and z.
 *  - Moments (rows scaled by rho0, the entropy rows also by c_p; |c|^2 = c.c, each pattern times
 *    lambda^k for its degree k): rho, J; e = 19|c|^2 - 30, pxx = 3cx^2 - |c|^2, pww = cy^2 - cz^2,
 *    pxy, pyz, pxz = cx cy, cy cz, cx cz; q = (5|c|^2 - 9) c; mx, my, mz = (cy^2 - cz^2) cx,
 *    (cz^2 - cx^2) cy, (cx^2 - cy^2) cz; eps = (21|c|^4 - 53|c|^2 + 24)/2, pixx = (3|c|^2 - 5)
 *    (3cx^2 - |c|^2), piww = (3|c|^2 - 5)(cy^2 - cz^2); zeta, psi = c, eps7 = 3|c|^2 - 6 (the
 *    one-dimensional row 3|c|^2 - 2d with d = 3), xixx = 3cx^2 - |c|^2, xiww = cy^2 - cz^2.
 *  - Equilibria, with p(rho, s) of eq. (gaz-parfait), Pi = rho u u + p I, Q_ab = Pi_aa Pi_bb / rho and
 *    E = s Pi + (rho c_p lambda^2 / (gamma beta)) log(T/T0) I: e = 19 tr Pi - 30 lambda^2 rho,
 *    pxx = 3 Pi_xx - tr Pi, pww = Pi_yy - Pi_zz, pab = Pi_ab, q = -(2/3) lambda^2 J, m = 0,
 *    eps = 12 lambda^4 rho - 16 lambda^2 tr Pi + 21 (Q_xy + Q_yz + Q_xz), pixx = 2 lambda^2 (tr Pi
 *    - 3 Pi_xx) + 3 (Q_xy + Q_xz) - 6 Q_yz, piww = -2 lambda^2 (Pi_yy - Pi_zz) + 3 (Q_xy - Q_xz),
 *    psi = zeta u, eps7 = 3 tr E - 6 lambda^2 zeta, xixx = 3 E_xx - tr E, xiww = E_yy - E_zz.
 *  - Rates: s_e (e and the five second-order deviators), s_q (q, m), s_h (eps, pixx, piww), s_psi,
 *    s_eps (eps7, xixx, xiww); sigma_psi = beta (gamma/Pr) sigma_e. beta = 3/2 (eq. lien-sigma-sigma)
 *    makes the scheme the D1Q3Q3 one on one-dimensional data along any axis but leaves its D3Q7
 *    part linearly unstable; the default is beta = 9, with s_q = 1.5, s_h = 1.2, s_eps = 1.0
 *    (linearly stable at rest for s_e up to 1.5 and s - s0 up to 0.05 c_p).
 *  - Production added to zeta after relaxation: dt [rho nu (2 D:D + (div u)^2) / (3T)
 *    + kappa |grad T|^2 / T^2], nu = sigma_e lambda dx, kappa = rho nu c_p / Pr, centred
 *    differences of u and T at time t; then streaming f_i(x + c_i dx) = f_i*(x).
 * Storage: 26 planes of nx * ny * nz values (x fastest, then y, then z), LBM_F64 / LBM_F64_DF or
 * LBM_F32_SHIFTED (populations less those of the rest state rho0, u = 0, s0, in units of rho0). Same status codes
 * and pointer conventions as the other schemes: arrays may be host or device memory. */
typedef struct {
  double gamma;   /* > 1 */
  double Pr;      /* > 0 */
  double cp;      /* > 0 */
  double rho0;    /* > 0 */
  double p0;      /* pressure at rho0, s0; <= 0 selects rho0 c0^2 / gamma with c0 = lambda / 2 */
  double s0;      /* reference entropy */
  double lambda;  /* > 0 */
  double dx;      /* > 0 */
  double beta;    /* coupling of sigma_psi; <= 0 selects 9 */
  double s_e;     /* rate of e and the second-order deviators, in (0, 2) */
  double s_psi;   /* <= 0: from beta */
  double s_eps;   /* <= 0 selects 1.0 */
  double s_q;     /* <= 0 selects 1.5 */
  double s_h;     /* <= 0 selects 1.2 */
  int32_t source_on;
  int32_t pad;
} lbm3d_params;

typedef struct lbm3d_ctx lbm3d_ctx;

/* nx, ny, nz >= 3 nodes (nx up to 2^30, ny up to 4 * 65535, nx ny nz up to 2^33), precision
 * LBM_F64, LBM_F32_SHIFTED or LBM_F64_DF (planes of 8-byte (hi, lo) FP32 pairs, the node update in
 * double-float on the FP32 pipes; FP64 accuracy). LBM_ERR_INVALID_ARG for another precision, a size out of range, a rate
 * outside (0, 2) or a non-positive constant; LBM_ERR_OOM if the two 26-plane state buffers cannot be
 * had. */
int lbm3d_create(lbm3d_ctx **out, int64_t nx, int64_t ny, int64_t nz, const lbm3d_params *params,
                 int32_t precision, void *stream);
void lbm3d_destroy(lbm3d_ctx *ctx);
const char *lbm3d_last_error(const lbm3d_ctx *ctx);
int64_t lbm3d_steps_done(const lbm3d_ctx *ctx);
/* The rates in use (s_e, s_psi, s_eps, s_q, s_h): host rates[5]. */
int lbm3d_rates(const lbm3d_ctx *ctx, double *rates);
/* Equilibrium state from the fields rho, ux, uy, uz, s (float64 [nz][ny][nx] each, host or device, all
 * of one kind), computed in FP64 and stored rounded to the storage type. Resets the step counter. */
int lbm3d_set_state(lbm3d_ctx *ctx, const double *rho, const double *ux, const double *uy, const double *uz,
                    const double *s);
/* Advances nsteps >= 0 time steps, one launch each (enqueued; no synchronisation). */
int lbm3d_step(lbm3d_ctx *ctx, int64_t nsteps);
/* Populations as float64, node-major [nz][ny][nx][26] in the order (f0..f18, g0..g6), shift removed, in
 * units of rho0 (the layout of the CPU reference); host or device. */
int lbm3d_get_populations(lbm3d_ctx *ctx, double *f);
/* The fields rho, ux, uy, uz, s (float64 [nz][ny][nx], host or device, any NULL). */
int lbm3d_fields(lbm3d_ctx *ctx, double *rho, double *ux, double *uy, double *uz, double *s);
/* Kernel configuration: tile rows ty in {4, 8}, or 16 for FP32 (tiles of 32 x ty columns); the number
 * of planes each CTA marches through along z (zc >= 1, capped at nz and raised to nz / 65535 where
 * the grid needs it); keep, where a thread holds its
 * populations of plane z across the kernel's barrier: 1 in registers, 2 in a shared buffer of its own
 * (FP32 with ty 4 only), 0 nowhere (it reads them again after the barrier). 0 keeps the current ty or
 * zc, -1 the current keep. Defaults: 4 rows; keep 2 for FP32 on 4 rows, else 0; zc from the lattice
 * so that the grid fills the GPU about eight times. Every configuration gives the same results bit
 * for bit. */
int lbm3d_set_config(lbm3d_ctx *ctx, int32_t ty, int32_t zc, int32_t keep);
int lbm3d_get_config(const lbm3d_ctx *ctx, int32_t *ty, int32_t *zc, int32_t *keep);

#ifdef __cplusplus
}
#endif

#endif /* LBM_D1Q3Q3_H */
