/* lbcad.h -- C ABI of the GB300 hybrid lattice-Boltzmann library for 3D active
 * cholesteric droplets (Carenza, Gonnella & Negro, arXiv:2011.00287).
 *
 * One timestep ("hybrid step") advances, on a periodic nx*ny*nz lattice:
 *   - the D3Q19 populations f_i by BGK collision with a body force and streaming
 *     (Sec. 3, Eqs. 6-8; Eq. 7 read as BGK with Guo forcing, Eq. 9-11 read as a
 *     second-order equilibrium with the whole stress divergence entering as the force);
 *   - the tensor order parameter Q (traceless symmetric) by the Beris-Edwards equation
 *     with advection and co-rotation (Sec. 2, Eq. 2);
 *   - the concentration psi = phi - 1 by the Cahn-Hilliard equation (Sec. 2, Eq. 1);
 * with the molecular field H, chemical potential mu and stresses derived from the free
 * energy of Eq. 5 (Landau-de Gennes bulk, one-constant elasticity with the chiral q0 term,
 * binary mixture, interface and anchoring terms) plus the active stress of Eq. 4.
 *
 * All work runs in CUDA kernels on one GPU.  Every call returns LBCAD_OK (0) or a
 * negative LBCAD_E_* code; no C++ exception crosses this boundary.  After an error,
 * lbcad_last_error(ctx) returns a message (valid until the next call on ctx).
 *
 * Field layout.  Every field is row-major [component][z][y][x] (x fastest) with
 * n = nx*ny*nz sites per component.  Field masks select, in this order:
 *   LBCAD_FIELD_G   19 components (15 for LBCAD_D3Q15): pre-collision populations f_i at
 *                   the current time, unshifted, in the order of lbcad_velocity_set();
 *   LBCAD_FIELD_RHO  1 component : rho = sum_i f_i;
 *   LBCAD_FIELD_U    3 components: the fluid velocity u computed in the last step
 *                   ((sum_i f_i c_i + F/2)/rho of the previous time level, sum_i f_i c_i/rho
 *                   with LBCAD_LB_STRESS_EQ; 0 at t = 0);
 *   LBCAD_FIELD_Q    5 components: Q_xx, Q_xy, Q_xz, Q_yy, Q_yz (Q_zz = -Q_xx - Q_yy);
 *   LBCAD_FIELD_PSI  1 component : psi.
 * The exchange type is always double, whatever the compute precision.
 */
#ifndef LBCAD_H
#define LBCAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define LBCAD_OK 0
#define LBCAD_E_INVALID_ARG (-1) /* bad pointer, size, parameter or instance index       */
#define LBCAD_E_OOM (-2)         /* device allocation failed                             */
#define LBCAD_E_CUDA (-3)        /* a CUDA runtime call failed (message has the reason)  */
#define LBCAD_E_TIMEOUT (-4)     /* reserved: no kernel of this library waits on another */
#define LBCAD_E_NAN (-5)         /* a non-finite value was found in a reduction          */
#define LBCAD_E_UNSUPPORTED (-6) /* option not available on this path                    */

/* ---- options --------------------------------------------------------------------- */
#define LBCAD_FP32 0 /* FP32 storage and arithmetic; populations stored as f_i - w_i rho0 */
#define LBCAD_FP64 1 /* FP64 storage and arithmetic; populations stored unshifted         */
#define LBCAD_EULER 0
#define LBCAD_HEUN 1   /* predictor-corrector of Sec. 3 (Heun, velocity held fixed)       */
#define LBCAD_LAGGED 0 /* Q and psi advected with u of the previous step                  */
#define LBCAD_SYNC 1   /* advected with u of this step                                    */
/* Velocity set of the LB populations (the finite-difference stencils are D3Q19 in both). */
#define LBCAD_D3Q19 0  /* 19 velocities: rest, 6 faces, 12 edges                          */
#define LBCAD_D3Q15 1  /* 15 velocities: rest, 6 faces, 8 corners (Sec. 3, Fig. 1)          */
/* Where the stress enters the LB step. */
#define LBCAD_LB_BODY_FORCE 0 /* the whole stress as the force F = div sigma, BGK + Guo      */
#define LBCAD_LB_STRESS_EQ 1  /* Eqs. 9-11: f_eq carries the symmetric stress,
                               * sum f_eq c c = rho/3 I + rho u u - sigma^S; the antisymmetric
                               * stress enters as F_i = 3 w_i c . div sigma^A; rho u = sum f c  */
/* Finite-difference stencils of the order-parameter and stress derivatives (Sec. 3). */
#define LBCAD_STENCIL_ISO 0 /* isotropic D3Q19 gradient and Laplacian (radius 1)             */
#define LBCAD_STENCIL_R2 1  /* fourth-order central differences along the axes (radius 2)   */

#define LBCAD_FIELD_G 1u
#define LBCAD_FIELD_RHO 2u
#define LBCAD_FIELD_U 4u
#define LBCAD_FIELD_Q 8u
#define LBCAD_FIELD_PSI 16u

typedef struct {
  int32_t nx, ny, nz; /* each >= 4; periodic */
} lbcad_grid;

/* Device allocator callbacks: alloc returns a device pointer aligned to >= 256 bytes or
 * NULL; free releases it.  Both are called only from lbcad_create* / lbcad_destroy. */
typedef void* (*lbcad_alloc_fn)(size_t bytes, void* user);
typedef void (*lbcad_free_fn)(void* ptr, void* user);

/* Parameters of Eqs. 1-11 for one droplet instance (lattice units, dx = dt = 1). */
typedef struct {
  double tau;      /* BGK relaxation time (Eq. 7); viscosity (tau - 1/2)/3          */
  double rho0;     /* reference density                                              */
  double A0;       /* Landau-de Gennes scale (Eq. 5)                                 */
  double chi0;     /* chi(phi) = chi0 + chis * phi, phi = 1 + psi (Eq. 5)            */
  double chis;
  double K;        /* one-constant elastic modulus K_Q (Eq. 5)                       */
  double q0;       /* cholesteric wave number 2 pi / pitch (Eq. 5)                   */
  double gammaQ;   /* rotational mobility multiplying H (Eq. 2)                      */
  double xi;       /* flow-alignment parameter of the co-rotation term (Eq. 2)      */
  double a, b;     /* binary bulk -a psi^2/2 + b psi^4/4 (Eq. 5 with phi0 = 2)       */
  double kphi;     /* interface stiffness k_phi (Eq. 5)                              */
  double M;        /* Cahn-Hilliard mobility (Eq. 1)                                 */
  double W;        /* anchoring strength (Eq. 5), W > 0 tangential                  */
  double zeta;     /* activity (Eq. 4), > 0 extensile                                */
  double R;        /* droplet radius for the initial state                           */
  double centre[3];/* droplet centre (x, y, z) for the initial state                 */
  double S0;       /* scalar order of the initial helix inside the droplet           */
  double noise;    /* amplitude of the seeded uniform noise on Q inside the droplet  */
  int32_t precision;  /* LBCAD_FP32 or LBCAD_FP64                                     */
  int32_t integrator; /* LBCAD_EULER or LBCAD_HEUN; one value for all instances        */
  int32_t coupling;   /* LBCAD_LAGGED or LBCAD_SYNC; one value for all instances       */
  int32_t lattice;    /* LBCAD_D3Q19 or LBCAD_D3Q15; one value for all instances        */
  int32_t lb_form;    /* LBCAD_LB_BODY_FORCE or LBCAD_LB_STRESS_EQ; one for all         */
  int32_t stencil;    /* LBCAD_STENCIL_ISO or LBCAD_STENCIL_R2; one for all             */
  int32_t device;     /* CUDA device ordinal; -1 = the current device                 */
  void* stream;       /* cudaStream_t for all work; NULL = a private non-blocking stream */
  lbcad_alloc_fn alloc; /* NULL = cudaMalloc                                          */
  lbcad_free_fn free;   /* NULL = cudaFree                                            */
  void* alloc_user;
} lbcad_params;

/* FP64 conserved sums and centroid moments of one instance at the current time. */
typedef struct {
  double mass;       /* sum over sites of rho                                        */
  double sum_psi;    /* sum of psi                                                   */
  double mom[3];     /* sum over sites of sum_i f_i c_i (pre-collision)               */
  double cm_cos[3];  /* sum of phi_c cos(2 pi x_a / L_a), phi_c = (1 + psi)/2        */
  double cm_sin[3];  /* sum of phi_c sin(2 pi x_a / L_a)                              */
  double sum_phic;   /* sum of phi_c                                                 */
} lbcad_obs;

typedef struct lbcad_ctx lbcad_ctx;

/* The D3Q19 velocity order used by LBCAD_FIELD_G: c[3*i + a], weights w[i]. */
int lbcad_lattice(int32_t* c57, double* w19);

/* The velocity set `lattice` (LBCAD_D3Q19 or LBCAD_D3Q15) in the order of LBCAD_FIELD_G:
 * c[3*i + a] (room for 57 ints) and w[i] (room for 19 doubles).  Returns the number of
 * velocities (19 or 15), or LBCAD_E_INVALID_ARG. */
int lbcad_velocity_set(int32_t lattice, int32_t* c, double* w);

/* Create one instance: validates params, allocates its device state (through
 * params->alloc when given), builds the initial state on the host in FP64 and copies it
 * to the device once (the only host->device transfer).  Initial state: rho = rho0,
 * u = 0, psi = tanh((R - r)/2) with r the distance of the integer site to centre;
 * where r < R, Q = S0 (n n - I/3) + noise * U[-1,1) per stored component, with the
 * helix n = (cos q0 (z - cz), sin q0 (z - cz), 0); elsewhere Q = 0.  The uniform
 * variate for (seed, instance, site s, component c) is SplitMix64: output number
 * k = 1 + (instance << 40) + 5 s + c of the stream started from `seed`, mapped to
 * [-1, 1) as 2 (r >> 11) 2^-53 - 1.  On success *out owns the state; free it with
 * lbcad_destroy. */
int lbcad_create(const lbcad_grid* grid, const lbcad_params* params, uint64_t seed, lbcad_ctx** out);

/* Create n independent instances (uneven boxes and parameters allowed) advanced
 * together: every lbcad_step launch covers all of them.  grids[i], params[i] describe
 * instance i; precision, device, stream and allocator are taken from params[0] and must
 * agree across instances. */
int lbcad_create_batch(int32_t n, const lbcad_grid* grids, const lbcad_params* params, uint64_t seed,
                       lbcad_ctx** out);

/* Advance every instance by n >= 0 hybrid steps on the context's stream.  Asynchronous:
 * returns after enqueueing (errors of enqueued kernels surface at the next synchronising
 * call).  With graphs enabled (lbcad_set_graph), the steps replay a captured CUDA graph. */
int lbcad_step(lbcad_ctx* c, int64_t n);

/* Kernel path of lbcad_step.  LBCAD_PATH_FUSED (default): one persistent kernel per
 * step with shared-memory halo tiles.  LBCAD_PATH_TWO_KERNEL: a stencil kernel writing
 * H, mu and sigma to a per-site scratch (allocated on the first switch, 15 values per
 * site) and an update kernel; same arithmetic, kept as a cross-check.  Changing the path
 * drops a captured graph. */
#define LBCAD_PATH_FUSED 0
#define LBCAD_PATH_TWO_KERNEL 1
/* LBCAD_PATH_STAGED: per-site kernels in the order fields -> LB (force, pull, collision;
 * writes u of this step) -> order-parameter update, and for LBCAD_HEUN a second fields
 * pass at the predicted Q, psi and the corrector (Sec. 3).  The only path for
 * LBCAD_STENCIL_R2, selected at create (fused/two-kernel paths, tile shapes, autotune and the
 * adjoint return LBCAD_E_UNSUPPORTED there); other contexts may select it as a cross-check
 * (same per-site arithmetic).  Scratch: 15 values per site, 27 with LBCAD_HEUN.
 * LBCAD_SYNC or LBCAD_HEUN on the fused path (their default): the fused kernel on one fixed
 * tile shape does the LB half (u of this step; H and mu into the scratch), then tiled
 * z-marching order-parameter kernels on the same tiles (sync: the update; Heun: predictor,
 * fields at the predicted state, corrector); tile shapes, autotune, the two-kernel path and the adjoint return
 * LBCAD_E_UNSUPPORTED there.  LBCAD_D3Q15 and LBCAD_LB_STRESS_EQ run on the fused path (tile
 * shapes 0 and 3 only) and the staged path; the two-kernel path and the adjoint return
 * LBCAD_E_UNSUPPORTED for them. */
#define LBCAD_PATH_STAGED 2
int lbcad_set_path(lbcad_ctx* c, int32_t path);

/* Picks the fastest tile shape of the fused step for this context by timing each
 * candidate over `reps` launches that recompute the step from the current state into
 * the next-state buffers (the simulation does not advance; results are unchanged, only
 * speed), in three rounds that interleave the candidates; a candidate's time is its best
 * round.  Writes the chosen index to *chosen and, if ms_per_cfg is given, the measured
 * milliseconds per launch of up to ncfg candidates (-1 for a shape that does not fit).
 * Candidates: 0 = 32x8 tiles (the FP64 default), 1 = 32x16, 2 = 64x8, 3 (the FP32 default) and 4 = 32x8 software-pipelined
 * (sigma of plane k+1 on 8 or 6 warps while the other 8 or 10 warps output plane k-1, in
 * one phase), 5 and 6 = 32x6 software-pipelined (9 or 10 sigma warps, one round per
 * plane); 1-6 are FP32 only.  With LBCAD_D3Q15 or LBCAD_LB_STRESS_EQ only 0 and 3 are
 * candidates (-1 for the others). */
int lbcad_autotune(lbcad_ctx* c, int32_t reps, int32_t* chosen, float* ms_per_cfg, int32_t ncfg);

/* Selects tile shape `cfg` of the fused step explicitly (same candidates as above;
 * LBCAD_E_UNSUPPORTED for a shape the context's velocity set and LB form do not come in).
 * The arithmetic per site does not depend on the tile shape: results are identical. */
int lbcad_set_tiles(lbcad_ctx* c, int32_t cfg);

/* a6 in the fused step (on = 1, the default): each fused step also forms the FP64 mass,
 * psi, momentum and centroid sums of the state it writes (per-site shares, per-block sums in
 * shared memory, per-segment FP64 partials, and a last-block sum per instance), and
 * lbcad_observables after such a step only copies them.  on = 0 runs the step kernels without
 * the sums (about 5% faster on the 128^3 workload); lbcad_observables then runs a separate
 * reduction pass over the state.  Either way the state is the same.  Drops a captured graph. */
int lbcad_set_observe(lbcad_ctx* c, int32_t on);

/* Capture steps in a CUDA graph of `steps_per_graph` steps (0 disables; default 0).  The
 * state buffers alternate by step parity and a replay must leave the parity unchanged, so
 * steps_per_graph must be even: an odd or negative value returns LBCAD_E_INVALID_ARG and
 * leaves the previous setting.  lbcad_step(n) replays the graph n / steps_per_graph times
 * (after one plain step when the step count is odd) and launches the remaining steps plainly. */
int lbcad_set_graph(lbcad_ctx* c, int32_t steps_per_graph);

/* Copy the selected fields of instance `inst` to dst (FP64, layout above).  bytes must
 * be >= 8 * n * (number of selected components).  dst is a host pointer (pageable or
 * pinned) unless dst_is_device.  Synchronises the context's stream. */
int lbcad_get_fields(lbcad_ctx* c, int32_t inst, uint32_t mask, void* dst, size_t bytes, int32_t dst_is_device);

/* Overwrite the selected fields (G, U, Q, PSI; RHO is derived and rejected) of instance
 * `inst` from src (FP64, same layout).  G gives the pre-collision populations at the
 * current time.  Synchronises the context's stream. */
int lbcad_set_fields(lbcad_ctx* c, int32_t inst, uint32_t mask, const void* src, size_t bytes,
                     int32_t src_is_device);

/* FP64 reductions (deterministic order) of instance `inst` (a6): after a fused step with
 * the sums on (lbcad_set_observe) the sums that step formed, otherwise a separate pass over the
 * stored state.  Both sum the same quantities; they agree to rounding.  Returns LBCAD_E_NAN
 * when a reduced value is not finite.  Synchronises the context's stream. */
int lbcad_observables(lbcad_ctx* c, int32_t inst, lbcad_obs* out);

/* Raw state of instance `inst` in the context's storage precision (float for LBCAD_FP32,
 * double for LBCAD_FP64), for exact checkpoints and for moving the state without
 * conversion.  The layout is the library's own: the stored population array ([q][n], the
 * post-collision values of the previous step at their source sites; FP32 subtracts
 * w_i rho0), then Q [5][n], psi [n] and u [3][n], each [z][y][x].  lbcad_set_state of what
 * lbcad_get_state returned restores the instance bit for bit (the step counter is not part
 * of the state).  *bytes receives (q + 9) n times the element size.  dst/src are host
 * pointers (pageable or pinned) unless *_is_device; the copies run on the context's stream,
 * and both calls synchronise it before returning. */
int lbcad_state_bytes(lbcad_ctx* c, int32_t inst, size_t* bytes);
int lbcad_get_state(lbcad_ctx* c, int32_t inst, void* dst, size_t bytes, int32_t dst_is_device);
int lbcad_set_state(lbcad_ctx* c, int32_t inst, const void* src, size_t bytes, int32_t src_is_device);

/* Adjoint (reverse mode) of nsteps hybrid steps of a single-instance context.
 * Objective: J = |X(t0 + nsteps) - X(t0)|^2 / 2, X the droplet centroid (per-axis circular
 * mean of phi_c = (1 + psi)/2, minimum-image displacement), t0 the current step.
 * Runs the forward from the current state (the context advances by nsteps, as with
 * lbcad_step), storing a checkpoint every ckpt_every steps; then, segment by segment in
 * reverse, replays the segment's states and applies the vector-Jacobian product of each
 * step (per-site vector-Jacobian products by hand-written reverse sweeps through the
 * step's own arithmetic).  Writes dJ/dzeta and dJ/dq0 (accumulated in FP64; q0 enters through H and
 * sigma, the initial Q held fixed), dJ/dQ(t0) for the five stored Q components
 * ([5][z][y][x], host FP64, may be NULL) and J itself.  Device memory: (ceil(nsteps /
 * ckpt_every) + ckpt_every + 2) states of 28 values per site, plus 15 values per site for
 * each of the ckpt_every states of a segment (their sigma, mu and H, computed once in the
 * replay) and 139 values per site of work; owned by the context until lbcad_destroy and
 * reused by later calls that fit in them.  The paper has no adjoint; this is the differentiation form
 * of the step (gradient of the droplet's drift with respect to activity, chirality and
 * the initial order). */
int lbcad_adjoint(lbcad_ctx* c, int64_t nsteps, int32_t ckpt_every, double* dJ_dzeta, double* dJ_dq0,
                  double* dJ_dQ0, double* J);

/* Gradient of the last lbcad_adjoint's J with respect to the whole state at its start,
 * in the lbcad_get_fields layout and convention (G = pre-collision populations f_i, U =
 * velocity of the previous step, Q, PSI; RHO is not a state and is rejected).  FP64 host
 * buffer of >= 8 n (components) bytes. */
int lbcad_adjoint_fields(lbcad_ctx* c, uint32_t mask, void* dst, size_t bytes);

/* Number of instances, lattice of one instance, steps taken so far. */
int lbcad_num_instances(const lbcad_ctx* c);
int lbcad_instance_grid(const lbcad_ctx* c, int32_t inst, lbcad_grid* out);
int64_t lbcad_step_count(const lbcad_ctx* c);

/* The cudaStream_t all work of the context is enqueued on (created by the library,
 * non-blocking, when params->stream was NULL). */
void* lbcad_stream(const lbcad_ctx* c);

/* Block until all enqueued work of the context has finished; reports kernel errors. */
int lbcad_sync(lbcad_ctx* c);

/* ---- one step without any device allocation ------------------------------------- *
 * The paper has no counterpart of this call; it serves callers that must not have a
 * library allocate device memory (a host framework that owns all device memory through
 * its own pool, or a loop that cannot take the synchronisation cudaMalloc/cudaFree may
 * cause).  It advances ONE instance by ONE hybrid step with the two-kernel step and
 * keeps that step's scratch (H, mu and sigma: 15 values per site) in a fixed static
 * device array of LBCAD_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library
 * holds until the process exits.  It calls no cudaMalloc or cudaFree and creates no
 * stream.
 *
 * Buffers (device pointers, owned by the caller, in the library's storage layout,
 * element type float for LBCAD_FP32 and double for LBCAD_FP64, each [component][z][y][x]):
 *   g_in  [19][n]  post-collision populations of the previous step (FP32: f_i - w_i rho0;
 *                  FP64: f_i), so the initial state at rest is 0 (FP32) or w_i rho0 (FP64);
 *   q_in  [5][n], psi_in [n], u_in [3][n]: Q, psi and the velocity of the previous step;
 *   g_out, q_out, psi_out, u_out: the same fields after the step (must not alias inputs).
 * params supplies the physics, precision, device (-1 = current) and stream (NULL = the
 * legacy default stream); integrator/coupling must be Euler/lagged; alloc callbacks are
 * ignored.  Returns after enqueueing the work on that stream.
 *
 * Checks: the grid and params go through the same validation as lbcad_create (edges >= 4,
 * every floating-point parameter finite, tau > 1/2, rho0 > 0, known option codes), then the
 * size limit below, then the buffer pointers; all of these run on the host before any device
 * is touched, and a failure returns LBCAD_E_INVALID_ARG (LBCAD_E_UNSUPPORTED for an option
 * this call does not run) with a message in lbcad_last_error(NULL).
 * Limits: 15 * round_up_256(n * element size) bytes must fit in the scratch array, i.e.
 * up to 279,616 sites in FP32 (64^3 fits) and 139,808 in FP64; larger grids are rejected.
 * Work: two launches on the stream, one that writes the launch descriptor (passed by value
 * as a kernel argument, so no host memory is read after the call returns) into a second
 * static array of 512 bytes, then the step kernels.
 * Sharing: every call on a device uses the same scratch and descriptor, so calls whose
 * work overlaps on the GPU (different streams, or host threads) race and corrupt each
 * other; serialise them.  The array keeps the last call's contents; nothing needs to
 * start at zero because each call writes every scratch value before reading it.
 * Set-up: the first call on a device looks up the device addresses of the static arrays
 * with cudaGetSymbolAddress (a host-side runtime query, which may also load the library's
 * kernels) and keeps them for that device.  The addresses belong to the CUDA runtime's context of the device (its
 * primary context): call this only while that context is current, not under a context the
 * caller created with the driver API. */
#define LBCAD_NOALLOC_SCRATCH_BYTES (16u << 20)
int lbcad_step_noalloc(const lbcad_grid* grid, const lbcad_params* params, const void* g_in, const void* q_in,
                       const void* psi_in, const void* u_in, void* g_out, void* q_out, void* psi_out, void* u_out);

/* Release the context and its device memory.  NULL is a no-op. */
void lbcad_destroy(lbcad_ctx* c);

/* Message of the last error on c (or of the last failed create when c is NULL). */
const char* lbcad_last_error(const lbcad_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* LBCAD_H */
