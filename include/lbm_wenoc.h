/*
 * lbm_wenoc: one-GPU (GB300, sm_103a) coupled lattice-Boltzmann + WENO5 solver
 * for a settling particle concentration c in a Boussinesq fluid.
 *
 * The problem follows the paper's statement (arXiv 2106.07694):
 *   fluid      BGK lattice Boltzmann, D2Q9 (2D) or D3Q19 (3D), relaxation time tau
 *              with nu = (tau - 1/2)/3 (Sec. 2.3.1, Eqs. LBE, tau), Guo forcing
 *              (Eq. LBE_Guo), no-slip floor and lid by halfway bounce-back, periodic
 *              sides (Sec. 2.2.1);
 *   force      F = -A c e_v + body_force, A = gravity * density_contrast
 *              (Eq. forceterm with the density-altering scalar left out);
 *   particles  dc/dt + div[c (u - Vs e_v)] = kappa lap c (Eq. ADS), WENO5 with a
 *              global Lax-Friedrichs flux split, central diffusion, SSP-RK3
 *              (Supplement Sec. 1, Eqs. S4, S8-S23); the settling flux through the
 *              floor leaves the domain and is accumulated as deposited mass
 *              (Sec. 4, m_b).
 * Lattice units: dx = dt = 1.  e_v is the vertical axis: y in 2D, z in 3D.
 *
 * Memory: every device buffer belongs to the caller.  The library keeps only a
 * host-side handle (and the CUDA graphs and events it creates) and never calls
 * cudaMalloc.  All arrays are dense, C order, vertical axis slowest:
 * index = (z*ny + y)*nx + x.  Vectors are component-major: u[d*n + index].
 * The element type of c and u buffers is double when LW_FP64 is set, else float.
 *
 * Errors: every int-returning call returns LW_OK (0) or a negative LW_E* code;
 * nothing aborts, throws or traps across this boundary.  Work is asynchronous on
 * the stream given at create unless a call says it synchronises.
 * Threading: a handle is not thread-safe; use one handle per host thread/stream.
 */
#ifndef LBM_WENOC_H
#define LBM_WENOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LW_OK 0
#define LW_EINVAL -1    /* bad argument or parameter (e.g. tau <= 1/2, nx % 4 != 0, Q*nodes >= 2^31) */
#define LW_ENOMEM -2    /* workspace smaller than lbm_wenoc_workspace_bytes() */
#define LW_ECUDA -3     /* a CUDA runtime call failed */
#define LW_EUNSTABLE -4 /* device status: non-finite value or |u_d| > u_cap */
#define LW_ETIMEOUT -5  /* a bounded device wait gave up */
#define LW_ESTATE -6    /* call out of order (e.g. step before init) */

#define LW_FP64 0x1u              /* FP64 populations and arithmetic (validation build) */
#define LW_PERIODIC_VERTICAL 0x2u /* vertical axis periodic too: no walls, no deposit (tests) */
#define LW_FROZEN_VELOCITY 0x4u   /* fluid not advanced; c transported by the u given at init (tests) */
#define LW_NO_GRAPH 0x8u          /* launch kernels one by one instead of replaying CUDA graphs */
#define LW_FUSED_RK3 0x10u        /* 2D FP32: the three RK stages in one fused sweep kernel instead of
                                     three row-sweep launches (same results to rounding) */
#define LW_SUGAR 0x20u            /* second scalar S, the paper's sugar (Eqs. AD, forceterm, stokes_vel):
                                     force -g S* S (1 - phi0 c), settling velocity Vs (1 - kS S), S
                                     advected by first-order upwind (Supplement Eqs. S5, S6) with
                                     diffusion D_s; not with LW_FUSED_RK3, batches or the gradient */
#define LW_WENO3 0x40u            /* the paper's third-order WENO (Supplement Eqs. S10-S20, linear weights
                                     (2/3, 1/3) of Eq. S16) instead of WENO5; a compile-time variant of
                                     the FP32 sweep stage kernels (FP64: the generic ones) */
#define LW_SIGN_SPLIT 0x80u       /* whole flux w c reconstructed from the side the face velocity
                                     (w_i + w_{i+1})/2 comes from (ties left) instead of the
                                     Lax-Friedrichs split; stage kernels as for LW_WENO3.  Neither
                                     variant with LW_FUSED_RK3, batches or the gradient */
#define LW_ONE_COLUMN 0x100u      /* 2D FP32: the row-sweep stage kernels with one column per thread
                                     instead of four (bitwise the same c and u; the deposit's FP64
                                     partial sums are grouped differently).  For comparisons */

typedef struct lbm_wenoc lbm_wenoc; /* opaque host-side handle */

typedef struct {
  int32_t dim;               /* 2 (D2Q9) or 3 (D3Q19) */
  int32_t nx, ny, nz;        /* lattice extents; nz ignored in 2D; nx % 4 == 0, ny >= 4, nz >= 4 in 3D */
  double tau;                /* BGK relaxation time, > 1/2 (Eq. tau) */
  double gravity;            /* g, lattice units */
  double density_contrast;   /* (rho_p - rho_0)/rho_0; force = -gravity*density_contrast*c e_v (Eq. forceterm) */
  double settling_velocity;  /* Vs >= 0, directed down (Eq. ADS) */
  double diffusivity;        /* kappa >= 0 (D_c of Eq. ADS) */
  double lf_alpha;           /* Lax-Friedrichs split speed; 0 selects settling_velocity + u_cap */
  double u_cap;              /* bound on |u_d| checked on the device; 0 selects 0.1 */
  double body_force[3];      /* extra uniform force (e.g. a channel flow), added to the buoyancy */
  uint32_t flags;            /* LW_FP64 | LW_PERIODIC_VERTICAL | LW_FROZEN_VELOCITY | LW_NO_GRAPH | LW_FUSED_RK3
                                | LW_SUGAR | LW_WENO3 | LW_SIGN_SPLIT | LW_ONE_COLUMN */
  /* used with LW_SUGAR only (S normalised by its lower-layer value S0) */
  double sugar_contrast;     /* S* = rho(S0)/rho_0 - 1 (Eq. S_star): force -gravity*S* S (1 - phi0 c) e_v */
  double sugar_diffusivity;  /* D_s >= 0 */
  double phi0;               /* particle volume fraction at c = 1, in the (1 - phi) factor of Eq. forceterm */
  double vs_sugar;           /* kS: settling velocity Vs (1 - kS S) (Eq. stokes_vel with rho(S)) */
  /* polydisperse particles (Eqs. forceterm_poly, poly): n_classes >= 2 classes c_k, class k
   * settling at class_vs[k] (settling_velocity unused), each with its own deposit; the force
   * reads phi_tot = sum_k c_k.  0 or 1: one class.  At most 8; not with LW_FUSED_RK3,
   * batches or the gradient.  The default lf_alpha takes the largest class velocity. */
  int32_t n_classes;
  double class_vs[8];
} lbm_wenoc_params;

/* Bytes of device workspace a handle with these parameters needs (populations,
 * concentration, two Runge-Kutta stage fields, velocity, reduction scratch). */
int lbm_wenoc_workspace_bytes(const lbm_wenoc_params* p, size_t* bytes);

/* Create a handle over a caller-owned device workspace (256-byte aligned, at least
 * lbm_wenoc_workspace_bytes() long, kept alive until destroy).  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream); all work of the handle runs on it.
 * The handle binds to the current device.  Returns LW_EINVAL / LW_ENOMEM on bad input. */
int lbm_wenoc_create(const lbm_wenoc_params* p, void* dev_workspace, size_t bytes,
                     void* cuda_stream, lbm_wenoc** out);

/* Set the initial state (Sec. 2.2.1, Eqs. ini1/ini: fluid at rest, c given):
 * c0[n] is required; u0[dim*n] is optional (NULL = fluid at rest).  Populations
 * start at equilibrium f_i = f_i^eq(rho = 1, u0).  Either pointer may be host or
 * device memory (detected); host data are copied on the stream, so a pageable host
 * buffer may be reused when the call returns.  Resets the deposit and the step count. */
int lbm_wenoc_init(lbm_wenoc* h, const void* c0, const void* u0);

/* Advance nsteps >= 0 coupled time steps (asynchronous): per step, moments with the
 * half force, BGK-Guo collision and in-place streaming with bounce-back, then three
 * SSP-RK3 stages of the WENO5 transport of c with the velocity of that step, and the
 * deposit through the floor.  Returns LW_ESTATE before init. */
int lbm_wenoc_step(lbm_wenoc* h, int64_t nsteps);

/* Synchronise the stream and return the accumulated deposited mass (FP64): the sum
 * over steps of Vs * sum_floor(c/6 + c1/6 + 2 c2/3), i.e. the RK3-weighted settling
 * flux through the floor, so that total_mass + deposit is conserved.
 * Returns LW_EUNSTABLE if the device status word is set. */
int lbm_wenoc_deposited_mass(lbm_wenoc* h, double* out);

/* Synchronise and return sum of c over the domain (FP64, fixed summation order). */
int lbm_wenoc_total_mass(lbm_wenoc* h, double* out);

/* Particle mass below a horizontal plane (Sec. 4.2.3, Eq. flux): the sum of c over the
 * vertical levels 0 .. level-1 (FP64, fixed summation order; the sum of the classes with
 * several) plus the deposited mass, which has crossed every plane.  The mass flux through
 * the plane between two calls Delta t apart is J = (m(t) - m(t - Delta t)) / (A Delta t),
 * A = nx (2D) or nx ny (3D), in lattice units (m_i = c_i: unit cell volume and particle
 * density).  0 <= level <= ny (2D) or nz (3D), else LW_EINVAL; level = 0 gives the
 * deposit, the top level total_mass + deposit.  Synchronises the stream; LW_EUNSTABLE as
 * lbm_wenoc_deposited_mass (the value is still written). */
int lbm_wenoc_mass_below(lbm_wenoc* h, int32_t level, double* out);

/* Write the macroscopic state of the current step: rho[n], u[dim*n] (half-force
 * corrected velocity (sum f c + F/2)/rho with the current c), c[n].  Any pointer may
 * be NULL; each may be host or device memory.  Synchronises. */
int lbm_wenoc_fields(lbm_wenoc* h, void* rho, void* u, void* c);

/* Checkpoint and resume: the state a step reads -- populations, the current c (and S,
 * class fields), u, the FP64 deposits, the AA parity and the step count -- as one blob
 * with a header.  A handle with the same parameters (LW_NO_GRAPH aside) that loads it
 * continues bit for bit as the saved one would have.
 *   lbm_wenoc_state_bytes  blob size for this handle.
 *   lbm_wenoc_save_state   after the steps enqueued so far; dst host or device memory of at
 *                          least that size (LW_ENOMEM if smaller; LW_ESTATE before init).
 *   lbm_wenoc_load_state   src host or device memory; LW_EINVAL if the header is not a
 *                          state of a handle with these parameters.  Clears the status word.
 * Both synchronise the stream. */
int lbm_wenoc_state_bytes(const lbm_wenoc* h, size_t* bytes);
int lbm_wenoc_save_state(lbm_wenoc* h, void* dst, size_t bytes);
int lbm_wenoc_load_state(lbm_wenoc* h, const void* src, size_t bytes);

/* Synchronise and return LW_OK or LW_EUNSTABLE from the device status word. */
int lbm_wenoc_status(lbm_wenoc* h);

/* Steps taken since init. */
int64_t lbm_wenoc_steps(const lbm_wenoc* h);

/* Per-kernel timing with CUDA events on the handle's stream (off by default).
 * enable != 0 records an event pair around every kernel launched by later calls. */
int lbm_wenoc_profile_enable(lbm_wenoc* h, int enable);

typedef struct {
  char name[48];    /* kernel family name */
  int64_t launches; /* launches recorded */
  double total_ms;  /* summed device time between the event pairs */
} lbm_wenoc_kernel_stat;

/* Synchronise, fold pending event pairs into per-kernel totals, copy up to max
 * entries into out, set *count; reset = 1 clears the totals afterwards. */
int lbm_wenoc_profile_read(lbm_wenoc* h, lbm_wenoc_kernel_stat* out, int max, int* count,
                           int reset);

/* Number of kernel launches this handle has issued since create. */
int64_t lbm_wenoc_launch_count(const lbm_wenoc* h);

/* Tuning of the FP32 transport sweeps: rows per CTA segment of the 2D stage kernels (or
 * of the fused 2D kernel), or z levels per CTA segment of the 3D stage kernels (0 = default).  Results do not
 * depend on it (bitwise).  No effect on FP64 or periodic-vertical handles.  Drops
 * captured graphs; call between steps. */
int lbm_wenoc_set_segment_rows(lbm_wenoc* h, int32_t rows);

/* ---- Batched simulations (the paper's parameter sweep, Sec. 2.2 Table 1, as one job) ----
 * count independent 2D FP32 simulations with walls (no LW_FP64, LW_PERIODIC_VERTICAL,
 * LW_FROZEN_VELOCITY, LW_FUSED_RK3, LW_SUGAR, scheme variants, classes or LW_ONE_COLUMN),
 * each with its own size and parameters, in one caller-owned workspace.  By default they
 * advance together in one persistent cooperative launch per graph of up to 16 steps: as
 * many CTAs as the SMs hold at once take (instance, tile) work items of each phase of a
 * step (fluid part, three RK3 stages), with a grid barrier between phases whose waits are
 * bounded (a wait past the limit ends the launch and the batch status reads LW_ETIMEOUT).
 * Results are bitwise those of each instance stepped alone, the deposits included. */
typedef struct lbm_wenoc_batch lbm_wenoc_batch;

/* Workspace bytes for count instances with parameters p[0..count); LW_EINVAL if any
 * instance is not a 2D FP32 walled configuration of the default scheme. */
int lbm_wenoc_batch_workspace_bytes(const lbm_wenoc_params* p, int32_t count, size_t* bytes);

/* Create the batch over dev_workspace (256-byte aligned, at least the bytes above). */
int lbm_wenoc_batch_create(const lbm_wenoc_params* p, int32_t count, void* dev_workspace, size_t bytes,
                           void* cuda_stream, lbm_wenoc_batch** out);

/* Handle of instance i (owned by the batch: do not destroy it).  Use it for init,
 * fields, deposited_mass, total_mass and status; stepping it alone desynchronises it
 * from the batch (lbm_wenoc_batch_step then returns LW_ESTATE). */
lbm_wenoc* lbm_wenoc_batch_instance(lbm_wenoc_batch* b, int32_t i);

/* Advance every instance nsteps steps (asynchronous); all instances must be
 * initialised and at the same step count, else LW_ESTATE. */
int lbm_wenoc_batch_step(lbm_wenoc_batch* b, int64_t nsteps);

/* persistent = 1: the persistent launch (default where the device supports cooperative
 * launches; else LW_EINVAL); 2: per step the fluid part as one grouped launch, then the
 * three RK3 stages in one persistent launch; 0: one launch per kernel type and step.
 * Same results; other values LW_EINVAL.  Synchronises the stream; drops captured graphs. */
int lbm_wenoc_batch_set_persistent(lbm_wenoc_batch* b, int32_t persistent);

/* Bound of a grid-barrier wait of the persistent launch, in SM clock cycles (default
 * 2^31, about one second).  skip_cta >= 0 is for testing the timeout path: that CTA of the
 * next launch leaves before its first barrier, so the others' waits run out and the
 * batch status becomes LW_ETIMEOUT (the instances' fields are then undefined until
 * re-initialised).  -1: none.  Synchronises the stream. */
int lbm_wenoc_batch_set_wait_limit(lbm_wenoc_batch* b, int64_t cycles, int32_t skip_cta);

/* Synchronise; LW_ETIMEOUT if a barrier wait of a persistent launch gave up (launches
 * after that one do nothing until this call has reported it; it clears the flag, and the
 * instances must be initialised again), else the first non-OK instance status
 * (LW_EUNSTABLE), else LW_OK. */
int lbm_wenoc_batch_status(lbm_wenoc_batch* b);

/* Autotuner of the segment heights: starting from each instance's default, tries the
 * heights 4 .. 64 for each lattice size in turn (instances of one size share one), timing
 * steps_per_trial batched steps of the whole batch on a trial state, and keeps what is
 * fastest.  chosen_rows: NULL or count int32 slots for each instance's height.  Leaves every
 * instance uninitialised: call it before init. */
int lbm_wenoc_batch_autotune(lbm_wenoc_batch* b, int32_t steps_per_trial, int32_t* chosen_rows);

/* Kernel launches issued by lbm_wenoc_batch_step so far. */
int64_t lbm_wenoc_batch_launch_count(const lbm_wenoc_batch* b);

/* Destroy the batch and its instance handles (not the caller's workspace). */
void lbm_wenoc_batch_destroy(lbm_wenoc_batch* b);

/* ---- Gradient of the deposited mass (reverse mode, checkpoint-and-recompute) ----
 * J = deposited mass (Sec. 4, m_b) after nsteps steps from the initial state c0 (fluid
 * at rest).  lbm_wenoc_deposit_gradient runs the forward pass keeping the state every
 * `segment` steps, then for each segment in reverse recomputes its states and runs the
 * adjoint kernels backwards through every step (transport stages with the WENO5
 * nonlinear weights, streaming with bounce-back, BGK-Guo collision, buoyancy), giving
 *   grad_c0[n] = dJ/dc0   (caller buffer, host or device, element type of the handle)
 *   *dJ_dVs     = dJ/dVs  (FP64; lf_alpha is held fixed)
 *   *J          = the deposited mass of the forward pass (FP64).
 * Requires a 2D handle with walls, not frozen, without LW_FUSED_RK3, and an explicit
 * lf_alpha > 0 (LW_EINVAL otherwise).  adj_workspace: caller-owned device memory of at
 * least lbm_wenoc_gradient_workspace_bytes() (checkpoints + one segment of states +
 * adjoint fields, one stage's face records), 256-byte aligned.  Deterministic (no
 * atomics): the same inputs give the same bits for any segment.  The reverse steps run on
 * an internal stream at the device's greatest priority and the recompute of the next
 * segment on a second internal stream, both ordered after the work already queued on the
 * handle's stream and joined back to it; both are created and destroyed by the call.
 * Synchronises.  Afterwards the handle holds an intermediate state and must be
 * initialised again before stepping. */
int lbm_wenoc_gradient_workspace_bytes(const lbm_wenoc_params* p, int64_t nsteps, int32_t segment, size_t* bytes);
int lbm_wenoc_deposit_gradient(lbm_wenoc* h, const void* c0, int64_t nsteps, int32_t segment, void* adj_workspace,
                               size_t bytes, void* grad_c0, double* dJ_dVs, double* J);

/* Sugar field (LW_SUGAR handles): set after lbm_wenoc_init (which zeroes it) and before
 * or between steps, and read back; nx*ny(*nz) elements of the handle's element type, host
 * or device memory, natural layout.  LW_EINVAL without LW_SUGAR, LW_ESTATE before init.
 * Both synchronise. */
int lbm_wenoc_set_sugar(lbm_wenoc* h, const void* S0);
int lbm_wenoc_sugar(lbm_wenoc* h, void* S_out);

/* Particle classes (n_classes >= 2): lbm_wenoc_init puts c0 in class 0 and zeroes the
 * others; set class k (0 <= k < n_classes) after init, read it back, read its deposit.
 * lbm_wenoc_fields and lbm_wenoc_total_mass report the sum of the classes and
 * lbm_wenoc_deposited_mass the total deposit.  Host or device buffers; synchronise. */
int lbm_wenoc_set_class(lbm_wenoc* h, int32_t k, const void* ck);
int lbm_wenoc_class(lbm_wenoc* h, int32_t k, void* out);
int lbm_wenoc_class_deposit(lbm_wenoc* h, int32_t k, double* out);

/* Sum of a concentration field, FP64, for callers that cannot allocate device memory
 * (an application that owns a fixed device arena, a plugin inside another framework's
 * allocator, a tool holding only a pointer to someone else's field).  The paper has no
 * counterpart: this is a service of the library, the same reduction as
 * lbm_wenoc_total_mass() without a handle or workspace.
 *   c_dev    device array of n concentrations (double if fp64 != 0, else float)
 *   n        1 .. 67,108,864 (2048 blocks x 32768 elements); larger -> LW_EINVAL
 *   out_dev  device address of one double that receives the sum
 * Asynchronous on cuda_stream.  The partial sums live in a 16 KB static device array
 * that every GPU loading the library keeps until exit; no cudaMalloc or cudaFree is
 * called.  The first call on each device looks up that array's address, so make it
 * before any stream capture.  All calls share the array: calls that overlap on the GPU
 * race and must be ordered by the caller.  The looked-up address is kept for the life of
 * the process: after cudaDeviceReset (or any teardown of the device's primary context)
 * it is stale, and this entry point must not be used again in that process. */
int lbm_wenoc_total_mass_noalloc(const void* c_dev, int64_t n, int32_t fp64, void* cuda_stream,
                                 double* out_dev);

/* Destroy the handle (graphs, events).  Does not free the caller's workspace. */
void lbm_wenoc_destroy(lbm_wenoc* h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_WENOC_H */
