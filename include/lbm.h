/*
 * lbm.h - C ABI of the GB300 (sm_103a) implementation of the per-step update of the
 * central-moment pseudopotential lattice Boltzmann model for forced-convection boiling
 * on a heated cylinder (Saito, De Rosis, Fei, Luo, Ebihara, Kaneko, Abe,
 * arXiv:1912.02018).
 *
 * One time step (lbm_step) is, in this order:
 *   1. pull-streaming f_i(x) = f*_i(x - c_i)                     Eq. (streaming)
 *      with a Zou-He velocity inlet at x = 0, a convective outlet at x = nx-1 and a
 *      linear interpolated bounce-back (Bouzidi) on the cylinder  Sec. IV.A
 *   2. rho = sum_i f_i and the pseudopotential psi(rho, T) of     Eq. (potential)
 *      with the Peng-Robinson EOS                                 Eq. (eos)
 *   3. the interaction force on the 24-neighbour stencil           Eq. (interForce)
 *      plus gravity (rho - rho_l) g along -x                        Sec. IV.A
 *   4. u from rho u = sum f c + F/2 and the CM collision with the
 *      thermodynamic-consistency terms                             Eq. (postColl2)
 *   5. a wall heat-flux sample -lambda dT/dn averaged over the
 *      fluid nodes next to the cylinder                            Sec. IV.B
 *   6. the temperature equation by two-stage Runge-Kutta with
 *      third-order upwind convection and isotropic differences     Eq. (energy), Sec. II.C
 * During the first warmup_steps steps the force and steps 5-6 are skipped (Sec. IV.A).
 *
 * Conventions shared by every entry point:
 *   - Lattice units throughout.  The flow runs along +x; the domain is periodic in y
 *     (and in x too when lbm_domain.periodic_x is set, which removes inlet and outlet).
 *   - Host arrays are row-major [ny][nx] (node id = y*nx + x), populations
 *     [9][ny][nx] in the D2Q9 order c_x = {0,1,-1,0,0,1,-1,1,-1},
 *     c_y = {0,0,0,1,-1,1,-1,-1,1} of Eq. (velVec).  All host-side values are double.
 *   - The library owns all device memory it allocates (through the caller's
 *     allocator when one is given).  Buffers passed in are owned by the caller and
 *     are not retained after the call returns.
 *   - No exception crosses the ABI.  Every call returns an lbm_status; the text of the
 *     last error of a context is available from lbm_last_error.
 *   - lbm_step only enqueues work on the context's stream.  A fault detected by a
 *     kernel (non-finite density, non-positive psi radicand) is latched on the device
 *     and reported as LBM_EUNSTABLE by the next call that synchronises (lbm_sync,
 *     lbm_fields, lbm_get_state, lbm_wall_heat_flux); a bounded wait of a kernel that gave
 *     up is reported there as LBM_ETIMEOUT.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,    /* bad argument; nothing was changed */
    LBM_ENOMEM = -2,    /* device allocation failed */
    LBM_ECUDA = -3,     /* a CUDA runtime call failed */
    LBM_EUNSTABLE = -4, /* a kernel saw a non-finite density or psi radicand <= 0 */
    LBM_ETIMEOUT = -5,  /* a bounded device wait gave up (a shared-memory tile copy that did not land) */
    LBM_ESTATE = -6     /* call not valid in the context's current state */
} lbm_status;

/* Population storage.  Arithmetic is FP64 when compute_f64 is set (storage must then be
 * LBM_STORE_F64), FP32 otherwise, with populations stored as FP64, FP32 or shifted FP16
 * h_i = f_i - w_i rho_l (FP16 rounding is finest near zero, where liquid populations then
 * sit).  In the FP32 build the pseudopotential (Eq. potential) is evaluated with FP64-class
 * accuracy by default (see lbm_params.psi_mode); the wall heat flux is always accumulated
 * in FP64. */
typedef enum { LBM_STORE_F64 = 0, LBM_STORE_F32 = 1, LBM_STORE_F16S = 2 } lbm_storage;

typedef struct {
    int32_t nx, ny;     /* lattice size; nx, ny >= 5 */
    int32_t periodic_x; /* 0: Zou-He inlet at x=0, convective outlet at x=nx-1; 1: periodic in x */
    int32_t walls;      /* flat solid walls with halfway bounce-back (link fraction 1/2), their solid nodes at
                           T_w: bit 0 the column x = 0 (replaces the inlet; needs periodic_x = 0), as the
                           heated wall of the Stefan problem (Sec. III.E) turned to face +x; bit 1 the rows
                           y = 0 and y = ny-1, the no-slip planes of the Poiseuille flow (Sec. III.C) */
} lbm_domain;

typedef struct {
    double xc, yc;       /* centre; node (x, y) is solid iff (x-xc)^2 + (y-yc)^2 <= (D/2)^2 */
    double D;            /* diameter; D <= 0 means no cylinder */
    double superheat_Tc; /* wall superheat (T_w - T_sat) as a fraction of T_c, Sec. IV.A */
    double rho_solid;    /* density given to solid nodes for psi; 0 means rho_l */
    const double *wall_dT; /* optional: n_wall knots of extra superheat (fractions of T_c), equally spaced
                              in the angle from +x; a solid node at angle theta gets the periodic-linear
                              interpolation; NULL or n_wall = 0: uniform wall (copied at creation) */
    int32_t n_wall;
    int32_t reserved;
} lbm_cylinder;

typedef struct {
    /* Peng-Robinson EOS, Eq. (eos): a, b, R, acentric factor; T_c = 0.0778 a / (0.4572 b R) */
    double a, b, R, acentric;
    double G;           /* interaction strength of Eq. (interForce)/(potential); < 0; 0 = single phase */
    double sigma;       /* thermodynamic-consistency constant of Eq. (force2) */
    double Tr_sat;      /* T_sat / T_c */
    double Re;          /* Reynolds number u_in D / nu_l (used when nu_l == 0) */
    double u_in;        /* inlet speed (and initial speed) */
    double nu_l;        /* liquid kinematic viscosity; 0: u_in D / Re */
    double nu_ratio;    /* eta = nu_l / nu_v */
    double Pr_l, Pr_v;  /* Prandtl numbers: thermal diffusivity alpha = nu / Pr per phase */
    double c_v;         /* specific heat */
    double g;           /* gravity along -x; < 0: u_in^2 / (16 D), i.e. u_in / sqrt(g D) = 4 */
    double outlet_U;    /* convective-outlet speed; < 0: u_in */
    int64_t warmup_steps; /* steps with no force and no energy equation */
    int32_t energy;       /* 1: solve Eq. (energy); 0: keep T fixed */
    int32_t storage;      /* lbm_storage of the populations; must be LBM_STORE_F64 when compute_f64 = 1 */
    int32_t compute_f64;  /* 1: FP64 arithmetic throughout (the parity build) */
    int32_t psi_mode;     /* FP32 build only: how psi of Eq. (potential) is evaluated from FP32 rho, T:
                             0 double-float (FP32 pairs, ~2^-44 relative), 1 IEEE FP64, 2 FP32 */
    uint64_t seed;        /* SplitMix64 stream for the default density perturbation */
    double noise_amp;     /* amplitude of that perturbation (uniform in +/- noise_amp) */
    double body_fx;       /* uniform body force density along +x added to the force of Eq. (force), as the
                             driving force F_x = 8 nu U_0 / L_y^2 of the Poiseuille flow (Sec. III.C); 0: none */
    int32_t collision;    /* lbm_collision: LBM_COLL_CM, the central-moment collision of Sec. II.A (the method), or
                             LBM_COLL_BGK, the single-rate BGK operator the paper compares it with in Sec. III.B
                             (same equilibrium, Eq. (equi), and forcing, Eq. (forcingTerm); every central moment
                             relaxed at omega; no consistency term).  Batches and the adjoint take LBM_COLL_CM only */
    int32_t reserved;     /* must be 0 */
} lbm_params;

typedef enum { LBM_COLL_CM = 0, LBM_COLL_BGK = 1 } lbm_collision;

/* Optional initial fields (host, [ny][nx]); any pointer may be NULL.
 * rho0 = (rho ? rho : rho_l) + (drho ? drho : SplitMix64(seed) noise of amplitude noise_amp),
 * u0 = (ux, uy) or (u_in, 0), T0 = T or T_sat; solid nodes get rho_solid, u = 0 and their wall
 * temperature T_w(x), which they keep (the energy equation updates fluid nodes only).
 * Populations start at the fourth-order Hermite equilibrium of Eq. (equi). */
typedef struct {
    const double *rho, *drho, *ux, *uy, *T;
} lbm_init;

/* Device allocator: alloc returns a device pointer of at least `bytes` bytes (aligned
 * to 256 B) or NULL; free releases it.  NULL allocator: cudaMalloc / cudaFree. */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
} lbm_allocator;

/* Constants the library derived from the parameters (Sec. II.C, Sec. IV.A). */
typedef struct {
    double Tc, pc, T_sat, T_wall;
    double rho_l, rho_v, p_sat;  /* Maxwell equal-area coexistence at T_sat */
    double h_fg;                 /* latent heat T_sat (1/rho_v - 1/rho_l) dp_sat/dT (Clausius-Clapeyron; Sec. IV.A) */
    double nu_l, nu_v, alpha_l, alpha_v, lambda_v, g, outlet_U;
    int64_t steps;               /* steps taken so far */
    int64_t n_boundary;          /* fluid nodes with a D2Q9 link into the cylinder */
    int64_t kernel_launches;     /* kernels launched by this context so far */
    int64_t device_bytes;        /* device memory held by this context */
} lbm_info_t;

/*
 * Create a simulation.  Validates the parameters on the host (LBM_EINVAL: sizes,
 * 0 < omega < 2 in both phases, psi radicand > 0 at T_sat and T_w for densities
 * between rho_v and rho_l, cylinder at least 3 nodes from the inlet and outlet),
 * computes the derived constants, builds the geometry tables, allocates device
 * memory and writes the initial state.  cuda_stream is a cudaStream_t (NULL: the
 * legacy default stream); all work of the context is issued on it.
 * On success *out receives the handle, to be released with lbm_destroy.
 */
lbm_status lbm_create(const lbm_domain *domain, const lbm_cylinder *cyl, const lbm_params *params,
                      const lbm_init *init, const lbm_allocator *alloc, void *cuda_stream, lbm_ctx **out);

/* Enqueue n >= 0 time steps (the six parts listed at the top).  Asynchronous. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t n);

/* Wait for the context's stream; LBM_EUNSTABLE if a kernel latched a fault. */
lbm_status lbm_sync(lbm_ctx *ctx);

/*
 * Wall heat flux, Sec. IV.B: q(t) = mean over boundary fluid nodes b of
 * -lambda(rho_b) grad T(x_b) . n_b, n_b the outward unit normal from the cylinder
 * centre, grad T the isotropic gradient of the temperature entering the step.  One
 * sample per step after the warm-up (when energy = 1).  Returns the last sample,
 * the mean and standard deviation of the samples since creation or the last
 * lbm_reset_heat_flux, the mean Nusselt number D <q> / (lambda_v (T_w - T_sat)),
 * and the number of samples.  Any output pointer may be NULL.  Synchronises.
 */
lbm_status lbm_wall_heat_flux(lbm_ctx *ctx, double *q_now, double *q_mean, double *q_std, double *nu_mean,
                              int64_t *n_samples);

/* Restart the heat-flux averages (e.g. at the start of the quasi-steady window). */
lbm_status lbm_reset_heat_flux(lbm_ctx *ctx);

/* Field selection bits for lbm_fields. */
#define LBM_FIELD_RHO 1u
#define LBM_FIELD_UX 2u
#define LBM_FIELD_UY 4u
#define LBM_FIELD_T 8u
#define LBM_FIELD_PSI 16u
#define LBM_FIELD_SOLID 32u
#define LBM_FIELD_FX 64u
#define LBM_FIELD_FY 128u

/*
 * Copy macroscopic fields, as double, into dst: one [ny][nx] plane per set bit of
 * mask, in increasing bit order.  rho and u are those of the last collision, psi
 * that of the last step, T the current temperature; solid nodes report rho_solid,
 * u = 0, T_w; SOLID is 1.0 on solid nodes.  FX, FY: the force F = F_m + F_g (+ body_fx)
 * the last collision applied (the interaction force of Eq. (interForce) and gravity along
 * -x, Sec. IV.A), recomputed from the psi and rho it used, bit-equal to the collision's own;
 * zero on solid nodes, before the first step and after a warm-up step (no force).  bytes
 * must be at least popcount(mask) * nx * ny * 8.  dst_on_device: 1 if dst is device memory.
 * Synchronises.
 */
lbm_status lbm_fields(lbm_ctx *ctx, uint32_t mask, void *dst, size_t bytes, int dst_on_device);

/*
 * Checkpoint: post-collision populations f* ([9][ny][nx]), temperature ([ny][nx]),
 * the outlet's last streamed values of f_2, f_6, f_8 ([3][ny]) and the step
 * counter, as host doubles.  Any pointer may be NULL.  Synchronises.
 */
lbm_status lbm_get_state(lbm_ctx *ctx, double *f, double *T, double *side, int64_t *steps);

/* Restore (any subset of) a checkpoint written by lbm_get_state; NULL keeps that part.
 * steps < 0 keeps the step counter.  Host doubles are converted to the storage type.
 * T at solid nodes is the wall temperature from then on: pass the values lbm_get_state
 * returned there to keep the wall created with the context.  A restore also clears a latched
 * fault (LBM_EUNSTABLE, LBM_ETIMEOUT) and the energy pass's per-launch heat-flux
 * bookkeeping, so a context that reported one continues from the restored state; the
 * running heat-flux statistics are kept (lbm_reset_heat_flux clears them). */
lbm_status lbm_set_state(lbm_ctx *ctx, const double *f, const double *T, const double *side, int64_t steps);

/*
 * The same checkpoint in the context's own number formats, without conversion: f* in the
 * population storage type ([9][ny][nx]: double for LBM_STORE_F64, float for LBM_STORE_F32, IEEE
 * half for LBM_STORE_F16S holding f_i - w_i rho_l), T and the outlet rows in the compute type
 * (double with compute_f64, else float).  Half the bytes of the double form for an FP32
 * context; a native checkpoint restores bit-for-bit.  Same NULL, steps and sync rules as above.
 */
lbm_status lbm_get_state_native(lbm_ctx *ctx, void *f, void *T, void *side, int64_t *steps);
lbm_status lbm_set_state_native(lbm_ctx *ctx, const void *f, const void *T, const void *side, int64_t steps);

/*
 * Staged restore, for streaming states through one context (an ensemble kept in host memory,
 * checkpoints replayed in turn): the copy of the next state runs while the context steps.
 * lbm_stage_state_native starts copying a native-format state (the layouts and types of
 * lbm_get_state_native; f and T required, side may be NULL to keep the outlet rows) from host
 * memory into staging buffers of the context, on a copy stream of its own, and returns without
 * waiting.  lbm_take_staged makes the last staged state the current one: the context's stream
 * waits for that copy on the device (the host does not wait), the buffers are exchanged (no
 * device copy), and the rules of lbm_set_state_native apply (steps >= 0 given at staging sets the
 * step counter; a latched fault and the per-launch heat-flux bookkeeping are cleared).
 * Pinned host memory makes the copy asynchronous; the host arrays must stay unchanged until a
 * synchronising call that follows lbm_take_staged (lbm_sync, lbm_wall_heat_flux, lbm_fields,
 * lbm_get_state*) has returned.  Staging again before a take replaces the staged state.  The
 * first call allocates the staging buffers (9 population planes, one T plane, the outlet rows).
 * Errors: LBM_EINVAL (null ctx, f or T), LBM_ESTATE (a batch's domain; take with nothing
 * staged), LBM_ENOMEM, LBM_ECUDA.
 */
lbm_status lbm_stage_state_native(lbm_ctx *ctx, const void *f, const void *T, const void *side, int64_t steps);
lbm_status lbm_take_staged(lbm_ctx *ctx);

/* Derived constants and counters. */
lbm_status lbm_info(lbm_ctx *ctx, lbm_info_t *info);

/*
 * Test hook for the bounded device waits (the paper has no counterpart).  The next lbm_step
 * starves one pass: every tile of it that would be staged into shared memory by TMA arms its
 * barrier with the expected byte count but issues no copy, waits a short bound (64 tries)
 * that runs out, waits that bound once more and produces nothing.  No copy is ever in flight,
 * and the context stays usable: the next synchronising call reports LBM_ETIMEOUT with the pass
 * named in lbm_last_error, and lbm_set_state / lbm_set_state_native (which clear the latched
 * fault bits and the heat-flux bookkeeping) restore a state to continue from.
 * kind: LBM_FAULT_STARVE_COLLIDE or LBM_FAULT_STARVE_ENERGY.  LBM_EINVAL for another kind,
 * LBM_ESTATE when the context stages no tile (environment LBM_TMA=0 at creation) or, for the
 * energy pass, runs without the energy equation.
 */
typedef enum { LBM_FAULT_STARVE_COLLIDE = 1, LBM_FAULT_STARVE_ENERGY = 2 } lbm_fault;
lbm_status lbm_inject_fault(lbm_ctx *ctx, int32_t kind);

/*
 * Per-kernel timing with CUDA events on the context's stream.  lbm_profile(ctx, 1)
 * starts recording an event pair around every kernel launch; lbm_profile_read
 * synchronises and returns, for up to max_kernels kernels, the name (static
 * string), the number of launches and the total milliseconds since profiling was
 * enabled; *n_kernels receives the number of distinct kernels.
 */
lbm_status lbm_profile(lbm_ctx *ctx, int enable);
lbm_status lbm_profile_read(lbm_ctx *ctx, const char **names, int64_t *launches, double *total_ms,
                            int32_t max_kernels, int32_t *n_kernels);

/* ---------------------------------------------------------------------------------
 * Batches: many independent domains (uneven sizes allowed) stepped together.
 * Each step is one kernel launch per pass (psi, collision, energy) over the tiles of all
 * domains; once every domain is past its warm-up, pairs of steps are replayed from a
 * CUDA graph.  Not part of the paper's method (its boiling curve is a set of separate
 * runs, Sec. IV.B); it changes how the same per-domain step is scheduled, not what it
 * computes: every domain gives the same fields as its own context would.
 * ------------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch; /* opaque, owned by the library */

/* Create n >= 1 domains from arrays of n descriptors.  All must share compute_f64, with
 * storage F32 (FP32 build) or F64 (FP64 build) and psi_mode 0.  Errors as lbm_create;
 * cuda_stream: the caller's stream, on which lbm_batch_step orders its work. */
lbm_status lbm_batch_create(int32_t n, const lbm_domain *domains, const lbm_cylinder *cyls, const lbm_params *params,
                            const lbm_allocator *alloc, void *cuda_stream, lbm_batch **out);
/* Enqueue n >= 0 steps of every domain (asynchronous). */
lbm_status lbm_batch_step(lbm_batch *b, int64_t n);
/* Autotuner: time each tile-shape variant twice, in two interleaved rounds of
 * steps_per_variant real steps each (they advance the simulation: 2 x variants x
 * steps_per_variant steps), keep the variant with the fastest round; *variant (may be NULL)
 * receives its index.  The choice is cached per set of domains (their lattice, walls and
 * cylinder, energy and multiphase switches), precision and device (name, compute capability,
 * SM count) for the life of the process and, when the environment variable LBM_TUNE_CACHE
 * names a file, in that file across processes; a set tuned before is given the cached choice
 * without timing and without taking a step. */
lbm_status lbm_batch_tune(lbm_batch *b, int32_t steps_per_variant, int32_t *variant);
/* CUDA-graph replay on (1, default) or off (0). */
lbm_status lbm_batch_graph(lbm_batch *b, int enable);
/* Borrowed handle of domain i for lbm_fields, lbm_get_state, lbm_wall_heat_flux and
 * friends; lbm_step on it returns LBM_ESTATE and lbm_destroy on it does nothing. */
lbm_status lbm_batch_domain(lbm_batch *b, int32_t i, lbm_ctx **ctx);
/* Release the batch and all its domains.  NULL is a no-op. */
void lbm_batch_destroy(lbm_batch *b);

/*
 * Adjoint (reverse-mode derivative) of the time step.  The paper has no adjoint; these are
 * the exact transpose of the discrete update above (upwind switches and clamps take the
 * branch the forward took), for design and inverse problems on the wall heat flux of
 * Sec. IV.B.  Both need energy = 1, every step at or past the warm-up, and (FP32 build)
 * storage = LBM_STORE_F32; otherwise LBM_EINVAL / LBM_ESTATE.  Forward values are
 * recomputed in the context's precision; parameter gradients accumulate in FP64.
 *
 * Objective of a window of n steps from the current state:
 *   J = (1/n) sum_{s<n} q_s,  q_s the heat-flux sample of step s (lbm_wall_heat_flux),
 * with the solid nodes held at their wall temperature T_w from the first step on.
 * Parameters: T_w per solid node; superheat_Tc (T_w = T_sat + (superheat_Tc + profile) T_c);
 * the profile knots of lbm_cylinder.wall_dT; u_in, as the speed of the Zou-He inlet only
 * (nu_l, g and outlet_U stay at the context's values: pass them explicitly in
 * lbm_params when comparing with finite differences of u_in).
 */
typedef struct {
    double J;              /* out: the window's mean heat flux */
    double dJ_dsuperheat;  /* out: dJ / d superheat_Tc */
    double dJ_du_in;       /* out: dJ / d u_in */
    double *dJ_dwall_dT;   /* in: NULL or room for n_wall values; out: dJ / d knot k */
    double *dJ_dTw;        /* in: NULL or room for ny*nx doubles; out: dJ / dT_w at each solid
                              node, 0 at fluid nodes (host, [ny][nx]) */
} lbm_window_grad;

/*
 * Run the window's n_steps forward from the current state (the context advances exactly as
 * with lbm_step, heat-flux statistics included; T at solid nodes is first reset to T_w) and
 * return J and its gradient.  The reverse pass keeps a checkpoint every ckpt_every steps and
 * recomputes each segment from it: device memory (ckpt_every + 1 states, ckpt_every sets of
 * rho, psi, u and the stage-1 temperature, one state per checkpoint, 30 work planes) is
 * allocated on first use through the context's allocator and kept for later windows.
 * Synchronises.
 */
lbm_status lbm_adjoint_window(lbm_ctx *ctx, int64_t n_steps, int32_t ckpt_every, lbm_window_grad *out);

/*
 * Vector-Jacobian product of one step at the current state (the context does not advance).
 * Seeds on the step's outputs: fb ([9][ny][nx], on f* after the step), Tb ([ny][nx], on T
 * after the step), sb ([3][ny], on the outlet side values after the step) and q_weight (on
 * this step's heat-flux sample); NULL seeds are zero.  Results on the step's inputs: fb_out
 * (f* before the step), Tb_out (T before the step; at solid nodes it is the part that reaches
 * T_w through the state), sb_out, and the direct parameter parts dJ_dTw ([ny][nx], solid
 * nodes: through the Dirichlet values this step assigns) and dJ_du_in.  Host doubles; NULL
 * outputs are skipped.  Synchronises.
 */
lbm_status lbm_adjoint_step(lbm_ctx *ctx, const double *fb, const double *Tb, const double *sb, double q_weight,
                            double *fb_out, double *Tb_out, double *sb_out, double *dJ_dTw, double *dJ_du_in);

/*
 * Wall heat flux from caller-owned fields, with no context and no allocation.
 * The paper has no counterpart of this entry point; it exists for callers that cannot
 * allocate device memory: code whose device memory is a fixed pool handed out by an outer
 * framework, or a hook running where an allocation would synchronise the device or is
 * forbidden outright.  It computes the quantity lbm_wall_heat_flux samples, the mean over
 * the fluid nodes with a D2Q9 link into the cylinder of -lambda(rho) grad T . n (grad T the
 * isotropic 24-neighbour gradient, n the outward normal from the centre, lambda from the
 * parameters as in lbm_create), for the fields the caller passes in.
 *   T, rho  device arrays of doubles, dense [ny][nx] (as lbm_fields writes them)
 *   q_out   device pointer to one double receiving the mean; written on cuda_stream
 * Working memory is a fixed array inside the library (one partial sum and count per tile
 * of 32 x 8 nodes plus a completion counter, 512 KiB in all) that every GPU loading the
 * library keeps until the process exits: lattices above 8,388,608 nodes (more than
 * 32,768 tiles) are rejected with LBM_EINVAL, as are D <= 0 and nx or ny < 5.  The first
 * call on a device looks up that array's device address with the device current; make
 * that first call before any stream capture.  The address is kept with the id of the CUDA
 * context it was looked up in: after a device reset (cudaDeviceReset), which unloads the
 * library's device code, the next call on that device looks it up again (that call, too,
 * belongs outside a stream capture).  All calls share the one array, so calls
 * whose kernels overlap on the GPU race; serialise them (one stream, or events).  The
 * call allocates nothing and is asynchronous; synchronise cuda_stream before reading
 * q_out.  LBM_ECUDA if a CUDA call fails; lbm_last_error does not apply (no context).
 */
lbm_status lbm_wall_heat_flux_noalloc(const lbm_domain *domain, const lbm_cylinder *cyl, const lbm_params *params,
                                      const double *T, const double *rho, double *q_out, void *cuda_stream);

/* Text of the last error of ctx (never NULL); with ctx == NULL, that of the last
 * failed lbm_create on this thread. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Release the context and all its device memory.  NULL is a no-op. */
void lbm_destroy(lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
