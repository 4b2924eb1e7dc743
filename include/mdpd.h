/*
 * mdpd.h -- C ABI of the GB300 (sm_103a) many-body DPD hot path.
 *
 * Method: many-body dissipative particle dynamics (mDPD) as used in
 * arXiv:1903.10134.  Per time step the library bins the particles into a cell
 * lattice, evaluates the local density rho_i (Sec. 2.1), the pair forces
 * F^C + F^D + F^R of Sec. 2.1 and Eq. 1, and advances the velocity-Verlet
 * integrator in the order of Algorithm 1, reflecting particles off solid
 * voxels of a pore image (Sec. 2.2) and off non-periodic box faces.
 *
 * Conventions for every entry point:
 *   - Return 0 (MDPD_OK) on success or a negative MDPD_ERR_* code; the text of
 *     the last error of a handle is available from mdpd_last_error().
 *   - Host arrays are read or written before the call returns (inputs are
 *     copied, the caller keeps ownership).  *_dev variants take device
 *     pointers on the current CUDA device, borrowed for the duration of the
 *     call; their copies are ordered on the handle's stream.
 *   - Particle arrays are indexed by particle id: the caller's input order is
 *     0..n-1; wall particles added by mdpd_set_walls() follow as n, n+1, ...
 *     Vectors are interleaved xyz (element 3*i+k).
 *   - Units are DPD units with particle mass m = 1.
 *   - Work is enqueued on the handle's stream; errors raised on the device
 *     (non-finite values, particles outside a non-periodic box) are reported
 *     by the next call that synchronises (mdpd_sync, mdpd_get_state,
 *     mdpd_forces, mdpd_observables*).
 *   - A handle is used by one host thread at a time.
 */
#ifndef MDPD_H
#define MDPD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MDPD_MAX_TYPES 8
#define MDPD_NUM_OBS 16
#define MDPD_MAX_REPLICAS 65536

enum {
    MDPD_OK = 0,
    MDPD_ERR_INVALID_ARG = -1,   /* bad argument or unsupported geometry     */
    MDPD_ERR_OOM = -2,           /* device or host allocation failed         */
    MDPD_ERR_CUDA = -3,          /* a CUDA runtime call failed               */
    MDPD_ERR_NONFINITE = -4,     /* a position, velocity or force is NaN/inf */
    MDPD_ERR_OUT_OF_BOX = -5,    /* a particle left a non-periodic box       */
    MDPD_ERR_TILE_OVERFLOW = -6, /* a cell held more particles than a kernel
                                    tile can stage                           */
    MDPD_ERR_TIMEOUT = -7,       /* a bounded device wait gave up            */
    MDPD_ERR_BOUNDS = -8         /* an index check of the debug build failed
                                    (libmdpd_gb300_debug.so only)            */
};

/* System parameters (Sec. 2.1, Eq. 1).  Pair tables are indexed [type_i][type_j]
 * and must be symmetric.  sigma of the random force follows the
 * fluctuation-dissipation theorem, sigma^2 = 2 gamma kT (Sec. 2.1). */
typedef struct mdpd_params {
    double box_lo[3];        /* lower box corner                                */
    double box[3];           /* box edge lengths; periodic axes need >= 3 r_c    */
    int32_t periodic[3];     /* 1 periodic, 0 reflecting faces                  */
    int32_t ntypes;          /* 1..MDPD_MAX_TYPES                               */
    double rc;               /* cutoff of w_C = w_R = 1 - r/r_c                 */
    double rd;               /* many-body cutoff r_d < r_c (w_d, w_rho)         */
    double dt;               /* time step                                       */
    double kT;               /* temperature                                     */
    double A[MDPD_MAX_TYPES][MDPD_MAX_TYPES];     /* attraction, A < 0          */
    double B[MDPD_MAX_TYPES][MDPD_MAX_TYPES];     /* many-body repulsion, B > 0 */
    double gamma[MDPD_MAX_TYPES][MDPD_MAX_TYPES]; /* dissipation                */
    double g[3];             /* body acceleration on mobile particles           */
    uint32_t frozen_type_mask; /* bit t: type t is frozen (no motion, v = 0)    */
    int32_t precision;       /* 0: FP64 pair arithmetic; 1: FP32 pair arithmetic
                                on cell-relative offsets, FP64 integration     */
    int32_t xi_dist;         /* 0: xi uniform, unit variance; 1: Gaussian       */
    int32_t rho_self;        /* 1: rho_i also counts w_rho(0) for j = i (0 in
                                the paper, Sec. 2.1)                           */
} mdpd_params;

typedef struct mdpd_handle mdpd_handle;

/* Create a system of n particles on the current CUDA device.
 * pos, vel: host arrays of 3n doubles; type: n values in [0, ntypes).
 * seed keys the Philox-4x32-10 stream of the random force; the pair draw
 * for the force evaluation of step s uses counter (min id, max id, s_lo, s_hi)
 * so that xi_ij = xi_ji (Sec. 2.1).  cuda_stream: a cudaStream_t to run on,
 * or NULL for a stream the handle creates and owns.
 * The density and forces of the initial state are evaluated (step index 0).
 * At most 2^27 particles (including wall particles).
 * Errors: INVALID_ARG (n < 0, ntypes out of range, r_d > r_c, non-positive
 * dt/r_c/box, a periodic axis shorter than 3 r_c, a type out of range),
 * OOM, CUDA. */
int mdpd_create(const mdpd_params* params, int64_t n, const double* pos,
                const double* vel, const int32_t* type, uint64_t seed,
                void* cuda_stream, mdpd_handle** out);

/* Same as mdpd_create with device arrays pos, vel (3n doubles) and type (n). */
int mdpd_create_dev(const mdpd_params* params, int64_t n, const double* pos,
                    const double* vel, const int32_t* type, uint64_t seed,
                    void* cuda_stream, mdpd_handle** out);

/* Batch of nrep independent systems advanced together: every kernel of a
 * time step is one launch over all replicas (ensembles, parameter sweeps and
 * fits of A, B over many small boxes; the paper's single system is the case
 * nrep = 1).  Replica r has its own params[r] (box, periodicity, pair
 * tables, r_c, r_d, dt, kT, body force; precision must be equal), its own
 * seed seeds[r] and n[r] particles; the inputs pos, vel (3 N doubles), type
 * (N values), N = sum n[r], hold replica 0's particles first, then replica
 * 1's, and so on, and the batch's particle ids follow that order.  Within a
 * replica the random stream is keyed on the particle's index inside the
 * replica, so replica r evolves bit-identically to mdpd_create() of
 * (params[r], n[r] particles, seeds[r]) run alone with the same kernel
 * variant.  Walls and the wall density are not available on a batch handle;
 * the VJPs and windows are, with per-replica parameter gradients.
 * mdpd_step, mdpd_get_state/set_state(_dev), mdpd_forces(_dev),
 * mdpd_set_step, mdpd_sync, mdpd_pair_count (summed over replicas),
 * mdpd_profile, mdpd_set_option and mdpd_autotune apply to the whole batch;
 * the observables are per replica (mdpd_batch_observables).
 * Errors: INVALID_ARG (nrep outside 1..MDPD_MAX_REPLICAS, any replica's
 * params invalid as for mdpd_create, mixed precision, more than 2^27
 * particles or 16.7M cells in all), OOM, CUDA. */
int mdpd_create_batch(int32_t nrep, const mdpd_params* params, const int64_t* n,
                      const double* pos, const double* vel, const int32_t* type,
                      const uint64_t* seeds, void* cuda_stream, mdpd_handle** out);

/* Number of replicas (1 for a handle made by mdpd_create). */
int mdpd_num_replicas(const mdpd_handle* h, int32_t* nrep);

/* Per-replica observables of a batch handle, nrep * MDPD_NUM_OBS doubles
 * (replica-major, each record laid out as mdpd_observables): the last step's
 * values (mean = 0) or the running means since the last reset (mean = 1;
 * reset = 1 then clears the running sums).  INVALID_ARG on a single-system
 * handle.  Synchronises. */
int mdpd_batch_observables(mdpd_handle* h, double* out, int32_t mean, int32_t reset);

/* Replace every replica's parameters between steps (params: nrep records).
 * The boxes, periodicity, r_c, precision and ntypes must not change; the
 * seeds are kept.  Captured step graphs stay valid.  INVALID_ARG on a
 * single-system handle.  Synchronises. */
int mdpd_batch_set_params(mdpd_handle* h, const mdpd_params* params);

/* Walls from a voxel image (Sec. 2.2, 2.3).  solid: nx*ny*nz bytes, x
 * fastest, nonzero = solid, covering [origin, origin + n*voxel) per axis.
 * 1) The image becomes the reflection mask: a drift that lands in a solid
 *    voxel is undone and the half-step velocity negated.
 * 2) Solid voxels whose centre lies within shell_thickness of a pore voxel
 *    centre (periodic wrap on periodic axes) receive wall particles of
 *    wall_type (which should be frozen) at number density wall_density: a
 *    voxel gets floor(wall_density * voxel^3 + u) particles at uniform points,
 *    u and the points drawn from Philox-4x32-10 keyed by seed with counter
 *    (voxel id, k, 0x57414C4C, 0); they take ids n, n+1, ... by ascending
 *    voxel id.  Their velocity is 0.
 * May be called once per handle.  Densities and forces are re-evaluated.
 * Images up to 2^31 voxels.  Errors: INVALID_ARG (dims, voxel, type, a
 * periodic axis the image does not span exactly, more than 2^31 voxels, a
 * second call), OOM, CUDA. */
int mdpd_set_walls(mdpd_handle* h, const uint8_t* solid, int32_t nx, int32_t ny,
                   int32_t nz, double voxel, const double origin[3],
                   double wall_density, double shell_thickness, int32_t wall_type,
                   uint64_t seed);

/* Advance nsteps velocity-Verlet steps (Algorithm 1 without its
 * communication lines): v += dt/2 a; x += dt v; reflect; rho(x); a(x, v, rho);
 * v += dt/2 a.  Asynchronous on the handle's stream.  nsteps >= 0. */
int mdpd_step(mdpd_handle* h, int64_t nsteps);

/* Wait for the handle's stream and report device-side errors. */
int mdpd_sync(mdpd_handle* h);

/* Number of particles (including wall particles) and of steps taken. */
int mdpd_num_particles(const mdpd_handle* h, int64_t* n);
int mdpd_step_count(const mdpd_handle* h, int64_t* steps);

/* Copy the state to host arrays in id order: pos/vel 3N doubles, type N,
 * rho N (the local density of the last force evaluation).  This is the state
 * of Algorithm 1 after its last line: x(t + dt), v(t + dt) and the density
 * rho_i of Sec. 2.1 at x(t + dt).  Any pointer may be NULL.  Errors:
 * INVALID_ARG (NULL handle), NONFINITE / OUT_OF_BOX raised by the last steps,
 * CUDA.  Synchronises. */
int mdpd_get_state(mdpd_handle* h, double* pos, double* vel, int32_t* type,
                   double* rho);

/* Device-array variant of mdpd_get_state (no host synchronisation beyond the
 * error check). */
int mdpd_get_state_dev(mdpd_handle* h, double* pos, double* vel, int32_t* type,
                       double* rho);

/* Replace positions and velocities (3N doubles each, id order, host arrays);
 * types and step index are kept; densities and forces are re-evaluated at the
 * current step index.  Positions on periodic axes are wrapped into the box.
 * The frozen-frozen part of the wall particles' densities is kept when every
 * frozen particle is loaded at exactly the position it had when that part was
 * computed, and recomputed otherwise.  Synchronises. */
int mdpd_set_state(mdpd_handle* h, const double* pos, const double* vel);

/* Device-array variant of mdpd_set_state. */
int mdpd_set_state_dev(mdpd_handle* h, const double* pos, const double* vel);

/* Checkpoint and bit-exact resume.  mdpd_get_accel (host, N x 3, id order)
 * returns the accelerations the next step's first half-kick will use: those
 * of the last force evaluation, a(t + dt) computed with the half-step
 * velocity.  mdpd_set_state_accel loads positions, velocities and those
 * accelerations without evaluating the forces, so a run resumed from
 * (mdpd_get_state, mdpd_get_accel, mdpd_step_count, seed) with mdpd_create,
 * mdpd_set_step and mdpd_set_state_accel continues bit for bit (Philox is
 * keyed on the step, not on a running state).  Until the next step or force
 * evaluation the densities returned by mdpd_get_state are stale.
 * Errors: INVALID_ARG, NONFINITE, CUDA.  Synchronise. */
int mdpd_get_accel(mdpd_handle* h, double* accel);
int mdpd_set_state_accel(mdpd_handle* h, const double* pos, const double* vel,
                         const double* accel);

/* Evaluate, without stepping, the density and the forces at the current
 * positions and velocities with the current step index: the local density
 * rho_i of Sec. 2.1 and the pair forces F^C + F^D + F^R of Sec. 2.1 and Eq. 1
 * (Algorithm 1 lines 4 and 6 without the integration).  force gets 3N doubles
 * (sum_j F_ij + g for mobile particles, m = 1; 0 for frozen ones), rho N
 * doubles, id order.  Either pointer may be NULL.  Errors: INVALID_ARG,
 * NONFINITE, CUDA.  Synchronises. */
int mdpd_forces(mdpd_handle* h, double* force, double* rho);

/* Device-array variant of mdpd_forces. */
int mdpd_forces_dev(mdpd_handle* h, double* force, double* rho);

/* Observables of the last force evaluation (the pressure-tensor and
 * temperature checks of Sec. 4.1: the surface tension there is built from
 * the diagonal of the pressure tensor, kinetic part plus the virial below),
 * reduced in FP64 in a fixed order:
 * out[0..2] momentum, out[3] kinetic energy, out[4] kT = 2 KE / (3 (N_m - 1)),
 * out[5..10] conservative virial 1/2 sum_{i mobile} sum_j r_ij,a F^C_ij,b
 * (xx yy zz xy xz yz), out[11..13] sum v_a^2, out[14] N_m (mobile count),
 * out[15] step index.  Synchronises. */
int mdpd_observables(mdpd_handle* h, double out[MDPD_NUM_OBS]);

/* Mean of the per-step observables over the steps since the last reset
 * (reset != 0 clears the accumulator after reading).  Synchronises. */
int mdpd_observables_mean(mdpd_handle* h, double out[MDPD_NUM_OBS], int32_t reset);

/* Pair evaluations (0 < r < r_c) of the last force pass: every mobile
 * particle counts its partners, so a pair of two mobile particles counts
 * twice.  Synchronises. */
int mdpd_pair_count(mdpd_handle* h, int64_t* pairs);

/* Options (mdpd_set_option):
 *   MDPD_OPT_GRAPH     1 (default): replay each step as a captured CUDA graph;
 *                      0: launch kernels one by one.
 *   MDPD_OPT_PROFILE   k > 0: record CUDA events around every kernel class of
 *                      the next steps (up to k steps); 0: off.
 *   MDPD_OPT_KERNELS   MDPD_KERNELS_NLIST (default): a warp-per-cell density
 *                      pass records each mobile particle's partners within r_c
 *                      and the force pass walks that list;
 *                      MDPD_KERNELS_NLIST_THREAD: the same with a
 *                      thread-per-particle density pass; MDPD_KERNELS_SCAN:
 *                      both passes scan the 27 neighbour cells directly.
 *                      Same results up to FP summation order.
 *   MDPD_OPT_WALL_DENSITY  1: every density pass also accumulates the wall
 *                      density phi of each mobile particle (Sec. 3.2,
 *                      Algorithm 1 step 2; read with mdpd_get_wall_density);
 *                      the thread-per-particle density variant is used while
 *                      it is on.  0 (default): off.
 *   MDPD_OPT_FORCE_LANES  1, 2 or 4 (default 1): lanes that share one
 *                      particle's partner list in the force pass (more warps
 *                      for small systems; the partner sums are combined in a
 *                      fixed order, so results are reproducible for a given
 *                      setting but round differently from another setting).
 *                      A batch handle accepts 1 only.
 *   MDPD_OPT_PROFILE_EVERY  m >= 1: with MDPD_OPT_PROFILE on, record the events
 *                      on every m-th step only (default 1), which keeps their
 *                      cost out of most steps.
 *   MDPD_OPT_DENSITY_SHAPE  0 (default) or 1: code shape of the
 *                      thread-per-particle density kernel (candidate loop not
 *                      unrolled, or unrolled by two under a tighter register
 *                      budget).  Results are identical; only the speed
 *                      differs (mdpd_autotune picks the faster).
 */
enum { MDPD_OPT_GRAPH = 1, MDPD_OPT_PROFILE = 2, MDPD_OPT_KERNELS = 3,
       MDPD_OPT_PROFILE_EVERY = 4, MDPD_OPT_WALL_DENSITY = 5, MDPD_OPT_FORCE_LANES = 6,
       MDPD_OPT_DENSITY_SHAPE = 7 };
enum { MDPD_KERNELS_NLIST = 0, MDPD_KERNELS_SCAN = 1, MDPD_KERNELS_NLIST_THREAD = 2 };
int mdpd_set_option(mdpd_handle* h, int32_t option, int64_t value);

/* Kernel classes reported by mdpd_profile(). */
enum { MDPD_K_BIN = 0, MDPD_K_DENSITY = 1, MDPD_K_FORCE = 2, MDPD_K_OTHER = 3,
       MDPD_NUM_KCLASS = 4 };

/* Sum of the recorded kernel durations per class (ms) and the number of steps
 * recorded; clears the record.  Synchronises. */
int mdpd_profile(mdpd_handle* h, double ms[MDPD_NUM_KCLASS], int64_t* steps,
                 int64_t* launches);

/* Wall density of the last density pass (MDPD_OPT_WALL_DENSITY on): for each
 * mobile particle phi_i = sum over frozen particles j with 0 < r_ij < r_c of
 * 15/(2 pi r_c^3) (1 - r_ij/r_c)^2, the density of solid particles within the
 * particle's support (Sec. 3.2); 0 for frozen particles.  Host array of N
 * doubles, id order.  Synchronises. */
int mdpd_get_wall_density(mdpd_handle* h, double* phi);

/* Replace the parameters of a handle between steps.  Only A, B, gamma, kT, dt,
 * g, frozen_type_mask, xi_dist and rho_self may differ; box, periodicity, rc,
 * rd, ntypes and precision must match the handle's.  The next step (or
 * mdpd_forces / mdpd_set_state) uses the new values.  Synchronises. */
int mdpd_set_params(mdpd_handle* h, const mdpd_params* params);

/* Set the step index: the next force evaluation of mdpd_step uses step + 1,
 * mdpd_forces / mdpd_set_state / mdpd_force_vjp_dev use step (this selects the
 * Philox draws).  Synchronises. */
int mdpd_set_step(mdpd_handle* h, int64_t step);

/* Device copy (id order, 3N doubles) of the acceleration the next half-kick
 * will use: a(t) of the current state.  Synchronises. */
int mdpd_get_accel_dev(mdpd_handle* h, double* accel);

/* Vector-Jacobian product of one evaluation of Sec. 2.1 / Eq. 1 (the local
 * densities rho_i, the accelerations a_i = sum_j F_ij + g of mobile
 * particles and the conservative virial W of mdpd_observables, whose
 * diagonal builds the pressure tensor and surface tension of Sec. 4.1) at
 * the current positions, the current velocities (those the dissipative term
 * sees) and the current step index, with the random draws of that step held
 * fixed:  L = sum_i abar_i . a_i + sum_r sum_k cvir[6r + k] W_k(replica r)
 *            + sum_i rhobar_i rho_i.
 * Inputs (device, each may be NULL = zero): abar 3N doubles (id order; rows
 * of frozen particles are ignored), cvir 6 doubles per replica (xx yy zz xy
 * xz yz weights, the order of mdpd_observables), rhobar N doubles.
 * Outputs (device, may be NULL): xbar, ubar 3N doubles (id order): dL/dx
 * (including the path through the local densities) and dL/du; theta_bar
 * 3*8*8 doubles per replica (replica-major): the gradient with respect to
 * the symmetric tables A, B, gamma ([q][a][b] = [q][b][a] = dL/dP_ab; the
 * gamma entry includes sigma = sqrt(2 gamma kT)).  The parameter gradients
 * are reduced in a fixed order, so repeated calls agree bit for bit.  The
 * state is not changed.  Errors: INVALID_ARG (a host pointer),
 * TILE_OVERFLOW (a particle with more than 64 partners within r_c), CUDA.
 * Synchronises. */
int mdpd_eval_vjp_dev(mdpd_handle* h, const double* abar, const double* cvir,
                      const double* rhobar, double* xbar, double* ubar, double* theta_bar);

/* mdpd_eval_vjp_dev with abar only (the force VJP of Sec. 2.1 / Eq. 1);
 * abar is required. */
int mdpd_force_vjp_dev(mdpd_handle* h, const double* abar, double* xbar, double* ubar,
                       double* theta_bar);

/* mdpd_eval_vjp_dev with rhobar only: xbar (device, 3N, id order) =
 * d(sum_i rhobar_i rho_i)/dx of the local densities of Sec. 2.1; every
 * particle's density counts, frozen ones included.  Both pointers are
 * required. */
int mdpd_density_vjp_dev(mdpd_handle* h, const double* rhobar, double* xbar);

/* Record a velocity-Verlet window for its adjoint: advance nsteps steps of
 * Algorithm 1 (as mdpd_step) from the current state and step index s0,
 * keeping every step's positions x_k and half-step velocities
 * v'_k = v_k + (dt/2) a_k in device memory owned by the handle (48 N bytes
 * per step; the checkpoints of the adjoint), so that mdpd_window_vjp_dev can
 * run the chain rule backwards.  Reflection is not differentiable: handles
 * with walls or a non-periodic axis are refused.  The checkpoints stay valid
 * until the parameters or the particles change (mdpd_set_params,
 * mdpd_batch_set_params, mdpd_set_walls) or another window is recorded;
 * stepping or setting the state in between does not disturb them.
 * Errors: INVALID_ARG, OOM, CUDA and the errors of mdpd_step.  Synchronises. */
int mdpd_window_forward(mdpd_handle* h, int32_t nsteps);

/* Adjoint of the recorded window (Algorithm 1 run backwards with the VJP of
 * each step's force evaluation, random draws fixed): given the adjoints of
 * the final state, xbar and vbar (device, 3N doubles, id order), and of the
 * final evaluation's virial and local densities (what mdpd_observables /
 * mdpd_batch_observables and mdpd_get_state report after the window), cvir
 * (device, 6 doubles per replica) and rhobar (device, N doubles) -- each NULL
 * for zero -- it returns x0bar, v0bar (device, 3N; may be NULL), the gradient with
 * respect to the window's initial positions and velocities, and theta_bar
 * (device, 3*8*8 doubles per replica; may be NULL), the gradient with
 * respect to A, B, gamma as in mdpd_eval_vjp_dev, every step's and every
 * replica's partials reduced in a fixed order.  Per step, with
 * (xb, vb, ab) the adjoints of (x_{k+1}, v_{k+1}, a_{k+1}) and h = dt/2:
 *   vhb = vb, ab += h vb;  xb += F_x^T ab, vhb += F_u^T ab;
 *   vhb += dt xb;  vb = vhb, ab = h vhb   (frozen particles: no kick, no drift)
 * and finally a_0 = F(x_0, v_0).  Afterwards the handle is back at the start
 * of the window (x_0, v_0, step index s0, accelerations re-evaluated) and the
 * window stays recorded, so it may be run again or differentiated with other
 * adjoints.  Errors: INVALID_ARG (no recorded window), TILE_OVERFLOW, CUDA.
 * Synchronises. */
int mdpd_window_vjp_dev(mdpd_handle* h, const double* xbar, const double* vbar,
                        const double* cvir, const double* rhobar, double* x0bar, double* v0bar,
                        double* theta_bar);

/* Time the density-pass variants (MDPD_KERNELS_NLIST, MDPD_KERNELS_NLIST_THREAD
 * in both code shapes of MDPD_OPT_DENSITY_SHAPE) and then the force pass at 1,
 * 2 and 4 lanes per particle (MDPD_OPT_FORCE_LANES; 1 only on a batch) on the
 * current state, reps launches each, and keep the fastest of each.  The
 * trajectory is not advanced.  chosen (may be NULL, 3 ints) receives the
 * density variant, the lanes per particle and the code shape kept; ms (may be
 * NULL, 5 doubles) the mean time of each density variant in that order (the
 * thread variant's faster shape), then of the force pass at 1, 2, 4 lanes (-1:
 * not tried).  Synchronises. */
int mdpd_autotune(mdpd_handle* h, int32_t reps, int32_t* chosen, double* ms);

/* Grid of the cell lattice (cells per axis) and the kernel launches one step
 * issues. */
int mdpd_describe(const mdpd_handle* h, int32_t ncell[3], int32_t* launches_per_step);

/* Local densities rho_i for callers that cannot allocate device memory.
 * There is no counterpart in the paper; this is a service of the library.
 * Some callers may not let a library allocate: a plugin inside a host
 * application that owns the whole device-memory budget and passes in only
 * its buffers, or code on a latency-critical path where cudaMalloc/cudaFree
 * (which can synchronise the device) are not allowed.  This entry point runs
 * the binning and density kernels with all temporaries in one fixed
 * __device__ array of the library (about 4.3 MB, held by every GPU that
 * loads the library until the process exits); it calls no allocator.
 * params: box, periodic, rc, rd, precision and rho_self are used.
 * pos: device array of 3n doubles (interleaved xyz); on non-periodic axes
 * positions must lie in [lo, lo + L] (the upper face included).  A particle
 * outside that range, or with a non-finite coordinate, gets rho = NaN, and
 * the densities of its neighbours are then undefined too.
 * rho: device array of n doubles, written in input order.
 * Limits: n <= 65536 and at most 32768 cells of edge >= rc; larger inputs
 * fail with MDPD_ERR_INVALID_ARG (message from mdpd_last_error(NULL)).
 * Errors: INVALID_ARG (the limits, NULL arrays, rd > rc, bad box),
 * CUDA (a CUDA error already pending before the call is reported, not
 * cleared; a failed launch is named in the message).
 * Asynchronous on cuda_stream (NULL = legacy default stream).  Outside
 * stream capture every call looks up the array's device address afresh, so
 * cudaDeviceReset between calls is harmless; a call made while cuda_stream is
 * being captured reuses the address found by the last uncaptured call on the
 * device, so make the first call on a device before any stream capture.  All
 * calls share the array: calls whose work overlaps on the GPU (other streams,
 * other host threads) race and give wrong results. */
int mdpd_density_noalloc(const mdpd_params* params, int64_t n, const double* pos,
                         double* rho, void* cuda_stream);

/* Measured FP32 issue rate of the current device, the denominator of the ALU
 * roofline that the density and force passes are reported against: a
 * full-occupancy grid of independent fused multiply-add chains, best of 4
 * timed launches (about 50 ms in all).  lane_ops_per_s receives FMA
 * lane-operations per second (one per lane per instruction), best_ms (may be
 * NULL) the best launch time.  Errors: INVALID_ARG (NULL output), CUDA. */
int mdpd_measure_fma_peak(double* lane_ops_per_s, double* best_ms);

/* Release a handle: waits for its stream, frees every device buffer and
 * captured graph it owns and, if it created its stream, that stream (the end
 * of the run of Algorithm 1; the paper's code leaves this to its host
 * framework).  NULL is accepted and ignored.  No error is reported. */
void mdpd_destroy(mdpd_handle* h);

/* Message of the last error on h (or of the last failed mdpd_create when h is
 * NULL).  Valid until the next call on the same handle. */
const char* mdpd_last_error(const mdpd_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* MDPD_H */
