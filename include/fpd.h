/*
 * fpd.h -- C ABI of the GB300 (sm_103a) extended fluid-particle-dynamics
 * (FPD) solver of arXiv 2212.14153: flexible bead-spring fibers in a confined
 * Couette flow, computed with a D2Q9 multiple-relaxation-time lattice
 * Boltzmann method in which every bead is a smoothed high-viscosity region.
 *
 * One call of fpd_step advances the method of Sec. 2.3 by one time step:
 *   (3) of the previous step  V_i = int phi_i v / int phi_i  (Eq. 5) and
 *       R_i <- R_i + dt V_i (forward Euler, dt = 1), skipped at step 0;
 *   (1) phi_i from R_i (Eq. 2), bead forces F_i (Eqs. 11-12 + excluded
 *       volume), force density f = sum_i phi_i F_i / int phi_i (Eq. 4),
 *       viscosity eta = eta_f + sum_i (eta_s - eta_f) phi_i (Eq. 1);
 *   (2) MRT collision with Guo forcing, streaming, and half-way moving-wall
 *       bounce-back at y = 0 (speed u_bottom) and y = H (speed u_top), x
 *       periodic (Sec. 4.1).
 * Everything is in lattice units: dx = dt = 1, rho_0 = 1, c_s^2 = 1/3.
 *
 * Conventions of every entry point:
 *  - Return value: an fpd_status (0 = FPD_OK, negative = error).  The text
 *    of the last error of a handle is returned by fpd_last_error(handle);
 *    fpd_last_error(NULL) returns the last error of fpd_create in the
 *    calling thread.  No exception crosses this boundary.
 *  - Host pointers are caller-owned and only read or written during the
 *    call.  The library owns all device memory of a handle (allocated by
 *    fpd_create, freed by fpd_destroy).
 *  - Work runs on the CUDA stream given to fpd_create (NULL = the legacy
 *    default stream).  fpd_step is asynchronous; the fpd_read_* calls and
 *    fpd_sync synchronise the stream and report any device-side error.
 *  - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef FPD_H
#define FPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FPD_ABI_VERSION 4

typedef enum {
    FPD_OK = 0,
    FPD_EINVAL = -1,   /* invalid argument or parameter set                 */
    FPD_ENOMEM = -2,   /* device or host allocation failed                  */
    FPD_ECUDA = -3,    /* a CUDA call failed (message has the CUDA error)   */
    FPD_ETIMEOUT = -4, /* a bounded wait gave up                            */
    FPD_ENAN = -5,     /* a non-finite value was found in the state         */
    FPD_EBUSY = -6     /* no free slot or memory for the request            */
} fpd_status;

typedef enum {
    FPD_F64 = 0,          /* FP64 storage and arithmetic (parity path)       */
    FPD_F32 = 1,          /* FP32 storage of f_k - w_k, FP32 arithmetic      */
    FPD_F32_F16STORE = 2  /* FP16 storage of (f_k - w_k) * 2^s_k, FP32 math  */
} fpd_precision;

typedef enum {
    FPD_MRT_MAGIC = 0, /* s_e = s_eps = s_nu, (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16 */
    FPD_MRT_LL = 1,    /* constant s_e, s_eps, s_q (Lallemand-Luo set)        */
    FPD_BGK = 2        /* every rate equal to s_nu (single relaxation time)   */
} fpd_collision;

/* Problem statement of Sec. 4.1 plus the numerical parameters of Sec. 2.
 * Negative values select the documented default where one is stated. */
typedef struct {
    int32_t nx, ny;         /* lattice cells: L_x = nx (periodic), H = ny      */
    double u_bottom;        /* wall speed at y = 0 (paper: -V0)                */
    double u_top;           /* wall speed at y = H (paper: +V0)                */
    double nu_f;            /* fluid kinematic viscosity; <= 0: from re        */
    double re;              /* Re = gamma_dot l_c^2 / nu_f, gamma_dot =
                               (u_top - u_bottom)/H, l_c = 2 a N; Re_ps = re/4 */
    double visc_ratio;      /* r_eta = eta_s / eta_f (Eq. 1)                   */
    double xi;              /* interface thickness of Eq. 2                    */
    double bead_radius;     /* a; spring rest length l_0 = d = 2a              */
    int32_t n_beads;        /* N beads per fiber (0: no fiber)                 */
    int32_t n_fibers;       /* number of fibers                                */
    double k_s;             /* spring constant of Eq. 9; < 0: 0.25 pi a^2 l0^2 */
    double k_b;             /* bending constant of Eq. 9 (used if K <= 0)      */
    double stiffness_K;     /* K = 2 k_b / (eta_f gamma_dot l_c^2) (Eq. 18);
                               > 0 overrides k_b                               */
    double k_ev;            /* excluded-volume stiffness; < 0: k_s / l0^2      */
    double phi_cut;         /* phi = 0 where |r - R_i| >= a + phi_cut xi       */
    double body_force_x;    /* uniform body-force density added to f           */
    double body_force_y;
    int32_t precision;      /* fpd_precision                                   */
    int32_t collision;      /* fpd_collision                                   */
    int32_t init_couette;   /* 1: start at equilibrium of the linear wall
                               profile; 0: fluid at rest                       */
    double s_e, s_eps, s_q; /* rates for FPD_MRT_LL                            */
    const double *centre_xy;/* n_fibers x 2: fiber centres (ignored if bead_xy) */
    const double *theta0;   /* n_fibers: fiber angles in radians               */
    const double *bead_xy;  /* optional (n_fibers*n_beads) x 2 explicit R_i^0  */
    double sandwich_zl;     /* > 0: static solid layers of the Couette benchmark
                               (Sec. 3.1, Eq. 14): phi(y) = (tanh((zl - y)/xi)
                               + 1)/2 for y <= H/2, (tanh((y - zr)/xi) + 1)/2
                               above, added to the bead profiles in Eq. 1   */
    double sandwich_zr;
    int32_t periodic_y;     /* 1: periodic in y as well, no walls (the driven
                               particle of Sec. 3.2); wall speeds then only
                               shape the init_couette start                   */
    double bead_force_x;    /* constant external force F_0 added to the force */
    double bead_force_y;    /* of every bead (Sec. 3.2), spread by Eq. 4       */
} fpd_params;

typedef struct fpd_sim fpd_sim;

/* ABI version (FPD_ABI_VERSION of the built library). */
int fpd_version(void);

/* Fill *p with defaults: 80 x 40, walls -/+0.01, re = 1, r_eta = 50, xi = 1,
 * a = 2, no fiber, phi_cut = 8, FP64, magic MRT, Couette start. */
void fpd_default_params(fpd_params *p);

/* Validate p, derive nu_f, k_s, k_b, k_ev, allocate the state on the device,
 * initialise the fluid (equilibrium at rho_0 = 1) and the fibers
 * (R_i = c + (i - (N+1)/2) l_0 (cos theta, sin theta), i = 1..N, Sec. 4.1:
 * fiber centred) and compute the first bead table.  stream: a cudaStream_t
 * or NULL.  On success *out owns the state.  Errors: FPD_EINVAL (bad
 * parameter, message names it), FPD_ENOMEM, FPD_ECUDA.
 * Environment read here (for the life of the instance; none changes a
 * result unless stated): FPD_NO_GRAPHS=1 launches every kernel directly
 * instead of replaying captured step chunks; FPD_NO_EARLY_COLD=1 makes
 * every tile of every sweep wait for its step's bead phase; for tests only,
 * FPD_TEST_COPY_SHORTFALL=1 has each staged-sweep block (tuning variants 3
 * and 4) expect 16 bytes more than its bulk copy moves, so that its
 * bounded wait runs out: those blocks are left unwritten and
 * FPD_FLAG_COPY_TIMEOUT is set. */
int fpd_create(const fpd_params *p, void *stream, fpd_sim **out);

/* Device bytes of the state of one instance with parameters p (populations,
 * both bead tables, tile masks, a counter and the instance record, each part
 * 256-byte aligned): the workspace fpd_create_ex needs.  FPD_EINVAL for
 * invalid parameters (as fpd_create). */
int fpd_workspace_bytes(const fpd_params *p, uint64_t *bytes);

/* As fpd_create, with the state placed in caller-owned device memory
 * `workspace` of workspace_bytes bytes (at least fpd_workspace_bytes, at a
 * 256-byte aligned address; e.g. the data of a torch tensor), which the
 * caller keeps valid until fpd_destroy and frees afterwards: the library
 * never frees it.  Buffers for reads (fpd_read_*, fpd_internal_flow) and
 * host staging are still allocated by the library on first use.  The paper
 * has no counterpart: this serves applications that own device memory.
 * FPD_EINVAL for a NULL or short or misaligned workspace. */
int fpd_create_ex(const fpd_params *p, void *stream, void *workspace, uint64_t workspace_bytes, fpd_sim **out);

/* Enqueue n_steps >= 0 time steps (Sec. 2.3 items (1)-(3)).  Asynchronous:
 * returns launch errors only.  Whole chunks of 32 steps (after the first
 * step) replay CUDA graphs, captured on first use. */
int fpd_step(fpd_sim *s, int64_t n_steps);

/* Capture now, and upload to the device, the step graphs that the next
 * fpd_step(s, n_steps) will replay (starting from the current step count),
 * so that that call only enqueues them; calls that find the graphs already
 * captured, or that use none (n_steps < 32, profiling on, graphs disabled),
 * do nothing.  Runs no kernel.  The paper has no counterpart: this serves callers
 * that time or bound the latency of fpd_step.  Graphs are dropped by
 * fpd_set_tuning and fpd_export_beads. */
int fpd_prepare(fpd_sim *s, int64_t n_steps);

/* Block until all work of s has finished; report device-side errors:
 * FPD_ECUDA for a failed launch or kernel, FPD_ENAN once FPD_FLAG_NONFINITE
 * is set (see fpd_flags). */
int fpd_sync(fpd_sim *s);

/* Sticky status bits of an instance, set on the device while it runs and
 * kept until fpd_load replaces its state.  The paper has no counterpart:
 * they guard the method's assumptions and report divergence.
 *   FPD_FLAG_FAST_BEAD: a bead velocity component reached 0.5 cells per
 *     step (Eq. 5 gave |V_x| or |V_y| >= 0.5), far outside the low-Mach
 *     range of the lattice Boltzmann fluid (c_s = 0.577).  The sweep's early
 *     update of tiles no bead marked assumes beads move less than a cell per
 *     step; from the step after the flag is set every tile of the instance
 *     waits for its bead phase instead, so results stay those of the
 *     waiting path.
 *   FPD_FLAG_NONFINITE: a non-finite bead velocity, or a non-finite
 *     population found by the watchdog, a pass over the populations that
 *     runs whenever the step count crosses a multiple of 1024.  fpd_sync and
 *     the calls that synchronise then return FPD_ENAN.
 *   FPD_FLAG_COPY_TIMEOUT: a CTA of the staged sweep (tuning variants 3
 *     and 4) waited 0.1 s for the bulk copy of its block into shared memory
 *     without seeing it complete, and left that block's cells unwritten for
 *     the step; fpd_sync and the calls that synchronise then return
 *     FPD_ECUDA. */
#define FPD_FLAG_FAST_BEAD 1u
#define FPD_FLAG_NONFINITE 2u
#define FPD_FLAG_COPY_TIMEOUT 4u

/* Synchronise and copy the status bits of s into *flags (no error for a
 * set bit).  FPD_EINVAL for a NULL argument. */
int fpd_flags(fpd_sim *s, uint32_t *flags);

/* Copy the macroscopic fields to caller-owned host arrays of ny*nx doubles
 * (row-major [j][i], cell centre (i + 1/2, j + 1/2)): velocity
 * u = (sum_k f_k c_k + f/2) / rho with f the force density of Eq. 4 for the
 * current bead table (the one used by the last collision; the velocity that
 * Eq. 5 averages), and rho = sum_k f_k.
 * Any pointer may be NULL.  Synchronises. */
int fpd_read_fields(fpd_sim *s, double *ux, double *uy, double *rho);

/* Copy the bead table to caller-owned host arrays of n_fibers*n_beads
 * entries (fiber-major): positions and velocities (x, y pairs) of the last
 * advance (V of Eq. 5; V = 0 before the first), forces F_i (Eqs. 11-12 +
 * excluded volume, x, y pairs) and support integrals S_i = sum_x phi_i,
 * the lattice form of the integral of phi_i in Eqs. 4-5 (one double
 * each).  Positions are unwrapped in x.  Any pointer may be NULL.
 * Synchronises. */
int fpd_read_beads(fpd_sim *s, double *pos, double *vel, double *force, double *support);

/* Stream-ordered bead read for callers that keep the device busy while they
 * consume results: enqueue, after the steps queued so far, a copy of the
 * current bead table (the table fpd_read_beads would read after those steps)
 * into the caller-owned host array dst of 7 * n_fibers * n_beads doubles --
 * the arrays R_x, R_y, V_x, V_y, F_x, F_y, S one after another, each in bead
 * order -- and return without waiting.  Steps queued afterwards run while
 * the copy is in flight.  dst holds the values once fpd_wait_read(s, *ticket)
 * has returned FPD_OK and must stay valid until then; page-locked (pinned)
 * host memory keeps the copy asynchronous, pageable memory may make this call
 * block.  FPD_EINVAL for a NULL dst or ticket. */
int fpd_read_beads_async(fpd_sim *s, double *dst, uint64_t *ticket);

/* Block until the read with this ticket, and every read before it, has
 * completed; report device-side errors.  FPD_EINVAL for a ticket this handle
 * has not issued. */
int fpd_wait_read(fpd_sim *s, uint64_t ticket);

/* Per-step bead export, for callers that take every step's beads while the
 * steps keep running: from the next step on, the bead phase of each step
 * also writes its finished table into a ring of `slots` (>= 2) entries of
 * page-locked host memory owned by the handle, from the device itself, so
 * that no copy is queued between the kernels of the step chain.
 * fpd_take_beads then hands over the table after a given step.  slots = 0
 * turns the export off.  Synchronises and drops captured step graphs.
 * FPD_EINVAL for slots < 0 or slots == 1; FPD_ENOMEM if the ring cannot be
 * allocated. */
int fpd_export_beads(fpd_sim *s, int32_t slots);

/* Copy the bead table after n completed steps (the layout of
 * fpd_read_beads_async: R_x, R_y, V_x, V_y, F_x, F_y, S, 7 * n_fibers *
 * n_beads doubles) from the export ring to dst, waiting until the device has
 * written it.  n counts the steps since fpd_create; the first exported n is
 * the step count at fpd_export_beads plus one (two if that count was 0: the
 * first step has no bead phase).  FPD_EBUSY if the ring has already reused
 * that entry (the caller fell `slots` or more steps behind); FPD_EINVAL if
 * export is off, n was not exported or not enqueued yet; FPD_ETIMEOUT if the
 * entry has not arrived within 60 s while the stream is still busy. */
int fpd_take_beads(fpd_sim *s, int64_t n, double *dst);

/* Copy the populations f_k (not the stored deviations) of the current time
 * into a caller-owned host array of 9*ny*nx doubles, layout [k][j][i] with
 * the velocity order (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1)
 * (1,-1).  Synchronises. */
int fpd_read_populations(fpd_sim *s, double *f);

/* Replace the populations of the current time by a caller-owned host array
 * of 9*ny*nx doubles (same layout as fpd_read_populations); stored at the
 * handle's precision.  The bead table is unchanged.  Synchronises. */
int fpd_write_populations(fpd_sim *s, const double *f);

/* out[0] = total mass sum f, out[1..2] = momentum sum f c (without the half
 * force), out[3] = completed steps.  FP64 reduction on the device.  Returns
 * FPD_ENAN if the state holds a non-finite value.  Synchronises. */
int fpd_diag(fpd_sim *s, double out[4]);

/* Checkpoint / resume (the paper has no counterpart: long runs, Sec. 4,
 * survive restarts).  fpd_save writes the whole device state of the handle
 * to the file `path` (created or truncated): the stored populations in their
 * storage precision, both bead tables, the tile masks, the step count and
 * the derived per-instance constants, behind a header with a format tag and
 * the ABI version.  fpd_load reads such a file into a handle created with
 * the same parameters (same lattice, precision, beads and derived
 * constants; the stream may differ) and replaces its state: the run then
 * continues exactly as the saved one would have, bit for bit.  Both
 * synchronise.  FPD_EINVAL for a NULL argument, a file that cannot be
 * opened, read or written, a file that is not a checkpoint of this format
 * or ABI version, or one written with other parameters (the handle is then
 * unchanged). */
int fpd_save(fpd_sim *s, const char *path);
int fpd_load(fpd_sim *s, const char *path);

/* Same result as fpd_diag, computed without allocating any device memory.
 * The paper has no counterpart: this is a library service.  fpd_diag keeps
 * its per-block partial sums in a buffer it allocates (cudaMalloc) on first
 * use; callers that must not allocate device memory when they run the check
 * (a serving loop whose device memory is all committed to resident
 * instances, code running while other work is being captured or replayed on
 * the device, an application whose own allocator owns device memory) call
 * this instead.  Its scratch is a fixed device array of 4 * 1024 + 4 doubles
 * (32 800 bytes) that every device loading the library holds until exit;
 * the reduction uses at most 1024 blocks, so any lattice size is accepted
 * (a larger block count would be refused with FPD_EINVAL).  The first call
 * on each device looks up that array's device address (cudaGetSymbolAddress
 * with the handle's device current); make that first call before any
 * stream capture.  All calls share the array and every call overwrites what
 * it reads, so nothing needs clearing; calls whose device work overlaps
 * (other streams, handles or threads on the same device) race on the array
 * and must not overlap.  Returns FPD_ENAN like fpd_diag.  Synchronises. */
int fpd_diag_noalloc(fpd_sim *s, double out[4]);

/* Residual flow inside each bead (Sec. 3.2): eps[i] = sum_x phi_i (v - V_i)^2
 * / sum_x phi_i over the bead's support at its current position, v the
 * velocity of fpd_read_fields and V_i the bead's latest velocity.  eps:
 * caller-owned host array of n_beads * n_fibers doubles.  Evaluated in FP64
 * from the stored populations whatever the storage precision.  FPD_EINVAL
 * for a NULL pointer; synchronises. */
int fpd_internal_flow(fpd_sim *s, double *eps);

/* Kernel tuning (same arithmetic, same results up to rounding: the
 * compiler may contract multiply-adds differently in each variant):
 * variant 0 runs the lattice sweep with one cell per thread (32 x 8 threads
 * per 32 x 8 tile), variant 1 with two cells per thread along x, adjacent
 * (FP32, FP16 storage; paired accesses) or 16 cells apart (FP64) (16 x 8
 * threads), variant 2 with 2 (FP64) or 4 (FP32, FP16 storage) consecutive
 * cells per thread along x, each plane moved with one 16-byte (8-byte for
 * FP16) access; variant 2 needs nx to be a multiple of that width, and an
 * instance whose nx is not runs variant 0 instead.  Variants 3 and 4 run
 * variant 1's threads on blocks of 2 or 4 (FP32 storage) or 4 or 8 (FP16
 * storage) tiles stacked in y, whose populations one bulk copy per block
 * stages in shared memory; FP64 storage and batches run variant 1 for
 * them.  Chosen per workload by
 * an autotuner that times them.  fpd_set_tuning synchronises and drops
 * captured step graphs; FPD_EINVAL for an unknown variant.  fpd_get_tuning:
 * current variant and count. */
int fpd_set_tuning(fpd_sim *s, int32_t variant);
int fpd_get_tuning(const fpd_sim *s, int32_t *variant, int32_t *n_variants);
/* Number of sweep variants (host only: needs no device or handle).  The
 * paper has no counterpart: launch shapes are an implementation choice. */
int32_t fpd_sweep_variants(void);

/* Derived parameters: out[0] nu_f, [1] k_s, [2] k_b, [3] k_ev, [4] l_0,
 * [5] support radius a + phi_cut xi, [6] gamma_dot, [7] stored bytes per
 * cell update (2 x 9 x storage size). */
int fpd_derived(const fpd_sim *s, double out[8]);

/* Kernel timing (CUDA events around every launch on the handle's stream).
 * on = 1 starts recording and clears the totals; 0 stops. */
int fpd_set_profiling(fpd_sim *s, int on);

/* Profiling totals: out[0] lattice-kernel milliseconds, out[1] lattice
 * launches, out[2] bead-kernel milliseconds, out[3] bead launches.
 * Synchronises. */
int fpd_kernel_times(fpd_sim *s, double out[4]);

/* ------------------------------------------------------------------------
 * Batched instances.  Many independent instances (points of a confinement /
 * Reynolds-number / stiffness sweep, or serving requests) of possibly
 * different lattice sizes share one device pool and advance together: each
 * time step is one bead-phase launch over the beads of all active instances
 * and one lattice sweep over a packed list of all their tiles.  Instances
 * never interact, and an instance computes the same numbers alone or in a
 * batch (the same kernels, per-instance reductions in a fixed order).
 * ------------------------------------------------------------------------ */
typedef struct fpd_batch fpd_batch;

/* Create an empty batch: every instance uses `precision`; at most
 * max_slots instances at a time; a device pool of pool_bytes for their
 * populations and room for max_beads beads in total.  stream: cudaStream_t
 * or NULL.  Errors: FPD_EINVAL, FPD_ENOMEM, FPD_ECUDA. */
int fpd_batch_create(int32_t precision, int32_t max_slots, int64_t pool_bytes, int32_t max_beads, void *stream,
                     fpd_batch **out);

/* Admit an instance (same parameters and placement rules as fpd_create)
 * that is to run n_steps time steps; *slot receives its slot index.  It
 * starts at its own step 0 on the next fpd_batch_run.  FPD_EBUSY when no slot
 * or no contiguous pool / bead room is free; FPD_EINVAL for bad parameters
 * or a precision other than the batch's. */
int fpd_batch_add(fpd_batch *b, const fpd_params *p, int64_t n_steps, int32_t *slot);

/* Advance every active instance by the same number of steps: max_steps, or
 * fewer so that no instance passes its requested count (*steps_done gets
 * the count).  Instances that reach their count become finished.  Enqueues
 * the work asynchronously (the call may synchronise after admissions). */
int fpd_batch_run(fpd_batch *b, int64_t max_steps, int64_t *steps_done);

/* Lattice sweep variant of the batch (as fpd_set_tuning; under variant 2
 * an instance whose nx is not a multiple of the vector width runs its tiles
 * with that many cells per thread along y instead). */
int fpd_batch_set_tuning(fpd_batch *b, int32_t variant);

/* Block until the batch's work has finished. */
int fpd_batch_sync(fpd_batch *b);

/* Synchronise, then list up to `capacity` instances that finished or
 * failed and were not listed before (done_slots may be NULL to only count
 * them).  An instance whose status has FPD_FLAG_NONFINITE set (a non-finite
 * bead velocity, or a non-finite population found by the watchdog pass that
 * every fpd_batch_run ends with and that also runs each time the global
 * step count crosses a multiple of 1024) is stopped and listed as failed
 * (state 3 in fpd_batch_slot_info); the other instances run on unchanged. */
int fpd_batch_poll(fpd_batch *b, int32_t *done_slots, int32_t capacity, int32_t *n_done);

/* out = {nx, ny, beads, steps done, steps requested, state (0 free,
 * 1 running, 2 finished, 3 failed: non-finite state)}. */
int fpd_batch_slot_info(fpd_batch *b, int32_t slot, int64_t out[6]);

/* As fpd_flags for one slot (running, finished or failed). */
int fpd_batch_slot_flags(fpd_batch *b, int32_t slot, uint32_t *flags);

/* As fpd_read_fields / fpd_read_beads / fpd_read_populations for one slot
 * (running or finished).  Synchronise. */
int fpd_batch_read_fields(fpd_batch *b, int32_t slot, double *ux, double *uy, double *rho);
int fpd_batch_read_beads(fpd_batch *b, int32_t slot, double *pos, double *vel, double *force, double *support);

/* Advance every active instance by up to n steps (n >= 0): fpd_batch_run
 * repeated until n steps are done or no instance is active any more (a run
 * stops where an instance reaches its requested count, which then finishes).
 * Each step is the coupled step of Sec. 2.3 for every instance; the batch as
 * a whole is the sweep over independent problems of Sec. 4 (Fig. 10).
 * FPD_EINVAL for n < 0; launch errors as fpd_batch_run. */
int fpd_batch_step(fpd_batch *b, int64_t n);

/* Velocity field (ux, uy: ny*nx doubles, row-major, as fpd_read_fields:
 * the velocity of Eq. 5) and bead positions (pos: n_fibers*n_beads x, y
 * pairs, unwrapped in x) of one slot, running or finished, into
 * caller-owned host arrays; any pointer may be NULL.  Synchronises.
 * FPD_EINVAL for a slot that holds no instance. */
int fpd_batch_read(fpd_batch *b, int32_t slot, double *ux, double *uy, double *pos);
int fpd_batch_read_populations(fpd_batch *b, int32_t slot, double *f);
/* As fpd_internal_flow for one slot (running or finished).  Synchronises. */
int fpd_batch_internal_flow(fpd_batch *b, int32_t slot, double *eps);

/* Release a slot and its pool and bead room. */
int fpd_batch_remove(fpd_batch *b, int32_t slot);

/* out = {running instances, their cells, finished instances, pool bytes in
 * use, pool bytes, global steps, cell updates done, beads in use}. */
int fpd_batch_stats(fpd_batch *b, double out[8]);

/* Text of the batch's last error; never NULL. */
const char *fpd_batch_last_error(const fpd_batch *b);

/* Free the batch (NULL-safe).  Synchronises. */
int fpd_batch_destroy(fpd_batch *b);

/* Text of the last error on s (or of fpd_create in this thread if s is
 * NULL); never NULL; valid until the next call on s. */
const char *fpd_last_error(const fpd_sim *s);

/* Free all device memory of s.  NULL-safe.  Synchronises. */
int fpd_destroy(fpd_sim *s);

#ifdef __cplusplus
}
#endif
#endif /* FPD_H */
