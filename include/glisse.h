/*
 * glisse.h -- C ABI of the GB300 (sm_103a) implementation of the GLISSE
 * test-particle map (Zhang & Gladman, "GLISSE: A GPU-optimized planetary
 * system integrator", arXiv 2011.03484).
 *
 * The library advances N massless test particles through the mixed-variable
 * symplectic (Wisdom-Holman) map of section 2.2 under a central star and
 * N_p <= GLISSE_MAX_PLANETS planets, removing particles on close encounter
 * or escape.  All arithmetic is IEEE binary64 on the GPU.  Units are AU, yr
 * and M_sun with G = 4 pi^2.
 *
 * Conventions
 *   - Every function returns GLISSE_OK (0) or a negative GLISSE_E_* code;
 *     glisse_strerror() names it.  After a GLISSE_E_CUDA error the context
 *     should be destroyed.
 *   - Host buffers are owned by the caller; the library copies them during
 *     the call and keeps no pointer to them.  Device buffers passed to the
 *     *_device functions are owned by the caller and must stay valid until
 *     the call returns (the calls synchronise their stream before returning).
 *   - A context belongs to the CUDA device that was current at
 *     glisse_create() and to the stream given in its options (or a stream
 *     the library creates).  Contexts are not thread-safe; distinct contexts
 *     may be used from distinct threads.
 *   - Particle ids are input indices 0..n-1; outputs are indexed by id.
 */
#ifndef GLISSE_H
#define GLISSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GLISSE_MAX_PLANETS 8

/* status codes */
#define GLISSE_OK 0
#define GLISSE_E_INVAL -1   /* bad argument (NULL, size, order, non-finite, unbound planet) */
#define GLISSE_E_NOMEM -2   /* device or host allocation failed */
#define GLISSE_E_CUDA -3    /* a CUDA call failed (no device, launch error, ...) */
#define GLISSE_E_KEPLER -4  /* a planet's Kepler solve did not converge */
#define GLISSE_E_TIMEOUT -5 /* a bounded wait on the device gave up (glisse_advance: a particle task waited seconds for the task before it) */
#define GLISSE_E_STATE -6   /* call not valid in the context's current state */

/* removal reasons reported by glisse_read() */
#define GLISSE_ALIVE 0
/* 1..N_p: close encounter with planet j (1-based, in input order) */
#define GLISSE_REMOVED_ESCAPE -1
#define GLISSE_REMOVED_KEPLER -2
#define GLISSE_REMOVED_NONFINITE -3

/* Kepler solver modes */
#define GLISSE_KEPLER_CONVERGE 0    /* iterate to convergence (default) */
#define GLISSE_KEPLER_PAPER_FIXED 1 /* fixed iteration count, deactivate if not converged (section 2.2) */
/* PAPER_FIXED: kepler_iters Newton steps on Kepler's equation in the eccentric
 * anomaly, started at x0 = dM / (1 - e cos E0); a particle whose last step
 * exceeds GLISSE_PAPER_KEPLER_TOL (the 1e-14 convergence section 2.2 quotes)
 * is removed with GLISSE_REMOVED_KEPLER, keeping its state from before the
 * drift.  Unbound or nearly radial orbits (r alpha < 1e-3), which the paper
 * does not treat, use the converged universal-variable solve.  Only
 * glisse_create accepts it (and GLISSE_SORT_COST); the batched and
 * differentiable entry points return GLISSE_E_INVAL for either. */
#define GLISSE_PAPER_KEPLER_TOL 1e-14
#define GLISSE_MAX_KEPLER_ITERS 64

/* encounter criterion (section 2.2, close-encounter paragraph) */
#define GLISSE_ENC_HILL 0  /* R_crit,j = enc_value * a_j (m_j / 3 m0)^(1/3) */
#define GLISSE_ENC_FIXED 1 /* R_crit,j = enc_value (AU) for every planet */

/* particle order (section 2.2 suggests sorting particles by the expected work
 * of their Kepler solve so that the threads of a block do similar work, the
 * costliest group first).  GLISSE_SORT_COST orders the live particles at every
 * compaction (and before the first step) by the tier of their pericentre
 * value of z = beta s^2 ~ (n dt / (1 - e))^2, which sets the fast path's
 * polynomial degree (tiers <= 2^-9, <= 2^-5, <= 0.1, beyond / unbound: the
 * general solver), costliest tier first, stable within a tier.  Results per
 * particle change only by rounding (a warp's polynomial degree depends on its
 * members). */
#define GLISSE_SORT_NONE 0
#define GLISSE_SORT_COST 1

/* launch shape of the particle map (results are bit-identical in every shape).
 * PLAIN: one thread per particle slot, one launch per segment.  TASKS: a
 * persistent grid of a few warps per SM partition that take (32-slot group,
 * 32-step sub-chunk) tasks in order from a device counter, so every partition
 * keeps the same number of busy warps to the end of the segment; a task waits
 * (bounded: GLISSE_E_TIMEOUT after seconds) for its group's previous
 * sub-chunk.  AUTO picks TASKS when the live groups outnumber the resident
 * warps (two to four per partition) by half again, PLAIN otherwise.  The
 * fixed-iteration Kepler mode always uses PLAIN. */
#define GLISSE_LAUNCH_AUTO 0
#define GLISSE_LAUNCH_PLAIN 1
#define GLISSE_LAUNCH_TASKS 2

/* element frames for glisse_set_sampling */
#define GLISSE_FRAME_HELIO 0 /* heliocentric; mu = G m0 (particles), G (m0 + m_j) (planet j) */
#define GLISSE_FRAME_BARY 1  /* barycentre of star and planets; mu = G (m0 + sum m_j) for every body */

typedef struct glisse_ctx glisse_ctx; /* opaque; owned by the library */

typedef struct {
    int32_t chunk_steps;   /* steps per planet chunk C (section 2.2), default 1024 */
    int32_t resync_chunks; /* compact live particles every R chunks (section 2.2), default 1 */
    int32_t kepler_mode;   /* GLISSE_KEPLER_*, default CONVERGE */
    int32_t kepler_iters;  /* iterations for PAPER_FIXED (1..GLISSE_MAX_KEPLER_ITERS), default 5 (section 2.2) */
    int32_t enc_mode;      /* GLISSE_ENC_*, default HILL */
    int32_t timing;        /* non-zero: time every launch with CUDA events (see glisse_timings) */
    int32_t sort_mode;     /* GLISSE_SORT_*, default NONE */
    int32_t launch_mode;   /* GLISSE_LAUNCH_*, default AUTO (a performance choice: not saved in checkpoints) */
    double enc_value;      /* Hill multiple k (default 1.0) or fixed distance in AU */
    double r_max;          /* escape radius in AU, default 1000; <= 0 disables the escape test */
    void* cuda_stream;     /* cudaStream_t to run on; NULL = the library creates one */
} glisse_opts;

/* Fill *opts with the defaults listed above. */
void glisse_opts_default(glisse_opts* opts);

/*
 * Create a context and copy the initial conditions to the device.
 *   star_mass  : m0 in M_sun (> 0)
 *   planets    : host [n_planets][7] = m, x, y, z, vx, vy, vz (heliocentric),
 *                ordered by increasing initial osculating semi-major axis
 *                (Jacobi indexing, section 2.2); 0 <= n_planets <= GLISSE_MAX_PLANETS
 *   particles  : host [n_particles][6] = x, y, z, vx, vy, vz (heliocentric); may be
 *                NULL when n_particles == 0
 *   dt         : step in yr (non-zero, finite; negative integrates backwards)
 *   opts       : NULL for defaults
 * The removal test at t_0 (section 2.2: particles already inside R_crit or
 * beyond r_max) is applied by the first glisse_advance() call.
 * Errors: INVAL (sizes, ordering, non-finite planets, unbound planet), NOMEM, CUDA.
 */
int glisse_create(glisse_ctx** out, double star_mass, const double* planets, int32_t n_planets,
                  const double* particles, int64_t n_particles, double dt, const glisse_opts* opts);

/*
 * Advance every live particle by n_steps steps of kick(dt/2) - Kepler drift(dt) -
 * kick(dt/2) (section 2.2), integrating the planets on the GPU one chunk ahead.
 * Returns after the work has finished on the context's stream.  In the first
 * chunk the host launches the particles' segments as the planet kernel (started
 * by glisse_create) reports its progress through host-mapped memory; if that
 * progress does not come within 0.5 s (the GPU busy with other work), the rest
 * of the chunk waits for the whole planet chunk instead.  A call longer than a
 * few chunks lets the planets run ahead of the particles up to its last chunk:
 * the planet-log buffers then grow (once, kept until glisse_destroy) to up to
 * 512 MB, (C + 1) x (4 (N_p + 1) + 6 N_p) doubles per chunk held.
 * Splitting a run into calls changes nothing: advance(a) then advance(b) gives
 * bit for bit what advance(a + b) gives.  Between calls the device keeps each
 * live particle's velocity with the next step's opening half kick already
 * applied (as an uncut run has it there), and every call ends by computing the
 * synchronised state that glisse_read returns.  Live particles are compacted
 * (section 2.2's resync) at chunk boundaries only, every resync_chunks chunks,
 * so at the same steps however the run is split.
 * Errors: INVAL (n_steps < 0), STATE (external ephemeris too short), KEPLER, CUDA.
 */
int glisse_advance(glisse_ctx* ctx, int64_t n_steps);

/*
 * Copy results to host buffers indexed by particle id (any pointer may be NULL):
 *   state        : [n][6] x, y, z, vx, vy, vz.  Live particles: synchronised state at
 *                  the current time.  Removed particles: the state at removal
 *                  (after the drift, before the closing half kick).
 *   alive        : [n] 1 = live, 0 = removed
 *   removal_step : [n] step index of removal, -1 while live
 *   removal_reason: [n] GLISSE_ALIVE, planet 1..N_p, or GLISSE_REMOVED_*
 */
int glisse_read(glisse_ctx* ctx, double* state, uint8_t* alive, int64_t* removal_step, int32_t* removal_reason);

/* Number of live particles, current step index and time (t = step * dt); pointers may be NULL. */
int glisse_status(glisse_ctx* ctx, int64_t* n_live, int64_t* step, double* t);

/*
 * Planets at the particles' current time: host [n_planets][7] m, x, y, z, vx, vy, vz
 * (heliocentric).  *t receives the time (may be NULL).
 * Errors: STATE while an external ephemeris (below) is installed.
 */
int glisse_read_planets(glisse_ctx* ctx, double* planets, double* t);

/*
 * Test hook (section 2.2 notes any source of planet positions will do, e.g.
 * interpolation from a history file): install planet positions for the next
 * n_steps steps instead of the built-in integrator.
 *   log : host [n_steps+1][n_planets][3] heliocentric positions at t_k .. t_{k+n}
 *         where t_k is the current time.
 * The common term h0 = -sum_j G m_j r_j / |r_j|^3 is computed from these positions.
 * After these steps are consumed, glisse_advance() returns STATE until another
 * log is installed; the built-in planets are no longer valid for this context.
 * Installed after some steps have run, the positions at t_k take part from the
 * next step on: the kick at t_k was applied, with the positions then in force,
 * when the previous call ended.
 * Returns STATE while element sampling is set (glisse_set_sampling).
 */
int glisse_set_ephemeris(glisse_ctx* ctx, const double* log, int64_t n_steps);

/* Device time spent per stage since glisse_create (or the last reset), collected
 * when opts.timing != 0 from CUDA events recorded on the stream each kernel runs
 * on.  particle_steps is the exact number of steps the live particles advanced
 * (a removed particle counts the steps up to its removal). */
typedef struct {
    double particle_ms;        /* particle-map kernel */
    int64_t particle_launches;
    int64_t particle_steps;
    double ephemeris_ms;       /* planet kernel (side stream, overlaps the particles) */
    int64_t ephemeris_launches;
    double compact_ms;         /* stable partition (three kernels) */
    int64_t compact_launches;
} glisse_timing;

/* Copy the counters to *out (may be NULL) and zero them when reset != 0.
 * Errors: STATE when the context was created without opts.timing. */
int glisse_timings(glisse_ctx* ctx, glisse_timing* out, int32_t reset);

/*
 * Checkpoint and resume.  The paper continues runs from their output states
 * (sections 4.2.2 and 4.3.2: the librating particles integrated for another
 * 1 Myr from the states a 4 Gyr run left).  A checkpoint holds everything the
 * map needs to go on exactly as the context would have: the star, dt and the
 * map options, the planet constants
 * (masses, encounter radii fixed at create), the planets' Jacobi state at the
 * start of the current planet chunk (the chunk is recomputed on resume, bit
 * for bit), the step counter, and the particle arrays as laid out on the device
 * (so warps keep their members), with every removed particle's frozen state,
 * step and reason, and, when element sampling is set, its settings, the kept
 * samples and the libration flags and counts.  A context resumed from it and
 * advanced gives results identical to the original context advanced by the
 * same calls.
 *
 * glisse_checkpoint_size: *bytes receives the size of a checkpoint of ctx now.
 * glisse_checkpoint: write it to the caller's host buffer `buf` of `bytes`
 *   bytes (at least the size above).  Synchronises the context's streams.
 * glisse_resume: create a context from a checkpoint (host buffer, not kept).
 *   opts may be NULL; only its cuda_stream and timing fields are used (every
 *   option that shapes the map comes from the checkpoint).  Runs on the
 *   current device.
 * The buffer is plain bytes in the byte order of the machine that wrote it
 * (little-endian on every supported host).
 * Errors: INVAL (NULL pointers, a buffer too small, or not a checkpoint of this
 *   format: wrong magic, version or inconsistent sizes), STATE (an external
 *   ephemeris installed: it is not saved), NOMEM, CUDA.
 */
int glisse_checkpoint_size(glisse_ctx* ctx, int64_t* bytes);
int glisse_checkpoint(glisse_ctx* ctx, void* buf, int64_t bytes);
int glisse_resume(glisse_ctx** out, const void* buf, int64_t bytes, const glisse_opts* opts);

/* Sizes fixed at create (or resume): particles (all ids, live or not) and
 * planets; pointers may be NULL. */
int glisse_sizes(glisse_ctx* ctx, int64_t* n_particles, int32_t* n_planets);

/* Release all device and host resources of the context (NULL is ignored). */
void glisse_destroy(glisse_ctx* ctx);

/* Static string naming a status code. */
const char* glisse_strerror(int code);

/*
 * Device-level stable partition of live particles (section 2.2 moves
 * deactivated particles to the end of the arrays with an order-preserving
 * partition, so live ones keep their relative order).  All pointers are device pointers:
 *   alive   : [n] uint8, non-zero = keep
 *   src     : [6][ld] doubles (x, y, z, vx, vy, vz planes, leading dimension ld >= n)
 *   src_id  : [n] int32
 *   dst     : [6][ld] doubles, dst_id: [n] int32 (must not overlap src)
 *   n_out   : [1] int64 (device) receives the number of kept entries
 * Kept entries appear in dst in their original relative order.  Scratch memory
 * is allocated and freed by the call.  Runs on `stream` (cudaStream_t, NULL =
 * legacy default stream) and synchronises it before returning.
 * Errors: INVAL, NOMEM, CUDA.
 */
int glisse_partition_device(int64_t n, int64_t ld, const uint8_t* alive, const double* src, const int32_t* src_id,
                            double* dst, int32_t* dst_id, int64_t* n_out, void* stream);

/*
 * Same stable partition as glisse_partition_device, for callers that must not
 * allocate device memory (for example under a framework or pool allocator that
 * owns all device memory, with a memory budget fixed at start-up, or in a loop
 * that cannot afford an allocation's synchronisation or its failure).
 * The paper has no counterpart; this is a property of this library only.
 *   - Makes no cudaMalloc / cudaFree or allocating library call.  Its
 *     scratch is a fixed array of GLISSE_PARTITION_NOALLOC_MAX / 2048 int64
 *     (256 KiB) inside the library's device image.  The array is placed in a
 *     device's memory when the CUDA driver loads the library's module there.
 *     Under lazy module loading (CUDA's default) that may happen during the
 *     first call on the device, so the first call may allocate through the
 *     driver; every later call on that device allocates nothing.  A call with
 *     n = 0 does this set-up and nothing else.  The array then stays until
 *     the process exits or the device's context is destroyed.
 *   - n above GLISSE_PARTITION_NOALLOC_MAX returns GLISSE_E_INVAL.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress,
 *     with the caller's device current); the first call on each device also
 *     sets the module up as above, so make that first call before any stream
 *     capture.
 *   - All calls on a device share the one array (its contents are left over
 *     from the previous call and are never assumed to be zero).  Calls whose
 *     GPU work overlaps -- e.g. from two host threads on two streams -- race on
 *     it and give wrong results; serialise them.  Each call synchronises its
 *     stream before returning.
 * Arguments, results and errors are those of glisse_partition_device.
 */
#define GLISSE_PARTITION_NOALLOC_MAX 67108864
int glisse_partition_device_noalloc(int64_t n, int64_t ld, const uint8_t* alive, const double* src,
                                    const int32_t* src_id, double* dst, int32_t* dst_id, int64_t* n_out,
                                    void* stream);

/* Test hook: evaluate one of the device arithmetic helpers elementwise,
 * out[i] = fn(a[i], b[i]) for device arrays of n doubles (b may be NULL:
 * 1.0).  The helpers stand in for library division and square root on the
 * hot path, so the tests check each against exact arithmetic:
 *   RSQRT  a^(-1/2) (MUFU seed, one correction);  RCP  1/a (same);
 *   RCP40  1/a to about 2^-40;  KRCUBE  b a^(-3/2) (integer seed powers);
 *   FLOAT_SQUARE / FLOAT_CUBE  s^2 / s^3 of s = (float)a (integer products);
 *   D2F  a truncated to float by bit operations.
 * Not part of the method (the paper has no counterpart).  Synchronises the
 * stream.  Errors: INVAL, CUDA. */
#define GLISSE_MATH_RSQRT 0
#define GLISSE_MATH_RCP 1
#define GLISSE_MATH_RCP40 2
#define GLISSE_MATH_KRCUBE 3
#define GLISSE_MATH_FLOAT_SQUARE 4
#define GLISSE_MATH_FLOAT_CUBE 5
#define GLISSE_MATH_D2F 6
int glisse_selftest_math(int32_t fn, const double* a, const double* b, double* out, int64_t n, void* stream);

/* Test hook: make one task launch's bounded wait run out.  The task launches
 * of glisse_advance (which = PARTICLE_TASKS), of the differentiable forward
 * pass (DIFF_FORWARD) and of the reverse sweep (DIFF_BACKWARD) order a
 * particle group's sub-chunks with a device-side wait on the group's counter,
 * limited to seconds of polling.  Here the same kernel runs on two groups of
 * 32 slots whose first sub-chunks no task runs, with the limit set to `polls`
 * polls (>= 1, each ~64 ns or more): every wait gives up, the kernel writes
 * GLISSE_E_TIMEOUT to its status word and returns without touching particle
 * data.  *status receives that word (GLISSE_E_TIMEOUT expected, 0 if no wait
 * gave up).  Allocates and frees a few bytes of device memory; synchronises
 * the stream.  Not part of the method.  Errors: INVAL, CUDA. */
#define GLISSE_WAIT_PARTICLE_TASKS 0
#define GLISSE_WAIT_DIFF_FORWARD 1
#define GLISSE_WAIT_DIFF_BACKWARD 2
int glisse_selftest_wait(int32_t which, int32_t polls, int32_t* status, void* stream);

/*
 * FP64 throughput probe: runs independent chains of fused multiply-adds on
 * every SM for about `iterations` x 8 operations per thread and reports the
 * achieved rate (FMA instructions per second per GPU) in *dfma_per_s and the
 * mean SM clock in MHz seen by the kernel in *sm_mhz (either may be NULL).
 * Used to state the FP64 roofline the particle kernel is measured against.
 */
int glisse_fp64_peak(int32_t iterations, double* dfma_per_s, double* sm_mhz);

/* ------------------------------------------------------------------------ */
/* Derivatives of the map (tangent and adjoint).                              */
/* The map of section 2.2 is differentiated with respect to the particles'   */
/* initial states (planet positions are data).  A glisse_diff object holds   */
/* the planet log of a fixed run of n_steps and the checkpoint storage; the */
/* forward pass maps initial to final states and can carry tangent vectors   */
/* (J t); the backward pass returns J^T g for a cotangent g of the final     */
/* states, recomputing each checkpoint interval from its stored state.       */
/* All state arrays are device pointers in [n][6] layout (x, y, z, vx, vy,   */
/* vz per particle); tangents are [n_tangents][n][6].                        */
/* ------------------------------------------------------------------------ */
typedef struct glisse_diff glisse_diff; /* opaque; owned by the library */

/* Planets as in glisse_create; n_particles states per forward call; the planet
 * log of n_steps steps is computed on the device here.  checkpoint_every >= 1:
 * the backward pass recomputes that many steps per segment (storage: 48 B per
 * particle per checkpoint plus 112 + 16 n_planets B per particle per step of
 * one segment).  checkpoint_every = 0 (tape mode): the forward pass records
 * every step (112 + 16 n_planets B per particle per step, e.g. 115 GB for
 * 65536 particles and 4 planets over 10^4 steps) and the backward pass does
 * not recompute; NOMEM if the device cannot hold it.
 * checkpoint_every = GLISSE_DIFF_AUTO: tape mode when its record takes at
 * most half of the device memory free at the call, else checkpoints every
 * 256 steps (glisse_diff_checkpoint_every tells which).
 * checkpoint_every = GLISSE_DIFF_TAPE_TANGENT: tape mode whose record also
 * keeps tangent 0 (184 + 16 n_planets B per particle per step), written by a
 * forward call with at least one tangent, so that glisse_diff_backward_growth
 * needs no recompute either.
 * n_steps <= INT32_MAX (the planet log is one chunk of that many steps).
 * opts: enc_mode, enc_value and r_max apply.  Errors: INVAL, NOMEM, CUDA, KEPLER. */
#define GLISSE_DIFF_AUTO (-1)
#define GLISSE_DIFF_TAPE_TANGENT (-2)
int glisse_diff_create(glisse_diff** out, double star_mass, const double* planets, int32_t n_planets,
                       int64_t n_particles, double dt, int64_t n_steps, int32_t checkpoint_every,
                       const glisse_opts* opts);

/* The checkpoint interval in effect (0: tape mode; GLISSE_DIFF_TAPE_TANGENT),
 * e.g. after GLISSE_DIFF_AUTO.
 * Errors: INVAL. */
int glisse_diff_checkpoint_every(glisse_diff* d, int32_t* checkpoint_every);

/* state0 -> state1 over n_steps (explicit half kicks; removal as in glisse_advance, a
 * removed particle's output being its frozen state).  n_tangents (0..6) tangent
 * vectors tangent0 are carried to tangent1 = J tangent0.  log_growth[i] (may be
 * NULL) receives log(|J t_0| / |t_0|) of tangent 0, a stability indicator.
 * removal_step / removal_reason (device, may be NULL) as in glisse_read.
 * Synchronises `stream` (cudaStream_t).  Errors: INVAL, CUDA. */
int glisse_diff_forward(glisse_diff* d, const double* state0, double* state1, int32_t n_tangents,
                        const double* tangent0, double* tangent1, double* log_growth, int64_t* removal_step,
                        int32_t* removal_reason, void* stream);

/* grad_state0 = J^T grad_state1 for the states of the last forward call (J of each
 * particle's own map).  Errors: STATE before any forward call, INVAL, CUDA. */
int glisse_diff_backward(glisse_diff* d, const double* grad_state1, double* grad_state0, void* stream);

/* Reverse pass for the map extended by the tangent of the last forward call's
 * tangent 0 (the growth seed t_0): one sweep back through the checkpoints gives
 *   grad_state0   = J^T grad_state1 + grad_growth * dg/dstate0 (t_0 held fixed)
 *   grad_tangent0 = grad_growth * dg/dt_0 = grad_growth * (J^T (J t_0) / |J t_0|^2 - t_0 / |t_0|^2)
 * for g = log(|J t_0| / |t_0|) (per particle).  Each kick and drift runs its
 * adjoint in dual numbers, the state carrying the tangent and the cotangent
 * (growth part, state part): the second-order term is (dM[t])^T of the step's
 * Jacobian M, by the symmetry of the map's second derivative.
 *   grad_state1   : device [n][6] or NULL (zero)
 *   grad_growth   : device [n] or NULL (zero)
 *   tangent1      : device [n][6], J t_0 as returned by that forward call
 *   grad_state0, grad_tangent0 : device [n][6] out
 * Needs checkpoints (checkpoint_every >= 1) or GLISSE_DIFF_TAPE_TANGENT, and a
 * forward call with at least one tangent.  With checkpoints, the extended
 * recompute takes 184 B per particle per step of one segment on first use;
 * with GLISSE_DIFF_TAPE_TANGENT the sweep reads the forward call's record and
 * recomputes nothing.  Errors: STATE (no such forward call, or plain tape
 * mode), INVAL, NOMEM, CUDA. */
int glisse_diff_backward_growth(glisse_diff* d, const double* grad_state1, const double* grad_growth,
                                const double* tangent1, double* grad_state0, double* grad_tangent0, void* stream);

/* Gradient of the tangent-growth indicator g = log(|J t_0| / |t_0|) with respect to
 * the initial state, the tangent seed t_0 held fixed (the part through t_0 is
 * J^T (J t_0) / |J t_0|^2 - t_0 / |t_0|^2, which glisse_diff_backward gives).
 *   state0, tangent0 : device [n][6]; grad_state0 : device [n][6] out,
 *                      grad_state0[i][c] = dg_i / d state0[i][c]
 *   log_growth       : device [n] out, g_i (may be NULL)
 * Forward mode: for each particle and each of the 6 state coordinates, the map,
 * its tangent along that coordinate and the growth tangent with its derivative
 * (the second derivative of the map contracted with t_0) run through the same
 * steps, kick merging and removals as glisse_diff_forward; about 6 forward
 * passes with two tangents, one of them in dual numbers.  Independent of any
 * forward call.  Synchronises `stream`.  Errors: INVAL, CUDA. */
int glisse_diff_growth_gradient(glisse_diff* d, const double* state0, const double* tangent0,
                                double* grad_state0, double* log_growth, void* stream);

/* Release the object (NULL is ignored). */
void glisse_diff_destroy(glisse_diff* d);

/* ------------------------------------------------------------------------ */
/* Element sampling and resonance libration (section 3: osculating elements */
/* are logged at a fixed interval, and a particle librates in the p:q       */
/* resonance with a planet when                                             */
/*     phi = p lambda - q lambda_planet - (p - q) varpi                     */
/* never comes within avoid_deg of 0, or never within avoid_deg of 180     */
/* degrees, over the samples; lambda = varpi + M, varpi = Omega + omega).   */
/* A sample is taken at every global step that is a multiple of `every`,   */
/* on the particles live at that step, by a kernel that runs between the   */
/* particle segments (glisse_advance ends a segment at each sample step).  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t every;       /* steps between samples, >= 1 */
    int32_t frame;       /* GLISSE_FRAME_HELIO or GLISSE_FRAME_BARY */
    int64_t max_samples; /* samples of elements kept on the device (0: none, flags only);
                            needs 48 B per particle per sample */
    int32_t res_planet;  /* 0-based planet of the resonance (e.g. 3 for the 4th), -1: no libration test */
    int32_t res_p;       /* p >= 1 of the p:q resonance (3 for 3:1, 5 for 5:2) */
    int32_t res_q;       /* q >= 0 */
    int32_t pad_;
    double avoid_deg;    /* window half-width in degrees, 0 < avoid_deg < 90 (10 in section 3) */
} glisse_sampling;

/* Start sampling with *s (replacing earlier settings and discarding their
 * samples and flags), or stop it with s == NULL.  Needs the internal planet
 * integration (GLISSE_E_STATE after glisse_set_ephemeris: no planet
 * velocities).  Errors: INVAL (bad field), STATE, NOMEM, CUDA. */
int glisse_set_sampling(glisse_ctx* ctx, const glisse_sampling* s);

/* Copy up to max_samples samples to host memory: elements [max_samples][n][6]
 * (a, e, i, Omega, omega, M per particle id, angles in radians; NaN rows for
 * particles not live at the sample) and sample_steps [max_samples] (global
 * step of each sample; may be NULL).  *n_samples receives the number copied.
 * Samples past the max_samples given to glisse_set_sampling are not kept.
 * Errors: INVAL, STATE (sampling not set), CUDA. */
int glisse_read_elements(glisse_ctx* ctx, double* elements, int64_t* sample_steps, int64_t max_samples,
                         int64_t* n_samples);

/* Copy the libration flags per particle id to host memory: near0[n] / near180[n]
 * = 1 if phi came within the window of 0 / 180 degrees in some sample,
 * count[n] = samples that entered the test (bound particle and planet).  A
 * particle librates when count > 0 and (near0 == 0 or near180 == 0).  Any
 * pointer may be NULL.  Errors: INVAL, STATE (no libration test set), CUDA. */
int glisse_read_libration(glisse_ctx* ctx, uint8_t* near0, uint8_t* near180, int32_t* count);

/* ------------------------------------------------------------------------ */
/* Many independent systems in one context (a batch).                        */
/* Each system has its own star, 0..GLISSE_MAX_PLANETS planets, particles    */
/* and step dt; all advance the same number of steps (each of its own dt).   */
/* The per-chunk work -- planet chunks of every system (one warp each), one  */
/* persistent particle launch that takes 32-particle tasks from a device    */
/* work counter, compaction and the task-table rebuild -- keeps every size   */
/* on the device and is replayed as a captured CUDA graph.                   */
/* ------------------------------------------------------------------------ */
typedef struct glisse_batch glisse_batch; /* opaque; owned by the library */

/*
 * Create a batch.  Host arrays, systems concatenated in order:
 *   star_mass  : [n_systems]
 *   n_planets  : [n_systems]  (0..GLISSE_MAX_PLANETS; each system's planets
 *                ordered by increasing initial semi-major axis)
 *   planets    : [sum n_planets][7] m, x, y, z, vx, vy, vz (heliocentric)
 *   n_particles: [n_systems]  (>= 0)
 *   particles  : [sum n_particles][6] heliocentric (particle id = row index)
 *   dt         : [n_systems] non-zero
 *   opts       : NULL for defaults; chunk_steps, enc_mode, enc_value, r_max,
 *                timing and cuda_stream apply to every system.
 * Errors: INVAL, NOMEM, CUDA.
 */
int glisse_batch_create(glisse_batch** out, int32_t n_systems, const double* star_mass, const int32_t* n_planets,
                        const double* planets, const int64_t* n_particles, const double* particles, const double* dt,
                        const glisse_opts* opts);

/* Advance every system by n_steps steps (section 2.2 map per system).  Errors: INVAL, KEPLER, CUDA. */
int glisse_batch_advance(glisse_batch* b, int64_t n_steps);

/* Results by particle id (rows of the create call's particle array); pointers may be NULL.
 * Same meaning as glisse_read. */
int glisse_batch_read(glisse_batch* b, double* state, uint8_t* alive, int64_t* removal_step,
                      int32_t* removal_reason);

/* Live particles over all systems and the step index (pointers may be NULL). */
int glisse_batch_status(glisse_batch* b, int64_t* n_live, int64_t* step);

/* Particle-steps advanced since creation over all systems (each particle counts
 * the steps it actually advanced; exact in every mode).  Synchronises the batch's
 * stream.  Errors: INVAL, CUDA. */
int glisse_batch_steps_done(glisse_batch* b, int64_t* steps);

/* Stage timings of the batch (opts.timing != 0), as glisse_timings. */
int glisse_batch_timings(glisse_batch* b, glisse_timing* out, int32_t reset);

/*
 * Autotuner: tries particle-kernel block sizes {64, 128, 256}, then 2 lanes per
 * particle instead of 1 at the best block size, then chunk lengths {256, 512,
 * 1024, 2048} (up to the creation chunk), on a scratch copy of the batch
 * (trial_steps steps each, <= 0 for 256), and keeps the fastest in live
 * particle-steps per second.  The batch itself does not move.  *chunk_steps,
 * *block_threads and *threads_per_particle (may be NULL) receive the choice.
 * Errors: INVAL, NOMEM, CUDA.
 */
int glisse_batch_tune(glisse_batch* b, int32_t trial_steps, int32_t* chunk_steps, int32_t* block_threads,
                      int32_t* threads_per_particle);

/*
 * Set the particle kernel's launch shape directly: block_threads in {32, 64,
 * ..., 256}, threads_per_particle 1 (one lane per particle) or 2 (a lane pair
 * per particle, each lane taking half of the planets in the kick: shorter steps
 * per particle, more FP64 work in all, for batches too small to fill the GPU).
 * Errors: INVAL.
 */
int glisse_batch_set_launch(glisse_batch* b, int32_t block_threads, int32_t threads_per_particle);

/*
 * Checkpoint and resume of a batch (the continuation runs of sections 4.2.2
 * and 4.3.2, as for glisse_checkpoint): every system's constants, dt and
 * current Jacobi planet state, the live particles per system, the particle
 * slots as laid out on the device, the per-id results, the step and the
 * removal test at t_0 still pending or not, the chunk length and the launch
 * shape.  A batch resumed from it and advanced by the same calls gives
 * results identical to the original.  glisse_batch_checkpoint writes to the
 * caller's host buffer (at least glisse_batch_checkpoint_size bytes) and
 * synchronises the batch's stream; glisse_batch_resume creates a batch on the
 * current device, taking only cuda_stream and timing from opts (may be NULL).
 * Errors: INVAL (NULL pointers, a buffer too small or not a batch checkpoint:
 * wrong magic, version or inconsistent sizes, ids or counts), NOMEM, CUDA.
 */
int glisse_batch_checkpoint_size(glisse_batch* b, int64_t* bytes);
int glisse_batch_checkpoint(glisse_batch* b, void* buf, int64_t bytes);
int glisse_batch_resume(glisse_batch** out, const void* buf, int64_t bytes, const glisse_opts* opts);

/* Sizes fixed at create (or resume): particles over all systems and systems;
 * pointers may be NULL. */
int glisse_batch_sizes(glisse_batch* b, int64_t* n_particles, int32_t* n_systems);

/* Release the batch (NULL is ignored). */
void glisse_batch_destroy(glisse_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* GLISSE_H */
