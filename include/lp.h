/*
 * lp.h - C ABI of the GB300 (sm_103a) Lagrangian-particle granular-flow step.
 *
 * The library implements, on one GPU, the per-time-step particle hot path of
 * the Lagrangian particle (LP) method with mu(I) rheology of Zepeda & Samulyak,
 * "Computational Model for Granular Flows based on the Lagrangian Particle
 * Method" (arXiv 2206.14061):
 *   neighbour search and stencils          (Sec. 3.1 items 4-6)
 *   GFD least-squares derivative fits      (Sec. 3.1 item 7)
 *   strain-rate norm and mu(I) closure     (Sec. 2.2, 2.3)
 *   stress-divergence update of V, u, x    (Sec. 3.1 items 8, 10)
 *   floor mirror particles                 (Sec. 3.1 item 9, solid boundary)
 * plus a hand-written adjoint of the step (not in the paper).
 *
 * Conventions (all entry points):
 *   - Every call returns an lp_status. LP_OK is 0.
 *   - Particle arrays are CALLER-OWNED DEVICE pointers, FP64, structure of
 *     arrays, length n, in the caller's particle order (lp_step also takes
 *     HOST arrays, see there). The library never frees them and never keeps
 *     them beyond the call.
 *   - The library owns its workspace through an opaque lp_ctx (one context
 *     per device; not thread-safe: serialise calls on one context).
 *   - Work is enqueued on the given CUDA stream (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream) and returns before it
 *     finishes, except where a call says it synchronises.
 *   - Null pointers, negative sizes and sizes beyond the context's capacity
 *     fail on the host with LP_ERR_INVALID_ARG and enqueue nothing.
 *   - Errors detected on the device (stencil overflow, non-finite values,
 *     bounded-wait timeouts) are accumulated in the context and reported by
 *     lp_ctx_sync(), which returns the first such error and clears them.
 *
 * Neighbour encoding: an entry j (0 <= j < 2^31) is particle j; j | 2^31 is
 * the floor mirror of particle j, located at (x_j, y_j, 2 floor_z - z_j).
 */
#ifndef LP_H
#define LP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lp_status;
#define LP_OK 0
#define LP_ERR_INVALID_ARG 1
#define LP_ERR_STENCIL_OVERFLOW 2
#define LP_ERR_NONFINITE 3
#define LP_ERR_TIMEOUT 4
#define LP_ERR_CUDA 5
#define LP_ERR_OOM 6
#define LP_ERR_UNIMPLEMENTED 7

/* arithmetic of the least-squares fits */
#define LP_FP64 0  /* FP64 moments, Cholesky and solve (QR fallback in FP64)   */
#define LP_MIXED 1 /* FP32 moments and Cholesky + one FP64 refinement step     */
#define LP_MIXED_FF 2 /* FP32 only on the stencil rows: offsets, moments and   */
                      /* right-hand sides accumulated as float-float (FP32     */
                      /* pairs, error-free transformations), the Gram matrix   */
                      /* factored and solved in float-float (Cholesky); the    */
                      /* derived values and the inertial closure in            */
                      /* float-float, rounded to FP64 once; FP64 for the       */
                      /* regime test, the update and the pivoted-QR fallback.  */
                      /* lp_step and lp_fit_derivatives.                       */

/* time integration (lp_params.time_scheme) */
#define LP_TIME_PAPER 0
#define LP_TIME_HEUN 1

/* floor mirror particles (Sec. 3.1 item 9) */
#define LP_MIRROR_NONE 0
#define LP_MIRROR_NOSLIP 1   /* mirror velocity -u (all components)            */
#define LP_MIRROR_FREESLIP 2 /* mirror velocity (u, v, -w): normal component flipped */

/* how lp_step issues a step */
#define LP_LAUNCH_KERNELS 0    /* one kernel per phase                               */
#define LP_LAUNCH_GRAPH 1      /* the per-phase kernels replayed as a CUDA graph     */
#define LP_LAUNCH_PERSISTENT 2 /* one cooperative persistent launch per step, phases */
                               /* separated by a bounded grid barrier               */

/* bits of lp_diag.flags */
#define LP_FLAG_OVERFLOW 0x1u  /* a stencil had more neighbours than cap       */
#define LP_FLAG_NONFINITE 0x2u /* a new state value was NaN or infinite        */
#define LP_FLAG_TIMEOUT 0x4u   /* a bounded device wait gave up                */
#define LP_FLAG_BELOW_FLOOR 0x8u /* a particle ended below the floor           */

#define LP_MAX_CAP 64 /* largest stencil capacity */

/* phases timed by lp_ctx_phase_times */
#define LP_PHASE_SORT 0      /* cell keys, scan, scatter, in-cell sort, gather   */
#define LP_PHASE_NEIGHBORS 1 /* stencil search                                   */
#define LP_PHASE_PASS1 2     /* fits of u, v, w (+ QR fallback kernel)           */
#define LP_PHASE_PASS2 3     /* fits of |gdot|, V^{n+1}; acceleration; update    */
#define LP_NPHASES 4

typedef struct lp_ctx lp_ctx;

typedef struct {
  int32_t device;        /* CUDA device ordinal the context lives on          */
  int32_t max_columns;   /* largest number of independent columns per call    */
  int64_t max_particles; /* largest n of any call on this context             */
  int32_t cap;           /* stencil capacity (1..LP_MAX_CAP) used by lp_step  */
  int32_t pad;
} lp_ctx_desc;

/* A set of particles. Columns are independent problems (their particles never
 * neighbour each other); column c holds particles
 * [column_offsets[c], column_offsets[c+1]). */
typedef struct {
  double *x, *y, *z;    /* positions (m)                                      */
  double *u, *v, *w;    /* velocity (m/s)                                      */
  double *V;            /* specific volume V = 1/phi (dimensionless)           */
  int64_t n;
  const int32_t* column_offsets; /* HOST array of ncolumns+1 ints, or NULL for one column */
  int32_t ncolumns;              /* >= 1                                        */
  int32_t pad;
} lp_particles;

/* mu(I) law (Sec. 2.2): mu(I) = mu_s + (mu_2 - mu_s)/(I0/I + 1), grain
 * diameter d (m), grain density rho_s = phi_s (kg/m^3). */
typedef struct {
  double mu_s, mu_2, I0, d, rho_s;
} lp_mui;

/* pressure law (Sec. 2.2.1): P = 0 for phi <= phi_min; Bagnold-type inertial
 * pressure for phi_min < phi <= phi_max; phi_s (alpha + beta phi) above. */
typedef struct {
  double phi_c, phi_min, phi_max, alpha, beta;
} lp_eos;

typedef struct {
  double h;           /* lattice spacing: offsets are scaled by 1/h in the fits */
  double radius;      /* stencil radius: all neighbours with d <= radius        */
  double gx, gy, gz;  /* body force (m/s^2)                                     */
  double floor_z;     /* height of the floor plane for mirrors                  */
  int32_t mirror_mode;   /* LP_MIRROR_*                                         */
  int32_t precision;     /* LP_FP64, LP_MIXED or LP_MIXED_FF                    */
  int32_t rebuild_every; /* rebuild stencils every k steps (1 = every step)     */
  int32_t launch_mode;   /* LP_LAUNCH_*                                         */
  double skin;           /* > 0 (with rebuild_every == 1): Verlet candidate lists.
                          * A full search collects all neighbours within
                          * radius + skin; every step filters them with the exact
                          * radius test (same stencils as a full search); a new
                          * search runs once some particle has moved more than
                          * skin/2 since the last one. 0: full search every step.
                          * The lists live for one lp_step call; calls of fewer
                          * than 3 steps search every step (same stencils).
                          * All launch modes; the persistent launch takes the
                          * search branch inside the kernel.                      */
  int32_t free_surface;  /* 1: ghost particles at free boundaries (Sec. 3.1 items
                          * 6 and 9). A particle whose stencil is one-sided (its
                          * weighted mean offset, weights r^2 - d^2, exceeds
                          * 0.22 h) gets ghosts at the point reflections of its
                          * entries at least h/2 on the inner side, none within
                          * h/2 of an entry or below a mirrored floor. A ghost
                          * carries the particle's velocity, solid fraction
                          * phi_min (1 - 1e-3) and the |gdot| that keeps the
                          * inertial pressure continuous. Stencil entries plus
                          * ghosts must fit in cap (else LP_ERR_STENCIL_OVERFLOW).
                          * lp_step_adjoint covers them (flags frozen like the
                          * stencils, ghost regime frozen).                     */
  int32_t time_scheme;   /* LP_TIME_PAPER: the paper's step (Sec. 3.1 items 8,
                          * 10: V first, momentum with V^{n+1}, x with the mean
                          * velocity; first order). LP_TIME_HEUN: Heun's method
                          * on the semi-discrete system (second order; the paper
                          * plans a second-order scheme): two stages on the
                          * step's stencils, y* = y + dt F(y), y** = y* +
                          * dt F(y*), y^{n+1} = (y + y**) / 2, F taking V at its
                          * own time level. lp_step_adjoint covers it (both
                          * stages on the segment's stencils, then the average). */
  double period_x, period_y; /* > 0: periodic boundaries along x / y (Sec. 3.1
                          * item 9). lp_step first maps positions into [0, L)
                          * (values already there are kept bit for bit); every
                          * offset along the axis takes its nearest image, the
                          * neighbour grid wraps, and each step moves positions
                          * back into [0, L). Must be >= 3 (radius + skin).
                          * Heun's average takes the two positions on the same
                          * image. The floor and ghosts are unchanged (ghost
                          * offsets wrap modulo round(K L) with K the fixed-
                          * point scale). 0: not periodic. lp_build_neighbors
                          * and lp_fit_derivatives are not periodic;
                          * lp_step_adjoint is (offsets shift by whole
                          * periods, so the derivatives are unchanged).        */
  int32_t keep_lists;    /* 1 (with skin > 0, rebuild_every == 1): the Verlet
                          * candidate lists, their reference positions and the
                          * sorted order of this call are kept on the context
                          * for the next lp_step call, which then searches only
                          * if some particle moved more than skin/2 since the
                          * last search (checked on the device; stencils are
                          * those of a full search either way). They are kept
                          * while the particle count, the column offsets,
                          * radius, skin, floor, mirror mode and periods stay
                          * the same and no other entry point uses the
                          * context. Results then depend on the earlier calls
                          * only through the summation order of the stencils.
                          * 0: lists live for one call.                        */
  int32_t pad;
} lp_params;

/* Stencils produced by lp_build_neighbors: library-owned device memory, valid
 * until the next lp_build_neighbors / lp_step / lp_step_adjoint call on the
 * same context. nbr is k-major: nbr[k*n + i], k < min(cnt[i], cap), in
 * caller indices with the mirror bit. */
typedef struct {
  const int32_t* nbr;
  const int32_t* cnt;
  int64_t n;
  int32_t cap;
  int32_t pad;
} lp_neighbors;

typedef struct {
  uint32_t flags;        /* LP_FLAG_* seen since the last lp_ctx_sync            */
  int32_t min_stencil, max_stencil;
  int32_t pad;
  int64_t n_overflow;    /* particle-steps whose stencil exceeded cap            */
  int64_t n_fallback;    /* fits that used the pivoted-QR path                   */
  int64_t n_gas, n_quasistatic, n_over_c; /* particle-steps per regime (phi > phi_c) */
  int64_t n_nonfinite, n_below_floor;
  int64_t n_stencil_rows;  /* sum of stencil sizes over all stencils built     */
  int64_t n_stencils;      /* number of stencils built                          */
  int64_t n_ghosts;        /* ghost entries added to stencils (free_surface)    */
} lp_diag;

/* Version string of the library build. Never fails. */
const char* lp_version(void);
/* Human-readable name of a status code. Never fails. */
const char* lp_status_string(lp_status s);

/* Create a context on desc->device: allocates the workspace for
 * desc->max_particles particles (about 1 kB each). Makes desc->device current
 * for the calling thread. LP_ERR_OOM if the allocation fails. */
lp_status lp_ctx_create(const lp_ctx_desc* desc, lp_ctx** out);
/* Free the workspace. Waits for all work of the context to finish. */
lp_status lp_ctx_destroy(lp_ctx* ctx);
/* Wait for `stream`, copy the device diagnostics into *diag (may be NULL),
 * clear them, and return the first device-detected error (overflow ->
 * LP_ERR_STENCIL_OVERFLOW, non-finite -> LP_ERR_NONFINITE, timeout ->
 * LP_ERR_TIMEOUT) or LP_OK. Synchronises. */
lp_status lp_ctx_sync(lp_ctx* ctx, void* stream, lp_diag* diag);

/* Bounded waits of the persistent launch (failure detection, not in the
 * paper). Every grid barrier of LP_LAUNCH_PERSISTENT spins at most max_spins
 * rounds of __nanosleep(64) (default 2^25, about 2 s), then sets
 * LP_FLAG_TIMEOUT and leaves the kernel; lp_ctx_sync then returns
 * LP_ERR_TIMEOUT and the context stays usable. extra_arrivals > 0 makes each
 * barrier wait for that many blocks that do not exist, so the wait runs out:
 * a test aid only (0 restores normal operation). */
lp_status lp_ctx_set_wait_limit(lp_ctx* ctx, int64_t max_spins, int32_t extra_arrivals);

/* Device memory that lp_step_adjoint may use to keep a whole run's states,
 * fit data and stencils (not in the paper): max_bytes < 0 (the default) means
 * half of the device memory free at the call, 0 means never (re-run each
 * checkpoint segment). About 930 bytes per particle and step. */
lp_status lp_ctx_set_adjoint_memory(lp_ctx* ctx, int64_t max_bytes);

/* Per-phase timing (profiling aid, not in the paper). While enabled, lp_step
 * records a CUDA event pair around each phase of every step and does not use
 * graph replay. A persistent launch (one kernel per step) times its phases
 * inside the kernel instead: thread 0 of block 0 reads the GPU's global timer
 * after the grid barrier that closes each phase (two extra barriers while
 * profiling). */
lp_status lp_ctx_profile(lp_ctx* ctx, int32_t enable);
/* Wait for `stream`; ms[LP_NPHASES] receives the device time of each phase
 * accumulated since the last call (0 where profiling was off); *launches
 * (may be NULL) the number of kernels the library launched since the last
 * call, *steps (may be NULL) the number of LP steps. Resets all three.
 * Synchronises. */
lp_status lp_ctx_phase_times(lp_ctx* ctx, void* stream, double* ms, int64_t* launches,
                             int64_t* steps);

/* truncation rules of lp_build_neighbors (keep_nearest) */
#define LP_KEEP_ALL 0      /* every neighbour; longer than cap: overflow         */
#define LP_KEEP_NEAREST 1  /* the cap nearest                                    */
#define LP_KEEP_OCTANTS 2  /* the first cap of the octant-balanced ordering      */

/* Neighbour search (Sec. 3.1 items 5-6, mirrors item 9). For every particle i:
 * all j != i of the same column with ((dx*dx)+(dy*dy))+(dz*dz) <= r_i*r_i in
 * FP64 without contraction (d = x_j - x_i), and, if mirror_mode != NONE, every
 * mirror j* (including i*) passing the same test. r_i = radius[i] if radius
 * (device, length n) is non-NULL, else r_const. keep_nearest:
 *   LP_KEEP_ALL: cnt[i] is the full count and stencils longer than cap set
 *     LP_FLAG_OVERFLOW;
 *   LP_KEEP_NEAREST: only the min(cap, m_i) nearest are kept (ties by index,
 *     real before mirror) and cnt[i] is that number;
 *   LP_KEEP_OCTANTS: octant-balanced stencils (Sec. 3.1 item 6, the first
 *     entries of a list lie in all neighbouring octants): a candidate's round
 *     is its rank, in the nearest-first order above, among the candidates in
 *     its own octant (bit 0: dx >= 0, bit 1: dy >= 0, bit 2: dz >= 0); the
 *     min(cap, m_i) first by (round, nearest-first order) are kept.
 * At most 128 candidates per particle are considered by the two truncating
 * rules (more set LP_FLAG_OVERFLOW). Other values are LP_ERR_INVALID_ARG.
 * Order within a stencil is unspecified. Result in *out (library-owned). */
lp_status lp_build_neighbors(lp_ctx* ctx, const lp_particles* p, const double* radius,
                             double r_const, int32_t mirror_mode, double floor_z, int32_t cap,
                             int32_t keep_nearest, lp_neighbors* out, void* stream);

/* Copy stencils to host in canonical order: host_nbr is n x cap row-major,
 * real neighbours first then mirrors, each ascending; host_cnt[i] =
 * min(cnt[i], cap). Synchronises. */
lp_status lp_neighbors_export(lp_ctx* ctx, const lp_neighbors* nb, int32_t* host_nbr,
                              int32_t* host_cnt, void* stream);

/* GFD least-squares derivatives (Sec. 3.1 item 7) of nf fields on the given
 * stencils. fields: HOST array of nf DEVICE pointers (length n each);
 * mirror_sign: HOST array of nf factors applied to a field at a floor mirror
 * (+1 even, -1 odd, 0 zero). Rows: offsets d = (x_k - x_i)/h, columns
 * [dx, dy, dz, dx^2/2, dy^2/2, dz^2/2, dx dy, dx dz, dy dz], right-hand side
 * s_k - s_i. coeffs (device, n*nf*9 doubles, row-major [i][f][c]) receives
 * d/dx, d/dy, d/dz, d2/dx2, d2/dy2, d2/dz2, d2/dxdy, d2/dxdz, d2/dydz.
 * precision: LP_FP64, LP_MIXED or LP_MIXED_FF (moments, factor and
 * right-hand sides in float-float on positions relative to the first
 * particle; 8 B per particle and field of extra workspace, up to 16 fields,
 * allocated on first use). 1 <= nf <= 16. With n = 0 nothing is enqueued and
 * the field and coeffs pointers may be NULL. */
lp_status lp_fit_derivatives(lp_ctx* ctx, const lp_particles* p, const lp_neighbors* nb,
                             const double* const* fields, const double* mirror_sign, int32_t nf,
                             double h, double floor_z, double* coeffs, int32_t precision,
                             void* stream);

/* Largest n accepted by lp_fit_derivatives_noalloc. */
#define LP_NOALLOC_MAX_PARTICLES (1 << 20)

/* lp_fit_derivatives for callers that cannot allocate device memory (code
 * running inside an allocator or memory-pool hook, which must not re-enter the
 * allocator; plug-ins whose host application owns every device allocation;
 * loops that forbid allocation after start-up). The paper has no counterpart;
 * this is a deployment variant of the same fit. Needs no lp_ctx and calls no
 * cudaMalloc/cudaFree or allocating routine: its only scratch (the
 * pivoted-QR fallback queue, its counter and a diagnostics word, about 4 MB)
 * is a file-scope __device__ array that every GPU loading the library holds
 * until the process exits.
 * Inputs and output are as in lp_fit_derivatives, with the stencils passed
 * directly: nbr (device, k-major nbr[k*n + i], k < min(cnt[i], cap), particle
 * index j or j | 2^31 for the floor mirror of j; an index outside [0, n) is
 * skipped, as if the entry were absent) and cnt (device, n). Works on the
 * current CUDA device. Accepted: precision LP_FP64 or LP_MIXED (LP_MIXED_FF
 * needs per-particle workspace and is LP_ERR_INVALID_ARG here);
 * n <= LP_NOALLOC_MAX_PARTICLES (larger n is LP_ERR_INVALID_ARG).
 * diag (HOST, may be NULL): if non-NULL, the call waits for `stream` and
 * fills diag->n_fallback (stencils solved by the pivoted-QR fallback) and
 * diag->flags; the other fields are 0. With diag NULL the call is
 * asynchronous and reports no device-side counts.
 * First call on a device: it looks up the array's device address
 * (cudaGetSymbolAddress), which under CUDA's lazy module loading may also
 * load the library's module and place the array and kernels in device
 * memory. Make that first call at start-up, outside any allocator hook and
 * before any stream capture. All calls share the array and clear its counter
 * and diagnostics on entry, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race: serialise them. */
lp_status lp_fit_derivatives_noalloc(int64_t n, const double* x, const double* y, const double* z,
                                     const int32_t* nbr, const int32_t* cnt, int32_t cap,
                                     const double* const* fields, const double* mirror_sign,
                                     int32_t nf, double h, double floor_z, double* coeffs,
                                     int32_t precision, void* stream, lp_diag* diag);

/* Pointwise mu(I) stress (Sec. 2.2, 2.2.1) from V and the velocity gradient
 * grad_u (device, n x 9 row-major, grad_u[9i + 3a + b] = d u_a / d x_b):
 * gdot = D - (div u / 3) I as (xx, yy, zz, xy, xz, yz) (device, n x 6),
 * |gdot| = sqrt(gdot:gdot / 2), pressure P, effective viscosity eta
 * (tau = eta gdot) and regime (0 gas, 1 inertial, 2 quasi-static) chosen
 * from phi = 1/V. Any output pointer may be NULL. */
lp_status lp_mui_stress(lp_ctx* ctx, const lp_mui* mui, const lp_eos* eos, int64_t n,
                        const double* V, const double* grad_u, double* gdot, double* gdot_norm,
                        double* P, double* eta, int8_t* regime, void* stream);

/* nsteps explicit LP steps in place (Sec. 3.1 items 4-10). mui points to
 * p->ncolumns entries (HOST), one per column. Per step: stencils from the
 * current positions (every params->rebuild_every steps), pass 1 fits u, v, w
 * and gives gdot, |gdot|, div u, (1/2) Lap u + (1/6) grad div u and
 * V^{n+1} = V^n + dt V^n div u^n; pass 2 fits |gdot| and V^{n+1} and gives the
 * acceleration from the pressure law and mu(I) stress at phi^{n+1}; then
 * u^{n+1} = u^n + dt a and x^{n+1} = x^n + dt (u^n + u^{n+1})/2.
 * The seven state arrays are either all device arrays (stepped in place) or
 * all HOST arrays: the call then copies them to a staging block of the
 * context on the stream (one copy if they lie one after the other in the
 * order x, y, z, u, v, w, V, each of n doubles), steps there and copies the
 * result back on the stream; the arrays may be read once the stream has
 * finished (pinned memory makes the copies asynchronous). A mix of host and
 * device arrays is LP_ERR_INVALID_ARG. */
lp_status lp_step(lp_ctx* ctx, lp_particles* p, const lp_mui* mui, const lp_eos* eos,
                  const lp_params* params, double dt, int32_t nsteps, void* stream);

/* Launch configuration of lp_step (not in the paper). Block sizes are threads
 * per block of the neighbour search and of the two fit passes (64, 128 or
 * 256); launch_mode is the faster of LP_LAUNCH_GRAPH and LP_LAUNCH_PERSISTENT
 * for the tuned workload, for the caller to pass in lp_params. */
typedef struct {
  int32_t block_neighbors, block_pass1, block_pass2;
  int32_t launch_mode;
  double ms_per_step;  /* step time measured with this configuration          */
  int32_t from_table;  /* 1: read from the table, 0: measured by this call     */
  int32_t pad;
} lp_tuning;

/* Apply a launch configuration to the context. */
lp_status lp_ctx_set_tuning(lp_ctx* ctx, const lp_tuning* tuning);

/* Autotuner (not in the paper): times steps_per_trial steps of the given
 * workload (from the caller's particles, which are not modified) for each
 * candidate block size, keeps the fastest per phase, then times graph replay
 * against the persistent launch. The choice is applied to the context and
 * returned in *out. If table_path is non-NULL, a table line keyed by device
 * name, log2 n, log2 columns, precision and radius/h is looked up first
 * (then nothing is measured) and a new measurement is appended to it.
 * Synchronises. */
lp_status lp_autotune(lp_ctx* ctx, const lp_particles* p, const lp_mui* mui, const lp_eos* eos,
                      const lp_params* params, double dt, int32_t steps_per_trial,
                      const char* table_path, lp_tuning* out, void* stream);

/* Adjoint of nsteps lp_step steps (FP64) from `initial` (not modified). The
 * forward run being differentiated rebuilds stencils only at the start of each
 * segment of checkpoint_every steps and holds them fixed within it; regimes
 * are frozen at their forward values and d|gdot|/d gdot is taken as 0 where
 * |gdot| = 0. seed holds dL/d(final x, y, z, u, v, w, V) (device). On return
 * dL_dmui (device, 3 doubles) holds dL/d(mu_s, mu_2, I0) summed over all
 * columns, and if dL_dinitial is non-NULL its arrays receive dL/d(initial
 * state). Synchronises. Requires p->ncolumns == 1 in this version.
 * Workspace (allocated and freed by the call): the checkpoints, the
 * adjoints and, for the paper's step, each step's fit data (about 860 bytes
 * per particle and step) so that the reverse sweep need not compute it again:
 *  - when every segment's states, fit data and stencils fit in the limit set
 *    by lp_ctx_set_adjoint_memory, the forward sweep keeps them all and the
 *    reverse sweep recomputes nothing (one forward run in all);
 *  - otherwise the reverse sweep re-runs each segment from its checkpoint and
 *    keeps that segment's data (two forward runs); when even that cannot be
 *    allocated, each reverse step recomputes its own.
 * The three give the same result to rounding. Heun's method always takes the
 * last. */
lp_status lp_step_adjoint(lp_ctx* ctx, const lp_particles* initial, const lp_mui* mui,
                          const lp_eos* eos, const lp_params* params, double dt, int32_t nsteps,
                          int32_t checkpoint_every, const lp_particles* seed, double* dL_dmui,
                          lp_particles* dL_dinitial, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LP_H */
