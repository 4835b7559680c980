/*
 * smrt.h -- C ABI of libsmrt, a GB300 (sm_103a) implementation of the D2Q9
 * Single MRT-featured Lattice Boltzmann Method (SmrtLBM) of
 * J. G. Zhou, arXiv 2409.01076.
 *
 * The library advances a 2-D lattice of nx x ny nodes with the fused
 * stream-and-collide update of Eq. (SmrtLBM-1):
 *
 *   f_a(x + e_a, t + 1) = f_a^eq(x, t)
 *       + (-1)^a (1 - 1/tau) sum_{k=1}^{8} (-1)^k / 4
 *             [1_{1234}(a, k) + 1_{5678}(a, k)] (f_k(x, t) - f_k^eq(x, t)),
 *
 * with f^eq of Eq. (feq-full), rho and u of Eq. (fea-0), the indicator of
 * Eq. (indicator-fn), and the D2Q9 velocities e_a in the paper's order
 * (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1).  The SRT-LBM
 * update of Eq. (lb.srt) and the two-relaxation-time form of
 * Eq. (SmrtLBM-lb.1.5) are selectable collision kinds of the same kernels.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns an smrt_status; on failure smrt_last_error() explains.
 *   Nothing is freed that the caller owns; the library owns only what
 *   smrt_create/smrt_destroy manage.
 * - Node (i, j): i = 0..nx-1 along x, j = 0..ny-1 along y, the top side at
 *   j = ny-1.  Field arrays are row-major, index j*nx + i, with no padding.
 *     f   : double[9][ny][nx]       (population a, row j, column i)
 *     rho : double[ny][nx]
 *     u   : double[2][ny][nx]       (the u_x plane, then the u_y plane)
 * - Pointers may be host memory (pageable or pinned) or device memory of the
 *   current CUDA device; the library tells them apart with
 *   cudaPointerGetAttributes.  Device-pointer calls run on the handle's
 *   stream; host-pointer calls return after the transfer completed.  Page-locked
 *   host memory (cudaHostAlloc / cudaHostRegister, e.g. pinned torch tensors)
 *   is read or written by the kernels themselves over the host link, with no
 *   staging copy, so the transfer overlaps the arithmetic; pageable host memory
 *   goes through a device staging buffer in chunks of up to 64 MB.
 * - The canonical state f(t) is the post-streaming, pre-collision field, i.e.
 *   the left-hand side of Eq. (SmrtLBM-1) after t updates; rho(t), u(t) are its
 *   moments (Eq. fea-0).  t counts applications of the update.
 * - Boundaries (the paper's cavity: "standard bounce-back" on three walls, a
 *   lid moving with u_x = u0, u_y = 0): halfway (link) bounce-back; a moving
 *   wall adds -6 w_a rho_w (e_a . u_w) to the returning population, with
 *   rho_w = 1.  A link that leaves through a bottom/top wall and a left/right
 *   side at once takes the bottom/top wall's velocity; a link that leaves
 *   through a wall in one axis bounces back even if the other axis is
 *   periodic.
 * - Not thread-safe per handle: one host thread at a time per smrt_t.
 */
#ifndef SMRT_H
#define SMRT_H

#include <stddef.h>

#if defined(__GNUC__)
#define SMRT_API __attribute__((visibility("default")))
#else
#define SMRT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smrt_t smrt_t; /* opaque; owns device buffers, stream binding, flags */

enum smrt_status {
    SMRT_OK = 0,
    SMRT_ERR_ARG = -1,      /* invalid argument; nothing was changed          */
    SMRT_ERR_OOM = -2,      /* device allocation failed or exceeds MEM_LIMIT  */
    SMRT_ERR_CUDA = -3,     /* a CUDA runtime call failed (message has it)    */
    SMRT_ERR_DIVERGED = -4, /* some node had rho <= 0 or a non-finite rho     */
    SMRT_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up             */
    SMRT_ERR_STATE = -6     /* call not valid in the handle's current state   */
};

/* Boundary kind of one side; bc_flags packs 2 bits per side:
 * left (bits 0-1), right (2-3), bottom (4-5), top (6-7).
 * A moving wall slides with speed u_lid along its tangent: +x for the bottom
 * and top sides, +y for the left and right sides.  Periodic sides come in
 * pairs (left with right, bottom with top). */
enum smrt_bc { SMRT_BC_PERIODIC = 0, SMRT_BC_WALL = 1, SMRT_BC_MOVING = 2 };
#define SMRT_BC_FLAGS(left, right, bottom, top) \
    ((unsigned)(left) | ((unsigned)(right) << 2) | ((unsigned)(bottom) << 4) | ((unsigned)(top) << 6))
/* lid-driven cavity: resting walls left, right, bottom; moving lid on top */
#define SMRT_BC_CAVITY SMRT_BC_FLAGS(SMRT_BC_WALL, SMRT_BC_WALL, SMRT_BC_WALL, SMRT_BC_MOVING)

/* smrt_set_option keys and values. */
enum smrt_option {
    SMRT_OPT_COLLISION = 1,   /* SMRT_COLLISION_*; any time                               */
    SMRT_OPT_TAU_S = 2,       /* tau_s of the two-relaxation-time form (> 0.5); any time  */
    SMRT_OPT_LAYOUT = 3,      /* SMRT_LAYOUT_*; only before the state is first touched    */
    SMRT_OPT_PRECISION = 4,   /* SMRT_PREC_*;   only before the state is first touched    */
    SMRT_OPT_CHECK_DIVERGENCE = 5, /* 1 (default): smrt_step syncs and reports DIVERGED;
                                      0: smrt_step only enqueues                           */
    SMRT_OPT_MEM_LIMIT = 6,   /* bytes the handle may allocate on the device; 0 = no limit;
                                 only before the state is first touched                  */
    SMRT_OPT_TAU = 7,         /* change tau (> 0.5); any time                              */
    SMRT_OPT_ROUNDING = 8     /* SMRT_ROUND_*: how F16/BF16 storage rounds; any time       */
};
/* Rounding of the stored offsets in the 16-bit formats (FP32 and FP64 storage keep the
 * arithmetic's own result and ignore it).  NEAREST (default): round to nearest even.  In a
 * smooth, slowly changing flow neighbouring nodes then round the same way step after step, a
 * coherent error that grows to ~9e-2 U (FP16) and ~0.45 U (BF16) after 20,000 updates of a
 * 1024^2 cavity at Re 5,000.  STOCHASTIC: each stored value rounds up or down with the
 * probabilities that make its expected value exact, from counter-based random bits keyed by
 * (node, population, t) -- reproducible, identical in both layouts, restored with t from a
 * checkpoint -- so the rounding errors are uncorrelated and largely average out, at the cost
 * of ~60 more integer operations per node. */
enum smrt_rounding {
    SMRT_ROUND_NEAREST = 0,
    SMRT_ROUND_STOCHASTIC = 1
};
enum smrt_collision {
    SMRT_COLLISION_SMRT = 0,    /* Eq. (SmrtLBM-1)                                   */
    SMRT_COLLISION_SRT = 1,     /* Eq. (lb.srt)                                      */
    SMRT_COLLISION_TWO_TAU = 2  /* Eq. (SmrtLBM-lb.1.5) with tau_s from SMRT_OPT_TAU_S */
};
enum smrt_layout {
    SMRT_LAYOUT_AB = 0, /* two buffers: pull-stream from A, collide, store to B, swap     */
    SMRT_LAYOUT_AA = 1  /* one buffer, in place: alternating local / neighbour-swap steps */
};
enum smrt_precision {
    SMRT_PREC_F64 = 0,  /* stored f - w_a in double, double arithmetic         */
    SMRT_PREC_F32 = 1,  /* stored f - w_a in float, float arithmetic           */
    SMRT_PREC_F16 = 2,  /* stored f - w_a in IEEE half, float arithmetic       */
    SMRT_PREC_BF16 = 3  /* stored f - w_a in bfloat16, float arithmetic        */
};

/* Create a handle for an nx x ny lattice with relaxation time tau (Eq. SmrtLBM-1;
 * the kinematic viscosity is nu = (2 tau - 1) e dx / 6, Eq. relation-chapman-viscosity),
 * moving-wall speed u_lid (lattice units) and boundary kinds bc_flags.
 * Requires nx, ny >= 2, tau > 0.5 (finite), |u_lid| < 1/sqrt(3), valid paired
 * bc_flags, and 9 * pitch * ny elements addressable.  No CUDA call is made
 * here: device memory is allocated on the first call that touches the state,
 * which initialises f(0) = f^eq(rho = 1, u = 0) and t = 0.
 * On success *out receives the handle; on failure *out is set to NULL and
 * smrt_last_error(NULL) explains.  Defaults: SMRT collision, AB layout, F64,
 * divergence check on, legacy default stream. */
SMRT_API int smrt_create(int nx, int ny, double tau, double u_lid, unsigned bc_flags, smrt_t **out);

/* Set one option (see enum smrt_option).  Options marked "before the state is
 * first touched" return SMRT_ERR_STATE afterwards. */
SMRT_API int smrt_set_option(smrt_t *h, int key, double value);

/* Read one option's current value. */
SMRT_API int smrt_get_option(const smrt_t *h, int key, double *value);

/* Bind the CUDA stream (a cudaStream_t, passed as void*) that every later
 * launch and copy of this handle uses; NULL selects the legacy default stream.
 * The caller keeps ownership of the stream and must keep it alive. */
SMRT_API int smrt_set_stream(smrt_t *h, void *stream);

/* Apply the update n >= 0 times (t += n).  Launches are enqueued on the
 * handle's stream.  With the divergence check on, the call then waits for the
 * stream and returns SMRT_ERR_DIVERGED if any node had rho <= 0 or a
 * non-finite rho during these or earlier unchecked steps (t still advanced);
 * the flag clears on smrt_set_f / smrt_init_macros. */
SMRT_API int smrt_step(smrt_t *h, long long n);

/* Wait for the handle's stream; returns SMRT_ERR_DIVERGED if the divergence
 * flag is set (see smrt_step), else SMRT_OK or SMRT_ERR_CUDA. */
SMRT_API int smrt_sync(smrt_t *h);

/* Moments rho(t) and u(t) of the canonical state (Eq. fea-0), accumulated in
 * double.  rho: double[ny][nx]; u: double[2][ny][nx]; either may be NULL. */
SMRT_API int smrt_macros(smrt_t *h, double *rho, double *u);

/* Steady-state residual without advancing t:
 *   r = ||u(t+1) - u(t)||_2 / ||u(t+1)||_2 over all nodes (0 when both vanish),
 * where u(t+1) is what the next update would produce.  The paper states no
 * criterion; this is the definition used for "steady".  r (host, may be NULL)
 * receives r; sums (host, may be NULL) receives double[3] =
 * {sum rho(t), sum rho u_x(t), sum rho u_y(t)}.  All accumulation is double. */
SMRT_API int smrt_residual(smrt_t *h, double *r, double *sums);

/* The residual of smrt_residual for a lattice the caller holds, computed
 * without allocating any memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- for example code that
 * runs while a framework's caching allocator owns the device memory budget
 * (a raw cudaMalloc there can fail or fragment the pool), or latency-critical
 * loops where cudaMalloc/cudaFree would synchronize the device -- and who
 * therefore cannot create an smrt_t either (its state is allocated on first use).
 *
 * f:   the canonical f(t) in DEVICE memory of the current device,
 *      double[9][ny][nx] (the layout of smrt_get_f); read only.
 * out: double[4] = {r, sum rho, sum rho u_x, sum rho u_y}, host or device
 *      memory.  r and the sums are defined as for smrt_residual, evaluated in
 *      FP64 with the update given by tau, u_lid, bc_flags, collision and tau_s
 *      (tau_s is read only for SMRT_COLLISION_TWO_TAU).
 * stream: the cudaStream_t to run on (NULL: legacy default stream).  With a
 *      device `out` the call only enqueues work; with a host `out` it waits.
 *
 * Scratch: the per-block partial sums live in one file-scope device array of
 * 1216 x 5 + 4 doubles (48,672 bytes), which every GPU that loads the library
 * holds until the process exits.  Every call looks up that array's device
 * address (cudaGetSymbolAddress) in the current context, so a context that was
 * reset and created again is handled; the first call on a device also loads the
 * library's device code there, so make that first call before any stream
 * capture.  Every call on a device shares the
 * array and leaves its contents behind; nothing in it needs to start at zero
 * (each call writes every slot it later reads).  Calls whose work overlaps on
 * the GPU -- on different streams, or from different host threads -- race on
 * the array: serialise them.
 * Limits: nx, ny >= 2 and nx * ny <= SMRT_NOALLOC_MAX_NODES; larger lattices
 * return SMRT_ERR_ARG.  Errors are reported through smrt_last_error(NULL).
 * Calls no cudaMalloc, cudaFree or other allocating routine. */
#define SMRT_NOALLOC_MAX_NODES (1LL << 30)
SMRT_API int smrt_residual_noalloc(const double *f, int nx, int ny, double tau, double u_lid,
                                   unsigned bc_flags, int collision, double tau_s, double *out,
                                   void *stream);

/* Copy the canonical state f(t) out as double[9][ny][nx]. */
SMRT_API int smrt_get_f(smrt_t *h, double *f);

/* Replace the canonical state by f (double[9][ny][nx]); t is unchanged and the
 * divergence flag clears.  Values are rounded to the storage precision. */
SMRT_API int smrt_set_f(smrt_t *h, const double *f);

/* Replace the state by f = f^eq(rho, u) of Eq. (feq-full) at every node
 * (rho: double[ny][nx], u: double[2][ny][nx]); t is unchanged, the divergence
 * flag clears. */
SMRT_API int smrt_init_macros(smrt_t *h, const double *rho, const double *u);

/* Number of updates applied so far (t); -1 for a NULL handle. */
SMRT_API long long smrt_time(const smrt_t *h);

/* Set t (>= 0) without touching the populations.  With the AA layout the
 * stored arrangement depends on the parity of t, so this is allowed only
 * while the parity stays the same (else SMRT_ERR_STATE). */
SMRT_API int smrt_set_time(smrt_t *h, long long t);

/* Bytes of device memory the handle holds (0 before the state is touched). */
SMRT_API size_t smrt_device_bytes(const smrt_t *h);

/* Last error message of h, or of the calling thread's last failed
 * smrt_create when h is NULL.  Never NULL; valid until the next call on h. */
SMRT_API const char *smrt_last_error(const smrt_t *h);

/* Free the handle's device memory and the handle.  NULL is ignored. */
SMRT_API void smrt_destroy(smrt_t *h);

/* ---- batches of independent lattices ------------------------------------------
 * Many lattices ("cavities") of uneven size and relaxation time, advanced by the
 * same update as smrt_step (bit for bit: the same per-block kernel code) in one
 * launch per step: a persistent work-list kernel walks the step blocks of every
 * active lattice.  Lattice k has nx[k] x ny[k] nodes, tau[k], u_lid[k]; all share
 * bc_flags, the collision kind (SMRT or SRT), the precision (F32 or F64) and the
 * layout.  Each lattice starts at f = f^eq(1, 0), t = 0.  Lattices retire
 * (stop advancing) in smrt_batch_run when converged, capped or diverged.
 * The paper runs one cavity at a time; batching is this library's addition. */
typedef struct smrt_batch_t smrt_batch_t;
enum smrt_batch_state {
    SMRT_BATCH_ACTIVE = 0, SMRT_BATCH_CONVERGED = 1, SMRT_BATCH_CAPPED = 2, SMRT_BATCH_DIVERGED = 3
};

/* Allocates all lattices in one buffer (two for the AB layout) on the current
 * device.  Host arrays of length count.  Errors: SMRT_ERR_ARG (invalid sizes,
 * tau <= 0.5, |u_lid| >= 1/sqrt(3), flags, precision other than F32/F64,
 * collision other than SMRT/SRT), SMRT_ERR_OOM; message in smrt_last_error(NULL). */
SMRT_API int smrt_batch_create(int count, const int *nx, const int *ny, const double *tau, const double *u_lid,
                               unsigned bc_flags, int precision, int layout, int collision, smrt_batch_t **out);

/* Stream for every later launch and copy (NULL: legacy default stream). */
SMRT_API int smrt_batch_set_stream(smrt_batch_t *b, void *stream);

/* Times each candidate tile shape of the work-list kernel (nodes per thread x
 * threads per block, with or without a 64-register bound, each without (index k)
 * and with (index k + 5 for FP32 storage, k + 4 for FP64) the edge column groups
 * of the two-buffer layout in the vector path; then row-segmented shapes, whose
 * warps cover several rows of a narrow lattice at once (indices 10 to 14 for
 * FP32, 13 and 14 with each block walking one contiguous run of the work list;
 * 8 for FP64); FP32: 15 candidates, FP64: 9) on
 * `steps` steps of this batch, run on a copy of the state so no lattice advances,
 * and keeps the fastest; *choice (may be NULL) receives its index.  Allocates one
 * scratch copy of the populations for the duration. */
SMRT_API int smrt_batch_autotune(smrt_batch_t *b, int steps, int *choice);

/* Selects tile shape `shape` (an index as returned by smrt_batch_autotune) without
 * timing anything; SMRT_ERR_ARG if it is not a candidate of the batch's precision.
 * The lattices' state is untouched: every shape computes the same bits. */
SMRT_API int smrt_batch_set_shape(smrt_batch_t *b, int shape);

/* n >= 0 updates of every active lattice (one work-list launch each); waits,
 * then marks lattices whose divergence word is set as SMRT_BATCH_DIVERGED. */
SMRT_API int smrt_batch_step(smrt_batch_t *b, long long n);

/* Runs until no lattice is active: replays a CUDA graph of check_every updates
 * (rounded up to even) plus a residual pass, then retires each active lattice
 * whose residual r_k is below tol (CONVERGED), that reached max_steps (CAPPED),
 * or whose divergence word is set or r_k is not finite (DIVERGED).
 * residual_kind SMRT_BATCH_RESIDUAL_STEP: the one-step residual of smrt_residual,
 *   r_k = ||u(t+1) - u(t)||_2 / ||u(t+1)||_2 at the last update of each chunk.
 * residual_kind SMRT_BATCH_RESIDUAL_STRIDE: the mean change per update over the
 *   chunk, r_k = ||u(t) - u(t - check_every)||_2 / (check_every ||u(t)||_2); the
 *   first check of a run compares with zero velocity.  With FP32 storage the
 *   one-step residual stops falling near 1e-7..1e-6 (rounding), and a period-two
 *   oscillation that halfway bounce-back keeps alive at the lid corners can hold
 *   it near 1e-5; the even stride averages both out.
 * *n_active (may be NULL) receives the active count at return (0). */
enum smrt_batch_residual { SMRT_BATCH_RESIDUAL_STEP = 0, SMRT_BATCH_RESIDUAL_STRIDE = 1 };
SMRT_API int smrt_batch_run(smrt_batch_t *b, double tol, long long check_every, long long max_steps,
                            int residual_kind, int *n_active);

/* Per-lattice host arrays of length count (each may be NULL): updates applied,
 * last residual of smrt_batch_run (-1 before the first check), smrt_batch_state. */
SMRT_API int smrt_batch_status(const smrt_batch_t *b, long long *steps, double *residual, int *state);

/* Canonical f(t) of lattice k as double[9][ny][nx] (host or device memory). */
SMRT_API int smrt_batch_get_f(smrt_batch_t *b, int k, double *f);

/* rho(t), u(t) of lattice k: double[ny][nx] and double[2][ny][nx], host or device. */
SMRT_API int smrt_batch_macros(smrt_batch_t *b, int k, double *rho, double *u);

/* f = f^eq(rho, u) in lattice k (a warm start); only while k is active and in step
 * with the others.  rho, u: host or device, as in smrt_init_macros. */
SMRT_API int smrt_batch_init_macros(smrt_batch_t *b, int k, const double *rho, const double *u);

/* Total nodes of the batch (-1 for NULL). */
SMRT_API long long smrt_batch_nodes(const smrt_batch_t *b);

/* Last error message of b (of the thread's last failed create when b is NULL). */
SMRT_API const char *smrt_batch_last_error(const smrt_batch_t *b);

/* Frees the batch.  NULL is ignored. */
SMRT_API void smrt_batch_destroy(smrt_batch_t *b);

#ifdef __cplusplus
}
#endif

#endif /* SMRT_H */
