/* btdf.h - C ABI of the GB300 (sm_103a) implementation of the boundary
 * thickening direct-forcing immersed-boundary lattice Boltzmann method
 * (BTDF-IB/LBM) of M. Jiang and Z. Liu, arXiv 1806.09403.
 *
 * One call of btdf_step advances the flow by whole time steps of the paper's
 * Algorithm 1 (with NF forcing passes):
 *   IB stage   - density and unforced velocity at the marker supports
 *                (Eqs. 9-10), interpolation to the Lagrangian markers with the
 *                regularized delta function (Eqs. 12, 14, 37-39), the explicit
 *                direct-forcing force F_b = 2 rho (U_b - D_I u*) (Eq. 20) and
 *                the force on each body (Eq. 27), reduced in FP64.
 *   LBM stage  - spreading of F_b with the thickened solid shell drs
 *                (Eqs. 13, 15), velocity correction u = u* + f / (2 rho)
 *                (Eq. 11), BGK collision with the Guo forcing term
 *                (Eqs. 5-7) and streaming, fused in one kernel.
 *
 * Units: lattice units, dh = dt = c = 1, reference density rho0 = 1.
 * Fields: row-major, x fastest, node (x, y) at integer coordinates
 * 0..nx-1, 0..ny-1.  D2Q9 population order (Eq. 8):
 *   0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 *
 * Conventions shared by every entry point:
 *   - Every function returns a btdf_status (0 on success, < 0 on error);
 *     btdf_last_error() gives a message for the last failure of a context.
 *   - The caller owns every pointer it passes; the library copies what it
 *     needs and never frees or retains caller memory.  Pointers are host
 *     pointers unless stated otherwise.
 *   - A context owns the device memory it allocates and frees it in
 *     btdf_destroy.  All device work is issued on the stream given to
 *     btdf_create; calls that return data to the host synchronize it.
 *   - A context is not thread-safe: serialize calls on one context.
 *   - Device-side failures (an unstable density at a marker, a bounded wait
 *     that gave up) are recorded in a status word and reported by the next
 *     btdf_sync or read call, and are sticky.
 */
#ifndef BTDF_H
#define BTDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct btdf_ctx btdf_ctx;

typedef enum {
    BTDF_OK = 0,
    BTDF_EINVAL = -1,     /* bad argument or configuration */
    BTDF_ENOMEM = -2,     /* device or host allocation failed */
    BTDF_ECUDA = -3,      /* a CUDA runtime call failed (message in last_error) */
    BTDF_EUNSTABLE = -4,  /* non-positive or non-finite density/force at a marker */
    BTDF_ETIMEOUT = -5,   /* a bounded device wait gave up */
    BTDF_ESTATE = -6      /* call not valid in the current state (e.g. no fields) */
} btdf_status;

/* Regularized delta functions of Sec. 4.3: 2-point (Eq. 37), 3-point (Eq. 38),
 * 4-point (Eq. 39), and a 4-point cosine kernel that the paper does not print. */
typedef enum {
    BTDF_DELTA2 = 2,
    BTDF_DELTA3 = 3,
    BTDF_DELTA4 = 4,
    BTDF_DELTA4COS = 5
} btdf_delta;

/* Population storage.  All forms store deviations f_a - f_eq_a(1, (u_in, 0))
 * from the equilibrium of the reference state (unit density, velocity
 * (u_in, 0)), so rounding scales with the departure of the flow from that
 * state; arithmetic is FP32 in every form. */
typedef enum {
    BTDF_F32 = 0,
    BTDF_F16DEV = 1,
    BTDF_BF16DEV = 2
} btdf_storage;

/* x boundaries: periodic, or inlet at x = 0 (non-equilibrium extrapolation to
 * velocity (u_in, 0)) with a zero-gradient or convective outlet at x = nx-1
 * (Sec. 5.2 names a convective outlet). */
typedef enum {
    BTDF_BCX_PERIODIC = 0,
    BTDF_BCX_INOUT = 1,      /* inlet + zero-gradient outlet (copy of column nx-2) */
    BTDF_BCX_CONVECTIVE = 2, /* inlet + convective outlet: d f / dt + u_in d f / dx = 0,
                                implicit upwind, f(nx-1, t+1) = (f(nx-1, t) + u_in f(nx-2, t+1)) / (1 + u_in);
                                markers must keep off the outlet column; not for the batch */
    BTDF_BCX_BOX = 3         /* prescribed-velocity box: every outer node (all four sides) gets
                                the velocity set by btdf_set_boundary_velocity, by
                                non-equilibrium extrapolation from its nearest interior node
                                (Sec. 5.1); bc_y is ignored; not for the batch or the adjoint */
} btdf_bc_x;
/* y boundaries: periodic, free-slip walls (half-way specular reflection) or
 * no-slip walls (half-way bounce-back); walls sit half a node outside rows
 * 0 and ny-1. */
typedef enum { BTDF_BCY_PERIODIC = 0, BTDF_BCY_FREESLIP = 1, BTDF_BCY_NOSLIP = 2 } btdf_bc_y;

/* Device layout of the population buffers (elements of the storage type):
 * planes: [9][ny][nxp]; rows: [ny][9][nxp] (the nine planes of one row are
 * adjacent), with nxp = nx rounded up to a multiple of 32. */
typedef enum { BTDF_LAYOUT_PLANES = 0, BTDF_LAYOUT_ROWS = 1 } btdf_layout;

typedef enum {
    BTDF_FIELD_RHO = 0,   /* density, Eq. 9 (ny*nx floats) */
    BTDF_FIELD_UX = 1,    /* unforced velocity u*, Eq. 10 (ny*nx floats) */
    BTDF_FIELD_UY = 2,
    BTDF_FIELD_POPS = 3,  /* populations f (not deviations), [9][ny][nx] floats */
    BTDF_FIELD_FX = 4,    /* immersed-boundary force density of the last step, Eq. 15 */
    BTDF_FIELD_FY = 5     /* (without the uniform body force gx, gy), ny*nx floats */
} btdf_field;

typedef struct {
    int32_t nx, ny;        /* lattice size, >= 4 each */
    double tau;            /* BGK relaxation time, > 0.5 (tau = 0.5 + 3 nu) */
    double u_in;           /* inlet speed for BTDF_BCX_INOUT; the value at creation is
                              also the reference velocity of the stored deviations */
    int32_t delta;         /* btdf_delta */
    int32_t nf;            /* forcing passes per step, 1 = BTDF/DF, > 1 = MDF (Sec. 3.2) */
    int32_t storage;       /* btdf_storage */
    int32_t bc_x, bc_y;    /* btdf_bc_x, btdf_bc_y */
    int32_t history_len;   /* steps of body-force history kept on the device (>= 1) */
    double gx, gy;         /* uniform body force added to the IB force everywhere */
    int32_t layout;        /* btdf_layout */
    int32_t reserved;      /* must be 0 */
} btdf_config;

/* Fills *cfg with a 64 x 64 periodic FP32 lattice, tau = 0.6, 3-point delta,
 * nf = 1, history_len = 4096, row-interleaved layout. */
int btdf_config_default(btdf_config *cfg);

/* Validates *cfg, allocates the two population buffers and per-context
 * scratch on the device, and binds the context to `stream` (a cudaStream_t;
 * NULL = the legacy default stream).  On success *out receives the context.
 * Errors: EINVAL (bad configuration; nothing allocated), ENOMEM, ECUDA. */
int btdf_create(const btdf_config *cfg, void *stream, btdf_ctx **out);
int btdf_destroy(btdf_ctx *ctx);

/* Sets f = f_eq(rho, u) at every node (Eq. 6).  rho, ux, uy are host arrays
 * of ny*nx doubles.  Resets the step counter and the force history. */
int btdf_init_fields(btdf_ctx *ctx, const double *rho, const double *ux, const double *uy);

/* Adds one rigid body of n markers at (X[l], Y[l]) with prescribed velocity
 * (Ubx[l], Uby[l]) (NULL = at rest), arc length ds per marker and solid-shell
 * thickness drs (Eq. 15; drs <= 0 takes the value suggested in Sec. 4.4 for
 * the configured delta: 1.4, 1.9, 2.6 for 2, 3, 4 points, 2.6 for the cosine
 * kernel).  Interpolation weights delta(x_e - X) delta(y_e - Y) (Eq. 14) are
 * evaluated once here in FP64; markers are static.  Every marker's support
 * must lie at least partly inside the lattice; under BTDF_BCX_CONVECTIVE no
 * support may reach the outlet column x = nx-1.  *body_id receives the index.
 * Errors: EINVAL (n < 1, ds <= 0, marker outside the lattice, support on the
 * convective outlet column). */
int btdf_add_markers(btdf_ctx *ctx, int32_t n, const double *X, const double *Y,
                     const double *Ubx, const double *Uby, double ds, double drs,
                     int32_t *body_id);

/* Velocities of the outer nodes of a BTDF_BCX_BOX lattice (the Dirichlet
 * boundary of the Taylor-Green test, Sec. 5.1), host arrays of
 * 2 nx + 2 (ny - 2) doubles in perimeter order: row 0 (x = 0..nx-1), row
 * ny-1 (x = 0..nx-1), column 0 (y = 1..ny-2), column nx-1 (y = 1..ny-2).  The
 * values apply from the next step on; zero until first set.  Asynchronous on
 * the context stream (the arrays are read before the call returns).
 * Errors: ESTATE (no box), EINVAL (null, not finite, |u| >= 0.5). */
int btdf_set_boundary_velocity(btdf_ctx *ctx, const double *ubx, const double *uby);

/* Adds a circular body: n markers equally spaced on the circle of diameter D
 * about (cx, cy), X_l = cx + (D/2) cos(2 pi l / n), Y_l = cy + (D/2) sin(2 pi l / n),
 * at rest, with arc length ds = pi D / n per marker and thickness drs (<= 0:
 * the value of Sec. 4.4, as btdf_add_markers).  Errors: EINVAL (n < 1,
 * D <= 0, support outside the lattice). */
int btdf_add_cylinder(btdf_ctx *ctx, double cx, double cy, double D, int32_t n, double drs,
                      int32_t *body_id);

/* Replaces the prescribed marker velocities U_b of one body (host arrays of
 * that body's marker count, read before the call returns), or, with
 * body = -1, of every body at once (arrays of all markers, in the order the
 * bodies were added; one copy to the device).  The upload is
 * asynchronous on the context stream through one of four page-locked
 * staging slots; a call waits only when the upload four calls back has not
 * run yet. */
int btdf_set_marker_velocity(btdf_ctx *ctx, int32_t body, const double *Ubx, const double *Uby);

/* Changes the inlet speed of BTDF_BCX_INOUT (the non-equilibrium
 * extrapolation target, Sec. 5.2 inflow) without touching the stored state:
 * the reference velocity of the stored deviations stays the creation-time
 * u_in, so a checkpoint still loads as the same physical state.
 * Synchronizes.  Errors: EINVAL (|u_in| >= 0.5 or not finite). */
int btdf_set_inflow(btdf_ctx *ctx, double u_in);

/* Moves the markers of one body to (X[l], Y[l]) (host arrays of the body's
 * marker count) and re-evaluates its weights and the spreading table; ds,
 * drs and the velocities are kept.  The force history restarts at the
 * current step.  Synchronizes.  The positions are checked as in
 * btdf_add_markers (convective outlet column included) before anything
 * changes.  Errors: EINVAL (bad body, marker outside, support on the
 * convective outlet column). */
int btdf_move_markers(btdf_ctx *ctx, int32_t body, const double *X, const double *Y);

/* Advances nsteps time steps (Algorithm 1), asynchronously on the context
 * stream.  Requires btdf_init_fields or btdf_load_state first (ESTATE). */
int btdf_step(btdf_ctx *ctx, int64_t nsteps);

/* Waits for the context stream and returns the sticky device status
 * (OK, EUNSTABLE or ETIMEOUT). */
int btdf_sync(btdf_ctx *ctx);

/* Force on one body (Eq. 27, force exerted by the fluid on the body) for the
 * steps first .. first+n-1, into host arrays Fx, Fy of n doubles; with
 * body = -1 the forces on every body, n x nbody doubles each, step-major
 * (Fx[i * nbody + b]).  The steps must have been taken and must still be
 * inside the device history ring.  Synchronizes.  Errors: EINVAL (body or
 * step range). */
int btdf_read_forces(btdf_ctx *ctx, int32_t body, int64_t first, int64_t n,
                     double *Fx, double *Fy);

/* As btdf_read_forces, without waiting: enqueues the copy of the steps
 * first .. first+n-1 into F[2 i] = Fx, F[2 i + 1] = Fy (body = -1: into
 * F[2 (i * nbody + b)], F[2 (i * nbody + b) + 1]) on the context stream and
 * returns.  F must stay valid until the stream reaches the copy
 * (btdf_sync); page-locked memory (cudaMallocHost, a pinned torch tensor)
 * makes it a DMA transfer that overlaps host work, pageable memory makes
 * the call wait for the copy.  Device status is reported by btdf_sync. */
int btdf_read_forces_async(btdf_ctx *ctx, int32_t body, int64_t first, int64_t n, double *F);

/* Per-marker results of the last step for one body, host arrays of the body's
 * marker count (any may be NULL): interpolated unforced velocity D_I u*
 * (Eq. 14) and the Lagrangian force F_b summed over the forcing passes
 * (Eq. 20). Synchronizes. */
int btdf_read_markers(btdf_ctx *ctx, int32_t body, float *Usx, float *Usy,
                      float *Fbx, float *Fby);

/* Macroscopic field or populations of the current state (after the last
 * step's streaming and boundary rules), as floats.  dst is a host pointer, or
 * a device pointer when dst_is_device != 0.  Synchronizes. */
int btdf_read_field(btdf_ctx *ctx, int32_t kind, float *dst, int32_t dst_is_device);

int64_t btdf_step_count(const btdf_ctx *ctx);

/* Checkpoint of the populations and the step counter (not the force
 * history), plus the outlet column buffer under the convective outlet.
 * Byte image: a 48-byte header (uint64 magic; int32 nx, ny, nxp, storage;
 * int32 at byte 24: 1 if the populations are post-streaming, 0 if
 * post-collision; int32 layout; int64 step counter; double at byte 40: the
 * reference velocity u_ref of the stored deviations, i.e. the creation-time
 * u_in), then the population buffer in the device layout, then the outlet
 * column ([9][ny] floats) under the convective outlet.
 * btdf_state_size gives the byte count; save copies to a host buffer of at
 * least that size; load restores a checkpoint of a context with the same nx,
 * ny, storage, layout, x boundary and creation-time u_in.  Errors: EINVAL
 * (size, shape or reference-velocity mismatch). */
int btdf_state_size(btdf_ctx *ctx, size_t *bytes);
int btdf_save_state(btdf_ctx *ctx, void *dst, size_t cap, size_t *used);
int btdf_load_state(btdf_ctx *ctx, const void *src, size_t len);

/* Profiling hooks for benchmarks: while enabled, btdf_step launches every
 * kernel directly (no CUDA graph) between CUDA events on the context stream;
 * btdf_profile_read synchronizes and returns the summed device time of the
 * IB-stage kernels and of the fused collide-stream kernel, and the number of
 * kernel launches, since profiling was enabled.  Enabling resets the sums. */
int btdf_profile_enable(btdf_ctx *ctx, int32_t on);
int btdf_profile_read(btdf_ctx *ctx, double *ms_ib, double *ms_lbm, int64_t *launches_ib,
                      int64_t *launches_lbm);

/* Number of collide-stream variants, 0 (automatic) included: the length of
 * btdf_autotune's ms output. */
#define BTDF_VARIANT_COUNT 14

/* Variant of the fused collide-stream kernel.  Results do not depend on it.
 *   0 automatic: on lattices of at least 2^23 nodes 11 for FP32 and 12 for
 *     FP16 / BF16 storage (11 where no tensor maps could be encoded), on
 *     smaller ones 2 for FP32 and 11 for FP16 / BF16 (the autotuner's usual
 *     picks on a GB300)
 *   1 register-pipelined warps, 4 nodes per lane (16-byte FP32 vectors)
 *   2 register-pipelined warps, 2 nodes per lane
 *   3 TMA-tiled CTAs: 128 x 8 node tiles, 2 pipeline stages
 *   4 TMA-tiled CTAs: 128 x 8 node tiles, 3 pipeline stages
 *   5 TMA-tiled CTAs: 128 x 16 node tiles, 2 pipeline stages
 *   6 register warps, 4 nodes per lane, next segment's loads issued early
 *   7 register warps, 2 nodes per lane, next segment's loads issued early
 *   8 register warps, 1 node per lane, 6 resident blocks per SM
 *   9 register warps, 2 nodes per lane, 5 resident blocks per SM
 *  10 as 9, and each warp prefetches into L2 the row segment that a warp
 *     half a wave later will process
 *  11 as 1, with the L2 prefetch of 10
 *  12 warp-specialized TMA CTAs: 128 x 8 node tiles handed out one at a time
 *     from a device counter, one producer warp issuing the loads, 8 warps
 *     computing rows, 2 pipeline stages, 3 resident blocks per SM
 *  13 as 12 with 128 x 7 node tiles, 7 computing warps and 3 pipeline
 *     stages, 3 resident blocks per SM
 * grid_blocks caps the grid, counted in blocks of the variant: 256 threads,
 * or 128 for variant 2 and, with FP16 / BF16 storage, variants 1 and 8-11,
 * or 288 for variant 12.  0 = default:
 * one 32 x NPL-node row segment per warp for variants 1, 2 and 8-11, so the
 * block scheduler balances the SMs; SM count x resident blocks per SM for
 * the persistent variants 3-7, 12 and 13.
 * The TMA variants (3-5, 12, 13) run pulling steps only: the first step after
 * btdf_init_fields (which streams in place) runs variant 1 instead, as do all
 * steps of a lattice with the Taylor-Green box (BTDF_BCX_BOX), where variants
 * 6 and 7 also give way to variant 1.
 * Synchronizes and drops cached CUDA graphs.
 * Errors: EINVAL (unknown variant, TMA variant without tensor maps). */
int btdf_tune(btdf_ctx *ctx, int32_t variant, int32_t grid_blocks);

/* Bound of the TMA-tiled variants' (3-5, 12, 13) per-stage waits, in polls of the
 * stage's mbarrier: polls < 0 restores the default (about a second of
 * polling); 0 makes every such wait give up at once.  A wait that gives up
 * records BTDF_ETIMEOUT in the status word (reported by the next btdf_sync),
 * and its CTA waits, with the default bound, for the copies it has in flight
 * before it leaves; the populations of that step are then invalid.  Meant for
 * testing the timeout path of failure detection.  Synchronizes and drops
 * cached CUDA graphs. */
int btdf_set_wait_limit(btdf_ctx *ctx, int32_t polls);

/* Bytes of device memory the context holds. */
int btdf_device_bytes(const btdf_ctx *ctx, size_t *bytes);

/* Autotuner of the collide-stream launch: times every available variant of
 * btdf_tune (1..BTDF_VARIANT_COUNT-1; the TMA variants only where tensor maps were encoded) on
 * this context's own lattice, `steps` steps each after 3 untimed ones, every
 * step (IB and LBM stage, overlapped as in btdf_step) between CUDA events on
 * the context stream, with the L2 cache evicted before each step when
 * flush_l2 != 0.  Keeps the variant with the lowest interquartile mean step
 * time (the mean of the middle half of the sorted times).  The
 * populations, the step counter, the force history and the last step's
 * marker results are restored afterwards, so the simulation does not
 * advance.  Outputs (may be NULL): *chosen, and ms[v] = that mean, in ms per step, of
 * variant v for v = 0..BTDF_VARIANT_COUNT-1 (-1 where not timed).  Needs temporary device memory
 * for one copy of the populations and, with flush_l2, four times the L2 size.
 * Synchronizes.  Errors: EINVAL (steps outside 1..100000), ESTATE (no fields),
 * ENOMEM / ECUDA. */
int btdf_autotune(btdf_ctx *ctx, int32_t steps, int32_t flush_l2, int32_t *chosen, float *ms);

/* ---- discrete adjoint of a time window -----------------------------------
 * Objective: the drag coefficient averaged over the next nsteps steps from the
 * current state,
 *   J = (1 / nsteps) sum_n Cd^n,   Cd^n = Fx^n / (u_in^2 dref / 2),
 * with Fx^n the x force on the selected body (Eq. 27; body = -1: the sum over
 * all bodies) in step n.  Gradients are taken with respect to the inlet speed
 * u_in (entering the inlet extrapolation and the normalization; tau fixed)
 * and every marker position (through the delta functions of Eq. 14 in both
 * interpolation and spreading; ds and drs fixed).  The reverse sweep is the
 * exact discrete adjoint of the FP32 step (collision with the Guo term, pull
 * streaming with the wall, inlet and outlet rules, Eqs. 14, 15, 20).
 *
 * btdf_adjoint_forward runs the window from the current state on private
 * buffers, keeping a checkpoint every `every` steps and the Lagrangian forces
 * of every step, and returns J.  The context's own state, step counter and
 * force history are not changed.  Requires nf = 1, FP32 storage, at least
 * one body, dref > 0, u_in != 0, and, with an inlet, no marker support on
 * columns 0 or nx-1.  Device memory: (ceil(nsteps/every) + every + 2) states
 * of 36 * nxp * ny bytes plus 8 * nsteps * markers bytes, held until
 * btdf_adjoint_release or btdf_destroy.
 * Errors: EINVAL, ESTATE (no fields or no bodies), ENOMEM, EUNSTABLE.
 *
 * btdf_adjoint_backward reverses the last forward window: segments are
 * recomputed from their checkpoints, then each step is reversed by three
 * kernels (collision and boundary folds, marker forces and positions,
 * interpolation at the band nodes).  Outputs (host, any may be NULL):
 * dJdU = dJ/du_in, dJdX[l], dJdY[l] = dJ/dX_l, dJ/dY_l for every marker in the
 * order the markers were added.  Setting the inflow, moving markers or
 * changing marker velocities invalidates the window (ESTATE).  Synchronizes.
 * Both passes are replayed as CUDA graphs captured on first use (on an
 * internal stream) and updated in place when the window, the markers or the
 * inflow change. */
int btdf_adjoint_forward(btdf_ctx *ctx, int64_t nsteps, int32_t every, int32_t body, double dref,
                         double *J);
int btdf_adjoint_backward(btdf_ctx *ctx, double *dJdU, double *dJdX, double *dJdY);
int btdf_adjoint_release(btdf_ctx *ctx);

/* ---- batched form --------------------------------------------------------
 * Many independent lattices (each with its own size, relaxation time,
 * inflow, boundary kinds and bodies) advanced together: one IB launch over
 * the markers of all lattices and one persistent collide-stream launch over
 * all lattices per step, replayed through CUDA graphs.  Each lattice computes
 * exactly what a single context with the same configuration computes.  All
 * lattices share storage, layout, delta function, history_len and nf = 1.
 * Fields and markers are set before the first step.  Body ids count bodies in
 * the order they were added, over all lattices. */
typedef struct btdf_batch btdf_batch;

/* cfgs: n configurations.  Errors: EINVAL (a bad configuration or mixed
 * storage / layout / delta / history_len, nf != 1), ENOMEM, ECUDA. */
int btdf_batch_create(const btdf_config *cfgs, int32_t n, void *stream, btdf_batch **out);
int btdf_batch_destroy(btdf_batch *b);
/* As btdf_init_fields, for lattice `lattice`. */
int btdf_batch_init_fields(btdf_batch *b, int32_t lattice, const double *rho, const double *ux,
                           const double *uy);
/* As btdf_add_markers, for lattice `lattice`; *body_id receives the batch-wide
 * body id. */
int btdf_batch_add_markers(btdf_batch *b, int32_t lattice, int32_t n, const double *X,
                           const double *Y, const double *Ubx, const double *Uby, double ds,
                           double drs, int32_t *body_id);
int btdf_batch_body_count(const btdf_batch *b, int32_t *n);
int btdf_batch_body_lattice(const btdf_batch *b, int32_t body, int32_t *lattice);
/* Collide-stream launch shape: 1 = 4 nodes per lane, 2 = 2 nodes per lane,
 * on a persistent grid whose CTAs own balanced ranges of 8-row units;
 * 3 = 4, 4 = 2 nodes per lane with one unit per CTA (the block scheduler
 * balances the SMs); 0 = default (1).  Results do not depend on it. */
int btdf_batch_tune(btdf_batch *b, int32_t variant);
/* As btdf_autotune, over the batch's launch shapes 1..4; ms[0..4]. */
int btdf_batch_autotune(btdf_batch *b, int32_t steps, int32_t flush_l2, int32_t *chosen, float *ms);
int btdf_batch_step(btdf_batch *b, int64_t nsteps);
int btdf_batch_sync(btdf_batch *b);
int64_t btdf_batch_step_count(const btdf_batch *b);
/* As btdf_read_forces, for a batch-wide body id. */
int btdf_batch_read_forces(btdf_batch *b, int32_t body, int64_t first, int64_t n, double *Fx,
                           double *Fy);
/* As btdf_read_field, for lattice `lattice`. */
int btdf_batch_read_field(btdf_batch *b, int32_t lattice, int32_t kind, float *dst,
                          int32_t dst_is_device);
const char *btdf_batch_last_error(const btdf_batch *b);

/* ---- IB force stage without device allocation ----------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot call cudaMalloc: code that runs inside another framework's memory
 * budget (a caching allocator owns the device memory), or real-time loops
 * that must not enter the driver's allocator.  The call copies its host
 * inputs from pageable memory and synchronizes `stream` before returning.
 *
 * For one body of n markers it runs the IB stage of one step on a population
 * buffer the caller owns: interpolation of rho and u* to the markers
 * (Eqs. 9-10, 12, 14), the force F_b = 2 rho_l (U_b - D_I u*) (Eq. 20) and
 * the force on the body F_p = -sum F_b ds drs in FP64 (Eq. 27).  It uses the
 * same kernel as btdf_step's IB stage.
 *   cfg    lattice description (nx, ny, u_in, delta, storage, bc_x, bc_y,
 *          layout; tau, nf, history_len and g are not used).  cfg->u_in is
 *          the inlet speed the pull's inlet rule extrapolates to.
 *   pops   device pointer to populations in the library's layout: the
 *          storage type, deviations f_a - f_eq_a(1, (u_ref, 0)), rows of
 *          nxp = nx rounded up to 32, planar or row-interleaved per
 *          cfg->layout, aligned to the storage element.  This is the byte
 *          image btdf_save_state writes after its 48-byte header.
 *   pull   0: pops holds post-streaming populations; 1: post-collision ones
 *          (streaming and the boundary rules are applied while reading).  A
 *          checkpoint's header says which (its int32 at byte 24 is 1 for
 *          post-streaming).
 *   u_ref  reference velocity (u_ref, 0) of the stored deviations: the
 *          creation-time u_in of the context that wrote them (a checkpoint's
 *          double at byte 40); it differs from cfg->u_in after
 *          btdf_set_inflow.
 *   X, Y, Ubx, Uby, ds, drs  as in btdf_add_markers (host arrays of n
 *          doubles; Ubx/Uby may be NULL; drs <= 0 takes Sec. 4.4's value).
 *   Fb     device output, 2n floats (F_b per marker, x and y interleaved),
 *          8-byte aligned.
 *   Fp     host output, 2 doubles (force on the body).
 *   stream cudaStream_t to run on (NULL = legacy default stream).
 * No device memory is allocated: the marker tables and the reduction scratch
 * live in one file-scope device array of about 320 KB, which every GPU that
 * loads the library holds until the process exits.  n may not exceed
 * BTDF_STATIC_MAX_MARKERS (EINVAL).  The first call on a device (and the
 * first after its CUDA context was re-created) looks up that array's device
 * address with cudaGetSymbolAddress.  Every call reuses the same array, so
 * calls that overlap on the GPU (two streams, two host threads) race:
 * serialize them.
 * Errors: EINVAL (arguments, n out of range, misaligned Fb or pops), ECUDA,
 * EUNSTABLE (density or force at a marker non-positive or non-finite). */
#define BTDF_STATIC_MAX_MARKERS 2048
int btdf_ib_forces_static(const btdf_config *cfg, const void *pops, int32_t pull, double u_ref,
                          int32_t n, const double *X, const double *Y, const double *Ubx,
                          const double *Uby, double ds, double drs, float *Fb, double *Fp,
                          void *stream);

const char *btdf_last_error(const btdf_ctx *ctx);
const char *btdf_status_string(int status);
int btdf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BTDF_H */
