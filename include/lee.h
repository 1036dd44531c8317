/*
 * lee.h -- C ABI of the B300 ghost-point IBM / ADE impedance / 2D linearized
 * Euler solver (liblee.so).
 *
 * The library computes the method of "A high-order ghost-point immersed
 * boundary method coupled with auxiliary differential equations for
 * time-domain impedance walls": one 2N-storage Runge-Kutta stage of the LEE
 * (Sec. 2.1 Eq. 1, Sec. 2.2 Eq. DRP_s) coupled to the normal-stencil ghost
 * points (Sec. 3.1, Eqs. ns-rotation .. ns-ghost) and the mass-spring-damper
 * ADE (Sec. 2.5), with the six coupling steps of Sec. 3.2 at every stage.
 *
 * Conventions used by every entry point
 *  - Grid: nx x ny nodes, node (i, j) at x = x0 + i h, y = y0 + j h; c0 = rho0 = 1,
 *    dt = cfl * h.  Lengths and times are physical (same unit as h), so the
 *    impedance R, M, K is in units of rho0 c0 with that length unit.
 *  - Status: every function returns LEE_OK (0) or one of LEE_ERR_*; after an
 *    error lee_last_error() returns a message.  No entry point aborts.
 *  - Memory: the library never allocates device memory.  lee_plan() reports
 *    the device bytes it needs; the caller allocates them (PyTorch in the
 *    Python binding) and passes the pointer to lee_bind().  Host arrays passed
 *    in are copied before the call returns (caller keeps ownership); host
 *    output buffers are caller-owned and must hold the documented number of
 *    elements.
 *  - Streams: all device work is enqueued on the stream given to lee_bind();
 *    entry points that return host data synchronise that stream.
 *  - Thread safety: a context is used by one host thread at a time.
 */
#ifndef LEE_H
#define LEE_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LEE_OK               0
#define LEE_ERR_ARG          1  /* bad argument or call order                        */
#define LEE_ERR_GEOMETRY     2  /* wall geometry not representable on this grid      */
#define LEE_ERR_RANK         3  /* an elliptical cloud is rank deficient at degree 1 */
#define LEE_ERR_ADE_UNSTABLE 4  /* an admittance pole lies outside the RK4 region    */
#define LEE_ERR_BUDGET       5  /* device buffer too small / over budget             */
#define LEE_ERR_CUDA         6  /* a CUDA call failed (message has the CUDA error)   */
#define LEE_ERR_DIVERGED     7  /* field is no longer finite                         */
#define LEE_ERR_TIMEOUT      8  /* a bounded device wait gave up                     */

/* bulk field precision (ghost weights, ghost projections and ADE are FP64 always) */
#define LEE_FP64 0
#define LEE_FP32 1

/* outer boundary treatment per axis */
#define LEE_BC_RADIATION 0      /* one-sided DRP stencils + radiation condition in 3 layers */
#define LEE_BC_PERIODIC  1

/* field selectors */
#define LEE_P 0
#define LEE_U 1
#define LEE_V 2

typedef struct lee_ctx lee_ctx;
typedef struct lee_batch lee_batch;

typedef struct {
    int nx, ny;            /* nodes per axis, >= 8 (radiation) or >= 7 (periodic)  */
    double h;              /* grid spacing, > 0                                    */
    double cfl;            /* dt = cfl * h (c0 = 1), 0 < cfl                        */
    double x0, y0;         /* coordinates of node (0, 0)                            */
    int precision;         /* LEE_FP64 or LEE_FP32                                  */
    int bc_x, bc_y;        /* LEE_BC_RADIATION or LEE_BC_PERIODIC                   */
} lee_grid;

typedef struct {
    long long device_bytes;   /* bytes of device memory lee_bind() needs (256-B aligned) */
    int n_ghost;              /* ghost points (Sec. 3.1)                                 */
    int n_fluid;              /* fluid nodes advanced per stage                          */
    long long n_entries;      /* total cloud entries over all ghosts                     */
    int n_reduced;            /* ghosts whose LSQ degree was lowered below k = 4         */
    int regime;               /* 0 rigid, 1 complex pair, 2 real poles, 3 double pole,
                                 4 rational admittance                                   */
    double dt;                /* time step                                               */
    double ade_amplification; /* max |P(pole dt)| of the RK4 polynomial over the poles  */
    int n_tiles;              /* stencil tiles                                           */
    int n_states;             /* ADE states per ghost: 2 (MSD or rigid wall), N + 2M     */
} lee_sizes;

/* ---- context life cycle ------------------------------------------------- */
/* Create a context for one solve on grid g.  *out receives the handle. */
int lee_create(lee_ctx **out, const lee_grid *g);
/* Destroy a context (does not free the caller's device buffer). */
int lee_destroy(lee_ctx *ctx);
/* Message of the last error on ctx (or of the last lee_create failure if ctx is NULL). */
const char *lee_last_error(const lee_ctx *ctx);

/* ---- geometry and impedance (before lee_plan) -------------------------- */
/* No immersed wall: every node is fluid. */
int lee_set_wall_none(lee_ctx *ctx);
/* Straight wall through (xw, yw) at angle `angle` (radians) to the x-axis; the
 * wall normal n = (-sin angle, cos angle) points into the fluid, i.e. node x is
 * fluid when (x - xw) . n > 0 (Sec. 4.1, App. A). */
int lee_set_wall_line(lee_ctx *ctx, double xw, double yw, double angle);
/* Circular cylinder of radius r (> 3.5 h) centred at (xc, yc): nodes with
 * |x - c| > r are fluid (Sec. 4.2). */
int lee_set_wall_cylinder(lee_ctx *ctx, double xc, double yc, double r);
/* Mass-spring-damper wall Z(s) = M s + R + K/s, M, R, K > 0 (Sec. 2.5).  The
 * three pole regimes (complex pair, two real poles, double pole at
 * R = 2 sqrt(KM)) are all supported. */
int lee_set_impedance(lee_ctx *ctx, double R, double M, double K);
/* Rigid wall, the limit Y -> 0: u_n = 0 and dp/dn = 0 (Sec. 2.4). */
int lee_set_rigid(lee_ctx *ctx);
/* Broadband wall: the rational admittance of Sec. 2.3 (Eq. Yrational)
 *   Y(s) = sum_k A_k / (s - lam_k) + sum_k [q_k / (s - s_k) + conj(q_k) / (s - conj(s_k))],
 * s_k = alpha_k + i beta_k, q_k = B_k + i C_k, advanced by one real state per
 * real pole and two per pair (Eq. ADEgeneral), u_n by Eq. unGeneral.
 *   real   n_real x 2 doubles (lam_k < 0, A_k), host, copied;
 *   pairs  n_pairs x 4 doubles (alpha_k < 0, beta_k > 0, B_k, C_k), host, copied.
 * 1 <= n_real + 2 n_pairs <= 8.  The direct term Y_inf of Eq. Yrational is
 * not supported: with Y_inf != 0 the Neumann datum du_n/dt of Sec. 3.2 step 4
 * needs dp/dt at the boundary point, which the coupling does not provide.
 * The RK4 stability check of lee_plan covers every pole.  LEE_ERR_ARG for
 * counts out of range, a pole off the left half-plane or a non-finite
 * residue.  Before lee_plan.  A batch that holds such an instance runs the
 * general ADE for all its members (two-state walls then agree with their solo
 * runs to rounding instead of bitwise). */
int lee_set_impedance_rational(lee_ctx *ctx, int n_real, const double *real, int n_pairs, const double *pairs);
/* Outer boundary of a non-periodic axis (Secs. 2.2, 4.1, 4.2): the three outer
 * layers use the one-sided 7-point DRP stencils of Tam and Webb (1993) and
 * their radiation condition dq/dt = -(cos th dq/dx + sin th dq/dy + q/(2 rho)),
 * polar about the domain centre, with no damping, as in the paper.  That
 * closure has grid-scale modes that grow by about 0.3% per step, so rounding
 * errors become visible after several thousand steps (sooner in FP32).
 * lee_set_sponge adds, as an opt-in departure from the paper, an absorbing
 * ramp over the `width` outer layers: damping rate
 * (kappa / h) ((width - d) / width)^2 at d < width cells from the nearest
 * non-periodic edge (width 12, kappa 0.04 damp 2% per step at the edge at
 * CFL 0.5).  width = 0 (the default) turns it off.  Before lee_plan;
 * LEE_ERR_ARG for width < 0, kappa < 0 or a ramp wider than half the grid. */
int lee_set_sponge(lee_ctx *ctx, int width, double kappa);

/* ---- plan and bind ------------------------------------------------------ */
/* Tile shape of the FP32 TMA stencil (columns x rows of outputs per tile),
 * before lee_plan; 0, 0 restores the default.  Supported shapes: 128x28,
 * 64x60, 64x40, 64x32 and 64x24 (warp-specialised kernel).  LEE_ERR_ARG for
 * another shape, after lee_plan, or for FP64 / periodic instances (their
 * shared-memory kernel has one shape).  Batch members must share the shape. */
int lee_set_tile(lee_ctx *ctx, int tile_w, int tile_h);
/* Host set-up (Sec. 3.1): mask, ghost set, boundary points, elliptical clouds,
 * FP64 Householder-QR least squares, Lagrange factors, combined weight rows;
 * ADE poles/residues (Sec. 2.5) and the RK4 stability check of the poles.
 * Fills *out.  Returns LEE_ERR_ADE_UNSTABLE if a pole times dt lies outside
 * the RK4 stability region, LEE_ERR_RANK / LEE_ERR_GEOMETRY on bad geometry.
 * Probes (lee_set_probes) must be set before lee_plan. */
int lee_plan(lee_ctx *ctx, lee_sizes *out);
/* Attach caller-owned device memory (dev_ptr, 256-byte aligned, dev_bytes >=
 * sizes.device_bytes) and a cudaStream_t (passed as void*, NULL = legacy
 * default stream).  Uploads the tables, zeroes the fields and ADE state. */
int lee_bind(lee_ctx *ctx, void *dev_ptr, long long dev_bytes, void *stream);

/* ---- initial state and source ------------------------------------------- */
/* Gaussian pulse p = amp exp(-ln2 |x - xs|^2 / w^2), u = v = 0 at fluid nodes
 * (Sec. 4.2); resets ADE states, step counter and probe records. */
int lee_init_pulse(lee_ctx *ctx, double xs, double ys, double amp, double halfwidth);
/* Wave packet of Sec. 4.1 along direction `angle`: s = (x - xs).d,
 * p = amp/2 exp(-alpha^2 s^2) cos(2 pi k s), (u, v) = p d; resets as above. */
int lee_init_packet(lee_ctx *ctx, double xs, double ys, double angle, double amp, double k, double alpha);
/* Harmonic monopole s = amp exp(-ln2 |x - xs|^2 / w^2) sin(omega t) (Sec. 4.3).
 * The time factor enters each stage as its moment over the step, which keeps
 * the four-stage scheme 4th order.  amp = 0 removes the source.  May be called
 * before or after lee_bind. */
int lee_set_monopole(lee_ctx *ctx, double xs, double ys, double amp, double halfwidth, double omega);
/* Overwrite one field (LEE_P/U/V) from a host array of nx*ny doubles (row-major,
 * j slowest).  Values at non-fluid nodes are ignored. */
int lee_write_field(lee_ctx *ctx, int which, const double *host);

/* ---- probes --------------------------------------------------------------- */
/* n pressure probes at (xy[2i], xy[2i+1]), recorded after every step into a
 * device history of `capacity` records (4x4 Lagrange interpolation of degree 3
 * when all 16 nodes are fluid, else the nearest fluid node).  Before lee_plan. */
int lee_set_probes(lee_ctx *ctx, int n, const double *xy, int capacity);
/* Copy the recorded probe history (records x n doubles) to host; *nrec gets the
 * number of records (<= capacity). */
int lee_read_probes(lee_ctx *ctx, double *host, long long *nrec);

/* ---- time stepping ------------------------------------------------------- */
/* Advance nsteps time steps (4 stages each) on the bound stream; asynchronous.
 * Each stage runs the ghost/ADE kernel (steps 1-5 of Sec. 3.2) and the fused
 * stencil + stage-update kernel (step 6).  The first call captures one step in
 * a CUDA graph that later calls replay. */
int lee_step(lee_ctx *ctx, long long nsteps);
/* Wait for the bound stream, then read the instance's status word: returns
 * LEE_ERR_DIVERGED once a ghost pressure, ADE state or probe sample has been
 * non-finite (checked on the device every stage), LEE_ERR_TIMEOUT if a stencil
 * kernel gave up a bounded wait for a tile copy (the step is then incomplete).
 * The status stays set until the state is rewritten (lee_write_state,
 * lee_init_*). */
int lee_sync(lee_ctx *ctx);

/* ---- read back ------------------------------------------------------------ */
/* Field LEE_P/U/V of Q^n as nx*ny doubles (FP32 storage is widened). */
int lee_read_field(lee_ctx *ctx, int which, double *host);
/* Node kinds, nx*ny bytes: 0 solid, 1 fluid, 2 ghost. */
int lee_read_mask(lee_ctx *ctx, unsigned char *host);
/* Stencil tile classes after lee_plan (host arrays; test hook): *tiles_x and
 * *tiles_y receive the tile grid of the plan's tile shape and, when host is
 * not NULL, host receives tiles_x*tiles_y flag words, row-major: bit 0 the
 * tile's outputs meet the three outer layers (band), bit 1 some output is
 * not fluid or lies past the grid, bit 2 the tile meets the absorbing ramp,
 * bit 3 every band node of the tile and every node of its 7-node windows is
 * fluid, bit 5 every node is solid and none is a ghost (inert: no kernel
 * visits it at the ends of a tile column, its values stay zero).  Sec. 3.1
 * defines the node kinds the classes follow.  LEE_ERR_ARG for a NULL context
 * or tile-count pointer, or before lee_plan; host is caller-owned. */
int lee_tile_flags(lee_ctx *ctx, unsigned int *host, int *tiles_x, int *tiles_y);
/* ADE states X^n, n_ghost x n_states doubles, in the ghost order of lee_ghost_info. */
int lee_read_ade(lee_ctx *ctx, double *host);
/* Completed time steps. */
int lee_get_step(lee_ctx *ctx, long long *steps);
/* Acoustic energy 1/2 h^2 sum_fluid (p^2 + u^2 + v^2) of Q^n (FP64 sum). */
int lee_energy(lee_ctx *ctx, double *out);

/* ---- checkpoint ----------------------------------------------------------- */
/* Bytes of a state blob: Q^n at fluid nodes, ADE states, step counter, probes. */
int lee_state_bytes(lee_ctx *ctx, long long *bytes);
int lee_read_state(lee_ctx *ctx, void *host_blob);
int lee_write_state(lee_ctx *ctx, const void *host_blob);

/* Asynchronous variants for streaming use (no synchronisation; the host
 * memory must stay valid until the bound stream has passed the copy; use
 * page-locked memory for overlap).  The blob layout is lee_read_state's. */
int lee_upload_state_async(lee_ctx *ctx, const void *host_blob);
/* Copy probe records [first, first + count) to host asynchronously. */
int lee_download_probes_async(lee_ctx *ctx, double *host, long long first, long long count);

/* ---- test hooks ----------------------------------------------------------- */
/* Ghost g of the plan: target node index (j*nx + i), boundary point, normal,
 * r = d/h, degree m of the normal extrapolation (= the cloud-fit degree,
 * 4 down to 1; a cloud whose nodes lie on one line takes the constant fit,
 * its mean, with m = 1), cloud size. meta = {bpx, bpy, nx, ny, r}. */
int lee_ghost_info(lee_ctx *ctx, int g, int *target, double *meta, int *m, int *ncloud);
/* Cloud of ghost g: node indices and the combined FP64 weight rows
 * w[4*e + {0,1,2,3}] = {L0, w_p, w_d, w_f}; kappa = {kappa_p, kappa_u} such that
 * p_g = w_p.p + kappa_p dp/dn, w_g = w_d.(u.n) + kappa_u w_BP, t_g = w_f.(u.tau),
 * p_BP = L0.p. */
int lee_ghost_weights(lee_ctx *ctx, int g, int *idx, double *w, double *kappa);

/* Steps 4-5 of Sec. 3.2 alone, through the product's ghost kernel: fill the
 * ghost nodes of Q^n from given boundary data instead of the ADE's, with
 * bc[2g] = u.n and bc[2g+1] = dp/dn at the boundary point of ghost g (normal
 * from the wall into the fluid, ghost order of lee_ghost_info; n_ghost x 2
 * host doubles, copied before the call returns).  Fluid nodes, ADE states and
 * the step counter are untouched; synchronises the bound stream.  With exact
 * boundary data of a polynomial field of degree <= 4 the ghost values equal
 * the polynomial (Sec. 3.1).  LEE_ERR_ARG before lee_bind. */
int lee_fill_ghosts_with_bc(lee_ctx *ctx, const double *bc);

/* ---- batches: many instances per launch ---------------------------------- */
/* A batch advances several bound contexts (any sizes, precisions must match)
 * with one ghost launch and one stencil launch per stage over all of them. */
int lee_batch_create(lee_batch **out, int precision);
int lee_batch_destroy(lee_batch *b);
/* Add a bound context; the batch uses the context's own device buffers. */
int lee_batch_add(lee_batch *b, lee_ctx *ctx);
/* Remove a context (at a step boundary). */
int lee_batch_remove(lee_batch *b, lee_ctx *ctx);
/* Device bytes the batch tables need for its current members. */
int lee_batch_plan(lee_batch *b, long long *device_bytes);
/* Attach caller-owned device memory for the batch tables and a stream. */
int lee_batch_bind(lee_batch *b, void *dev_ptr, long long dev_bytes, void *stream);
/* Advance every member nsteps steps. */
int lee_batch_step(lee_batch *b, long long nsteps);
const char *lee_batch_last_error(const lee_batch *b);
/* Wait for the batch stream and copy every member's status word into
 * host[0..n-1] (caller-owned, n = member count, member order = order of
 * lee_batch_add): 0 = healthy, bit 0 = a bounded tile wait gave up (timeout),
 * bit 1 = a ghost, ADE or probe value became non-finite (diverged).  One small
 * gather kernel and one copy; LEE_ERR_ARG if n differs from the member count. */
int lee_batch_status(lee_batch *b, long long *host, int n);
/* Packing of the batch's stencil work: columns of tiles are cut into strips of
 * at most ceil(total tiles / (strips x SMs)) tiles, dealt longest first to the
 * persistent CTAs; more strips balance better, fewer keep more halo rows in
 * L2 down a strip.  strips = 1..64, 0 restores the default (2). */
int lee_batch_set_strips_per_sm(lee_batch *b, int strips);
/* Temporal blocking of stages 1 and 2 (on = 1; 0, the default, turns it off):
 * tiles whose region widened by 3 nodes is fluid, outside the three outer
 * layers and the absorbing ramp, of instances without a source, run both
 * stages in one pass over Q^n (the stage-1 values of the region widened by 4
 * stay in shared memory): 9 words of HBM traffic per node for the two stages
 * instead of 15; the other tiles keep one pass per stage.  The ghost fill
 * between the two stages touches nothing those tiles read, so the results are
 * bitwise those of the unfused stages.  Applies to FP32 batches with the
 * default 64 x 40 warp-specialised stencil, otherwise has no effect.  At a
 * step boundary. */
int lee_batch_set_stage_fusion(lee_batch *b, int on);
/* Where the band nodes (the three outer layers: one-sided DRP rows, Tam-Webb
 * radiation condition, Sec. 2.2 and Sec. 4.1) of an FP32 batch on the
 * warp-specialised stencil are updated, per stage: bit k of stage_mask (k =
 * 2..4) set = inside the stencil's band tiles, from the tile's shared-memory
 * box, stored with the tile's other nodes; clear = by a separate band pass
 * over the global planes after the stencil (stage 1 always: its shared copy
 * of Q^n is the box itself).  Both give bitwise the same values; the
 * separate pass is the faster on large batches.  -1 restores the default (0:
 * the separate pass in every stage; the environment variable LEE_BAND_TILE, a
 * bit mask, overrides it).  LEE_ERR_ARG for bits outside 2..4.  At a step
 * boundary; no effect on other kernels. */
int lee_batch_set_band_in_tile(lee_batch *b, int stage_mask);
/* The stage mask in effect (see lee_batch_set_band_in_tile); LEE_ERR_ARG for
 * a NULL argument. */
int lee_batch_band_in_tile(lee_batch *b, int *stage_mask);
/* Tiles that the fused pass covers and the batch's total tiles (after the
 * members are final; refreshes the batch's tables). */
int lee_batch_fused_tiles(lee_batch *b, long long *fused, long long *total);
/* The latest probe record of every member with probes (record steps-1 of
 * each, Sec. 4 microphones; NaN before the first), members in batch order,
 * each member's probes in its lee_set_probes order, written to host (count
 * doubles; pinned memory keeps the copy asynchronous) by one gather kernel and
 * one copy on the batch stream: it is complete after the stream drains.
 * host = NULL returns the count only.  LEE_ERR_ARG for a NULL batch or count
 * or an unbound batch, LEE_ERR_CUDA if the launch or copy fails. */
int lee_batch_read_latest_probes_async(lee_batch *b, double *host, long long *count);
/* Name of the stencil kernel variant the batch launches (static string; ""
 * before lee_batch_bind or without members). */
const char *lee_batch_stencil_kernel(lee_batch *b);
/* Measurement hook: enqueue only one kernel of stage `stage` (1..4) for every
 * member: what = 0 ghost/ADE kernel, 1 stencil kernel.  Stages 2..4 read and
 * write disjoint buffers, so repeated launches are idempotent. */
int lee_batch_launch(lee_batch *b, int stage, int what);

/* ---- energy without device allocation ----------------------------------- */
/* Maximum grid rows accepted by lee_energy_noalloc (its static scratch). */
#define LEE_NOALLOC_MAX_ROWS 16384
/* Acoustic energy 1/2 h^2 sum (p^2 + u^2 + v^2) over the nodes whose kind is
 * fluid (1), written to *out (one double in device memory), for callers that
 * cannot allocate device memory: their fields live in memory owned by another
 * runtime or pool that hands out pointers but allows no cudaMalloc (nor an
 * allocating library call) on their side.  The paper has no counterpart; this
 * is a library utility.
 *   p, u, v  device arrays of ny rows of `pitch` elements (FP64 or FP32 per
 *            `precision`), mask: ny x pitch bytes (node kinds), nx <= pitch.
 *   stream   cudaStream_t (void*, NULL = legacy default stream); asynchronous.
 * The entry point allocates nothing: its scratch is a static device array of
 * LEE_NOALLOC_MAX_ROWS doubles (128 KiB), held by every GPU that loads the
 * library until the process exits.  ny > LEE_NOALLOC_MAX_ROWS is rejected with
 * LEE_ERR_ARG and a message (lee_last_error(NULL)).  The first call on a
 * device looks up the scratch's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for the life of the process, so make the
 * first call on each device before any stream capture, and do not reset a
 * device (cudaDeviceReset) after its first call: the kept address would then
 * be stale.  All calls share the scratch; each call rewrites every entry it
 * reads, so nothing needs clearing, but calls that overlap on the GPU (two
 * streams, two host threads) race on it.  The summation order is fixed: two
 * calls on the same data give bitwise the same result. */
int lee_energy_noalloc(const void *p, const void *u, const void *v, const unsigned char *mask, int nx, int ny,
                       long long pitch, int precision, double h, double *out, void *stream);

/* ---- measurement ----------------------------------------------------------- */
/* Enqueue on `stream` (cudaStream_t as void*, NULL = legacy default stream) a
 * kernel of `blocks` x 256 threads that issues only FP64 fused multiply-adds:
 * 8 independent chains of `iters` FMAs per thread, i.e. blocks * 256 * 8 *
 * iters FMAs (2 flops each).  `sink` is a device double written only if the
 * arithmetic left its bounded range (never), so the work is not optimised
 * away.  The caller times the launch (CUDA events) to measure the FP64 FMA
 * rate, the bound of the FP64 stencil path.  A measurement utility: the paper
 * has no counterpart.  LEE_ERR_ARG for blocks < 1, iters < 1 or sink NULL. */
int lee_fp64_fma_probe(int blocks, long long iters, double *sink, void *stream);

/* ---- library --------------------------------------------------------------- */
/* Kernel launches enqueued by this process so far (all contexts and batches). */
long long lee_launch_count(void);
/* Version string. */
const char *lee_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LEE_H */
