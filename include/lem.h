/*
 * lem.h -- C ABI of the GB300 (sm_103a) landscape-evolution time step.
 *
 * Implements, on one GPU, the per-timestep method of Barnes, "Accelerating a
 * Landscape Evolution Model with Parallelism" (arXiv:1803.02977), Section
 * "The Algorithm": receivers (Alg 1), donors (Alg 2), the breadth-first
 * queue of levels (Alg 3), flow accumulation (Alg 4, Eq. 2), uplift (Alg 5)
 * and implicit stream-power erosion (Alg 6, Eq. 1: the closed form for
 * n-hat = 1, Newton-Raphson for other exponents), repeated ("Rinse,
 * Repeat").
 *
 * Conventions shared by every entry point
 *  - Grid: width nx, height ny, cell (x, y) at address c = y*nx + x, rows
 *    growing southward (Section "Step 1: Initialization").  Perimeter cells
 *    are fixed base level and never have a receiver.
 *  - Neighbour code k = 0..7 in ascending address order:
 *      0=NW 1=N 2=NE 3=W 4=E 5=SW 6=S 7=SE.
 *  - "No receiver" (NoFlow) is exported as rec[c] = c.
 *  - Pointers named dev_* are CUDA device pointers owned by the caller;
 *    the library never frees them.  Host pointers are named plainly.
 *  - Every call is asynchronous on the context's stream except those that
 *    return a host value computed on the device (lem_levels, lem_sync),
 *    which synchronise that stream.
 *  - Every call returns a status (LEM_OK or a negative LEM_E* code) and
 *    never throws.  Errors found by a kernel (a receiver cycle, a timed-out
 *    device wait, a non-finite elevation) are sticky and reported by the
 *    next synchronising call.
 *  - Elevations must be finite.  Alg 1 checks every value it reads while
 *    computing the receivers of interior cells: a NaN or infinity is
 *    reported as LEM_EINVAL, and lem_step then stops before it changes any
 *    elevation of that step (lem_receivers still writes its outputs).
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef LEM_H
#define LEM_H

#include <stdint.h>

/* Symbols of the shared library are exported explicitly. */
#if defined(__GNUC__)
#define LEM_API __attribute__((visibility("default")))
#else
#define LEM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lem_ctx lem_ctx;

/* Status codes. */
enum {
  LEM_OK = 0,
  LEM_EINVAL = -1,    /* bad argument, or a frozen receiver graph with a cycle */
  LEM_ENOMEM = -2,    /* device allocation failed                              */
  LEM_ECUDA = -3,     /* a CUDA runtime call failed                            */
  LEM_ETIMEOUT = -4,  /* a bounded device-side wait ran out                    */
  LEM_ESTATE = -5,    /* a stage was called before its inputs were computed    */
  LEM_EOVERFLOW = -6, /* grid too large for 32-bit cell addresses              */
  LEM_EBOUNDS = -7    /* an index check of the LEM_DEBUG build failed (the      */
                      /* access was skipped; liblem_debug.so only)              */
};

/* Elevation element types. */
enum { LEM_F64 = 0, LEM_F32 = 1 };

/* Model parameters (Section "Step 1: Initialization"; Eq. 1 with n-hat = 1).
 *  nx, ny      grid width and height, each >= 3, nx*ny < 2^31
 *  dx          cell spacing in metres (dy = dx), > 0
 *  K           erodibility, >= 0 (K = 0 leaves pure uplift)
 *  m           area exponent m-hat, finite
 *  U           uplift rate u-hat in m/yr, finite (Alg 5)
 *  dt          time step in years, > 0
 *  area_scale  drainage area per counted cell: A = count * area_scale in the
 *              erosion factor; <= 0 selects dx*dx (Alg 4 initialises A to
 *              dx*dy)
 *  dtype       LEM_F64 or LEM_F32: element type of the bound elevations.
 *              Receiver slopes are always compared in FP64.
 *  count_bits  32 or 64: integer width of the cell counts (Alg 4). */
typedef struct {
  int nx, ny;
  double dx, K, m, U, dt;
  double area_scale;
  int dtype;
  int count_bits;
} lem_params;

/* Create a context for an nx-by-ny FP64 grid with 32-bit counts and
 * area_scale = dx*dx.  Allocates the context's device scratch (about
 * 15 bytes per cell plus a 1 MiB erosion table) on the current device.
 * On failure *out is set to NULL. */
LEM_API int lem_create(lem_ctx** out, int nx, int ny, double dx, double K, double m, double U,
               double dt);

/* Create a context from a full parameter set (see lem_params). */
LEM_API int lem_create_ex(lem_ctx** out, const lem_params* p);

/* Free the context and its device scratch.  NULL is ignored. */
LEM_API void lem_destroy(lem_ctx* ctx);

/* Issue all later work on `stream` (a cudaStream_t; NULL = legacy default). */
LEM_API int lem_set_stream(lem_ctx* ctx, void* stream);

/* Bind the caller's elevation array: nx*ny elements of `dtype` (which must
 * match the context's), row-major, updated in place by lem_erode/lem_step.
 * Binding invalidates every derived stage. */
LEM_API int lem_bind_elevation(lem_ctx* ctx, void* dev_h, int dtype);

/* Per-cell uplift rate (nx*ny doubles, m/yr) replacing the scalar U of
 * Alg 5 (whose text notes spatially varying uplift stays trivially
 * parallel); NULL restores the scalar. Perimeter entries are ignored. */
LEM_API int lem_set_uplift_field(lem_ctx* ctx, const double* dev_U);

/* Alg 1 (Step 2, Determine Receivers): for each interior cell, the
 * neighbour of greatest strictly positive slope (h[c]-h[n])/dist, lowest k
 * on ties, else NoFlow.  Slopes are compared as (h[c]-h[n])*w in FP64 with
 * w = 1 (cardinal) or the double nearest 1/sqrt(2) (diagonal).  Also
 * computes the donor masks of Alg 2.  If dev_rec is not NULL it receives
 * nx*ny int32 receiver addresses (self = NoFlow).  On a frozen context
 * (lem_set_receivers) the frozen graph is exported instead. */
LEM_API int lem_receivers(lem_ctx* ctx, int32_t* dev_rec);

/* Alg 2 (Step 3, Determine Donors), the inverse of the receivers, over every
 * cell including the perimeter.  dev_dnum (nx*ny int32) receives the donor
 * counts; dev_donor (8*nx*ny int32, Dmax = 8 per cell) receives the donor
 * addresses of cell c at [8c, 8c+dnum[c]) in k order, the rest set to -1.
 * Either pointer may be NULL.  Requires lem_receivers. */
LEM_API int lem_donors(lem_ctx* ctx, int32_t* dev_dnum, int32_t* dev_donor);

/* Alg 3 (Step 4, Generate Queue): breadth-first levels grown from the cells
 * without receivers.  Level 0 lists those cells in ascending address order;
 * level l+1 lists the donors of level l's cells, in queue order, each cell's
 * donors in k order.  *nlevels receives L (synchronises the stream).
 * Optional outputs: dev_queue (nx*ny int32), dev_levels (L+1 int64 offsets,
 * levels[0] = 0, levels[L] = nx*ny; size the buffer nx*ny+1), dev_depth
 * (nx*ny int32, the level of each cell).  Returns LEM_EINVAL if a frozen
 * receiver graph leaves cells unreached (a cycle).  Requires lem_receivers. */
LEM_API int lem_levels(lem_ctx* ctx, int64_t* nlevels, int32_t* dev_queue, int64_t* dev_levels,
               int32_t* dev_depth);

/* Alg 4 (Step 5, Flow Accumulation, Eq. 2 with w = 1): integer cell counts
 * A(c) = 1 + sum of the donors' counts, swept from the highest level down.
 * If dev_counts is not NULL it receives nx*ny counts of the context's
 * count width (int32 or int64).  Requires lem_levels. */
LEM_API int lem_accumulate(lem_ctx* ctx, void* dev_counts);

/* Flow accumulation with multiple flow directions (Section "Multiple Flow
 * Directions"; Eq. 2 with a general split alpha and source w), from the
 * bound elevations.  Receivers of an interior cell are all its strictly
 * lower neighbours (perimeter cells and pits have none); cell d sends
 *     alpha(d -> n_k) = s_k^p / (sum over its receivers of s^p),
 * s_k = (h_d - h_n_k) * w_k with Alg 1's weights (1 cardinal, the double
 * nearest 1/sqrt2 diagonal), the sum in k order (Freeman's slope-weighted
 * split; p = 1 is proportional to slope, large p approaches steepest
 * descent).  Then A(c) = w(c) + sum over the donors d of c, in k order of
 * c's neighbours, of alpha(d -> c) * A(d), in FP64 with each operation
 * rounded separately, every donor before its receivers (Kahn's levels on
 * the donor graph, which multiple flow directions require).  A does not
 * depend on the order of cells within a level; for p = 1 it is bit-exact
 * against a serial evaluation.
 *  p          split exponent, > 0 and finite
 *  dev_w      nx*ny doubles of source w(c), or NULL for 1 per cell (A then
 *             in cells; scale by dx*dx for area)
 *  dev_A      nx*ny doubles receiving A
 *  nlevels    if not NULL, receives the number of levels
 * The D8 stages (receivers, levels, counts, erosion) are not affected.  The
 * first call allocates 16 bytes of scratch per cell.  Synchronises the
 * stream and returns the kernel's status.  LEM_EINVAL for a NULL context
 * or dev_A or a p that is not finite and positive; LEM_ESTATE without bound
 * elevations. */
LEM_API int lem_accumulate_mfd(lem_ctx* ctx, double p, const double* dev_w, double* dev_A,
                               int64_t* nlevels);

/* Alg 5 + Alg 6 (Steps 6-7) for n-hat = 1, fused: interior cells without a
 * receiver are uplifted, h += dt*U; then, level 1 upward, every cell takes
 * h = (h + dt*U + F*h_r) / (1 + F), F = K*dt*(count*area_scale)^m / d,
 * d = dx (cardinal receiver) or dx*sqrt(2) (diagonal), h_r the receiver's
 * updated elevation.  The update is evaluated in the algebraically identical
 * increment form h0 - g*(h0 - h_r), h0 = h + dt*U, g = F/(1+F) from a table
 * computed in FP64 (rounded once to float for FP32 contexts); FP64 results
 * are within a few units in the last place of the closed form.  With a
 * slope exponent other than 1 (lem_set_slope_exponent) each cell's update is
 * Alg 6's Newton-Raphson iteration instead.
 * Updates the bound elevations in place.  Requires lem_accumulate. */
LEM_API int lem_erode(lem_ctx* ctx);

/* "Rinse, Repeat": nsteps full time steps (receivers through erosion) in
 * one cooperative persistent launch with device-wide barriers between
 * levels; no host round trip between levels or steps.  With depression
 * filling on (lem_set_fill) each step is a flood launch and a step launch. */
LEM_API int lem_step(lem_ctx* ctx, int nsteps);

/* Alg 6 (Step 7) for a general slope exponent n-hat (Eq. 1, erosion rate
 * K A^m S^n-hat).  Later lem_erode and lem_step calls solve each eroding
 * cell's implicit update
 *     h - h0 + F (h - h_r)^n = 0,   F = K*dt*(count*area_scale)^m / d^n,
 * h0 = h + dt*U, d = dx or dx*sqrt(2), h_r the receiver's new elevation, by
 * Alg 6's Newton-Raphson iteration from h = h0, in FP64 for either elevation
 * type (FP32 results are rounded once).  The iteration stops once an update
 * changes h by at most eps metres, or after max_iter updates (Alg 6's text
 * allows a fixed count in place of the tolerance test).  A cell whose h0 is
 * not above h_r keeps h0: the power of a non-positive slope is undefined for
 * non-integer n.
 *  n         slope exponent, finite and >= 1.  Then f(h) is convex and
 *            increasing above h_r, so the iterates fall monotonically to the
 *            root and stay above h_r; for n < 1 the first update can cross
 *            below h_r, so n < 1 is rejected.  n = 1 restores the closed
 *            form of lem_erode (the default); eps and max_iter are then
 *            ignored.
 *  eps       tolerance in metres, finite and > 0
 *  max_iter  1 .. 1000
 * Returns LEM_EINVAL for other values.  While n != 1 the step kernel's own
 * instantiation for the general exponent runs, in every tier and stage
 * call, and lem_adjoint returns LEM_EINVAL.  Takes effect at the next
 * launch; no device work. */
LEM_API int lem_set_slope_exponent(lem_ctx* ctx, double n, double eps, int max_iter);

/* Depression filling before Alg 1 (Section "Local Minima": depressions
 * filled to the level of their outlets by Priority-Flood, the flats this
 * leaves resolved as part of the flood).  Replaces the bound elevations, in
 * place, by the least surface w with w >= h, w = h on the perimeter and every
 * interior cell strictly above its lowest neighbour:
 *     w[c] = max(h[c], next representable value above min over the eight
 *            neighbours of w),
 * so that Alg 1 then finds a receiver for every interior cell and all flow
 * reaches the perimeter.  Increments are one unit in the last place of the
 * elevation type (double or float).  The result is unique and bit-exact;
 * elevations must be finite.  One cooperative launch, asynchronous on the
 * context's stream; the first call allocates a scratch of nx*ny elevations
 * and nx*ny int32 plus two bytes per 32 x 32 tile.  LEM_EINVAL for a NULL
 * context, LEM_ESTATE without bound elevations; LEM_ETIMEOUT (reported by
 * the next synchronising call) if a device wait ran out.  Invalidates the
 * derived stages. */
LEM_API int lem_fill(lem_ctx* ctx);

/* With on = 1, every later lem_step step begins with lem_fill (each step is
 * then its own launches); on = 0 (the default) turns it off. */
LEM_API int lem_set_fill(lem_ctx* ctx, int on);

/* Work of the last lem_fill (zeros if none ran; synchronises the stream):
 * stats[0] rounds (grid barriers between tile sweeps), stats[1] tile visits,
 * stats[2] relaxation passes over all visits, stats[3] visits that ran out
 * of passes and were revisited in the next round.  stats holds 4 entries. */
LEM_API int lem_fill_stats(lem_ctx* ctx, int64_t* stats);

/* Freeze the receiver graph: dev_rec (nx*ny int32, self = NoFlow, every
 * other entry an in-grid neighbour, perimeter cells self) replaces Alg 1 in
 * every later stage and step until called again with NULL.  The graph is
 * copied.  Returns LEM_EINVAL for an out-of-range entry (checked on the
 * device; reported by the next synchronising call). */
LEM_API int lem_set_receivers(lem_ctx* ctx, const int32_t* dev_rec);

/* The receiver graph (Alg 1) and donor masks (Alg 2) that the last
 * lem_step step -- or the last lem_receivers call, whichever ran later --
 * computed from its input elevations.  dev_rec (nx*ny int32, self = NoFlow)
 * and dev_mask (nx*ny bytes, bit k set iff neighbour k drains into the cell,
 * k in the neighbour order above) may each be NULL.  Asynchronous;
 * LEM_ESTATE if no step or receivers call has run yet. */
LEM_API int lem_last_graph(lem_ctx* ctx, int32_t* dev_rec, uint8_t* dev_mask);

/* Checkpoint / resume.  A state is a byte blob of *bytes = 32 + nx*ny *
 * (8 or 4) bytes (lem_state_size): a header (format tag, grid size,
 * element type, the number of lem_step steps taken, and whether the device
 * tier's next deep step starts by pointer jumping) followed by the bound
 * elevations.  lem_get_state writes it to buf, lem_set_state copies it back
 * into the bound elevations and restores the step count and the hint, so
 * that the steps after a resume equal, bit for bit, those the saved context
 * would have taken.  buf may be host or device memory (the copies use
 * unified addressing); both calls synchronise the context's stream.
 * LEM_EINVAL for a NULL pointer, a buffer smaller than the state, or (set)
 * a header of another grid or element type; LEM_ESTATE without bound
 * elevations.  The receiver graph, parameters, uplift field and step mode
 * are not part of the state. */
LEM_API int lem_state_size(lem_ctx* ctx, int64_t* bytes);
LEM_API int lem_get_state(lem_ctx* ctx, void* buf, int64_t bytes);
LEM_API int lem_set_state(lem_ctx* ctx, const void* buf, int64_t bytes);

/* Synchronise the context's stream and return the sticky device status
 * (then cleared). */
LEM_API int lem_sync(lem_ctx* ctx);

/* Upper bound, in seconds, on every device-side wait (grid barriers);
 * default 2 s.  A wait that runs out makes its kernel return early with
 * LEM_ETIMEOUT recorded. */
LEM_API int lem_set_wait_limit(lem_ctx* ctx, double seconds);

/* Launch one kernel that waits, bounded by the wait limit, on a device flag
 * that nothing sets; returns LEM_ETIMEOUT once the limit has run out and
 * the context stays usable.  Exercises the timeout path without a fault. */
LEM_API int lem_selftest_wait(lem_ctx* ctx);

/* How lem_step runs Algs 3-6.  Mode 0 (default): the trees are grown,
 * accumulated and eroded privately (the paper's private queues, Section
 * "Independent Parallelism").  The grid is cut into 32x8 tiles; a warp takes
 * the trees rooted in one tile and runs Algs 3-6 on them in its own slice of
 * shared memory with warp barriers only (up to 384 cells and 127 levels with
 * FP64 elevations, 512 cells with FP32).  Trees that do not fit go to their
 * thread block's private queue in global memory (block barriers; up to twice
 * the block's fair share of cells and 2048 levels), and what still does not
 * fit to device-wide levels (one grid barrier per level).  Mode 1:
 * device-wide levels only (the paper's level-synchronous queue).  Both give
 * the same elevations; the integer stages are identical. */
LEM_API int lem_set_step_mode(lem_ctx* ctx, int mode);

/* Work decomposition of lem_step (mode 0), for the package's autotuner.
 *  strip_rows   rows per strip of the codes pass (Algs 1-2; each warp takes
 *               strips of 30 columns): 8, 16 or 32 (32 with FP32 elevations
 *               only), or 0 for the default (32 for FP32 when every warp of
 *               the grid gets two strips, else 16).
 *  half_tiles   1: the warp tier claims every 32-column tile as two
 *               half-height items (8 -> 4 rows with FP64 elevations, 12 -> 6
 *               with FP32); 0 (the default): only the last tiles of a step.
 * Receivers and masks do not depend on either; elevations do not either
 * while no tree needs the device tier's pointer-jumping form (whose sums
 * associate differently, within a few units in the last place).
 * LEM_EINVAL for other values.  lem_get_tiling returns the values in use. */
LEM_API int lem_set_tiling(lem_ctx* ctx, int strip_rows, int half_tiles);
LEM_API int lem_get_tiling(lem_ctx* ctx, int* strip_rows, int* half_tiles);

/* Number of lem_step steps completed without and with device-wide levels
 * since the context was created (synchronises). */
LEM_API int lem_step_stats(lem_ctx* ctx, int64_t* private_steps, int64_t* device_wide_steps);

/* Cells handled by lem_step (mode 0) since the context was created, per
 * tier: cells[0] warp tiles in shared memory, cells[1] block-private queues,
 * cells[2] device-wide levels (synchronises).  cells must hold 3 entries. */
LEM_API int lem_tier_stats(lem_ctx* ctx, int64_t* cells);

/* The device-wide tier's pointer-jumping form (mode 0, n-hat = 1): trees
 * deeper than the device tier's level limit (max(64, nx*ny/2^15)
 * breadth-first levels) are counted by ranking their Euler tours and eroded
 * by composing each cell's affine update along its receivers, in O(log
 * depth) device-wide rounds instead of one per level; once a step needed
 * it, the next step's deep trees go to it directly (and block-private
 * queues hold at most 256 levels).  Counts are exact; elevations are within
 * a few units in the last place of the level-by-level sweep (FP64
 * accumulation for either elevation type).  stats[0]: steps that used it
 * since the context was created; stats[1]: erosion rounds of the latest
 * (synchronises).  The first lem_step in mode 0 allocates its scratch, 44
 * bytes per cell (grids below 2^30 cells). */
LEM_API int lem_jump_stats(lem_ctx* ctx, int64_t* stats);

/* Device-side tracing of the step kernel's timeline: with capacity > 0,
 * later launches record, after every device-wide barrier, the GPU global
 * timer (ns) and a tag (phase << 16 | level); capacity 0 turns tracing off.
 * Tracing costs one store per barrier. */
LEM_API int lem_trace_enable(lem_ctx* ctx, int capacity);

/* Copy up to `cap` recorded entries to host arrays ns[] and tags[] and clear
 * the record (synchronises the stream).  *n receives the number of entries
 * recorded since the last read (entries beyond the capacity are dropped).
 * Tags: 1 start, 2 receivers, 3 level 0, 4 wide level, 5 narrow levels,
 * 6 wide accumulation, 7 narrow accumulation, 8 uplift, 9 wide erosion,
 * 10 narrow erosion, 11-13 block-private levels, accumulation, erosion,
 * 14 step end, 15 block 0 reached a barrier, 16 warp and block tiers done,
 * 17 jumping tier: tour built, 18 one ranking round, 19 counts and factors,
 * 20 one erosion-jumping round, 21 block tier done on every block. */
LEM_API int lem_trace_read(lem_ctx* ctx, int64_t* ns, int32_t* tags, int cap, int* n);

/* Reverse-mode gradient of nsteps time steps (Alg 5 + Alg 6, n-hat = 1)
 * started from dev_h0, for the inverse problems the paper's introduction
 * motivates; the paper itself has no adjoint.  Each step's receiver graph is
 * frozen (its derivative is zero almost everywhere).  With mu the adjoint of
 * a step's output, swept donors first, mu_c = lambda_c + sum over donors d of
 * mu_d F_d/(1+F_d); then dL/dh_c = mu_c/(1+F_c), dL/dU_c += dt mu_c/(1+F_c)
 * and dL/dK += mu_c (h'_r - h'_c)/(1+F_c) dt A_c^m/d_c for eroding cells
 * (pits: mu_c and dt mu_c; perimeter: mu_c).
 *  dev_h0        nx*ny doubles, the run's initial elevations (not modified)
 *  dev_lambda_T  nx*ny doubles, dL/dh after the last step
 *  nsteps        number of steps (>= 1); the context's parameters and uplift
 *                field (lem_set_uplift_field) define them
 *  ckpt_every    the forward is recomputed from a checkpoint kept every
 *                ckpt_every steps; at most ckpt_every+1 states are stored
 *  dev_dLdU      nx*ny doubles receiving dL/dU per cell (zero on the
 *                perimeter)
 *  dLdK          host double receiving dL/dK
 *  dev_lambda_0  optional nx*ny doubles receiving dL/dh0
 * FP64 contexts with 32-bit counts only.  Allocates and frees its
 * checkpoint and segment buffers; synchronises the stream.  The context's
 * elevation binding is restored on return. */
LEM_API int lem_adjoint(lem_ctx* ctx, const double* dev_h0, const double* dev_lambda_T,
                        int nsteps, int ckpt_every, double* dev_dLdU, double* dLdK,
                        double* dev_lambda_0);

/* ---- Many realizations in one launch ------------------------------------
 * The paper motivates its algorithm by the many model realizations that
 * inverse problems and statistical studies need (abstract; Section
 * "Introduction"), and notes that a GPU's spare capacity can process other
 * models simultaneously (Section "GPU Implementation").  A batch holds R
 * independent grids of any sizes and parameters, FP32 elevations packed
 * back to back (realization r at offsets[r] .. offsets[r+1]), and advances
 * all of them in one launch: each thread block claims the largest grid not
 * yet taken and runs its time steps alone with block barriers.  Receivers
 * use FP64 slope tests as in lem_receivers; erosion uses the FP32 increment
 * form with 32-bit cell counts and area = dx*dx. */
typedef struct lem_batch lem_batch;

/* Create a batch of R grids; nx, ny, dx, K, m, U, dt are host arrays of R
 * entries (same meaning and limits as lem_params).  dtype must be LEM_F32.
 * Allocates about 20 bytes of device scratch per cell. */
LEM_API int lem_batch_create(lem_batch** out, int R, const int* nx, const int* ny,
                             const double* dx, const double* K, const double* m,
                             const double* U, const double* dt, int dtype);

/* Free the batch.  NULL is ignored. */
LEM_API void lem_batch_destroy(lem_batch* batch);

/* Host array of R+1 cell offsets of the packed layout (offsets[R] = total). */
LEM_API int lem_batch_offsets(const lem_batch* batch, int64_t* offsets);

/* Issue later work on `stream` (a cudaStream_t; NULL = legacy default). */
LEM_API int lem_batch_set_stream(lem_batch* batch, void* stream);

/* Bind the caller's packed FP32 elevations (offsets[R] floats), updated in
 * place by lem_batch_step. */
LEM_API int lem_batch_bind_elevation(lem_batch* batch, float* dev_h);

/* Kernel shape: threads per block (256, 512 or 1024) and breadth-first
 * entries per thread per round (4 or 8).  Default 1024 x 4.  The package's
 * autotuner picks it by timing; any shape gives the same results. */
LEM_API int lem_batch_set_config(lem_batch* batch, int block_threads, int items_per_thread);

/* Advance every realization by nsteps time steps (asynchronous). */
LEM_API int lem_batch_step(lem_batch* batch, int nsteps);

/* Synchronise the batch's stream; returns LEM_ECUDA if a kernel failed. */
LEM_API int lem_batch_sync(lem_batch* batch);

/* Largest grid (nx*ny cells) accepted by lem_step_noalloc. */
#define LEM_NOALLOC_MAX_CELLS (1 << 18)

/* Allocation-free form of lem_step, for callers that must not allocate
 * device memory -- for instance code embedded in a framework whose caching
 * allocator owns the GPU's memory, or a latency-critical loop where
 * cudaMalloc/cudaFree are off limits because they may block and implicitly
 * synchronise the device.  The paper has no counterpart: this is a
 * deployment convenience around the same step kernel.
 *
 * Runs nsteps FP64 steps (32-bit counts, area = dx*dx, scalar uplift) on the
 * caller's device array dev_h (nx*ny doubles, updated in place) on `stream`
 * (a cudaStream_t, NULL = legacy default), then synchronises that stream and
 * returns the kernel's status.  No context is created and nothing is
 * allocated or freed: the working memory is one fixed array of about 20 MiB
 * in the library's device image, held by every GPU that loads the library
 * until the process exits.
 *  - Grids with nx*ny > LEM_NOALLOC_MAX_CELLS (or nx, ny < 3, or invalid
 *    parameters) are rejected with LEM_EINVAL before any device work, and so
 *    is a dev_h that is not memory of the current device.
 *  - Every device-side wait (grid barriers) is bounded by a fixed 2 s; a
 *    wait that runs out makes the call return LEM_ETIMEOUT.
 *  - The first call on each device looks up the array's device address with
 *    that device current; make that first call before any stream capture.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; each call clears what must start at zero.  Calls that overlap on
 *    the GPU (from two host threads or two streams) race on it: serialise
 *    them. */
LEM_API int lem_step_noalloc(int nx, int ny, double* dev_h, double dx, double K, double m,
                             double U, double dt, int nsteps, void* stream);

/* Static description of a status code. */
LEM_API const char* lem_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* LEM_H */
