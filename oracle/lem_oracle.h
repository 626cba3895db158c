/*
 * lem_oracle.h -- serial FP64 statement of the landscape-evolution time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct CPU
 * restatement of Barnes, "Accelerating a Landscape Evolution Model with
 * Parallelism" (arXiv:1803.02977) against which the CUDA library is checked.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or constant generator with
 * the CUDA library; the two are written independently from the paper.
 *
 * Grid convention (Section "Step 1: Initialization"): a cell at column x and
 * row y of a width-by-height raster has address c = y*width + x.  Rows grow
 * southward.  Perimeter cells are fixed base level and have no receiver.
 *
 * Neighbour code k = 0..7 walks the 3x3 window in ascending address order:
 *   k : 0=NW 1=N 2=NE 3=W 4=E 5=SW 6=S 7=SE
 * Cardinal k in {1,3,4,6}; diagonal k in {0,2,5,7}.
 *
 * "No receiver" (NoFlow) is stored as rec[c] = c.
 *
 * Parity status of every function is recorded beside it.
 */
#ifndef LEM_ORACLE_H
#define LEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double dx;          /* grid spacing (dy = dx), metres                      */
  double K;           /* erodibility, 1/yr                                   */
  double m;           /* area exponent m-hat of Eq. 1                        */
  double U;           /* uplift rate u-hat (used when Ufield == NULL), m/yr  */
  double dt;          /* time step, yr                                       */
  double area_scale;  /* A = count * area_scale (dx*dy = Alg 4's init)      */
  const double* Ufield; /* optional per-cell uplift rate, length width*height */
} orc_params;

/* Alg 1 (Step 2, Determine Receivers).  Steepest descent with strict '>'
 * against an initial maximum slope of zero; ties keep the lowest k.
 * Slope is evaluated divide-free as (h[c]-h[n]) * w_k, w = 1 (cardinal) or
 * the double nearest 1/sqrt(2) (diagonal): the common factor 1/dx does not
 * change the argmax.  Pinned: exact-rational argmax on integer-valued grids,
 * near-argmax on real grids, descent and acyclicity invariants. */
void orc_receivers(int nx, int ny, const double* h, int32_t* rec);

/* Alg 1 on FP32 elevations: each value is promoted to double first and the
 * same expression as orc_receivers is used. */
void orc_receivers_f32(int nx, int ny, const float* h, int32_t* rec);

/* Alg 2 (Step 3, Determine Donors) on the grid, looping over every cell
 * (perimeter included) and its in-grid neighbours in k order.
 * donor has 8 entries per cell (Dmax = 8); dnum[c] of them are used.
 * Pinned: exact inverse of rec; Table 1 through orc_donors_graph. */
void orc_donors_grid(int nx, int ny, const int32_t* rec, int32_t* dnum, int32_t* donor);

/* Alg 2 on a general graph of n nodes (used for the worked example of
 * Table 1): donors of c are the nodes n != c with rec[n] == c, in ascending
 * node order.  donor has dmax entries per node. Returns 0, or -1 if a node
 * has more than dmax donors. */
int orc_donors_graph(int n, const int32_t* rec, int dmax, int32_t* dnum, int32_t* donor);

/* Alg 3 (Step 4, Generate Queue), breadth first.  Level 0 holds every cell
 * with rec[c] == c in ascending address order; level l+1 holds, for each
 * cell of level l in queue order, its donors in stored order.  Levels
 * (length >= n+1) receives L+1 offsets with Levels[0] = 0; depth[c] receives
 * the level of c (or -1 if c is never reached, which only a cyclic rec can
 * cause).  Returns L, the number of non-empty levels.
 * Pinned: Table 1; depth invariants on brute-force grids. */
int64_t orc_queue(int64_t n, const int32_t* rec, int dmax, const int32_t* dnum,
                  const int32_t* donor, int32_t* queue, int64_t* levels, int32_t* depth);

/* Alg 4 (Step 5, Flow Accumulation) with w(c) = 1 and alpha in {0,1}
 * (Eq. 2 for D8): integer cell counts, swept from level L-2 down to 0,
 * indexing cells through the queue.  Pinned: Table 1; brute-force path
 * counting; sum over sinks equals n. */
void orc_accumulate(int64_t n, const int32_t* queue, const int64_t* levels, int64_t nlevels,
                    int dmax, const int32_t* dnum, const int32_t* donor, int64_t* cnt);

/* Alg 5 (Step 6, Uplift): h[c] += U_c * dt on interior cells. */
void orc_uplift(int nx, int ny, double* h, const orc_params* p);

/* Alg 6 (Step 7, Calculate Erosion) for n-hat = 1, where one Newton step
 * from h0 is exact: h = (h0 + F*h_r) / (1 + F),
 * F = K*dt*A^m / d,  A = cnt*area_scale, d = dx (cardinal) or dx*sqrt(2).
 * Levels 1..L-1 ascending, each cell using its receiver's updated value.
 * h must already hold the uplifted elevations (call orc_uplift first).
 * Pinned: dense linear solve of the implicit system on tiny grids; closed-form
 * steady state of a 1-D channel; K = 0 and U = 0 special cases. */
void orc_erode(int nx, int ny, double* h, const int32_t* rec, const int32_t* queue,
               const int64_t* levels, int64_t nlevels, const int64_t* cnt, const orc_params* p);

/* Alg 6 for general n-hat: the Newton-Raphson iteration of Alg 6 from
 * h_new = h0 until |delta| <= eps or max_iter iterations, with
 * F = K dt A^m / dist^n-hat.  For n-hat = 1 it reaches the closed form after
 * one step (up to rounding).  Reading: a cell whose uplifted elevation h0 is
 * not above its receiver's new elevation keeps h0 (the power of a
 * non-positive slope is undefined for non-integer n-hat; with a uniform
 * uplift this never happens, since the sweep preserves strict descent).
 * Pinned: n-hat = 1 agreement with orc_erode; n-hat = 2 against the root of
 * the quadratic at every cell; one iteration against one Newton update
 * written out; the 1-D channel steady state (slope/d)^n = U/(K A^m) for
 * n-hat = 1.5 and 3; residual of the implicit equation at every cell. */
void orc_erode_newton(int nx, int ny, double* h, const int32_t* rec, const int32_t* queue,
                      const int64_t* levels, int64_t nlevels, const int64_t* cnt,
                      const orc_params* p, double n_exp, double eps, int max_iter);

/* Flow accumulation with multiple flow directions (Section "Multiple Flow
 * Directions"; Eq. 2 with general alpha and w).  Receivers of an interior
 * cell are all its strictly lower neighbours (perimeter cells and pits have
 * none); cell c sends the fraction alpha(c -> n_k) = s_k^p / sum of s^p over
 * its receivers (sum in k order), s_k = (h_c - h_n_k) * w_k as in Alg 1
 * (Freeman's slope-weighted split; p = 1 is proportional to slope).
 * A(c) = w(c) + sum over its donors d, in k order, of alpha(d -> c) * A(d);
 * w NULL means w = 1.  Cells are taken level by level: level 0 are the cells
 * without donors, a cell joins the level after its last donor's (Kahn's
 * order on the donor graph, which the paper's figure on multiple flow
 * directions requires: all of a cell's donors before it).  level (optional)
 * receives each cell's level.  Returns the number of levels, or -1 on
 * allocation failure.
 * Pinned: dense linear solve (I - M^T) A = w on tiny grids; mass balance
 * (the A of cells without receivers sum to the sum of w); a hand-computed
 * 3x3 example; the level of every cell is one more than its deepest
 * donor's. */
int64_t orc_accumulate_mfd(int nx, int ny, const double* h, const double* w, double p,
                           double* A, int32_t* level);

/* Depression filling before Alg 1 (Section "Local Minima": fill depressions
 * to their outlets by Priority-Flood, resolving the resulting flats as part
 * of the flood).  w receives the least surface with w >= h, w = h on the
 * perimeter, and every interior cell strictly above its lowest neighbour:
 *     w[c] = max(h[c], next double above min over the 8 neighbours of w),
 * so Alg 1 on w finds a receiver for every interior cell.  Elevations must
 * be finite.  Priority-Flood with one priority queue (ties by address).
 * Returns 0, or -1 on allocation failure.
 * Pinned: the fixed-point equation at every cell; Bellman-Ford relaxation
 * on tiny grids; hand-computed nested basins; no interior sink remains;
 * a surface already draining to the perimeter is unchanged. */
int orc_fill_eps(int nx, int ny, const double* h, double* w);

/* The same for FP32 elevations: w and its increments in float (next float
 * above). */
int orc_fill_eps_f32(int nx, int ny, const float* h, float* w);

/* "Rinse, Repeat": nsteps full time steps in place on h.  If frozen_rec is
 * non-NULL it replaces Alg 1 in every step.  If nlevels_out is non-NULL it
 * receives L for each step.  Returns 0, or -1 on allocation failure. */
int orc_run(int nx, int ny, double* h, int nsteps, const orc_params* p,
            const int32_t* frozen_rec, int64_t* nlevels_out);

/* Adjoint of one n-hat = 1 step over its frozen graph (not in the paper;
 * the exact transpose of the step's linearisation in h, U and K).
 *   h_next     : the step's output elevations
 *   lam        : dL/dh_next (in), overwritten by nothing
 *   lam_prev   : receives dL/dh_prev through this step
 *   dLdU       : accumulated (+=) per-cell gradient wrt the uplift rate
 *   dLdK       : accumulated (+=) gradient wrt K
 * The graph arguments are those the step computed from its input h.
 * Pinned: dot-product test against the tangent-linear step and central
 * finite differences of orc_run. */
void orc_adjoint_step(int nx, int ny, const double* h_next, const int32_t* rec,
                      const int32_t* queue, const int64_t* levels, int64_t nlevels,
                      const int64_t* cnt, const orc_params* p, const double* lam,
                      double* lam_prev, double* dLdU, double* dLdK);

/* Tangent-linear of one n-hat = 1 step over its frozen graph: given
 * perturbations dh (of the input), dU (per cell) and dK, returns dh_next.
 * h_next is the step's output.  Used to pin the adjoint. */
void orc_tangent_step(int nx, int ny, const double* h_next, const int32_t* rec,
                      const int32_t* queue, const int64_t* levels, int64_t nlevels,
                      const int64_t* cnt, const orc_params* p, const double* dh,
                      const double* dU, double dK, double* dh_next);

#ifdef __cplusplus
}
#endif
#endif
