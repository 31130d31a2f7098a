/*
 * mwdg_adjoint.h -- C ABI of the discrete adjoint of the DG2 step on a
 * uniform grid and on a frozen non-uniform grid (static graded, or MWDG2
 * held fixed over a segment; mwdg_adj_create_frozen) (GB300, sm_103a; FP64
 * and FP32).
 *
 * The step is the DG2 shallow-water step of Sharifian & Kesserwani, arXiv
 * 2107.02750, Sect. 2.1.1 (Eq. 1-4) on a uniform grid of nx x ny cells:
 * rain depth and split implicit Manning friction at the start of the step,
 * stage-input limiting (partial-wet reduction, minmod), hydrostatic face
 * revision and HLL fluxes, two RK2 stages with the positivity clip, the
 * time step from the CFL condition (Courant number cfl).  The same step as
 * mwdg.h's uniform mode in FP64, rounded the same way.
 *
 * The adjoint is the derivative of a run of K such steps,
 *   U_K = S_{dt_K} o ... o S_{dt_1}(U_0; z, n, Q),
 * with the time steps held at the values recorded by the forward run (a
 * perturbation of the parameters does not move dt), and every branch (wet
 * or dry, reduced, minmod selection, HLL region, clip) as the forward run
 * took it.  At an interface whose two bed limits agree to within
 * 1e-10 max(1, |z_L|, |z_R|) the derivative of max(z_L, z_R) is split in
 * halves between the sides (the mean of the one-sided derivatives).  Where
 * the step is not differentiable (still water, where the limiter's
 * differences vanish) the derivative is that of the branch taken.
 *
 * Precision (mwdg_adj_params.precision): MWDG_F64 runs every cell in FP64
 * and reproduces the solver's FP64 step bit for bit; MWDG_F32 runs the cells
 * in FP32 (depth form) with time, time steps, the hydrograph and its
 * gradient in FP64.  "Coefficient arrays" below are double for MWDG_F64 and
 * float for MWDG_F32; time steps, knots and gQ are double in both.
 *
 * Layout (device memory, caller-owned):
 *   U   9 x n coefficient array, component-major: component m of cell
 *       k = j nx + i at U[m n + k]; components (h0, h1x, h1y, qx0, qx1x, qx1y, qy0, qy1x,
 *       qy1y), the average and the two scaled-Legendre slope coefficients
 *       of depth and unit discharges (Eq. 2-3);
 *   z   3 x n, the bed planes (z0, z1x, z1y) in the same layout;
 *   n   n Manning coefficients;
 *   knot_t, knot_Q  the inflow hydrograph, piecewise linear, constant
 *       outside its knots (nknots >= 1 when an inflow edge is set);
 *   dts K time steps; vertex rasters (ny+1) x (nx+1), row j south to north.
 * Rows run south to north, columns west to east; edges 0 W, 1 E, 2 S, 3 N.
 *
 * Work is queued on the given CUDA stream (NULL: the legacy default stream);
 * no call synchronises it, except mwdg_adj_create and mwdg_adj_destroy.  A
 * context holds a tape of max_steps + 1 states (9 n coefficients each), with
 * tape_views 42 n more per step, and about 100 n coefficients of work
 * arrays; one host thread uses it at a time, and its calls on one stream run
 * in order.  Statuses are those of mwdg.h.
 */
#ifndef MWDG_ADJOINT_H
#define MWDG_ADJOINT_H

#include <stdint.h>

#include "mwdg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mwdg_adj mwdg_adj;

typedef struct {
  int32_t nx, ny;          /* cells                                          */
  double dx;               /* cell size (m)                                  */
  double g, h_dry;         /* gravity, dry-depth tolerance                   */
  double cfl, dt_max;      /* Courant number (0.33 for DG2), dt bound        */
  int32_t limiter;         /* 0 off, 1 minmod                                */
  int32_t bc[4];           /* MWDG_WALL / MWDG_OPEN per edge W, E, S, N      */
  int32_t inflow_edge;     /* -1 none, else the edge carrying the hydrograph */
  int32_t inflow_c0, inflow_c1; /* cells along that edge, inclusive          */
  double rain_rate, rain_t_end; /* m/s while t < rain_t_end                  */
  int32_t max_steps;       /* tape capacity: steps per forward/backward call */
  int32_t precision;       /* MWDG_F64 or MWDG_F32                           */
  int32_t tape_views;      /* 1: the tape also keeps each step's two stage   */
                           /* inputs and flux views (42 n coefficients per   */
                           /* step more), so the reverse sweep recomputes    */
                           /* nothing; 0: it recomputes them step by step    */
} mwdg_adj_params;

/* Defaults: g = 9.80665, h_dry = 1e-3, cfl = 0.33, dt_max = 1, limiter on,
 * walls, no inflow, no rain, max_steps = 200, FP64, tape of states only;
 * nx, ny, dx must be set. */
MWDG_API mwdg_status mwdg_adj_params_default(mwdg_adj_params *p);

/* Allocates the context on the current device.  MWDG_ERR_DIMS when nx or ny
 * < 1, nx ny > 2^28, dx <= 0 or max_steps < 1; MWDG_ERR_ARG on a bad edge,
 * inflow range or parameter; MWDG_ERR_CUDA when the allocation fails. */
MWDG_API mwdg_status mwdg_adj_create(const mwdg_adj_params *p, mwdg_adj **out);

/* The adjoint on a frozen non-uniform grid: a static graded grid (mode
 * MWDG_STATIC, Sect. 2.2.1) or an MWDG2 grid held fixed over the segment
 * (MWDG_ADAPTIVE, Sect. 2.3).  M x N roots, L levels below them; p->nx =
 * M 2^L, p->ny = N 2^L and p->dx describe the finest level (p->inflow_c0,
 * c1 in finest cells).  The n_leaves active leaves are (level[q], i[q],
 * j[q]) (host arrays, read during the call): level 0..L, column i west to
 * east and row j south to north among the level's (M 2^l) x (N 2^l) nodes.
 * They must tile the domain (every finest cell under exactly one leaf),
 * else MWDG_ERR_ARG; MWDG_ERR_DIMS when nx, ny disagree with M, N, L.
 *
 * The step is the DG2 step of mwdg_adj_create on the leaves, each with its
 * own cell size, with the interface rule of the grid's kind: a leaf reads
 * across each face the view of the same-level node there -- a leaf's flux
 * view, a coarser leaf's planes prolonged to that level (Eq. 10 with zero
 * details), a refined node's leaves encoded up to it (Eq. 9; MWDG2) or on a
 * static grid the mean of the face limits of its two children on the face.
 * Limiting uses same-level leaf neighbours only; the bed of a level is the
 * encoding of the finest bed planes (Eq. 9), Manning's n the mean of the
 * children's.  No regridding: it is the map that the adaptive solver's
 * steps follow between two adaptations.
 *
 * With such a context, mwdg_adj_forward and mwdg_adj_backward take U0,
 * U_out, gU_K and gU0 as 9 x n_leaves coefficient arrays (component m of
 * leaf q at [m n_leaves + q], leaves in the order given here) and z, n, gz,
 * gn on the finest level (3 x nx ny and nx ny) as before; the dts are the
 * CFL steps over the leaves or given ones.  The tape and work arrays cover
 * every node of every level (4/3 nx ny at most). */
MWDG_API mwdg_status mwdg_adj_create_frozen(const mwdg_adj_params *p, int32_t M, int32_t N, int32_t L,
                                            int32_t mode, int64_t n_leaves, const int32_t *level,
                                            const int32_t *i, const int32_t *j, mwdg_adj **out);
MWDG_API void mwdg_adj_destroy(mwdg_adj *a);

/* Eq. 8: vertex raster (ny+1) x (nx+1), double -> planes out (3 x n
 * coefficient array), on the device; computed in FP64. */
MWDG_API mwdg_status mwdg_adj_project(mwdg_adj *a, const double *vert, void *out, void *cuda_stream);

/* Forward run of `steps` steps from U0 at time t0 (all device pointers).
 * fixed_dt = 0: each dt from the CFL condition, written to dts[0..steps);
 * fixed_dt = 1: the steps dts[0..steps) are read.  U_out receives U_K (it
 * may alias U0).  MWDG_ERR_CAPACITY when steps > max_steps; MWDG_ERR_ARG on
 * NULL pointers (dts may be NULL when steps = 0), steps < 0, or nknots < 1
 * with an inflow edge. */
MWDG_API mwdg_status mwdg_adj_forward(mwdg_adj *a, const void *U0, const void *z, const void *n,
                                      int32_t nknots, const double *knot_t, const double *knot_Q, double t0,
                                      int32_t steps, int32_t fixed_dt, double *dts, void *U_out,
                                      void *cuda_stream);

/* Vector-Jacobian product of the run over the time steps dts[0..steps) from
 * U0 at t0: given gU_K (9 x n), the cotangent of U_K, writes gU0 (9 x n)
 * and ADDS to gz (3 x n), gn (n) and gQ (nknots), so that gradients of
 * several segments accumulate.  With reuse_tape = 0 the run's states are
 * recomputed from U0 into the tape (the segment's checkpoint is U0 itself).
 * reuse_tape = 1 states that the tape still holds this run: the last
 * forward call on the context ran these steps from the same U0, z, n,
 * knots, t0 and time steps, none of which changed since (no check is made
 * beyond the number of steps: MWDG_ERR_STATE when it differs).  gU0 may
 * alias gU_K.  Other errors as mwdg_adj_forward. */
MWDG_API mwdg_status mwdg_adj_backward(mwdg_adj *a, const void *U0, const void *z, const void *n,
                                       int32_t nknots, const double *knot_t, const double *knot_Q, double t0,
                                       int32_t steps, const double *dts, const void *gU_K, void *gU0,
                                       void *gz, void *gn, double *gQ, int32_t reuse_tape, void *cuda_stream);

/* Regridding at a checkpoint between two frozen MWDG2 grids (contexts of
 * mwdg_adj_create_frozen with the same M, N, L and precision): the state
 * transfer of the MWDG2 adaptation (Sect. 2.3) with its decision -- the new
 * grid, `to` -- held.  The old grid's state is prolonged below its leaves
 * (Eq. 10 with zero details; a depth plane's slopes are first scaled about
 * its average so that no child's average depth is negative, the scaling
 * limiter of Zhang & Shu 2010, and a child's rounding residue below zero
 * is set to zero) and encoded up its refined nodes (Eq. 9); each leaf of
 * the new grid takes the coefficients of its node: kept, coarsened or
 * refined.  U_from is 9 x (from's leaves), U_to 9 x (to's leaves).  The
 * transpose takes U_from too (the scaling's branches are recomputed from
 * it) and overwrites gU_from with the cotangent of U_from given gU_to.
 * Both use from's work arrays (not during a call on from).  MWDG_ERR_ARG on
 * a uniform context, NULL pointers or mixed precisions; MWDG_ERR_DIMS when
 * the grids differ in roots or levels. */
MWDG_API mwdg_status mwdg_adj_regrid(mwdg_adj *from, mwdg_adj *to, const void *U_from, void *U_to,
                                     void *cuda_stream);
MWDG_API mwdg_status mwdg_adj_regrid_transpose(mwdg_adj *from, mwdg_adj *to, const void *U_from,
                                               const void *gU_to, void *gU_from, void *cuda_stream);

/* Transpose of Eq. 8: plane cotangents (3 x n) -> vertex cotangents
 * ((ny+1) x (nx+1)), both coefficient arrays, overwritten. */
MWDG_API mwdg_status mwdg_adj_project_transpose(mwdg_adj *a, const void *g_planes, void *g_vert,
                                                void *cuda_stream);

/* Per-kernel timing.  mwdg_adj_profile(a, L) with L > 0 records a pair of
 * CUDA events around each of the next L launch groups (a group is one
 * kernel, or the two interface kernels of a stage); L = 0 stops recording.
 * It synchronises the device.  mwdg_adj_kernel_times waits for the recorded
 * events, writes per class the summed milliseconds and the number of
 * groups, and starts a new recording.  Classes, in order: */
enum {
  MWDG_ADJ_KC_CFL = 0,      /* CFL reduction and dt                         */
  MWDG_ADJ_KC_FRICTION,     /* rain and friction                            */
  MWDG_ADJ_KC_LIMIT,        /* stage-input limiting                         */
  MWDG_ADJ_KC_UPDATE,       /* RK2 stage update                             */
  MWDG_ADJ_KC_REV_FACE,     /* reverse: x and y interfaces                  */
  MWDG_ADJ_KC_REV_KNOTS,    /* reverse: hydrograph knots                    */
  MWDG_ADJ_KC_REV_LIMIT,    /* reverse: limiter                             */
  MWDG_ADJ_KC_REV_GATHER,   /* reverse: limiter's neighbour terms           */
  MWDG_ADJ_KC_REV_FRICTION, /* reverse: friction                            */
  MWDG_ADJ_KC_COUNT
};
MWDG_API mwdg_status mwdg_adj_profile(mwdg_adj *a, int32_t max_launches);
MWDG_API mwdg_status mwdg_adj_kernel_times(mwdg_adj *a, double *ms, int64_t *count);

/* Description of the context's most recent failure ("" if none). */
MWDG_API const char *mwdg_adj_last_error(const mwdg_adj *a);

#ifdef __cplusplus
}
#endif

#endif /* MWDG_ADJOINT_H */
