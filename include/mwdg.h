/*
 * mwdg.h -- C ABI of the GB300 (sm_103a) DG2 / multiwavelet-MRA flood solver.
 *
 * Method: Sharifian & Kesserwani, "Benchmarking (multi)wavelet-based dynamic
 * and static non-uniform grid solvers for flood inundation modelling",
 * arXiv 2107.02750.  Every computation behind these calls runs in CUDA
 * kernels of this library on one GPU; there is no CPU fallback.
 *
 * Conventions
 *  - SI units.  Rasters are row-major with row j running south to north and
 *    column i west to east.  A grid has nx = M 2^L by ny = N 2^L finest
 *    cells of size dx (Sect. 2.2); vertex rasters are (ny+1) x (nx+1).
 *  - Host pointers are owned by the caller and only read or written during
 *    the call (the data are copied).  Functions with the _dev suffix take
 *    device pointers that must stay valid until the work queued on
 *    params.cuda_stream has finished; the caller keeps ownership.
 *  - All device work is queued on params.cuda_stream (NULL: the legacy
 *    default stream).  Functions that return host data synchronise it.
 *    An adaptive context also owns a second stream: within each step the
 *    encode's coarsest levels run there, forked from params.cuda_stream
 *    by an event and joined back before the step continues, so work the
 *    caller orders on params.cuda_stream (or captures from it into a graph)
 *    stays ordered after the whole step.
 *  - Every function returns an mwdg_status; nothing throws or aborts across
 *    the boundary.  After MWDG_ERR_CUDA or MWDG_ERR_NONFINITE the context is
 *    in an error state: later calls on it return MWDG_ERR_STATE.
 *    mwdg_last_error() describes the most recent failure.
 *  - A context is used by one host thread at a time.
 */
#ifndef MWDG_H
#define MWDG_H

#include <stdint.h>

#if defined(__GNUC__)
#define MWDG_API __attribute__((visibility("default")))
#else
#define MWDG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mwdg_ctx mwdg_ctx;

typedef enum {
  MWDG_OK = 0,
  MWDG_ERR_ARG = -1,       /* invalid argument or NULL pointer            */
  MWDG_ERR_DIMS = -2,      /* sizes inconsistent with nx = M 2^L etc.     */
  MWDG_ERR_CUDA = -3,      /* a CUDA call failed                          */
  MWDG_ERR_NONFINITE = -4, /* non-finite input value or state             */
  MWDG_ERR_TIMEOUT = -5,   /* a bounded device wait ran out               */
  MWDG_ERR_STATE = -6,     /* call not valid in the current state         */
  MWDG_ERR_CAPACITY = -7   /* caller buffer or fixed capacity too small   */
} mwdg_status;

/* grid modes: uniform DG2 on the finest grid; static non-uniform DG2 on the
 * graded grid from one MRA of the topography (Sect. 2.2, 2.2.1); adaptive
 * MWDG2 with the MRA of flow and topography at every step (Sect. 2.3) */
enum { MWDG_UNIFORM = 0, MWDG_STATIC = 1, MWDG_ADAPTIVE = 2 };
/* arithmetic: FP64 coefficients (depth form), or FP32 coefficients in
 * free-surface form eta = h + z with FP64 time, volume sums and
 * detail-threshold comparisons */
enum { MWDG_F64 = 0, MWDG_F32 = 1 };
enum { MWDG_WALL = 0, MWDG_OPEN = 1 };
enum { MWDG_WEST = 0, MWDG_EAST = 1, MWDG_SOUTH = 2, MWDG_NORTH = 3 };
/* flux through a face between a leaf and a finer (refined) neighbour on a
 * static grid: PAPER, each side from its own same-level view (Sect. 2.2.1;
 * exactly well-balanced, mass moves at round-off only on homogeneous
 * faces); REFLUX, the coarse side takes the mean of the two fine leaves'
 * fluxes through their halves of the face (mass conserved to round-off,
 * lake at rest no longer exact at those faces).  Adaptive grids use PAPER. */
enum { MWDG_IFACE_PAPER = 0, MWDG_IFACE_REFLUX = 1 };
/* scheme: DG2 (piecewise planar, RK2, Sect. 2.1.1) or FV1 (piecewise
 * constant, forward Euler, Eq. 5-7, Sect. 2.1.2; Courant number 0.5).  On an
 * adaptive grid FV1 is HWFV1: the MRA uses Haar wavelets on the averages
 * (Sect. 2.3); a static FV1 grid comes from the multiwavelet MRA of the
 * planar topography like DG2's (Sect. 2.2).  ACC is the local inertial
 * solver (Sect. 2.1.3; Courant number 0.7) on uniform and static graded
 * grids: depth per element, a discharge per interface with semi-implicit
 * Manning resistance, the finer half-face discharges summed on a coarser
 * element (Sect. 2.2.1); open edges carry the discharge through. */
enum { MWDG_DG2 = 0, MWDG_FV1 = 1, MWDG_ACC = 2 };
#define MWDG_LMAX 15

typedef struct {
  int32_t M, N, L;     /* coarsest grid and maximum refinement level        */
  int32_t mode;        /* MWDG_UNIFORM / MWDG_STATIC / MWDG_ADAPTIVE        */
  int32_t precision;   /* MWDG_F64 / MWDG_F32                               */
  int32_t limiter;     /* 0 off, 1 minmod slope limiter                     */
  int32_t bc[4];       /* per edge (west, east, south, north): wall / open  */
  int32_t iface_rule;  /* static grids: MWDG_IFACE_PAPER or MWDG_IFACE_REFLUX */
  int32_t scheme;      /* MWDG_DG2, MWDG_FV1, MWDG_ACC (cfl 0.33, 0.5, 0.7) */
  double dx;           /* finest resolution R (m)                           */
  double eps;          /* MRA threshold (Sect. 2.2; 1e-3 recommended)      */
  double cfl;          /* Courant number (0.33 for DG2, Sect. 2.1.1)        */
  double g;            /* gravity (m/s^2)                                   */
  double h_dry;        /* dry-depth tolerance (m)                           */
  double dt_max;       /* upper bound on the time step (s)                  */
  void *cuda_stream;   /* cudaStream_t for all device work                  */
} mwdg_params;

/* Fills defaults: M=N=1, L=0, uniform, FP64, minmod, walls, PAPER interface
 * rule, dx=1, eps=1e-3, cfl=0.33, g=9.80665, h_dry=1e-3, dt_max=1, default
 * stream. */
MWDG_API mwdg_status mwdg_params_default(mwdg_params *p);

/* Creates a context and allocates its device memory (dense per-level
 * coefficient pyramids, about 4/3 of the finest grid per array).
 * MWDG_ERR_DIMS if L > MWDG_LMAX, M or N < 1, or dx <= 0. */
MWDG_API mwdg_status mwdg_create(const mwdg_params *p, mwdg_ctx **out);
MWDG_API void mwdg_destroy(mwdg_ctx *ctx);

/* Rasters are row-major, row j south to north, column i west to east, with
 * a row stride ld in elements (ld >= the row length; ld = 0: rows packed).
 * Host rasters are copied in and stay the caller's.  The _dev variants take
 * device pointers of the current device (e.g. torch data_ptr()s), read on
 * the context's stream; the caller keeps ownership and must not change them
 * until the call returns (every load synchronises the context's stream).
 * A raster with a non-finite value gives MWDG_ERR_NONFINITE (device rasters
 * are checked on the device); ld below the row length MWDG_ERR_ARG. */

/* Topography from a vertex raster z_vert[(ny+1) rows x (nx+1)]: planar
 * coefficients by Eq. 8 on the finest grid (the interface-centre values are
 * means of the two vertices, so z is continuous at interface centres), the
 * full static pyramid by Eq. 9 and each node's normalised topography detail
 * max|d| / max(1, max|z0|) (Sect. 2.2). */
MWDG_API mwdg_status mwdg_load_dem(mwdg_ctx *ctx, const double *z_vert, int64_t ld);
MWDG_API mwdg_status mwdg_load_dem_dev(mwdg_ctx *ctx, const double *z_vert, int64_t ld);

/* Manning coefficient n_M (Eq. 1) per finest cell, n_cell[ny rows x nx];
 * coarser elements use the mean of their finest cells. */
MWDG_API mwdg_status mwdg_load_roughness(mwdg_ctx *ctx, const double *n_cell, int64_t ld);
MWDG_API mwdg_status mwdg_load_roughness_dev(mwdg_ctx *ctx, const double *n_cell, int64_t ld);
MWDG_API mwdg_status mwdg_set_roughness_scalar(mwdg_ctx *ctx, double n);

/* Initial condition from vertex rasters ((ny+1) rows x (nx+1) each) of depth
 * h (or free surface eta = h + z when is_eta != 0) and discharges qx, qy,
 * projected like the topography (Sect. 2.1.4).  With is_eta, elements whose
 * average free surface is not above their average bed start dry.  Requires
 * mwdg_load_dem first.  Uniform and adaptive runs start on the finest grid;
 * a static run builds its graded grid here from the topography (as
 * mwdg_mra_adapt does) and encodes the state onto it.  Resets time to 0.
 * The host form takes packed rasters; the device form a common row stride
 * ld, and a non-finite value found in its second or third raster leaves the
 * context without an initial state. */
MWDG_API mwdg_status mwdg_load_initial(mwdg_ctx *ctx, const double *h_vert, const double *qx_vert,
                              const double *qy_vert, int32_t is_eta);
MWDG_API mwdg_status mwdg_load_initial_dev(mwdg_ctx *ctx, const double *h_vert, const double *qx_vert,
                                           const double *qy_vert, int64_t ld, int32_t is_eta);

/* Inflow hydrograph Q(t) (m^3/s, piecewise linear through nknots knots,
 * held constant outside) entering through finest cells c0..c1 of an edge;
 * each boundary face carries Q times its overlap with those cells divided
 * by their total width, as a critical-depth ghost state.  Faces of that
 * edge outside c0..c1 keep their bc.  nknots = 0 removes the inflow. */
MWDG_API mwdg_status mwdg_set_inflow(mwdg_ctx *ctx, int32_t edge, int32_t c0, int32_t c1, const double *t,
                            const double *Q, int32_t nknots);

/* Uniform rain rate (m/s) added to the depth at the start of each step
 * that begins before t_stop. */
MWDG_API mwdg_status mwdg_set_rain(mwdg_ctx *ctx, double rate, double t_stop);

/* Eq. 9 on the current flow state: scale coefficients of every refined node
 * (local encoding of its active leaves) and, per node, the flow details'
 * normalised maximum max_v max|d_v| / max(1, max|v0|) over h, qx, qy.
 * Adaptive mode only (MWDG_ERR_STATE otherwise). */
MWDG_API mwdg_status mwdg_mra_encode(mwdg_ctx *ctx);

/* Threshold, regularise and decode (Sect. 2.2, 2.3) with threshold eps:
 *  adaptive: after mwdg_mra_encode, a node is significant when its
 *    topography or flow normalised detail is >= eps; significant nodes flag
 *    their eight same-level neighbours; parents of flagged nodes are flagged;
 *    new active leaves take encoded or prolonged coefficients (Eq. 10).
 *  static: rebuilds the graded grid from the topography details alone
 *    (closure and 2:1 grading) and re-encodes the loaded initial state;
 *    valid only before the first step.
 * *n_active (may be NULL) receives the number of active leaves.  Synchronises. */
MWDG_API mwdg_status mwdg_mra_adapt(mwdg_ctx *ctx, double eps, int64_t *n_active);

/* One time step (Sect. 2.1.1, Eq. 4): [adaptive: encode + adapt], CFL time
 * step over the active leaves, rain, split implicit friction, RK2 stage 1 and
 * stage 2.  dt_out (may be NULL; if given the call synchronises) receives
 * the step's dt. */
MWDG_API mwdg_status mwdg_dg2_step(mwdg_ctx *ctx, double *dt_out);

/* One time step of the prescribed length dt (> 0, finite) instead of the
 * CFL step: otherwise exactly mwdg_dg2_step (Sect. 2.1.1, Eq. 4).  The paper
 * steps at the Courant number; a prescribed step serves comparisons of two
 * runs on one step sequence (the FP32 path on the FP64 path's steps) and
 * coupling to a caller's clock.  dt is not checked against the CFL
 * condition.  Queued without host synchronisation. */
MWDG_API mwdg_status mwdg_dg2_step_dt(mwdg_ctx *ctx, double dt);

/* nsteps steps queued without any host synchronisation. */
MWDG_API mwdg_status mwdg_run_steps(mwdg_ctx *ctx, int64_t nsteps);

/* Steps until the simulated time reaches t_end (the last step is shortened
 * to land on it).  *steps_out (may be NULL) receives the number of steps. */
MWDG_API mwdg_status mwdg_run_to_time(mwdg_ctx *ctx, double t_end, int64_t *steps_out);

/* Finest-resolution fields h, u, v (host, ny rows x nx with row stride ld,
 * ld = 0: packed; any may be NULL): each active leaf's plane evaluated at
 * the centres of the finest cells it covers; velocities are q/h where
 * h > h_dry, else 0.  Synchronises the context's stream.  MWDG_ERR_ARG when
 * ld is below nx. */
MWDG_API mwdg_status mwdg_read_fields(mwdg_ctx *ctx, double *h, double *u, double *v, int64_t ld);
/* Same into device buffers of the current device (FP64), queued on the
 * context's stream without synchronising; the caller keeps ownership. */
MWDG_API mwdg_status mwdg_read_fields_dev(mwdg_ctx *ctx, double *h, double *u, double *v, int64_t ld);

/* Gauge time series (Sect. 3, depth and velocity at gauge points): h, u, v
 * (host, n each, any may be NULL) at n finest cells given as (i, j) pairs in
 * ij (host, 2n int32, i west->east, j south->north), with the same values as
 * mwdg_read_fields at those cells.  MWDG_ERR_ARG if a cell is outside the
 * grid.  Device scratch grows to the largest n seen and is kept until
 * mwdg_destroy. */
MWDG_API mwdg_status mwdg_read_gauges(mwdg_ctx *ctx, const int32_t *ij, int32_t n, double *h, double *u,
                                      double *v);

/* Active leaves ordered by level, then row-major: level, i, j (any may be
 * NULL) and their nine coefficients (h0 h1x h1y qx0 qx1x qx1y qy0 qy1x qy1y,
 * depth form, may be NULL).  cap is the capacity of the buffers in leaves;
 * *n receives the count (MWDG_ERR_CAPACITY, with *n set, if cap < count). */
MWDG_API mwdg_status mwdg_read_active(mwdg_ctx *ctx, int32_t *level, int32_t *i, int32_t *j, double *coeffs,
                             int64_t cap, int64_t *n);

MWDG_API mwdg_status mwdg_get_time(mwdg_ctx *ctx, double *t, int64_t *steps);
/* Steps taken and active-leaf updates (one leaf advanced one step) summed
 * over them since mwdg_load_initial; either pointer may be NULL.
 * Synchronises. */
MWDG_API mwdg_status mwdg_get_counters(mwdg_ctx *ctx, int64_t *steps, int64_t *updates);

/* Volume sum over active leaves of h0 * area (FP64, fixed summation order)
 * and the mass budget terms since mwdg_load_initial: boundary inflow and
 * outflow volumes, rain volume, volume added by clipping negative depths and
 * the number of clipped leaves.  Any pointer may be NULL.  Synchronises. */
MWDG_API mwdg_status mwdg_get_volume(mwdg_ctx *ctx, double *V, double *V_in, double *V_out, double *V_rain,
                            double *V_clip, int64_t *n_clip);

/* Checkpoint / resume.  The state is the node kinds (the active tree), the
 * coefficients of every node, the static beds and roughness it was built
 * with, the simulated time and the mass-budget counters; a context with the
 * same parameters can resume from it.  mwdg_state_bytes gives the buffer
 * size; save writes into a host buffer of at least that size (synchronises);
 * load reads one (MWDG_ERR_DIMS if it belongs to another grid or precision,
 * MWDG_ERR_ARG if the buffer is not a state of this library). */
MWDG_API mwdg_status mwdg_state_bytes(mwdg_ctx *ctx, int64_t *bytes);
MWDG_API mwdg_status mwdg_save_state(mwdg_ctx *ctx, void *buf, int64_t cap);
MWDG_API mwdg_status mwdg_load_state(mwdg_ctx *ctx, const void *buf, int64_t size);

/* Per-kernel timing with CUDA events on the context stream: enable != 0
 * starts recording (and clears the totals).  mwdg_kernel_times fills up to
 * cap entries of names (static strings), total milliseconds and launch
 * counts, and returns the number of kernel classes in *n.  Synchronises. */
MWDG_API mwdg_status mwdg_profile(mwdg_ctx *ctx, int32_t enable);
MWDG_API mwdg_status mwdg_kernel_times(mwdg_ctx *ctx, const char **names, double *ms, int64_t *launches,
                              int32_t cap, int32_t *n);

/* Number of kernel launches this context has queued since creation. */
MWDG_API mwdg_status mwdg_launch_count(mwdg_ctx *ctx, int64_t *n);

/* Allocation-free volume sum, for callers that cannot allocate device memory
 * while they run (a host that gives all device memory to its own pool, a
 * real-time warning loop that must not meet an allocation failure, a
 * plug-in that only receives buffers).  The paper has no counterpart; this
 * is a service of the library.  It computes V = sum_k h0[k] * (dx 2^(L -
 * level[k]))^2 over n active leaves, in a fixed summation order, from device
 * arrays h0 (FP64 depth averages) and level (the leaves' levels, as
 * mwdg_read_active reports them), and writes V to the device pointer volume,
 * all queued on cuda_stream.  It allocates nothing: its per-block partial
 * sums live in a fixed file-scope device array (128 KB, held by every GPU
 * that loads the library until the process exits).  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress); with
 * lazy module loading that is also when the array is committed, so the
 * first call must come before the host hands all device memory to its own
 * pool (an n = 0 call at start-up does it).  Calls share the array: calls
 * whose work overlaps on the GPU race.  Every level must lie in 0..L: the
 * call waits for its own work on cuda_stream to check that, and a level
 * outside it makes the call return MWDG_ERR_ARG with *volume set to NaN.
 * Errors: MWDG_ERR_ARG (NULL pointer with n > 0, dx <= 0, L outside
 * 0..MWDG_LMAX, n < 0, a level outside 0..L), MWDG_ERR_CAPACITY when n
 * exceeds MWDG_VOLUME_NOALLOC_MAX, MWDG_ERR_CUDA when the address lookup or
 * one of its launches fails, or when a CUDA error from earlier work is
 * pending at entry (that error is not cleared, so its owner still sees
 * it). */
#define MWDG_VOLUME_NOALLOC_MAX 67108864LL
MWDG_API mwdg_status mwdg_volume_noalloc(const double *h0, const int32_t *level, int64_t n, double dx,
                                         int32_t L, double *volume, void *cuda_stream);

/* Measured arithmetic ceiling of the current device: the fused
 * multiply-add rate (2 flops each) that the FP64 (precision MWDG_F64) or FP32
 * (MWDG_F32) pipes sustain over all SMs, from a kernel of independent FMA
 * chains timed with CUDA events on cuda_stream, written to *flops_per_s.
 * Not part of the method (the paper has no counterpart): it gives the FP64
 * path, which GB300's FP64 pipes bound rather than its memory, a ceiling
 * measured on the same GPU.  Synchronises cuda_stream.  Errors:
 * MWDG_ERR_ARG (NULL pointer, another precision), MWDG_ERR_CUDA. */
MWDG_API mwdg_status mwdg_fma_rate(int32_t precision, void *cuda_stream, double *flops_per_s);

/* Launch shape of a context's step kernels: the number of blocks of the
 * leaf kernels (grid_leaves, 1..65535) and the size of the coarsest MRA
 * levels run by one block (coarse_nodes >= 1: levels with at most that many
 * nodes).  Neither changes the arithmetic of a leaf or node; both change
 * only how the work is spread.  Either argument <= 0 keeps the current
 * value.  By default grid_leaves is min(nodes / 256, 1216), and for a
 * static grid, once mwdg_load_initial has built it, about one block per 256
 * leaves (152 to 4864), unless set here before.  mwdg_get_launch_shape
 * reads them (any pointer may be NULL). */
MWDG_API mwdg_status mwdg_set_launch_shape(mwdg_ctx *ctx, int32_t grid_leaves, int64_t coarse_nodes);
MWDG_API mwdg_status mwdg_get_launch_shape(mwdg_ctx *ctx, int32_t *grid_leaves, int64_t *coarse_nodes);

/* Ensembles (batched scenarios of uneven sizes).  An ensemble steps n
 * independent contexts together: one CUDA graph per ensemble step holds
 * every member's step as a parallel branch (or, with
 * mwdg_ensemble_set_batched, groups of members as batched launches), so
 * small members share the GPU instead of each leaving most of it idle.  Members are created and loaded
 * as usual (any mode, precision and size, same device); the ensemble
 * borrows them (the caller keeps ownership and must not destroy a member
 * while the ensemble exists).  Each member keeps its own time step; in
 * mwdg_ensemble_run_to_time every member stops at t_end.  A member's own
 * calls may be interleaved with ensemble calls: ensemble work is ordered
 * after the member's earlier work on its stream and before its later work.
 * The graph is rebuilt when a member's parameters changed.  Results equal
 * those of the members stepped one by one.  cuda_stream orders the
 * ensemble's work (NULL: the ensemble creates a stream of its own; a
 * stream passed in must be capturable, i.e. not the legacy default
 * stream).  Errors: MWDG_ERR_ARG (NULL, n < 1, a member listed twice),
 * MWDG_ERR_STATE (a member without an initial state, in an error state or
 * with per-kernel timing on), MWDG_ERR_NONFINITE, MWDG_ERR_CUDA. */
typedef struct mwdg_ensemble mwdg_ensemble;
MWDG_API mwdg_status mwdg_ensemble_create(mwdg_ctx *const *members, int32_t n, void *cuda_stream,
                                          mwdg_ensemble **out);
MWDG_API void mwdg_ensemble_destroy(mwdg_ensemble *ens);
/* n ensemble steps (each member one step, queued, no host synchronisation) */
MWDG_API mwdg_status mwdg_ensemble_step(mwdg_ensemble *ens, int64_t n);
/* until every member's time reaches t_end (last steps shortened to land on
 * it); *graph_launches_out (may be NULL) receives the ensemble steps queued */
MWDG_API mwdg_status mwdg_ensemble_run_to_time(mwdg_ensemble *ens, double t_end, int64_t *graph_launches_out);
/* Autotuner: for each member, times `steps` steps of every candidate launch
 * shape (grid_leaves in {1, 2, 4, 8} x 152 blocks, coarse_nodes in {64,
 * 256, 1024}) from a saved state, restores the state, and keeps the fastest.
 * chosen (may be NULL) receives grid_leaves and coarse_nodes per member
 * (2n int64).  Members end with the state they had.  The results of later
 * steps are unchanged up to the FP32 contraction order of the coarsest MRA
 * levels (FP64: identical). */
MWDG_API mwdg_status mwdg_ensemble_tune(mwdg_ensemble *ens, int32_t steps, int64_t *chosen);
/* Batched launches: group = 2..64 puts the members on adaptive DG2 grids
 * (MWDG2, Sect. 2.3) of one precision in groups of up to `group`; each
 * group's step is one launch per kernel of the step (encode,
 * regularisation, decode, compaction, limiter, flux views, stage updates;
 * Eq. 9-10, Eq. 4) over a work list of (member, block): block b of the
 * launch works as block b - s_m of member m, whose blocks start at s_m, with
 * that member's own launch shape.  Groups and the other members are
 * parallel graph branches.  group = 0 (the default) or 1: one branch per
 * member.  Results are the same either way (each member's arithmetic and
 * order are its own); the member tables live in device memory of the
 * ensemble and are rebuilt with the graph.  MWDG_ERR_ARG for group outside
 * 0..64. */
MWDG_API mwdg_status mwdg_ensemble_set_batched(mwdg_ensemble *ens, int32_t group);
MWDG_API const char *mwdg_ensemble_last_error(const mwdg_ensemble *ens);

MWDG_API const char *mwdg_last_error(const mwdg_ctx *ctx);
MWDG_API const char *mwdg_status_string(mwdg_status s);

#ifdef __cplusplus
}
#endif
#endif /* MWDG_H */
