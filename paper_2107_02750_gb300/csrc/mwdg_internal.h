// Internal types shared by the host orchestration (mwdg_api.cu) and the
// per-precision kernel translation units (mwdg_f64.cu, mwdg_f32.cu).
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "mwdg.h"

namespace mwdg {

// Step control and diagnostics, resident in device memory so that a run of
// steps needs no host synchronisation.
struct Ctl {
  double t, dt, t_end;
  unsigned long long dtmin;    // bits of the smallest CFL candidate (positive double)
  unsigned long long vmax[3];  // bits of max |h0|, |qx0|, |qy0| over the leaves
  double bnd[2];               // outward boundary mass flux of each RK stage (m^3/s)
  double v_in, v_out, v_rain, v_clip;
  double volume;
  unsigned long long n_clip;
  long long steps;
  long long updates;           // active leaves advanced, summed over steps
  int nonfinite;
  int changed;                 // grading sweep made a change
  unsigned int blocks_done;    // completion tickets of the last kernel of a step
  unsigned int ticket;         // completion tickets of the multi-level MRA kernels (self-resetting)
  // set with dt at the start of a step, so that the FP32 kernels read them
  // without FP64 arithmetic: dt in FP32, and the rain depth of the step
  float dt_f, rain_inc_f;
  int rain_on;
  int pad_;
  double rain_inc;
  double dt_fixed;             // > 0: the next steps take this dt instead of the CFL step
  int bad_input;               // set by the finiteness check of a raster read from device memory
  int pad2_;
};

// Geometry and parameters of the level hierarchy (passed by value).
struct Geo {
  int L, M, N, mode, limiter, prec, iface, scheme;
  int nxl[MWDG_LMAX + 1], nyl[MWDG_LMAX + 1];
  long long off[MWDG_LMAX + 2];
  long long P;                 // nodes over all levels
  double dxl[MWDG_LMAX + 1];   // element size per level
  double g, hd, cfl, dt_max, eps, area;
  int bc[4];
  int inflow_edge, inflow_c0, inflow_c1, nknots;
  double rain_rate, rain_t_end;
  long long coarse_nodes;      // MRA levels up to this size run in one block
  // single-precision copies of g, h_dry and the element sizes, so that
  // FP32 kernels convert nothing from FP64 on the device
  float gf, hdf;
  float dxlf[MWDG_LMAX + 1];
};

// refresh the single-precision copies after any change of g, hd or dxl
inline void sync_single(Geo &g) {
  g.gf = (float)g.g;
  g.hdf = (float)g.hd;
  for (int l = 0; l <= MWDG_LMAX; l++) g.dxlf[l] = (float)g.dxl[l];
}

// Device arrays.  Coefficient arrays are component-major with stride P:
// component m of node k is at [m * P + k]; node (l, i, j) is
// k = off[l] + j * nxl[l] + i.
template <typename T>
struct Ptrs {
  T *U;     // state (9): leaves hold the solution, refined nodes its encoding
  T *Ui;    // RK2 intermediate state (9)
  T *Wn;    // limited stage-1 input in the stored view (9)
  T *Wi;    // limited stage-2 input in the stored view (9)
  T *FZ;    // flux view, one record of 12 per node: the limited stage input
            // (9) and its bed planes (3); refined nodes hold their encoding
  T *Z;     // static topography pyramid (3)
  T *NM;    // Manning n per node (1)
  double *DZ;   // normalised topography detail per node (compared with eps in FP64)
  uint8_t *kind, *flag, *flag2;
  uint8_t *kind_new;  // kinds of the next active set while the old ones are still read
  long long *leaves;  // active leaves, packed (level << 56 | j << 28 | i)
  long long *nbr;     // per active leaf, its four face-neighbour codes (E, W, N, S)
  int *nleaf;
  int *blk;         // compaction scratch: per-block counts / offsets
  double *part;     // volume partial sums
  Ctl *ctl;
  const double *knot_t, *knot_Q;
};

// Batched ensemble steps: members that share the adaptive DG2 pipeline step
// together, one launch per kernel (and MRA chunk) over all their blocks.
// Block b of such a launch belongs to the member whose block range
// [bstart, bstart + nblk) holds it and works as that member's block
// b - bstart of nblk; the members' records (geometry, arrays, the launch's
// per-member arguments) live in device memory, their first blocks in the
// kernel's parameters.
constexpr int BMAX = 64;  // members per batched launch
struct BStarts {
  int n;
  unsigned s[BMAX + 1];  // first block of each member, then the total
};
template <typename T>
struct BMember {
  Geo g;
  Ptrs<T> p;
  int a[4];  // per-member arguments: MRA chunk (top level, levels, tail), view tail
  unsigned bstart, nblk;
};
enum BKind { BK_SIG = 0, BK_REG, BK_DECODE, BK_SCATTER, BK_LIMIT1, BK_VIEW, BK_UPD1, BK_LIMIT2, BK_UPD2 };
struct BatchLaunch {
  int kind;
  BStarts bs;
  void *tab;  // device array of bs.n member records (owned by the ensemble)
};

// a fork of the launch stream: work queued on aux after fork is recorded on
// the launch stream runs beside what follows there, until the launch stream
// waits on join
struct Fork {
  cudaStream_t aux;
  cudaEvent_t fork, join;
};

// Launchers implemented per precision (explicit instantiations in
// mwdg_f64.cu and mwdg_f32.cu).  All queue work on `st` and return the
// number of kernels they launched.
template <typename T> struct Launch {
  static int project(const Geo &g, const Ptrs<T> &p, const double *vert, T *c0, T *c1x, T *c1y,
                     cudaStream_t st);
  static int load_dem_pyramid(const Geo &g, const Ptrs<T> &p, cudaStream_t st);
  static int roughness_pyramid(const Geo &g, const Ptrs<T> &p, cudaStream_t st);
  static int initial_finest(const Geo &g, const Ptrs<T> &p, int is_eta, cudaStream_t st);
  static int encode_dense_U(const Geo &g, const Ptrs<T> &p, cudaStream_t st);
  static int eta_rule_leaves(const Geo &g, const Ptrs<T> &p, cudaStream_t st);
  static int static_flags(const Geo &g, const Ptrs<T> &p, cudaStream_t st);
  static int closure(const Geo &g, uint8_t *flag, cudaStream_t st);
  static int grading_sweep(const Geo &g, const Ptrs<T> &p, cudaStream_t st);
  static int kinds(const Geo &g, const Ptrs<T> &p, const uint8_t *flag, cudaStream_t st);
  static int all_finest(const Geo &g, const Ptrs<T> &p, cudaStream_t st);
  static int compact(const Geo &g, const Ptrs<T> &p, cudaStream_t st);
  // begin: the adaptation's last kernel also starts the step that follows;
  // fk: a second stream and two events on which the encode's coarsest
  // levels run beside the regularisation (nullptr: all on st)
  static int adapt(const Geo &g, const Ptrs<T> &p, int encode_only, int with_maxabs,
                   cudaStream_t st, void (*mark)(void *, int), void *mark_arg, int begin = 0,
                   const Fork *fk = nullptr);
  // begun: the step was started by the adaptation
  static int step(const Geo &g, const Ptrs<T> &p, int grid_leaves, cudaStream_t st,
                  void (*mark)(void *, int), void *mark_arg, int begun = 0);
  // max |v0| and the CFL candidate over the current leaves (after a load,
  // a checkpoint restore or a stand-alone adaptation)
  static int prime(const Geo &g, const Ptrs<T> &p, int grid_leaves, cudaStream_t st);
  static int fields(const Geo &g, const Ptrs<T> &p, double *h, double *u, double *v,
                    cudaStream_t st);
  static int gauges(const Geo &g, const Ptrs<T> &p, const int32_t *ij, int n, double *out, cudaStream_t st);
  static int read_active(const Geo &g, const Ptrs<T> &p, int32_t *lev, int32_t *i, int32_t *j,
                         double *coef, cudaStream_t st);
  static int volume(const Geo &g, const Ptrs<T> &p, int grid_leaves, cudaStream_t st);
  static int dt_only(const Geo &g, const Ptrs<T> &p, int grid_leaves, cudaStream_t st);
  // the batched launches of one step of n <= BMAX adaptive DG2 members (the
  // sequence of adapt + step for each, with its own launch shapes); the
  // member tables are allocated and filled here (synchronous host work).
  // false when an allocation or copy fails (plan then holds what to free)
  static bool batch_plan(int n, const Geo *const *g, const Ptrs<T> *const *p, const int *grid_leaves,
                         std::vector<BatchLaunch> &plan);
  static int batch_step(const std::vector<BatchLaunch> &plan, cudaStream_t st);
};

// kernel classes reported by the per-kernel timer
enum KClass {
  KC_ENCODE = 0, KC_FLAGS, KC_DECODE, KC_COMPACT, KC_DT, KC_CONTROL, KC_FRICTION, KC_LIMIT,
  KC_VIEW, KC_UPDATE1, KC_UPDATE2, KC_COUNT
};

}  // namespace mwdg
