// Discrete adjoint of the uniform-grid DG2 step (include/mwdg_adjoint.h).
//
// The forward sweep is the DG2 step of Sect. 2.1.1 (Eq. 1-4) on a dense
// uniform grid, compiled without FMA contraction and written in the
// operation order of the step in mwdg_kernels.cuh, so that it rounds the
// same way.  The reverse sweep differentiates that step by hand, kernel by
// kernel, with every branch replayed from the recomputed forward values:
//
//   forward per step   friction -> limit(Un) -> update stage 1 -> limit(Ui)
//                      -> update stage 2 (+ the CFL dt when not given); the
//                      update computes each interface once per 16 x 16 tile
//   reverse per step   recompute friction, limit, stage 1, limit; then for
//                      stage 2 and stage 1 in turn:
//                        rev_face   per interface: both cells' operator
//                                   terms for it (post-stage masks, RK2
//                                   weights, flux weights, physical fluxes
//                                   and bed sources of the own revised
//                                   limits), then HLL and the two revisions,
//                                   the interface bed max, boundary ghosts
//                                   (and the hydrograph)
//                        rev_limit  the stored view's and the slope sources'
//                                   terms, the face-limit transpose and the
//                                   limiter (partial-wet reduction, minmod
//                                   picks)
//                        rev_gather neighbour terms of the limiter
//                      then friction.
//
// Every cotangent is gathered by the thread that owns it (a cell or a
// face) from buffers written by the kernel before: no atomics, so a run is
// deterministic.  The tape holds the state at the start of each step and
// the clip flags of each stage; nothing else is stored.
//
// Kernels are templated on the coefficient type T.  FP64 (T = double) is the
// reference: it reproduces the oracle's step bit for bit.  FP32 (T = float)
// keeps time, time steps, the hydrograph and its gradient in FP64 (a few
// operations per boundary cell) and everything else in FP32, so that the
// per-cell work runs on the FP32 pipes.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "dg2_math.cuh"
#include "mwdg_adjoint.h"

namespace mwdg {
namespace adj {

constexpr int TPB = 256;

// relative tolerance under which the two bed limits of an interface count as
// one (their rounding gap on a continuous DEM is a few units of the last place)
template <typename T> __device__ __forceinline__ T tie_rel();
template <> __device__ __forceinline__ double tie_rel<double>() { return 1e-10; }
template <> __device__ __forceinline__ float tie_rel<float>() { return 1e-5f; }

// parameters passed to the kernels by value.  On a frozen non-uniform grid
// every level is a dense array of nx x ny nodes (nx = M 2^l) in one
// coefficient array per component, levels one after another.  A kernel
// working on one level takes its pointers offset to the level's first node;
// one working on all levels (a Levels table) offsets them itself by off.
template <typename T>
struct Par {
  int nx, ny;
  long long n;          // nodes of this level (cells of a uniform grid)
  long long ns;         // stride between components (n on a uniform grid)
  long long off;        // the level's first node in the level arrays (0: uniform)
  long long fx, fy;     // its first x face and y face among all levels' faces
  long long fxp, fyp;   // the previous level's (its parents')
  long long lqo;        // its first boundary entry
  int sh;               // levels from this one down to the finest (0: uniform)
  int stat;             // 1: static graded grid (two-children mean, Sect. 2.2.1)
  const uint8_t *kind;  // per node of the level: K_BELOW, K_LEAF, K_SIG; NULL: all leaves
  long long dn, dp;     // nodes from this level's first to the next's, from the previous's to this
  T dx, g, hd;
  double dxd, cfl, dt_max;
  int limiter;
  int bc[4];
  int inflow_edge, c0, c1, nknots;
  double rain_rate, rain_t_end;
  const double *kt, *kQ;
};

// ---------------------------------------------------------------------------
// hydrograph (FP64 in both precisions)
// ---------------------------------------------------------------------------
// Q(t), piecewise linear over the knots and constant outside them; k0, k1
// and r give its weights: Q = (1 - r) Q[k0] + r Q[k1] in the derivative.
template <typename T>
__device__ double hydro(const Par<T> &P, double t, int &k0, int &k1, double &r) {
  const int n = P.nknots;
  if (t <= P.kt[0]) { k0 = k1 = 0; r = 0.0; return P.kQ[0]; }
  if (t >= P.kt[n - 1]) { k0 = k1 = n - 1; r = 0.0; return P.kQ[n - 1]; }
  int k = 0;
  while (k + 1 < n && !(t < P.kt[k + 1])) k++;
  const double tk = P.kt[k], tk1 = P.kt[k + 1], Qk = P.kQ[k], Qk1 = P.kQ[k + 1];
  k0 = k;
  k1 = k + 1;
  r = (t - tk) / (tk1 - tk);
  return Qk + (Qk1 - Qk) * (t - tk) / (tk1 - tk);
}

// finest inflow cells under the boundary face of node `along` of this level
// on edge e (0 or 1 on a uniform grid)
template <typename T>
__device__ __forceinline__ long long inflow_overlap(const Par<T> &P, int e, int along) {
  if (P.inflow_edge != e || P.nknots < 1) return 0;
  const long long a = (long long)along << P.sh, b = (long long)(along + 1) << P.sh;
  const long long lo = a > P.c0 ? a : (long long)P.c0, hi = b < (long long)P.c1 + 1 ? b : (long long)P.c1 + 1;
  return hi > lo ? hi - lo : 0;
}

// unit discharge through the boundary face of node `along` on edge e: the
// hydrograph spread over the inflow cells, times the face's overlap with them
template <typename T>
__device__ double inflow_unit(const Par<T> &P, int e, int along, double t) {
  const long long ov = inflow_overlap(P, e, along);
  if (ov <= 0) return 0.0;
  int k0, k1;
  double r;
  const double Q = hydro(P, t, k0, k1, r);
  return Q * (double)ov / ((double)(P.c1 - P.c0 + 1) * P.dxd);
}

// ---------------------------------------------------------------------------
// per-cell pieces shared by the sweeps
// ---------------------------------------------------------------------------
template <typename T>
struct Lim {
  T h, qx, qy, z;
};

template <typename T>
__device__ __forceinline__ Lim<T> cell_lim(const T *W, const T *Z, long long n, long long k, int f) {
  Lim<T> L;
  L.h = face_value(W[k], W[n + k], W[2 * n + k], f);
  L.qx = face_value(W[3 * n + k], W[4 * n + k], W[5 * n + k], f);
  L.qy = face_value(W[6 * n + k], W[7 * n + k], W[8 * n + k], f);
  L.z = face_value(Z[k], Z[n + k], Z[2 * n + k], f);
  return L;
}

// edge of the domain that face f of a boundary cell lies on
__device__ __forceinline__ int edge_of(int f) { return f == 0 ? 1 : f == 1 ? 0 : f == 2 ? 3 : 2; }

// ghost limit across a boundary face: inflow at the critical depth carrying
// the hydrograph, open (copy) or wall (mirror the normal discharge)
template <typename T>
__device__ Lim<T> ghost(const Par<T> &P, int e, int along, const Lim<T> &o, double t) {
  Lim<T> gl;
  gl.z = o.z;
  const T q = (T)inflow_unit(P, e, along, t);
  if (q > T(0)) {
    const T hc = tcbrt<T>(q * q / P.g);
    gl.h = tmax(o.h, hc);
    const T qn = (e == 0 || e == 2) ? q : -q;
    if (e < 2) { gl.qx = qn; gl.qy = T(0); }
    else { gl.qx = T(0); gl.qy = qn; }
    return gl;
  }
  if (P.bc[e] == MWDG_OPEN) {
    gl.h = o.h; gl.qx = o.qx; gl.qy = o.qy;
    return gl;
  }
  gl.h = o.h;
  if (e < 2) { gl.qx = -o.qx; gl.qy = o.qy; }
  else { gl.qx = o.qx; gl.qy = -o.qy; }
  return gl;
}

// node kinds of a frozen grid: below a coarser leaf, an active leaf, or
// refined (an ancestor of leaves)
constexpr uint8_t K_BELOW = 0, K_LEAF = 1, K_SIG = 2;

template <typename T>
__device__ __forceinline__ bool is_leaf(const Par<T> &P, long long k) {
  return !P.kind || P.kind[k] == K_LEAF;
}

// children (c = cx + 2 cy) of a node that touch its face f: E (cx = 1), W,
// N (cy = 1), S
__device__ __forceinline__ void face_children(int f, int &c1, int &c2) {
  c1 = f == 0 ? 1 : f == 1 ? 0 : f == 2 ? 2 : 0;
  c2 = f == 0 ? 3 : f == 1 ? 2 : f == 2 ? 3 : 1;
}

// index in the next level of child c of node (i, j)
template <typename T>
__device__ __forceinline__ long long child_of(const Par<T> &P, int i, int j, int c) {
  return P.dn + (long long)(2 * j + (c >> 1)) * (2 * P.nx) + (2 * i + (c & 1));
}

// What the other side of an interface sees of node (i, j) on the node's face
// f: the limits (h, qx, qy, z) of its view and the averages (h0, qx0, qy0)
// that the outflow limit takes when the node is the donor.  The view is the
// node's flux view (a leaf; on a frozen MWDG2 grid also the encoding of a
// refined node's leaves or the prolongation of a coarser leaf, Sect. 2.3),
// and on a static grid for a refined node the mean of its two children that
// touch the face (Sect. 2.2.1).
template <typename T>
__device__ __forceinline__ Lim<T> node_lim(const Par<T> &P, const T *W, const T *Z, int i, int j, int f, T avg[3]) {
  const long long k = (long long)j * P.nx + i, n = P.ns;
  if (P.stat && P.kind && P.kind[k] == K_SIG) {
    int c1, c2;
    face_children(f, c1, c2);
    const long long k1 = child_of(P, i, j, c1), k2 = child_of(P, i, j, c2);
    const Lim<T> a = cell_lim(W, Z, n, k1, f), b = cell_lim(W, Z, n, k2, f);
    Lim<T> m;
    m.h = T(0.5) * (a.h + b.h);
    m.qx = T(0.5) * (a.qx + b.qx);
    m.qy = T(0.5) * (a.qy + b.qy);
    m.z = T(0.5) * (a.z + b.z);
    avg[0] = T(0.5) * (W[k1] + W[k2]);
    avg[1] = T(0.5) * (W[3 * n + k1] + W[3 * n + k2]);
    avg[2] = T(0.5) * (W[6 * n + k1] + W[6 * n + k2]);
    return m;
  }
  avg[0] = W[k];
  avg[1] = W[3 * n + k];
  avg[2] = W[6 * n + k];
  return cell_lim(W, Z, n, k, f);
}

// limiter record of one cell: partial-wet reduction and, per direction and
// variable, 0 kept, 1 replaced by the forward difference, 2 by the backward
// difference, 3 by zero
struct LimRec {
  bool red;
  int8_t sel[2][3];
};

// Stage-input limiting of cell (i, j) of X (Sect. 2.1.1; the same reading
// as the solver's: partial-wet leaves drop to a flat free surface over the
// planar bed, seen by the fluxes as flat depth over a flat bed; minmod on
// the interface offsets of eta, qx, qy against the neighbours' averages).
template <typename T>
__device__ void limit_cell(const Par<T> &P, const T *X, const T *Z, int i, int j, T w_st[9], T w_fx[9], T ze[3],
                           LimRec &r) {
  const long long n = P.ns, k = (long long)j * P.nx + i;
  const T hd = P.hd, s3 = s3v<T>();
#pragma unroll
  for (int m = 0; m < 9; m++) w_st[m] = X[m * n + k];
#pragma unroll
  for (int m = 0; m < 3; m++) ze[m] = Z[m * n + k];
  r.red = false;
#pragma unroll
  for (int d = 0; d < 2; d++)
#pragma unroll
    for (int v = 0; v < 3; v++) r.sel[d][v] = 0;
  const T h0 = w_st[0];
  const T eta0 = h0 + ze[0];
  bool red = !(h0 > hd);
#pragma unroll
  for (int f = 0; f < 4; f++) {
    if (!(face_value(w_st[0], w_st[1], w_st[2], f) > hd)) red = true;
    if (!(eta0 - face_value(ze[0], ze[1], ze[2], f) > hd)) red = true;
  }
  if (red) {
    r.red = true;
    w_st[1] = -ze[1]; w_st[2] = -ze[2];
    w_st[4] = T(0); w_st[5] = T(0);
    w_st[7] = T(0); w_st[8] = T(0);
#pragma unroll
    for (int m = 0; m < 9; m++) w_fx[m] = w_st[m];
    w_fx[1] = T(0); w_fx[2] = T(0);
    ze[1] = T(0); ze[2] = T(0);
    return;
  }
  if (P.limiter) {
    for (int d = 0; d < 2; d++) {
      const int ia = i + (d == 0), ja = j + (d == 1), ib = i - (d == 0), jb = j - (d == 1);
      // neighbours: same-level leaves only (Sect. 2.2.1)
      const bool hasA = ia < P.nx && ja < P.ny && is_leaf(P, (long long)ja * P.nx + ia);
      const bool hasB = ib >= 0 && jb >= 0 && is_leaf(P, (long long)jb * P.nx + ib);
      if (!hasA && !hasB) continue;
      const long long ka = hasA ? (long long)ja * P.nx + ia : k, kb = hasB ? (long long)jb * P.nx + ib : k;
      const T hC = X[k], hA = X[ka], hB = X[kb];
      const bool wet = (hC > hd) && (!hasA || hA > hd) && (!hasB || hB > hd);
      const int cs = 1 + d;
      for (int v = 0; v < 3; v++) {
        if (v == 0 && !wet) continue;
        const T zs = Z[cs * n + k];
        T aC, a0, aB, slope;
        if (v == 0) {
          aC = hC + Z[k];
          a0 = hA + Z[ka];
          aB = hB + Z[kb];
          slope = X[cs * n + k] + zs;
        } else {
          aC = X[3 * v * n + k];
          a0 = X[3 * v * n + ka];
          aB = X[3 * v * n + kb];
          slope = X[(3 * v + cs) * n + k];
        }
        const T a = s3 * slope;
        const T d1 = a0 - aC, d2 = aC - aB;
        T mm;
        bool same;
        if (hasA && hasB) {
          same = (a > T(0) && d1 > T(0) && d2 > T(0)) || (a < T(0) && d1 < T(0) && d2 < T(0));
          mm = minmod3(a, d1, d2);
        } else {
          const T o = hasA ? d1 : d2;
          same = (a > T(0) && o > T(0)) || (a < T(0) && o < T(0));
          mm = minmod2(a, o);
        }
        if (mm != a) {
          const T ns = mm / s3;
          const int coef = v == 0 ? cs : 3 * v + cs;
          w_st[coef] = v == 0 ? ns - zs : ns;
          r.sel[d][v] = !same ? 3 : (hasA && hasB) ? (mm == d1 ? 1 : 2) : (hasA ? 1 : 2);
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 9; m++) w_fx[m] = w_st[m];
}

template <typename T>
__device__ __forceinline__ bool cell_of(const Par<T> &P, long long &k, int &i, int &j) {
  k = (long long)blockIdx.x * TPB + threadIdx.x;
  if (k >= P.n) return false;
  j = (int)(k / P.nx);
  i = (int)(k - (long long)j * P.nx);
  return true;
}

// One launch over every level of a frozen grid (one level on a uniform grid):
// the levels' parameters and, per level, its first block; each block works
// on one level.
constexpr int MAXLV = MWDG_LMAX + 1;
template <typename T>
struct Levels {
  int n;
  unsigned bstart[MAXLV + 1];
  Par<T> P[MAXLV];
};

// the level of this block (its parameters copied to shared memory) and the
// block's index within the level; ML = false: one level (a uniform grid),
// read in place
template <bool ML, typename T>
__device__ __forceinline__ const Par<T> &block_level(const Levels<T> &LV, Par<T> &sP, unsigned &b) {
  if (!ML) {
    b = blockIdx.x;
    return LV.P[0];
  }
  int l = 0;
  while (l + 1 < LV.n && blockIdx.x >= LV.bstart[l + 1]) l++;
  b = blockIdx.x - LV.bstart[l];
  if (threadIdx.x == 0) sP = LV.P[l];
  __syncthreads();
  return sP;
}

template <typename T>
__device__ __forceinline__ bool node_of(const Par<T> &P, unsigned b, long long &k, int &i, int &j) {
  k = (long long)b * TPB + threadIdx.x;
  if (k >= P.n) return false;
  j = (int)(k / P.nx);
  i = (int)(k - (long long)j * P.nx);
  return true;
}

// ---------------------------------------------------------------------------
// forward sweep
// ---------------------------------------------------------------------------
__global__ void k_set_t0(double *tt, double t0) { tt[0] = t0; }

__global__ void k_times(const double *dts, int steps, double *tt) {
  for (int s = 0; s < steps; s++) tt[s + 1] = tt[s] + dts[s];
}

// CFL candidate of every cell (Sect. 2.1.1), with the inflow ghost at the
// critical depth; the smallest goes to *best as the bits of a positive double
template <typename T, bool ML>
__global__ void __launch_bounds__(TPB) k_cfl(const Levels<T> LV, const T *U, const double *tt, int step,
                                             unsigned long long *best) {
  __shared__ T sh[TPB];
  __shared__ Par<T> sP;
  unsigned bl;
  const Par<T> &P = block_level<ML>(LV, sP, bl);
  U += P.off;
  long long k;
  int i, j;
  T c = tinf<T>();
  if (node_of(P, bl, k, i, j) && is_leaf(P, k)) {
    const long long n = P.ns;
    const T h0 = U[k], dx = P.dx, g = P.g;
    if (h0 > P.hd) {
      const T u = U[3 * n + k] / h0, v = U[6 * n + k] / h0;
      const T cc = tsqrt(g * h0);
      c = tmin(c, tmin(dx / (tabs(u) + cc), dx / (tabs(v) + cc)));
    }
    for (int e = 0; e < 4; e++) {
      const bool on = (e == 0 && i == 0) || (e == 1 && i == P.nx - 1) || (e == 2 && j == 0) ||
                      (e == 3 && j == P.ny - 1);
      if (!on) continue;
      const T q = (T)inflow_unit(P, e, e < 2 ? j : i, tt[step]);
      if (q > T(0)) {
        const T hc = tcbrt<T>(q * q / g);
        if (hc > P.hd) c = tmin(c, dx / (q / hc + tsqrt(g * hc)));
      }
    }
  }
  sh[threadIdx.x] = c;
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = tmin(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0 && sh[0] < tinf<T>())
    atomicMin(best, (unsigned long long)__double_as_longlong((double)sh[0]));
}

__global__ void k_dt(double cfl, double dt_max, unsigned long long *best, double *dts, double *tt, int step) {
  const double b = __longlong_as_double((long long)*best);
  double dt = dt_max;
  if (b < tinf<double>()) dt = fmin(dt, cfl * b);
  dts[step] = dt;
  tt[step + 1] = tt[step] + dt;
  *best = (unsigned long long)__double_as_longlong(tinf<double>());
}

// rain depth of the step, then split implicit Manning friction
template <typename T, bool ML>
__global__ void __launch_bounds__(TPB) k_friction(const Levels<T> LV, const T *U, const T *nman,
                                                  const double *dts, const double *tt, int step, T *Un) {
  __shared__ Par<T> sP;
  unsigned bl;
  const Par<T> &P = block_level<ML>(LV, sP, bl);
  U += P.off;
  nman += P.off;
  Un += P.off;
  long long k;
  int i, j;
  if (!node_of(P, bl, k, i, j)) return;
  const long long n = P.ns;
  const T dt = (T)dts[step], g = P.g;
  const double t = tt[step];
  const double rain = (t < P.rain_t_end) ? P.rain_rate : 0.0;
  T w[9];
#pragma unroll
  for (int m = 0; m < 9; m++) w[m] = U[m * n + k];
  if (!is_leaf(P, k)) {  // not a leaf of a frozen grid: still water, read by no leaf
#pragma unroll
    for (int m = 0; m < 9; m++) Un[m * n + k] = w[m];
    return;
  }
  if (rain > 0.0) w[0] = w[0] + (T)(rain * dts[step]);
  const T h0 = w[0];
  if (h0 > P.hd) {
    const T u = w[3] / h0, v = w[6] / h0;
    const T sp = tsqrt(u * u + v * v);
    const T nm = nman[k];
    const T den = T(1) + dt * g * nm * nm * sp / (h0 * tcbrt<T>(h0));
    const T f = T(1) / den;
#pragma unroll
    for (int m = 3; m < 9; m++) w[m] = w[m] * f;
  } else {
#pragma unroll
    for (int m = 3; m < 9; m++) w[m] = T(0);
  }
#pragma unroll
  for (int m = 0; m < 9; m++) Un[m * n + k] = w[m];
}

template <typename T, bool ML>
__global__ void __launch_bounds__(TPB) k_limit(const Levels<T> LV, const T *X, const T *Z, T *Wst, T *Wfx,
                                               T *Zfx) {
  __shared__ Par<T> sP;
  unsigned bl;
  const Par<T> &P = block_level<ML>(LV, sP, bl);
  X += P.off;
  Z += P.off;
  Wst += P.off;
  Wfx += P.off;
  Zfx += P.off;
  long long k;
  int i, j;
  // a frozen grid's non-leaf node gets its view from the view kernels
  if (!node_of(P, bl, k, i, j) || !is_leaf(P, k)) return;
  const long long n = P.ns;
  T ws[9], wf[9], ze[3];
  LimRec r;
  limit_cell(P, X, Z, i, j, ws, wf, ze, r);
#pragma unroll
  for (int m = 0; m < 9; m++) {
    Wst[m * n + k] = ws[m];
    Wfx[m * n + k] = wf[m];
  }
#pragma unroll
  for (int m = 0; m < 3; m++) Zfx[m * n + k] = ze[m];
}

// ---------------------------------------------------------------------------
// views of a frozen non-uniform grid (Sect. 2.3): every node of every level
// gets the same-level view that a neighbouring leaf reads -- a leaf its
// flux view (k_limit), a refined node the encoding of its children's views
// (Eq. 9, bottom-up), a node below a coarser leaf the prolongation of its
// parent's view (Eq. 10 with zero details, top-down).  V holds the 9 flow
// planes, Vz the 3 bed planes.  Sums run in the order of the oracle, so
// that FP64 rounds the same way.
// ---------------------------------------------------------------------------
// Eq. 9 (scale coefficients only): the parent's planes from its children's
// ch[c] = (c0, c1x, c1y), c = cx + 2 cy
template <typename T>
__device__ __forceinline__ void encode3(const T ch[4][3], T sp[3]) {
  const T H = T(0.5) * s3v<T>();
  sp[0] = T(0.25) * (((ch[0][0] + ch[1][0]) + ch[2][0]) + ch[3][0]);
  T a = (-H) * ch[0][0];
  a = a + T(0.5) * ch[0][1];
  a = a + H * ch[1][0];
  a = a + T(0.5) * ch[1][1];
  a = a + (-H) * ch[2][0];
  a = a + T(0.5) * ch[2][1];
  a = a + H * ch[3][0];
  a = a + T(0.5) * ch[3][1];
  sp[1] = T(0.25) * a;
  T b = (-H) * ch[0][0];
  b = b + T(0.5) * ch[0][2];
  b = b + (-H) * ch[1][0];
  b = b + T(0.5) * ch[1][2];
  b = b + H * ch[2][0];
  b = b + T(0.5) * ch[2][2];
  b = b + H * ch[3][0];
  b = b + T(0.5) * ch[3][2];
  sp[2] = T(0.25) * b;
}

// transpose of encode3: the children's cotangents (added) from the parent's
template <typename T>
__device__ __forceinline__ void encode3_t(const T gp[3], int c, T gc[3]) {
  const T H = T(0.5) * s3v<T>();
  const T sx = (c & 1) ? H : -H, sy = (c & 2) ? H : -H;
  gc[0] += T(0.25) * ((gp[0] + sx * gp[1]) + sy * gp[2]);
  gc[1] += T(0.125) * gp[1];
  gc[2] += T(0.125) * gp[2];
}

// Eq. 10 with zero details: child c's planes from its parent's
template <typename T>
__device__ __forceinline__ void prolong3(const T sp[3], int c, T sc[3]) {
  const T H = T(0.5) * s3v<T>();
  const T sx = (c & 1) ? H : -H, sy = (c & 2) ? H : -H;
  sc[0] = (sp[0] + sx * sp[1]) + sy * sp[2];
  sc[1] = T(0.5) * sp[1];
  sc[2] = T(0.5) * sp[2];
}

// transpose of prolong3: the parent's cotangents (added) from child c's
template <typename T>
__device__ __forceinline__ void prolong3_t(const T gc[3], int c, T gp[3]) {
  const T H = T(0.5) * s3v<T>();
  const T sx = (c & 1) ? H : -H, sy = (c & 2) ? H : -H;
  gp[0] += gc[0];
  gp[1] += sx * gc[0] + T(0.5) * gc[1];
  gp[2] += sy * gc[0] + T(0.5) * gc[2];
}

// refined nodes of this level: the encoding of their children's views
template <typename T>
__device__ __forceinline__ void view_encode_node(const Par<T> &P, T *V, T *Vz, long long k, int i, int j) {
  if (P.kind[k] != K_SIG) return;
  const long long n = P.ns;
#pragma unroll 1
  for (int v = 0; v < 4; v++) {
    T *A = v < 3 ? V + 3 * v * n : Vz;
    T ch[4][3], sp[3];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const long long kc = child_of(P, i, j, c);
#pragma unroll
      for (int m = 0; m < 3; m++) ch[c][m] = A[m * n + kc];
    }
    encode3(ch, sp);
#pragma unroll
    for (int m = 0; m < 3; m++) A[m * n + k] = sp[m];
  }
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_view_encode(Par<T> P, T *V, T *Vz) {
  long long k;
  int i, j;
  if (cell_of(P, k, i, j)) view_encode_node(P, V, Vz, k, i, j);
}

// nodes of this level below a coarser leaf: the prolongation of their
// parent's view
template <typename T>
__device__ __forceinline__ void view_prolong_node(const Par<T> &P, T *V, T *Vz, long long k, int i, int j) {
  if (P.kind[k] != K_BELOW) return;
  const long long n = P.ns;
  const long long kp = -P.dp + (long long)(j >> 1) * (P.nx >> 1) + (i >> 1);
  const int c = (i & 1) + 2 * (j & 1);
#pragma unroll 1
  for (int v = 0; v < 4; v++) {
    T *A = v < 3 ? V + 3 * v * n : Vz;
    T sp[3], sc[3];
#pragma unroll
    for (int m = 0; m < 3; m++) sp[m] = A[m * n + kp];
    prolong3(sp, c, sc);
#pragma unroll
    for (int m = 0; m < 3; m++) A[m * n + k] = sc[m];
  }
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_view_prolong(Par<T> P, T *V, T *Vz) {
  long long k;
  int i, j;
  if (cell_of(P, k, i, j)) view_prolong_node(P, V, Vz, k, i, j);
}

// One RK2 stage (Eq. 4a for stage 1, Eq. 4b for stage 2) on a tile of
// UT x UT cells: every interface of the tile (its own and the ones on its
// edge) is computed once into shared memory -- the flux and both sides'
// revised limits -- then each cell takes its four faces, forms the DG2
// operator, the stage combination and the positivity clip.  The clip is
// recorded in bit (stage - 1) of clip[k].  A face's values are the ones
// either cell would compute for it (the interface bed is the max of the two
// limits, HLL takes the west/south side first), so the result equals a
// per-cell evaluation bit for bit.
constexpr int UT = 16;
constexpr int UFX = (UT + 1) * UT, UFY = UT * (UT + 1);

template <typename T, bool ML>
__global__ void __launch_bounds__(UT * UT) k_update(const Levels<T> LV, int stage, const T *Wfx, const T *Zfx,
                                                    const T *Wst, const T *W1, const double *dts, const double *tt,
                                                    int step, T *Out, uint8_t *clip) {
  __shared__ T sF[UFX + UFY][3];
  __shared__ T sR[UFX + UFY][8];  // low side (hs, u, v, zr), high side (hs, u, v, zr)
  __shared__ Par<T> sP;
  unsigned bl;
  const Par<T> &P = block_level<ML>(LV, sP, bl);
  Wfx += P.off;
  Zfx += P.off;
  Wst += P.off;
  if (W1) W1 += P.off;
  Out += P.off;
  clip += P.off;
  const int tx = (P.nx + UT - 1) / UT;
  const int i0 = (int)(bl % tx) * UT, j0 = (int)(bl / tx) * UT;
  const long long n = P.ns;
  const double t = stage == 1 ? tt[step] : tt[step] + dts[step];
  for (int q = threadIdx.x; q < UFX + UFY; q += UT * UT) {
    const bool xf = q < UFX;
    int fi, fj;
    if (xf) { fj = q / (UT + 1); fi = q - fj * (UT + 1); }
    else { fj = (q - UFX) / UT; fi = (q - UFX) - fj * UT; }
    const int gi = i0 + fi, gj = j0 + fj;   // the face's high-side cell
    if (xf ? (gj >= P.ny || gi > P.nx) : (gi >= P.nx || gj > P.ny)) continue;
    const bool hasLo = xf ? gi > 0 : gj > 0;
    const bool hasHi = xf ? gi < P.nx : gj < P.ny;
    const int along = xf ? gj : gi;
    if (P.kind) {  // a frozen grid's face that no leaf reads
      const long long kH = (long long)gj * P.nx + gi, kL = xf ? kH - 1 : kH - P.nx;
      if (!(hasLo && P.kind[kL] == K_LEAF) && !(hasHi && P.kind[kH] == K_LEAF)) continue;
    }
    Lim<T> lo, hi;
    T aLo[3], aHi[3];  // the sides' averages for the outflow limit
    if (hasLo) lo = node_lim(P, Wfx, Zfx, xf ? gi - 1 : gi, xf ? gj : gj - 1, xf ? 0 : 2, aLo);
    if (hasHi) hi = node_lim(P, Wfx, Zfx, gi, gj, xf ? 1 : 3, aHi);
    if (!hasLo) lo = ghost(P, xf ? 0 : 2, along, hi, t);
    if (!hasHi) hi = ghost(P, xf ? 1 : 3, along, lo, t);
    const T zf = tmax(lo.z, hi.z);
    const Side<T> sl = revise_h(lo.h, lo.qx, lo.qy, lo.z, zf, P.hd);
    const Side<T> sh = revise_h(hi.h, hi.qx, hi.qy, hi.z, zf, P.hd);
    T H[3], F0, F1, F2;
    if (xf) {
      hll(sl.hs, sl.u, sl.v, sh.hs, sh.u, sh.v, P.g, P.hd, H);
      F0 = H[0]; F1 = H[1]; F2 = H[2];
    } else {
      hll(sl.hs, sl.v, sl.u, sh.hs, sh.v, sh.u, P.g, P.hd, H);
      F0 = H[0]; F1 = H[2]; F2 = H[1];
    }
    // outflow limit of the donor cell (never a boundary ghost)
    const bool dLo = F0 > T(0) && hasLo, dHi = F0 < T(0) && hasHi;
    if (dLo || dHi) {
      const T h0 = dLo ? aLo[0] : aHi[0], qx0 = dLo ? aLo[1] : aHi[1], qy0 = dLo ? aLo[2] : aHi[2];
      drain_limit(F0, F1, F2, h0, xf ? qx0 : qy0, xf ? qy0 : qx0, P.g, P.hd, P.dx, (T)dts[step]);
    }
    sF[q][0] = F0; sF[q][1] = F1; sF[q][2] = F2;
    sR[q][0] = sl.hs; sR[q][1] = sl.u; sR[q][2] = sl.v; sR[q][3] = sl.zr;
    sR[q][4] = sh.hs; sR[q][5] = sh.u; sR[q][6] = sh.v; sR[q][7] = sh.zr;
  }
  __syncthreads();
  const int ci = threadIdx.x % UT, cj = threadIdx.x / UT;
  const int i = i0 + ci, j = j0 + cj;
  if (i >= P.nx || j >= P.ny) return;
  const long long k = (long long)j * P.nx + i;
  if (!is_leaf(P, k)) {  // a node of a frozen grid that is not a leaf: still water
    Out[k] = T(1);
#pragma unroll
    for (int m = 1; m < 9; m++) Out[m * n + k] = T(0);
    clip[k] = 0;
    return;
  }
  const T dt = (T)dts[step];
  const T g = P.g, s3 = s3v<T>(), dxl = P.dx;
  // faces E, W (x faces (ci+1, cj), (ci, cj)) and N, S (y faces (ci, cj+1),
  // (ci, cj)); the cell is the low side of E and N, the high side of W and S
  const int qf[4] = {cj * (UT + 1) + ci + 1, cj * (UT + 1) + ci, UFX + (cj + 1) * UT + ci, UFX + cj * UT + ci};
  const int side[4] = {0, 4, 0, 4};
  T Fh[4][3], hs[4], us[4], vs[4], zr[4];
#pragma unroll
  for (int f = 0; f < 4; f++) {
    Fh[f][0] = sF[qf[f]][0]; Fh[f][1] = sF[qf[f]][1]; Fh[f][2] = sF[qf[f]][2];
    hs[f] = sR[qf[f]][side[f]];
    us[f] = sR[qf[f]][side[f] + 1];
    vs[f] = sR[qf[f]][side[f] + 2];
    zr[f] = sR[qf[f]][side[f] + 3];
  }
  T Fx[2][3], Gy[2][3];
#pragma unroll
  for (int a = 0; a < 2; a++) {
    int f = a;
    const T q = hs[f] * us[f];
    Fx[a][0] = q;
    Fx[a][1] = q * us[f] + T(0.5) * g * hs[f] * hs[f];
    Fx[a][2] = q * vs[f];
    f = 2 + a;
    const T r = hs[f] * vs[f];
    Gy[a][0] = r;
    Gy[a][1] = r * us[f];
    Gy[a][2] = r * vs[f] + T(0.5) * g * hs[f] * hs[f];
  }
  const T w1 = Wfx[n + k], w2 = Wfx[2 * n + k], zc1 = Zfx[n + k], zc2 = Zfx[2 * n + k];
  T o[9];
#pragma unroll
  for (int v = 0; v < 3; v++) {
    T L0 = -(Fh[0][v] - Fh[1][v]) / dxl - (Fh[2][v] - Fh[3][v]) / dxl;
    if (v == 1) L0 = L0 + -g * T(0.5) * (hs[0] + hs[1]) * (zr[0] - zr[1]) / dxl;
    if (v == 2) L0 = L0 + -g * T(0.5) * (hs[2] + hs[3]) * (zr[2] - zr[3]) / dxl;
    T L1x = -(s3 / dxl) * (Fh[0][v] + Fh[1][v] - Fx[0][v] - Fx[1][v]);
    T L1y = -(s3 / dxl) * (Fh[2][v] + Fh[3][v] - Gy[0][v] - Gy[1][v]);
    if (v == 1) L1x = L1x + -(T(2) * s3 * g / dxl) * w1 * (w1 + zc1);
    if (v == 2) L1y = L1y + -(T(2) * s3 * g / dxl) * w2 * (w2 + zc2);
    const T Lo[3] = {L0, L1x, L1y};
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const int m = 3 * v + c;
      if (stage == 1) o[m] = Wst[m * n + k] + dt * Lo[c];
      else o[m] = T(0.5) * (W1[m * n + k] + Wst[m * n + k] + dt * Lo[c]);
    }
  }
  // this stage's bit is written, the other stage's kept (a recomputed stage 1
  // must not erase the recorded stage-2 bit)
  const uint8_t mine = (uint8_t)(1u << (stage - 1));
  uint8_t bits = (uint8_t)(clip[k] & ~mine);
  if (o[0] < T(0)) {
    o[0] = T(0);
    bits |= mine;
  }
  if (!(o[0] > P.hd)) {
#pragma unroll
    for (int m = 1; m < 9; m++) o[m] = T(0);
  }
  clip[k] = bits;
#pragma unroll
  for (int m = 0; m < 9; m++) Out[m * n + k] = o[m];
}

// Eq. 8: vertex raster (FP64) -> planes, computed in FP64 and stored in T
template <typename T>
__global__ void __launch_bounds__(TPB) k_project(Par<T> P, const double *vert, T *out) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long w = P.nx + 1;
  const double s3 = s3v<double>();
  const double sw = vert[j * w + i], se = vert[j * w + i + 1];
  const double nw = vert[(j + 1) * w + i], ne = vert[(j + 1) * w + i + 1];
  const double zn = 0.5 * (nw + ne), zs = 0.5 * (sw + se);
  const double zE = 0.5 * (ne + se), zW = 0.5 * (nw + sw);
  out[k] = (T)(0.5 * (zE + zW));
  out[P.n + k] = (T)((zE - zW) / (2.0 * s3));
  out[2 * P.n + k] = (T)((zn - zs) / (2.0 * s3));
}

// transpose of k_project: each vertex gathers from the up to four cells
// that touch it
template <typename T>
__global__ void __launch_bounds__(TPB) k_project_t(Par<T> P, const T *gp, T *gv) {
  const long long w = P.nx + 1;
  const long long v = (long long)blockIdx.x * TPB + threadIdx.x;
  if (v >= w * (P.ny + 1)) return;
  const int j = (int)(v / w), i = (int)(v - (long long)j * w);
  const T s3 = s3v<T>();
  T acc = T(0);
  for (int cj = j - 1; cj <= j; cj++)
    for (int ci = i - 1; ci <= i; ci++) {
      if (ci < 0 || cj < 0 || ci >= P.nx || cj >= P.ny) continue;
      const long long k = (long long)cj * P.nx + ci;
      const T sx = ci == i ? T(-1) : T(1);   // west or east column of the cell
      const T sy = cj == j ? T(-1) : T(1);   // south or north row
      // c0 = (sw + se + nw + ne) / 4; c1x = (ne + se - nw - sw) / (4 s3);
      // c1y = (nw + ne - sw - se) / (4 s3)
      acc += T(0.25) * gp[k] + sx * gp[P.n + k] / (T(4) * s3) + sy * gp[2 * P.n + k] / (T(4) * s3);
    }
  gv[v] = acc;
}

// ---------------------------------------------------------------------------
// reverse sweep
// ---------------------------------------------------------------------------
// The cotangents a stage's output cotangent lY gives the cell's operator:
// lo = lY through the positivity clip and the dry reset (the clip recorded
// in bit stage - 1, the dry reset read off the stage's output Y), and
// lL = lo times the RK2 weight of the operator (dt, or dt / 2 in stage 2).
template <typename T>
__device__ __forceinline__ void stage_cot(const Par<T> &P, int stage, T dt, const T *lY, const T *Y,
                                          const uint8_t *clip, long long k, T lo[9], T lL[9]) {
  const long long n = P.ns;
  if (!is_leaf(P, k)) {  // a frozen grid's non-leaf node: its output is constant
#pragma unroll
    for (int m = 0; m < 9; m++) lo[m] = lL[m] = T(0);
    return;
  }
  const bool clipped = (clip[k] >> (stage - 1)) & 1u;
  const bool dry = !(Y[k] > P.hd);
  const T wL = stage == 2 ? T(0.5) * dt : dt;
#pragma unroll
  for (int m = 0; m < 9; m++) {
    T l = lY[m * n + k];
    if ((m == 0 && clipped) || (m > 0 && dry)) l = T(0);
    lo[m] = l;
    lL[m] = wL * l;
  }
}

// the cell's own revised limits at its face f (the other side's bed limit,
// or its own on the boundary, sets the interface bed)
template <typename T>
__device__ __forceinline__ Side<T> own_revised(const Par<T> &P, const T *W, const T *Z, int i, int j, int f) {
  const long long k = (long long)j * P.nx + i;
  const Lim<T> o = cell_lim(W, Z, P.ns, k, f);
  const int di = f == 0 ? 1 : f == 1 ? -1 : 0, dj = f == 2 ? 1 : f == 3 ? -1 : 0;
  const int a = i + di, b = j + dj;
  T zb = o.z;
  if (a >= 0 && b >= 0 && a < P.nx && b < P.ny) {
    T avg[3];
    zb = node_lim(P, W, Z, a, b, f ^ 1, avg).z;
  }
  return revise_h(o.h, o.qx, o.qy, o.z, tmax(o.z, zb), P.hd);
}

// What one cell's operator (Eq. 4, with lL its cotangent) gives its face f:
// the cotangent of the face flux (lF) and of the cell's own revised limits
// there (lr: hs, u, v, zr).  sf are those revised limits, so the ones at the
// opposite face (the bed source couples the two faces of a direction).
template <typename T>
__device__ __forceinline__ void cell_face_cot(const Par<T> &P, int f, const T lL[9], const Side<T> &sf,
                                              const Side<T> &so, T lF[3], T lr[4]) {
  const T g = P.g, rdx = T(1) / P.dx;
  const T kx = -(s3v<T>() * rdx);
  const T c = -g * T(0.5) * rdx;
  const bool xf = f < 2, plus = (f == 0 || f == 2);
  T lP[3];
#pragma unroll
  for (int v = 0; v < 3; v++) {
    const T l0 = lL[3 * v], ls = xf ? lL[3 * v + 1] : lL[3 * v + 2];
    lF[v] = (plus ? -l0 : l0) * rdx + kx * ls;   // L0 = -(F0 - F1)/dx - (F2 - F3)/dx; L1 = kx (F+ + F-)
    lP[v] = -kx * ls;                            // the physical flux of the own revised limits
  }
  lr[0] = lr[1] = lr[2] = lr[3] = T(0);
  if (xf) {
    const T q = sf.hs * sf.u;
    const T lq = lP[0] + lP[1] * sf.u + lP[2] * sf.v;
    lr[1] += lP[1] * q;
    lr[2] += lP[2] * q;
    lr[0] += lP[1] * g * sf.hs;
    lr[0] += lq * sf.u;
    lr[1] += lq * sf.hs;
  } else {
    const T r = sf.hs * sf.v;
    const T lq = lP[0] + lP[1] * sf.u + lP[2] * sf.v;
    lr[1] += lP[1] * r;
    lr[2] += lP[2] * r;
    lr[0] += lP[2] * g * sf.hs;
    lr[0] += lq * sf.v;
    lr[2] += lq * sf.hs;
  }
  // bed source of L0 in this direction: c (hs+ + hs-)(zr+ - zr-)
  const T l0s = xf ? lL[3] : lL[6];
  const T hsA = plus ? sf.hs : so.hs, hsB = plus ? so.hs : sf.hs;
  const T zrA = plus ? sf.zr : so.zr, zrB = plus ? so.zr : sf.zr;
  lr[0] += l0s * c * (zrA - zrB);
  lr[3] += (plus ? T(1) : T(-1)) * l0s * c * (hsA + hsB);
}

// reverse of hll(): cotangents of (hL, unL, utL, hR, unR, utR) from those of F
template <typename T>
__device__ void hll_rev(T hL, T unL, T utL, T hR, T unR, T utR, T g, T hd, const T lF[3], T l[6]) {
#pragma unroll
  for (int q = 0; q < 6; q++) l[q] = T(0);
  const bool dryL = !(hL > hd), dryR = !(hR > hd);
  if (dryL && dryR) return;
  const T cL = tsqrt(g * hL), cR = tsqrt(g * hR);
  T sL, sR;
  bool selA = false, selB = false;  // wet pair: sL from unL - cL, sR from unR + cR
  if (dryL) {
    sL = unR - T(2) * cR;
    sR = unR + cR;
  } else if (dryR) {
    sL = unL - cL;
    sR = unL + T(2) * cL;
  } else {
    const T us = T(0.5) * (unL + unR) + cL - cR;
    const T cs = T(0.5) * (cL + cR) + T(0.25) * (unL - unR);
    const T a1 = unL - cL, a2 = us - cs, b1 = unR + cR, b2 = us + cs;
    selA = a1 <= a2;
    selB = b1 >= b2;
    sL = selA ? a1 : a2;
    sR = selB ? b1 : b2;
  }
  const T qL = hL * unL, qR = hR * unR;
  T lqL = T(0), lqR = T(0), lhL = T(0), lhR = T(0), lunL = T(0), lunR = T(0), lutL = T(0), lutR = T(0);
  T lsL = T(0), lsR = T(0);
  T lFL[3] = {T(0), T(0), T(0)}, lFR[3] = {T(0), T(0), T(0)};
  if (sL >= T(0)) {
    lFL[0] = lF[0]; lFL[1] = lF[1]; lFL[2] = lF[2];
  } else if (sR <= T(0)) {
    lFR[0] = lF[0]; lFR[1] = lF[1]; lFR[2] = lF[2];
  } else {
    const T FL[3] = {qL, qL * unL + T(0.5) * g * hL * hL, qL * utL};
    const T FR[3] = {qR, qR * unR + T(0.5) * g * hR * hR, qR * utR};
    const T UL[3] = {hL, qL, hL * utL}, UR[3] = {hR, qR, hR * utR};
    const T rden = T(1) / (sR - sL);
    T lden = T(0), lUL[3], lUR[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const T N = sR * FL[c] - sL * FR[c] + sL * sR * (UR[c] - UL[c]);
      const T lN = lF[c] * rden;
      lden -= lN * N * rden;
      lsR += lN * (FL[c] + sL * (UR[c] - UL[c]));
      lsL += lN * (-FR[c] + sR * (UR[c] - UL[c]));
      lFL[c] += lN * sR;
      lFR[c] -= lN * sL;
      lUR[c] = lN * sL * sR;
      lUL[c] = -lN * sL * sR;
    }
    lsR += lden;
    lsL -= lden;
    lhL += lUL[0];
    lqL += lUL[1];
    lhL += lUL[2] * utL;
    lutL += lUL[2] * hL;
    lhR += lUR[0];
    lqR += lUR[1];
    lhR += lUR[2] * utR;
    lutR += lUR[2] * hR;
  }
  // physical fluxes of each side
  lqL += lFL[0] + lFL[1] * unL + lFL[2] * utL;
  lunL += lFL[1] * qL;
  lhL += lFL[1] * g * hL;
  lutL += lFL[2] * qL;
  lqR += lFR[0] + lFR[1] * unR + lFR[2] * utR;
  lunR += lFR[1] * qR;
  lhR += lFR[1] * g * hR;
  lutR += lFR[2] * qR;
  lhL += lqL * unL;
  lunL += lqL * hL;
  lhR += lqR * unR;
  lunR += lqR * hR;
  // wave speeds
  T lcL = T(0), lcR = T(0);
  if (dryL) {
    lunR += lsL + lsR;
    lcR += T(-2) * lsL + lsR;
  } else if (dryR) {
    lunL += lsL + lsR;
    lcL += -lsL + T(2) * lsR;
  } else {
    T lus = T(0), lcs = T(0);
    if (selA) { lunL += lsL; lcL -= lsL; }
    else { lus += lsL; lcs -= lsL; }
    if (selB) { lunR += lsR; lcR += lsR; }
    else { lus += lsR; lcs += lsR; }
    lunL += T(0.5) * lus;
    lunR += T(0.5) * lus;
    lcL += lus;
    lcR -= lus;
    lcL += T(0.5) * lcs;
    lcR += T(0.5) * lcs;
    lunL += T(0.25) * lcs;
    lunR -= T(0.25) * lcs;
  }
  if (!dryL) lhL += lcL * g * T(0.5) / cL;
  if (!dryR) lhR += lcR * g * T(0.5) / cR;
  l[0] = lhL; l[1] = lunL; l[2] = lutL;
  l[3] = lhR; l[4] = lunR; l[5] = lutR;
}

// reverse of revise_h(): cotangents of the limit (h, qx, qy, z) and of the
// interface bed zf from those of (hs, u, v, zr)
template <typename T>
__device__ __forceinline__ void revise_rev(const Lim<T> &s, T zf, T hd, T lhs, T lu, T lv, T lzr, T out[4], T &lzf) {
  const T eta = s.h + s.z;
  const T d = eta - zf;
  T leta = T(0), ld = T(0);
  if (d > hd) {
    ld = lhs;
    lzf += lzr;
  } else {
    leta += lzr;
  }
  leta += ld;
  lzf -= ld;
  out[0] = leta;
  out[3] = leta;
  out[1] = T(0);
  out[2] = T(0);
  if (s.h > hd) {
    const T rh = T(1) / s.h;
    out[1] = lu * rh;
    out[2] = lv * rh;
    out[0] -= (lu * s.qx + lv * s.qy) * rh * rh;
  }
}

// split of the cotangent of max(zL, zR)
template <typename T>
__device__ __forceinline__ void tiemax_rev(T zL, T zR, T lzf, T &lL, T &lR) {
  const T scale = tmax(T(1), tmax(tabs(zL), tabs(zR)));
  if (tabs(zL - zR) <= tie_rel<T>() * scale) {
    lL += T(0.5) * lzf;
    lR += T(0.5) * lzf;
  } else if (zL > zR) {
    lL += lzf;
  } else {
    lR += lzf;
  }
}

// reverse of ghost(): fold the ghost's cotangents into the own limit; the
// hydrograph's share (per unit of Q(t)) is returned
template <typename T>
__device__ double ghost_rev(const Par<T> &P, int e, int along, const Lim<T> &o, double t, const T lg[4], T lo[4]) {
  lo[3] += lg[3];
  const T q = (T)inflow_unit(P, e, along, t);
  if (q > T(0)) {
    const T x = q * q / P.g;
    const T hc = tcbrt<T>(x);
    T lq = T(0);
    if (o.h >= hc) lo[0] += lg[0];
    else lq += lg[0] / (T(3) * hc * hc) * (T(2) * q / P.g);
    const T sg = (e == 0 || e == 2) ? T(1) : T(-1);
    lq += sg * (e < 2 ? lg[1] : lg[2]);
    return (double)lq * (double)inflow_overlap(P, e, along) / ((double)(P.c1 - P.c0 + 1) * P.dxd);
  }
  if (P.bc[e] == MWDG_OPEN) {
    lo[0] += lg[0]; lo[1] += lg[1]; lo[2] += lg[2];
    return 0.0;
  }
  lo[0] += lg[0];
  if (e < 2) { lo[1] -= lg[1]; lo[2] += lg[2]; }
  else { lo[1] += lg[1]; lo[2] -= lg[2]; }
  return 0.0;
}

// reverse of drain_limit(): from the cotangent lG of the limited flux, the
// cotangent of the flux it limited (lF) and of the donor's averages (h0,
// q_n0, q_t0) in ld; F is the flux before the limit
template <typename T>
__device__ void drain_rev(const T F[3], T h0, T qn, T qt, T g, T hd, T dx, T dt, const T lG[3], T lF[3],
                          T ld[3]) {
  ld[0] = ld[1] = ld[2] = T(0);
  if (!(h0 > T(0))) {  // a donor without content passes nothing
    lF[0] = lF[1] = lF[2] = T(0);
    return;
  }
  T un = T(0), ut = T(0);
  const bool wet = h0 > hd;
  if (wet) {
    un = qn / h0;
    ut = qt / h0;
  }
  const T c = tsqrt(g * h0);
  const bool fwd = F[0] > T(0);
  const T out = fwd ? un : -un;
  const T e = tmax(out, T(0)) + c;
  const T S = (tabs(un) + tabs(ut)) + T(4) * c;
  const T R = h0 * dx / dt, Q = e / S;
  const T cap = R * Q;
  const T a = tabs(F[0]);
  if (!(a > cap)) {
    lF[0] = lG[0]; lF[1] = lG[1]; lF[2] = lG[2];
    return;
  }
  const T th = cap / a;
  const T sg = fwd ? T(1) : T(-1);
  T lcap = sg * lG[0];
  lF[1] = lG[1] * th;
  lF[2] = lG[2] * th;
  const T lth = lG[1] * F[1] + lG[2] * F[2];
  lcap += lth / a;
  lF[0] = -lth * th / a * sg;
  const T lR = lcap * Q, lQ = lcap * R;
  T lh0 = lR * dx / dt;
  const T le = lQ / S, lS = -lQ * Q / S;
  T lun = lS * (un > T(0) ? T(1) : un < T(0) ? T(-1) : T(0));
  const T lut = lS * (ut > T(0) ? T(1) : ut < T(0) ? T(-1) : T(0));
  T lc = T(4) * lS + le;
  if (out > T(0)) lun += fwd ? le : -le;
  lh0 += lc * g * T(0.5) / c;
  if (wet) {
    ld[1] = lun / h0;
    ld[2] = lut / h0;
    lh0 -= (lun * qn + lut * qt) / (h0 * h0);
  }
  ld[0] = lh0;
}

// Per interface: the flux cotangent from both cells, HLL and the two
// revisions in reverse, the interface bed split, the ghost folded into the
// boundary cell.  Output per face: the cotangents of the low side's limit
// (slots 0-3: h, qx, qy, z) and the high side's (slots 4-7), and those of the
// flux-view averages (h0, qx0, qy0) of the low (slots 8-10) and high (slots
// 11-13) cell through the outflow limit (non-zero for its donor only); `lq`,
// per boundary cell of the inflow edge, the cotangent of Q(t).
template <typename T, bool XF, bool ML>
__global__ void __launch_bounds__(TPB) k_rev_face(const Levels<T> LV, int stage, const double *dts, const double *tt,
                                                  int step, const T *Wfx, const T *Zfx, const T *lY, const T *Y,
                                                  const uint8_t *clip, T *lim, double *lq) {
  __shared__ Par<T> sP;
  unsigned bl;
  const Par<T> &P = block_level<ML>(LV, sP, bl);
  Wfx += P.off;
  Zfx += P.off;
  lY += P.off;
  Y += P.off;
  clip += P.off;
  lim += 14 * (XF ? P.fx : P.fy);
  lq += P.lqo;
  const long long nf = XF ? (long long)P.ny * (P.nx + 1) : (long long)(P.ny + 1) * P.nx;
  const long long fi = (long long)bl * TPB + threadIdx.x;
  if (fi >= nf) return;
  const double t = stage == 1 ? tt[step] : tt[step] + dts[step];
  int i, j;  // the high-side cell (i, j); the low side is (i-1, j) or (i, j-1)
  if (XF) { j = (int)(fi / (P.nx + 1)); i = (int)(fi - (long long)j * (P.nx + 1)); }
  else { j = (int)(fi / P.nx); i = (int)(fi - (long long)j * P.nx); }
  const int fLo = XF ? 0 : 2, fHi = XF ? 1 : 3;      // the low cell's face, the high cell's face
  const int eLo = XF ? 0 : 2, eHi = XF ? 1 : 3;      // edges W/S and E/N
  const bool hasLo = XF ? i > 0 : j > 0;
  const bool hasHi = XF ? i < P.nx : j < P.ny;
  const long long kLo = XF ? (long long)j * P.nx + (i - 1) : (long long)(j - 1) * P.nx + i;
  const long long kHi = (long long)j * P.nx + i;
  const int along = XF ? j : i;
  if (P.kind && !(hasLo && P.kind[kLo] == K_LEAF) && !(hasHi && P.kind[kHi] == K_LEAF)) {
    // a frozen grid's face between non-leaf nodes: no operator reads it
#pragma unroll
    for (int q = 0; q < 14; q++) lim[q * nf + fi] = T(0);
    if ((!hasLo && P.inflow_edge == eLo) || (!hasHi && P.inflow_edge == eHi)) lq[along] = 0.0;
    return;
  }
  Lim<T> lo, hi;
  T aLo[3], aHi[3];
  if (hasLo) lo = node_lim(P, Wfx, Zfx, XF ? i - 1 : i, XF ? j : j - 1, fLo, aLo);
  if (hasHi) hi = node_lim(P, Wfx, Zfx, i, j, fHi, aHi);
  if (!hasLo) lo = ghost(P, eLo, along, hi, t);
  if (!hasHi) hi = ghost(P, eHi, along, lo, t);
  const T zf = tmax(lo.z, hi.z);
  const Side<T> sLo = revise_h(lo.h, lo.qx, lo.qy, lo.z, zf, P.hd);
  const Side<T> sHi = revise_h(hi.h, hi.qx, hi.qy, hi.z, zf, P.hd);
  // each adjacent cell's operator: its share of the flux cotangent and the
  // cotangents of its own revised limits at this face
  const T dt = (T)dts[step];
  T lF[3] = {T(0), T(0), T(0)}, cLo[4] = {T(0), T(0), T(0), T(0)}, cHi[4] = {T(0), T(0), T(0), T(0)};
  if (hasLo && is_leaf(P, kLo)) {
    T lo_[9], lL[9], f3[3];
    stage_cot(P, stage, dt, lY, Y, clip, kLo, lo_, lL);
    const Side<T> opp = own_revised(P, Wfx, Zfx, XF ? i - 1 : i, XF ? j : j - 1, fLo ^ 1);
    cell_face_cot(P, fLo, lL, sLo, opp, f3, cLo);
    lF[0] += f3[0]; lF[1] += f3[1]; lF[2] += f3[2];
  }
  if (hasHi && is_leaf(P, kHi)) {
    T lo_[9], lL[9], f3[3];
    stage_cot(P, stage, dt, lY, Y, clip, kHi, lo_, lL);
    const Side<T> opp = own_revised(P, Wfx, Zfx, i, j, fHi ^ 1);
    cell_face_cot(P, fHi, lL, sHi, opp, f3, cHi);
    lF[0] += f3[0]; lF[1] += f3[1]; lF[2] += f3[2];
  }
  // the outflow limit in reverse: the flux before it and the donor's averages
  T dLo[3] = {T(0), T(0), T(0)}, dHi[3] = {T(0), T(0), T(0)};
  {
    T H[3], F[3];
    if (XF) {
      hll(sLo.hs, sLo.u, sLo.v, sHi.hs, sHi.u, sHi.v, P.g, P.hd, H);
      F[0] = H[0]; F[1] = H[1]; F[2] = H[2];
    } else {
      hll(sLo.hs, sLo.v, sLo.u, sHi.hs, sHi.v, sHi.u, P.g, P.hd, H);
      F[0] = H[0]; F[1] = H[2]; F[2] = H[1];
    }
    const bool donLo = F[0] > T(0) && hasLo, donHi = F[0] < T(0) && hasHi;
    if (donLo || donHi) {
      const T h0 = donLo ? aLo[0] : aHi[0], qx0 = donLo ? aLo[1] : aHi[1], qy0 = donLo ? aLo[2] : aHi[2];
      T lG[3] = {lF[0], lF[1], lF[2]}, ld[3];
      drain_rev(F, h0, XF ? qx0 : qy0, XF ? qy0 : qx0, P.g, P.hd, P.dx, dt, lG, lF, ld);
      T *dd = F[0] > T(0) ? dLo : dHi;  // the low side is the donor of an outflow along +x / +y
      dd[0] = ld[0];
      dd[1] = XF ? ld[1] : ld[2];
      dd[2] = XF ? ld[2] : ld[1];
    }
  }
  T l6[6];
  if (XF) {
    hll_rev(sLo.hs, sLo.u, sLo.v, sHi.hs, sHi.u, sHi.v, P.g, P.hd, lF, l6);
  } else {
    const T lH[3] = {lF[0], lF[2], lF[1]};
    hll_rev(sLo.hs, sLo.v, sLo.u, sHi.hs, sHi.v, sHi.u, P.g, P.hd, lH, l6);
  }
  // cotangents of (hs, u, v, zr) of each side
  T rLo[4], rHi[4];
  rLo[0] = l6[0];
  rHi[0] = l6[3];
  if (XF) { rLo[1] = l6[1]; rLo[2] = l6[2]; rHi[1] = l6[4]; rHi[2] = l6[5]; }
  else { rLo[2] = l6[1]; rLo[1] = l6[2]; rHi[2] = l6[4]; rHi[1] = l6[5]; }
  rLo[3] = T(0);
  rHi[3] = T(0);
#pragma unroll
  for (int q = 0; q < 4; q++) {
    rLo[q] += cLo[q];
    rHi[q] += cHi[q];
  }
  T gLo[4], gHi[4], lzf = T(0);
  revise_rev(lo, zf, P.hd, rLo[0], rLo[1], rLo[2], rLo[3], gLo, lzf);
  revise_rev(hi, zf, P.hd, rHi[0], rHi[1], rHi[2], rHi[3], gHi, lzf);
  tiemax_rev(lo.z, hi.z, lzf, gLo[3], gHi[3]);
  if (!hasLo) {
    T f4[4] = {T(0), T(0), T(0), T(0)};
    const double lQ = ghost_rev(P, eLo, along, hi, t, gLo, f4);
    for (int q = 0; q < 4; q++) { gHi[q] += f4[q]; gLo[q] = T(0); }
    if (P.inflow_edge == eLo) lq[along] = lQ;
  }
  if (!hasHi) {
    T f4[4] = {T(0), T(0), T(0), T(0)};
    const double lQ = ghost_rev(P, eHi, along, lo, t, gHi, f4);
    for (int q = 0; q < 4; q++) { gLo[q] += f4[q]; gHi[q] = T(0); }
    if (P.inflow_edge == eHi) lq[along] = lQ;
  }
#pragma unroll
  for (int q = 0; q < 4; q++) {
    lim[q * nf + fi] = gLo[q];
    lim[(4 + q) * nf + fi] = gHi[q];
  }
#pragma unroll
  for (int q = 0; q < 3; q++) {
    lim[(8 + q) * nf + fi] = dLo[q];
    lim[(11 + q) * nf + fi] = dHi[q];
  }
}

// hydrograph knots: the cotangent of Q(t) summed over the inflow edge in a
// fixed order, spread over the two knots around t
template <typename T>
__global__ void k_rev_knots(const Levels<T> LV, int stage, const double *dts, const double *tt, int step,
                            const double *lq, double *gQ) {
  __shared__ double sh[TPB];
  __shared__ Par<T> sP;
  for (int l = 0; l < LV.n; l++) {  // levels in order, each its own sum
    if (threadIdx.x == 0) sP = LV.P[l];
    __syncthreads();
    const Par<T> &P = sP;
    const int nedge = (P.inflow_edge < 2) ? P.ny : P.nx;
    double acc = 0.0;
    for (int a = threadIdx.x; a < nedge; a += TPB)
      if (inflow_overlap(P, P.inflow_edge, a) > 0) acc += lq[P.lqo + a];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = TPB / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double t = stage == 1 ? tt[step] : tt[step] + dts[step];
      int k0, k1;
      double r;
      hydro(P, t, k0, k1, r);
      const double v = sh[0];
      if (k0 == k1) {
        gQ[k0] += v;
      } else {
        gQ[k0] += v - v * r;
        gQ[k1] += v * r;
      }
    }
    __syncthreads();
  }
}

// The cotangents of a cell's flux-view planes (9 flow, 3 bed) from its four
// faces: the face-limit transpose of the limits' cotangents (E = low side of
// x face (j, i + 1), W = high side of x face (j, i), N = low side of y face
// (j + 1, i), S = high side of y face (j, i)) and the averages' cotangents
// from the outflow limit of the four interfaces.
template <typename T>
__device__ __forceinline__ void face_plane_cot(const Par<T> &P, int i, int j, const T *limx, const T *limy, T lw[9],
                                               T lz[3]) {
  const long long nfx = (long long)P.ny * (P.nx + 1), nfy = (long long)(P.ny + 1) * P.nx;
  const T s3 = s3v<T>();
  T lf[4][4];
  const long long fE = (long long)j * (P.nx + 1) + i + 1, fW = (long long)j * (P.nx + 1) + i;
  const long long fN = (long long)(j + 1) * P.nx + i, fS = (long long)j * P.nx + i;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    lf[0][q] = limx[q * nfx + fE];
    lf[1][q] = limx[(4 + q) * nfx + fW];
    lf[2][q] = limy[q * nfy + fN];
    lf[3][q] = limy[(4 + q) * nfy + fS];
  }
#pragma unroll
  for (int v = 0; v < 4; v++) {
    const T a = lf[0][v] + lf[1][v] + lf[2][v] + lf[3][v];
    const T bx = s3 * (lf[0][v] - lf[1][v]);
    const T by = s3 * (lf[2][v] - lf[3][v]);
    if (v < 3) { lw[3 * v] = a; lw[3 * v + 1] = bx; lw[3 * v + 2] = by; }
    else { lz[0] = a; lz[1] = bx; lz[2] = by; }
  }
#pragma unroll
  for (int v = 0; v < 3; v++)
    lw[3 * v] += ((limx[(8 + v) * nfx + fE] + limx[(11 + v) * nfx + fW]) + limy[(8 + v) * nfy + fN]) +
                 limy[(11 + v) * nfy + fS];
}

// Face-limit transpose and the limiter in reverse for one cell: the
// cotangent of the stage input X of this cell (lXo) and the shares of its
// neighbours' averages (lnb: direction, side A/B, variable), the bed's own
// cotangents added to gz.  GV: the flux-view planes' cotangents come
// gathered in gV (12 planes: a frozen grid, where views pass them between
// levels), else from the cell's four faces.
template <typename T, bool GV>
__global__ void __launch_bounds__(TPB) k_rev_limit(const Levels<T> LV, int stage, const double *dts, int step,
                                                   const T *X, const T *Z, const T *lY, const T *Y,
                                                   const uint8_t *clip, T *lW1, const T *limx, const T *limy,
                                                   const T *gV, T *lXo, T *lnb, T *gz) {
  __shared__ Par<T> sP;
  unsigned bl;
  const Par<T> &P = block_level<GV>(LV, sP, bl);
  X += P.off;
  Z += P.off;
  lY += P.off;
  Y += P.off;
  clip += P.off;
  lW1 += P.off;
  if (GV) gV += P.off;
  else {
    limx += 14 * P.fx;
    limy += 14 * P.fy;
  }
  lXo += P.off;
  lnb += P.off;
  gz += P.off;
  long long k;
  int i, j;
  if (!node_of(P, bl, k, i, j)) return;
  const long long n = P.ns;
  if (!is_leaf(P, k)) {  // no cotangent reaches a frozen grid's non-leaf node
#pragma unroll
    for (int m = 0; m < 9; m++) {
      lXo[m * n + k] = T(0);
      if (stage == 2) lW1[m * n + k] = T(0);
    }
#pragma unroll
    for (int m = 0; m < 12; m++) lnb[m * n + k] = T(0);
    return;
  }
  const T rs3 = T(1) / s3v<T>();
  T ws[9], wf[9], ze[3];
  LimRec r;
  limit_cell(P, X, Z, i, j, ws, wf, ze, r);
  T lw[9], lz[3];
  if (GV) {
#pragma unroll
    for (int m = 0; m < 9; m++) lw[m] = gV[m * n + k];
#pragma unroll
    for (int m = 0; m < 3; m++) lz[m] = gV[(9 + m) * n + k];
  } else {
    face_plane_cot(P, i, j, limx, limy, lw, lz);
  }
  // the stage's output cotangent: the stored view's share (stage 2 also
  // passes half to the stage-1 view) and the slope bed sources
  // S1 = c2 h1 (h1 + z1) of the flux view
  T lo_[9], lL[9], lsw[9];
  stage_cot(P, stage, (T)dts[step], lY, Y, clip, k, lo_, lL);
#pragma unroll
  for (int m = 0; m < 9; m++) {
    if (stage == 2) {
      lsw[m] = T(0.5) * lo_[m];
      lW1[m * n + k] = T(0.5) * lo_[m];
    } else {
      lsw[m] = lo_[m] + lW1[m * n + k];
    }
  }
  {
    const T c2 = -(T(2) * s3v<T>() * P.g / P.dx);
    lw[1] += lL[4] * c2 * (T(2) * wf[1] + ze[1]);
    lw[2] += lL[8] * c2 * (T(2) * wf[2] + ze[2]);
    lz[1] += lL[4] * c2 * wf[1];
    lz[2] += lL[8] * c2 * wf[2];
  }
  T lX[9], gzz[3] = {T(0), T(0), T(0)}, nb[2][2][3] = {};
  if (r.red) {
#pragma unroll
    for (int m = 0; m < 9; m++) lX[m] = T(0);
    lX[0] = lsw[0] + lw[0];
    lX[3] = lsw[3] + lw[3];
    lX[6] = lsw[6] + lw[6];
    gzz[1] -= lsw[1];
    gzz[2] -= lsw[2];
    gzz[0] += lz[0];
  } else {
    T lt[9];
#pragma unroll
    for (int m = 0; m < 9; m++) {
      lt[m] = lsw[m] + lw[m];
      lX[m] = lt[m];
    }
#pragma unroll
    for (int q = 0; q < 3; q++) gzz[q] += lz[q];
#pragma unroll
    for (int d = 0; d < 2; d++)
#pragma unroll
      for (int v = 0; v < 3; v++) {
        const int sel = r.sel[d][v];
        if (sel == 0) continue;
        const int cs = 1 + d, coef = v == 0 ? cs : 3 * v + cs;
        const T l = lt[coef];
        lX[coef] = T(0);
        if (v == 0) gzz[cs] -= l;
        const T lmm = l * rs3;
        T laC = T(0);
        if (sel == 1) { nb[d][0][v] += lmm; laC -= lmm; }
        else if (sel == 2) { laC += lmm; nb[d][1][v] -= lmm; }
        lX[3 * v] += laC;
        if (v == 0) gzz[0] += laC;
      }
  }
#pragma unroll
  for (int m = 0; m < 9; m++) lXo[m * n + k] = lX[m];
#pragma unroll
  for (int d = 0; d < 2; d++)
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
      for (int v = 0; v < 3; v++) lnb[((d * 2 + s) * 3 + v) * n + k] = nb[d][s][v];
#pragma unroll
  for (int q = 0; q < 3; q++) gz[q * n + k] += gzz[q];
}

// cotangent of the stage input: the cell's own share and its neighbours'
// (a cell's side-A neighbour in x is (i+1, j): the share it holds for this
// cell sits with (i-1, j) under side A, and so on); the average of eta in
// the limiter is h0 + z0, so the bed average takes the eta shares too
template <typename T, bool ML>
__global__ void __launch_bounds__(TPB) k_rev_gather(const Levels<T> LV, const T *lXo, const T *lnb, T *lX, T *gz) {
  __shared__ Par<T> sP;
  unsigned bl;
  const Par<T> &P = block_level<ML>(LV, sP, bl);
  lXo += P.off;
  lnb += P.off;
  lX += P.off;
  gz += P.off;
  long long k;
  int i, j;
  if (!node_of(P, bl, k, i, j)) return;
  const long long n = P.ns;
  if (!is_leaf(P, k)) {
#pragma unroll
    for (int m = 0; m < 9; m++) lX[m * n + k] = T(0);
    return;
  }
  T in[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int v = 0; v < 3; v++) {
    if (i > 0) in[v] += lnb[((0 * 2 + 0) * 3 + v) * n + k - 1];
    if (i < P.nx - 1) in[v] += lnb[((0 * 2 + 1) * 3 + v) * n + k + 1];
    if (j > 0) in[v] += lnb[((1 * 2 + 0) * 3 + v) * n + k - P.nx];
    if (j < P.ny - 1) in[v] += lnb[((1 * 2 + 1) * 3 + v) * n + k + P.nx];
  }
#pragma unroll
  for (int m = 0; m < 9; m++) {
    T l = lXo[m * n + k];
    if (m % 3 == 0) l += in[m / 3];
    lX[m * n + k] = l;
  }
  gz[k] += in[0];
}

// friction (and rain) in reverse: lU = cotangent of the step's input state,
// Manning n's share added to gn
template <typename T, bool ML>
__global__ void __launch_bounds__(TPB) k_rev_friction(const Levels<T> LV, const T *U, const T *nman,
                                                      const double *dts, const double *tt, int step, const T *lUn,
                                                      T *lU, T *gn) {
  __shared__ Par<T> sP;
  unsigned bl;
  const Par<T> &P = block_level<ML>(LV, sP, bl);
  U += P.off;
  nman += P.off;
  lUn += P.off;
  lU += P.off;
  gn += P.off;
  long long k;
  int i, j;
  if (!node_of(P, bl, k, i, j)) return;
  const long long n = P.ns;
  if (!is_leaf(P, k)) {
#pragma unroll
    for (int m = 0; m < 9; m++) lU[m * n + k] = T(0);
    return;
  }
  const T dt = (T)dts[step], g = P.g;
  const double t = tt[step];
  const double rain = (t < P.rain_t_end) ? P.rain_rate : 0.0;
  T w[9], l[9], lo[9];
#pragma unroll
  for (int m = 0; m < 9; m++) {
    w[m] = U[m * n + k];
    l[m] = lUn[m * n + k];
  }
  if (rain > 0.0) w[0] = w[0] + (T)(rain * dts[step]);
  const T h0 = w[0];
  lo[0] = l[0];
  lo[1] = l[1];
  lo[2] = l[2];
  T lnm = T(0);
  if (h0 > P.hd) {
    const T rh = T(1) / h0;
    const T u = w[3] * rh, v = w[6] * rh;
    const T sp = tsqrt(u * u + v * v);
    const T nm = nman[k];
    const T cr = tcbrt<T>(h0);
    const T B = h0 * cr, rB = T(1) / B;
    const T A = dt * g * nm * nm;
    const T den = T(1) + A * sp * rB;
    const T f = T(1) / den;
    T lf = T(0);
#pragma unroll
    for (int m = 3; m < 9; m++) {
      lo[m] = l[m] * f;
      lf += l[m] * w[m];
    }
    const T lden = -lf * f * f;
    const T lsp = lden * A * rB;
    const T lB = -lden * A * sp * rB * rB;
    lnm = lden * sp * rB * (dt * g * T(2) * nm);
    T lh = lB * (cr + h0 / (T(3) * cr * cr));
    if (sp > T(0)) {
      const T lu = lsp * u / sp, lv = lsp * v / sp;
      lo[3] += lu * rh;
      lo[6] += lv * rh;
      lh -= (lu * u + lv * v) * rh;
    }
    lo[0] += lh;
  } else {
#pragma unroll
    for (int m = 3; m < 9; m++) lo[m] = T(0);
  }
#pragma unroll
  for (int m = 0; m < 9; m++) lU[m * n + k] = lo[m];
  gn[k] += lnm;
}

// ---------------------------------------------------------------------------
// frozen non-uniform grids: the views in reverse, leaves in and out, and the
// level pyramids of the bed (Eq. 9) and of Manning's n (children's mean)
// ---------------------------------------------------------------------------
// The cotangent of every node's view planes (gV: 9 flow, 3 bed) from the
// interfaces of its level: its four faces (face_plane_cot), except where
// the node's faces show the mean of its children (a refined node of a static
// grid).  A child of such a node takes half of the cotangent of the mean on
// each of its parent's faces that it touches (the parent level's slots px,
// py).
template <typename T>
__global__ void __launch_bounds__(TPB) k_rev_view_gather(const Levels<T> LV, const T *limx, const T *limy,
                                                         T *gV) {
  __shared__ Par<T> sP;
  unsigned bl;
  const Par<T> &P = block_level<true>(LV, sP, bl);
  const T *px = limx + 14 * P.fxp, *py = limy + 14 * P.fyp;  // the parent level's faces
  limx += 14 * P.fx;
  limy += 14 * P.fy;
  gV += P.off;
  long long k;
  int i, j;
  if (!node_of(P, bl, k, i, j)) return;
  const long long n = P.ns;
  T lw[9], lz[3];
  if (P.stat && P.kind[k] == K_SIG) {
#pragma unroll
    for (int m = 0; m < 9; m++) lw[m] = T(0);
    lz[0] = lz[1] = lz[2] = T(0);
  } else {
    face_plane_cot(P, i, j, limx, limy, lw, lz);
  }
  if (P.stat && P.dp > 0) {
    const int pnx = P.nx >> 1, pny = P.ny >> 1, pi = i >> 1, pj = j >> 1;
    if (P.kind[-P.dp + (long long)pj * pnx + pi] == K_SIG) {
      const long long pfx = (long long)pny * (pnx + 1), pfy = (long long)(pny + 1) * pnx;
      const T s3 = s3v<T>();
      // the parent's face in x (E when the node is an east child: the low
      // side of x face (pj, pi + 1); else W, the high side of (pj, pi)) and
      // in y (N / S likewise)
      const bool east = i & 1, north = j & 1;
      const long long fx = (long long)pj * (pnx + 1) + pi + (east ? 1 : 0);
      const long long fy = (long long)(pj + (north ? 1 : 0)) * pnx + pi;
      const int sx = east ? 0 : 4, sy = north ? 0 : 4;     // limit slots of the parent's side
      const int ax = east ? 8 : 11, ay = north ? 8 : 11;   // average slots
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const T lx = T(0.5) * px[(sx + q) * pfx + fx], ly = T(0.5) * py[(sy + q) * pfy + fy];
        T *c = q < 3 ? lw + 3 * q : lz;
        c[0] += lx + ly;
        c[1] += east ? s3 * lx : -(s3 * lx);
        c[2] += north ? s3 * ly : -(s3 * ly);
      }
#pragma unroll
      for (int v = 0; v < 3; v++) lw[3 * v] += T(0.5) * px[(ax + v) * pfx + fx] + T(0.5) * py[(ay + v) * pfy + fy];
    }
  }
#pragma unroll
  for (int m = 0; m < 9; m++) gV[m * n + k] = lw[m];
#pragma unroll
  for (int m = 0; m < 3; m++) gV[(9 + m) * n + k] = lz[m];
}

// transpose of the prolongation: a leaf or a node below a coarser leaf (this
// level) takes the cotangents of its children that are below it (the next
// level); run from the finest level up
template <typename T>
__device__ __forceinline__ void rev_prolong_node(const Par<T> &P, T *gV, long long k, int i, int j) {
  if (P.kind[k] == K_SIG) return;
  const long long n = P.ns;
  T acc[12];
#pragma unroll
  for (int m = 0; m < 12; m++) acc[m] = gV[m * n + k];
  bool any = false;
#pragma unroll 1
  for (int c = 0; c < 4; c++) {
    const long long kc = child_of(P, i, j, c);
    if (P.kind[kc] != K_BELOW) continue;
    any = true;
#pragma unroll
    for (int v = 0; v < 4; v++) {
      T gc[3];
#pragma unroll
      for (int m = 0; m < 3; m++) gc[m] = gV[(3 * v + m) * n + kc];
      prolong3_t(gc, c, acc + 3 * v);
    }
  }
  if (!any) return;
#pragma unroll
  for (int m = 0; m < 12; m++) gV[m * n + k] = acc[m];
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_rev_prolong(Par<T> P, T *gV) {
  long long k;
  int i, j;
  if (cell_of(P, k, i, j)) rev_prolong_node(P, gV, k, i, j);
}

// transpose of the encoding: a child of a refined node (this level) takes
// its share of the parent's cotangents (the previous level); run from the
// coarsest level down
template <typename T>
__device__ __forceinline__ void rev_encode_node(const Par<T> &P, T *gV, long long k, int i, int j) {
  const long long kp = -P.dp + (long long)(j >> 1) * (P.nx >> 1) + (i >> 1);
  if (P.kind[kp] != K_SIG) return;
  const long long n = P.ns;
  const int c = (i & 1) + 2 * (j & 1);
#pragma unroll
  for (int v = 0; v < 4; v++) {
    T gp[3], gc[3];
#pragma unroll
    for (int m = 0; m < 3; m++) {
      gp[m] = gV[(3 * v + m) * n + kp];
      gc[m] = gV[(3 * v + m) * n + k];
    }
    encode3_t(gp, c, gc);
#pragma unroll
    for (int m = 0; m < 3; m++) gV[(3 * v + m) * n + k] = gc[m];
  }
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_rev_encode(Par<T> P, T *gV) {
  long long k;
  int i, j;
  if (cell_of(P, k, i, j)) rev_encode_node(P, gV, k, i, j);
}

// The view passes (and their transposes) of the coarse levels, one level
// after the other in one block: levels from l0 to l1 (step +1 or -1), each
// finished before the next starts.  A and B: the flow and bed view planes
// of the forward passes, or A the view cotangents of the reverse ones.
constexpr int VP_ENCODE = 0, VP_PROLONG = 1, VP_REV_PROLONG = 2, VP_REV_ENCODE = 3;
constexpr int CTPB = 512;
template <typename T, int PASS>
__global__ void __launch_bounds__(CTPB) k_views_coarse(const Levels<T> LV, T *A, T *B, int l0, int l1) {
  __shared__ Par<T> sP;
  const int step = l1 >= l0 ? 1 : -1;
  for (int l = l0;; l += step) {
    if (threadIdx.x == 0) sP = LV.P[l];
    __syncthreads();
    const Par<T> &P = sP;
    for (long long k = threadIdx.x; k < P.n; k += CTPB) {
      const int j = (int)(k / P.nx), i = (int)(k - (long long)j * P.nx);
      if (PASS == VP_ENCODE) view_encode_node(P, A + P.off, B + P.off, k, i, j);
      else if (PASS == VP_PROLONG) view_prolong_node(P, A + P.off, B + P.off, k, i, j);
      else if (PASS == VP_REV_PROLONG) rev_prolong_node(P, A + P.off, k, i, j);
      else rev_encode_node(P, A + P.off, k, i, j);
    }
    __syncthreads();
    if (l == l1) break;
  }
}

// every node of every level to still water (h0 = 1, the rest 0)
template <typename T>
__global__ void __launch_bounds__(TPB) k_still(long long nt, T *U) {
  const long long k = (long long)blockIdx.x * TPB + threadIdx.x;
  if (k >= nt) return;
  U[k] = T(1);
#pragma unroll
  for (int m = 1; m < 9; m++) U[m * nt + k] = T(0);
}

// leaf coefficients (9 x nl, component-major) to / from their nodes in the
// level arrays (9 x nt); `node` gives each leaf's node
template <typename T>
__global__ void __launch_bounds__(TPB) k_leaves_to_nodes(long long nl, long long nt, const long long *node,
                                                         const T *src, T *dst) {
  const long long q = (long long)blockIdx.x * TPB + threadIdx.x;
  if (q >= nl) return;
  const long long k = node[q];
#pragma unroll
  for (int m = 0; m < 9; m++) dst[m * nt + k] = src[m * nl + q];
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_nodes_to_leaves(long long nl, long long nt, const long long *node,
                                                         const T *src, T *dst) {
  const long long q = (long long)blockIdx.x * TPB + threadIdx.x;
  if (q >= nl) return;
  const long long k = node[q];
#pragma unroll
  for (int m = 0; m < 9; m++) dst[m * nl + q] = src[m * nt + k];
}

// the finest level's planes (C components of stride nfin) into the level
// arrays (stride nt, offset off), or back with add = 1 (dst += src)
template <typename T>
__global__ void __launch_bounds__(TPB) k_copy_planes(int C, long long cnt, const T *src, long long ss, T *dst,
                                                     long long ds, int add) {
  const long long k = (long long)blockIdx.x * TPB + threadIdx.x;
  if (k >= cnt) return;
  for (int m = 0; m < C; m++) dst[m * ds + k] = add ? dst[m * ds + k] + src[m * ss + k] : src[m * ss + k];
}

// one level of the bed pyramid (Eq. 9 on the bed planes) and of Manning's n
// (the mean of the children), from the next finer level
template <typename T>
__global__ void __launch_bounds__(TPB) k_pyramid_level(Par<T> P, T *Z, T *N) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long n = P.ns;
  T ch[4][3], sp[3], nc[4];
#pragma unroll
  for (int c = 0; c < 4; c++) {
    const long long kc = child_of(P, i, j, c);
#pragma unroll
    for (int m = 0; m < 3; m++) ch[c][m] = Z[m * n + kc];
    nc[c] = N[kc];
  }
  encode3(ch, sp);
#pragma unroll
  for (int m = 0; m < 3; m++) Z[m * n + k] = sp[m];
  N[k] = T(0.25) * (((nc[0] + nc[1]) + nc[2]) + nc[3]);
}

// its transpose: the children (this level) take their shares of the
// parent's (the previous level) bed and Manning cotangents; run from the
// coarsest level down
template <typename T>
__global__ void __launch_bounds__(TPB) k_pyramid_level_t(Par<T> P, T *gZ, T *gN) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long n = P.ns;
  const long long kp = -P.dp + (long long)(j >> 1) * (P.nx >> 1) + (i >> 1);
  const int c = (i & 1) + 2 * (j & 1);
  T gp[3], gc[3];
#pragma unroll
  for (int m = 0; m < 3; m++) {
    gp[m] = gZ[m * n + kp];
    gc[m] = gZ[m * n + k];
  }
  encode3_t(gp, c, gc);
#pragma unroll
  for (int m = 0; m < 3; m++) gZ[m * n + k] = gc[m];
  gN[k] = gN[k] + T(0.25) * gN[kp];
}

// ---------------------------------------------------------------------------
// regridding at a checkpoint: the MWDG2 adaptation's state transfer from one
// frozen grid to the next (Sect. 2.3), and its transpose.  D holds the state
// on every node of every level of the old grid: its leaves' coefficients,
// prolonged below them (Eq. 10 with zero details; a depth plane is first
// kept non-negative for its children) and encoded up its refined nodes
// (Eq. 9); the new grid's leaves read it at their nodes.
// ---------------------------------------------------------------------------
// The depth plane that a refinement prolongs: where a child's average would
// be negative, the slopes are scaled about the average so that the
// smallest child (the first in child order) is at zero depth (the scaling
// limiter of Zhang & Shu 2010), or dropped when the plane has no content.
// m and cm return that child's average and index (m >= 0: unchanged).
template <typename T>
__device__ __forceinline__ void depth_for_children(const T sp[3], T out[3], T &m, int &cm) {
  const T H = T(0.5) * s3v<T>();
  m = tinf<T>();
  cm = 0;
#pragma unroll
  for (int c = 0; c < 4; c++) {
    const T sx = (c & 1) ? H : -H, sy = (c & 2) ? H : -H;
    const T c0 = (sp[0] + sx * sp[1]) + sy * sp[2];
    if (c0 < m) { m = c0; cm = c; }
  }
  out[0] = sp[0];
  out[1] = sp[1];
  out[2] = sp[2];
  if (!(m < T(0))) return;
  if (sp[0] > T(0)) {
    const T th = sp[0] / (sp[0] - m);
    out[1] = sp[1] * th;
    out[2] = sp[2] * th;
  } else {
    out[1] = T(0);
    out[2] = T(0);
  }
}

// nodes of this level below a leaf of the old grid: the parent's planes
// prolonged, depth kept non-negative (top-down)
template <typename T>
__global__ void __launch_bounds__(TPB) k_regrid_prolong(Par<T> P, T *D) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j) || P.kind[k] != K_BELOW) return;
  const long long n = P.ns;
  const long long kp = -P.dp + (long long)(j >> 1) * (P.nx >> 1) + (i >> 1);
  const int c = (i & 1) + 2 * (j & 1);
#pragma unroll
  for (int v = 0; v < 3; v++) {
    T sp[3], sc[3];
#pragma unroll
    for (int q = 0; q < 3; q++) sp[q] = D[(3 * v + q) * n + kp];
    if (v == 0) {
      T dp[3], m;
      int cm;
      depth_for_children(sp, dp, m, cm);
      prolong3(dp, c, sc);
      if (sc[0] < T(0)) sc[0] = T(0);  // a rounding residue below zero depth
    } else {
      prolong3(sp, c, sc);
    }
#pragma unroll
    for (int q = 0; q < 3; q++) D[(3 * v + q) * n + k] = sc[q];
  }
}

// refined nodes of the old grid on this level: the encoding of their
// children (bottom-up)
template <typename T>
__global__ void __launch_bounds__(TPB) k_regrid_encode(Par<T> P, T *D) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j) || P.kind[k] != K_SIG) return;
  const long long n = P.ns;
#pragma unroll 1
  for (int v = 0; v < 3; v++) {
    T ch[4][3], sp[3];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const long long kc = child_of(P, i, j, c);
#pragma unroll
      for (int q = 0; q < 3; q++) ch[c][q] = D[(3 * v + q) * n + kc];
    }
    encode3(ch, sp);
#pragma unroll
    for (int q = 0; q < 3; q++) D[(3 * v + q) * n + k] = sp[q];
  }
}

// transpose of the encoding: a child of a refined node of the old grid (this
// level) takes its share of the parent's cotangent (top-down)
template <typename T>
__global__ void __launch_bounds__(TPB) k_regrid_encode_t(Par<T> P, T *gD) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long kp = -P.dp + (long long)(j >> 1) * (P.nx >> 1) + (i >> 1);
  if (P.kind[kp] != K_SIG) return;
  const long long n = P.ns;
  const int c = (i & 1) + 2 * (j & 1);
#pragma unroll
  for (int v = 0; v < 3; v++) {
    T gp[3], gc[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
      gp[q] = gD[(3 * v + q) * n + kp];
      gc[q] = gD[(3 * v + q) * n + k];
    }
    encode3_t(gp, c, gc);
#pragma unroll
    for (int q = 0; q < 3; q++) gD[(3 * v + q) * n + k] = gc[q];
  }
}

// transpose of the prolongation: a leaf or a node below a leaf of the old
// grid (this level) takes the cotangents of its children below it, through
// the children's zero-depth cut and the depth plane's scaling (bottom-up)
template <typename T>
__global__ void __launch_bounds__(TPB) k_regrid_prolong_t(Par<T> P, const T *D, T *gD) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j) || P.kind[k] == K_SIG) return;
  const long long n = P.ns;
  T sp[3], dp[3], m;
  int cm;
#pragma unroll
  for (int q = 0; q < 3; q++) sp[q] = D[q * n + k];
  depth_for_children(sp, dp, m, cm);
  T gd[3] = {T(0), T(0), T(0)}, gq[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  bool any = false;
#pragma unroll 1
  for (int c = 0; c < 4; c++) {
    const long long kc = child_of(P, i, j, c);
    if (P.kind[kc] != K_BELOW) continue;
    any = true;
    T g[3], sc[3];
#pragma unroll
    for (int q = 0; q < 3; q++) g[q] = gD[q * n + kc];
    prolong3(dp, c, sc);
    if (sc[0] < T(0)) g[0] = T(0);
    prolong3_t(g, c, gd);
#pragma unroll
    for (int v = 1; v < 3; v++) {
#pragma unroll
      for (int q = 0; q < 3; q++) g[q] = gD[(3 * v + q) * n + kc];
      prolong3_t(g, c, gq + 3 * (v - 1));
    }
  }
  if (!any) return;
  // the depth plane's scaling in reverse (the smallest child's index held)
  T gs[3] = {gd[0], gd[1], gd[2]};
  if (m < T(0)) {
    if (sp[0] > T(0)) {
      const T d = sp[0] - m, th = sp[0] / d;
      const T gth = gd[1] * sp[1] + gd[2] * sp[2];
      const T H = T(0.5) * s3v<T>();
      const T sx = (cm & 1) ? H : -H, sy = (cm & 2) ? H : -H;
      const T dsp0 = -m / (d * d), dm = sp[0] / (d * d);
      gs[1] = gd[1] * th + gth * dm * sx;
      gs[2] = gd[2] * th + gth * dm * sy;
      gs[0] = gd[0] + gth * dsp0 + gth * dm;
    } else {
      gs[1] = T(0);
      gs[2] = T(0);
    }
  }
#pragma unroll
  for (int q = 0; q < 3; q++) gD[q * n + k] += gs[q];
#pragma unroll
  for (int q = 0; q < 6; q++) gD[(3 + q) * n + k] += gq[q];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
inline unsigned blocks(long long items) { return (unsigned)((items + TPB - 1) / TPB); }

}  // namespace adj
}  // namespace mwdg

using namespace mwdg::adj;

struct mwdg_adj {
  mwdg_adj_params p{};
  // per-kernel timing: a pool of event pairs recorded around each launch
  std::vector<cudaEvent_t> evs;
  std::vector<int> ev_class;
  size_t ev_used = 0;
  int tape_steps = -1;         // steps of the run the tape holds (-1: none)
  bool views = false;          // the tape also keeps each step's stage inputs and flux views
  long long n = 0;
  size_t elem = 8;             // bytes per coefficient (8 FP64, 4 FP32)
  void *tape = nullptr;        // (max_steps + 1) x 9n: the state at the start of each step
  uint8_t *clip = nullptr;     // max_steps x n: bit s-1 set when stage s clipped
  double *tt = nullptr;        // max_steps + 1 step start times
  double *dtbuf = nullptr;     // max_steps time steps (fixed runs copy theirs here)
  unsigned long long *best = nullptr;
  void *Un = nullptr, *Ui = nullptr, *W1 = nullptr, *F1 = nullptr, *Z1 = nullptr;
  void *W2 = nullptr, *F2 = nullptr, *Z2 = nullptr;
  void *lU = nullptr, *lX = nullptr, *lW1 = nullptr, *limx = nullptr, *limy = nullptr, *lXo = nullptr,
       *lnb = nullptr;
  double *lq = nullptr;
  // a frozen non-uniform grid (levels = L + 1 > 0; 0 on a uniform grid):
  // per level its first node, x face, y face and boundary entry in the
  // concatenated arrays (the last entry: the totals)
  int levels = 0, mode = 0, gM = 0, gN = 0;
  std::vector<long long> off, fxo, fyo, lqo;
  long long nl = 0, nfin = 0;     // leaves; finest cells
  uint8_t *kind = nullptr;        // node kinds (K_BELOW, K_LEAF, K_SIG)
  long long *node = nullptr;      // each leaf's node
  void *zp = nullptr, *np = nullptr, *gzp = nullptr, *gnp = nullptr, *gV = nullptr;
  std::string err;
};

namespace {

void free_events(mwdg_adj *a) {
  for (cudaEvent_t e : a->evs) cudaEventDestroy(e);
  a->evs.clear();
  a->ev_class.clear();
  a->ev_used = 0;
}

// records an event pair around the launches of one scope when the profiler
// is on and its pool has room
struct Timed {
  mwdg_adj *a;
  cudaStream_t st;
  size_t slot;
  bool on;
  Timed(mwdg_adj *a_, int cls, cudaStream_t st_) : a(a_), st(st_), slot(0), on(false) {
    if (a->ev_used + 2 <= a->evs.size()) {
      slot = a->ev_used;
      a->ev_used += 2;
      a->ev_class[slot / 2] = cls;
      cudaEventRecord(a->evs[slot], st);
      on = true;
    }
  }
  ~Timed() {
    if (on) cudaEventRecord(a->evs[slot + 1], st);
  }
};

void free_all(mwdg_adj *a) {
  free_events(a);
  void *ptrs[] = {a->tape, a->clip, a->tt, a->dtbuf, a->best, a->Un, a->Ui, a->W1, a->F1, a->Z1, a->W2,
                  a->F2, a->Z2, a->lU, a->lX, a->lW1, a->limx, a->limy, a->lXo, a->lnb, a->lq,
                  a->kind, a->node, a->zp, a->np, a->gzp, a->gnp, a->gV};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

mwdg_status fail(mwdg_adj *a, mwdg_status s, const std::string &what) {
  if (a) a->err = what;
  return s;
}

mwdg_status cuda_check(mwdg_adj *a, const char *where) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return MWDG_OK;
  return fail(a, MWDG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// parameters of the finest (uniform) grid; for a frozen grid's level l see
// level_par
template <typename T>
Par<T> make_par(const mwdg_adj *a, int nknots, const double *kt, const double *kQ) {
  Par<T> P;
  const mwdg_adj_params &p = a->p;
  P.nx = p.nx;
  P.ny = p.ny;
  P.n = (long long)p.nx * p.ny;
  P.ns = P.n;
  P.off = P.fx = P.fy = P.fxp = P.fyp = P.lqo = 0;
  P.sh = 0;
  P.stat = 0;
  P.kind = nullptr;
  P.dn = P.dp = 0;
  P.dx = (T)p.dx;
  P.g = (T)p.g;
  P.hd = (T)p.h_dry;
  P.dxd = p.dx;
  P.cfl = p.cfl;
  P.dt_max = p.dt_max;
  P.limiter = p.limiter;
  for (int e = 0; e < 4; e++) P.bc[e] = p.bc[e];
  P.inflow_edge = p.inflow_edge;
  P.c0 = p.inflow_c0;
  P.c1 = p.inflow_c1;
  P.nknots = p.inflow_edge >= 0 ? nknots : 0;
  P.rain_rate = p.rain_rate;
  P.rain_t_end = p.rain_t_end;
  P.kt = kt;
  P.kQ = kQ;
  return P;
}

int nlev(const mwdg_adj *a) { return a->levels ? a->levels : 1; }
long long loff(const mwdg_adj *a, int l) { return a->levels ? a->off[l] : 0; }

// parameters of level l (the whole grid on a uniform grid)
template <typename T>
Par<T> level_par(const mwdg_adj *a, int l, int nknots, const double *kt, const double *kQ) {
  Par<T> P = make_par<T>(a, nknots, kt, kQ);
  if (!a->levels) return P;
  const int L = a->levels - 1;
  P.nx = a->gM << l;
  P.ny = a->gN << l;
  P.n = (long long)P.nx * P.ny;
  P.ns = a->n;
  P.sh = L - l;
  P.stat = a->mode == MWDG_STATIC;
  P.kind = a->kind + a->off[l];
  P.dn = l < L ? a->off[l + 1] - a->off[l] : 0;
  P.dp = l > 0 ? a->off[l] - a->off[l - 1] : 0;
  P.dxd = a->p.dx * (double)(1LL << (L - l));
  P.dx = (T)P.dxd;
  P.off = a->off[l];
  P.fx = a->fxo[l];
  P.fy = a->fyo[l];
  P.fxp = l > 0 ? a->fxo[l - 1] : 0;
  P.fyp = l > 0 ? a->fyo[l - 1] : 0;
  P.lqo = a->lqo[l];
  return P;
}

// launch tables over all levels: per level its first block
template <typename T, class F>
Levels<T> make_levels(const std::vector<Par<T>> &PL, F &&blocks_of, unsigned &total) {
  Levels<T> LV{};
  LV.n = (int)PL.size();
  unsigned b = 0;
  for (int l = 0; l < LV.n; l++) {
    LV.bstart[l] = b;
    LV.P[l] = PL[l];
    b += (unsigned)blocks_of(PL[l]);
  }
  LV.bstart[LV.n] = b;
  total = b;
  return LV;
}

template <typename T> T *ptr(void *p) { return static_cast<T *>(p); }

// where step s keeps its two stage inputs (Un, Ui) and their flux views
// (F1, Z1, F2, Z2): per-step slots of the tape when it keeps them, else one
// set of work arrays that the reverse sweep refills step by step
template <typename T>
struct StageArrays {
  T *Un, *Ui, *F1, *Z1, *F2, *Z2;
};

template <typename T>
StageArrays<T> stage_arrays(const mwdg_adj *a, int s) {
  const long long n = a->n, o9 = a->views ? (long long)s * 9 * n : 0, o3 = a->views ? (long long)s * 3 * n : 0;
  return StageArrays<T>{ptr<T>(a->Un) + o9, ptr<T>(a->Ui) + o9, ptr<T>(a->F1) + o9,
                        ptr<T>(a->Z1) + o3, ptr<T>(a->F2) + o9, ptr<T>(a->Z2) + o3};
}

// the views of the flux-view planes (F, Zf) of a frozen grid: encodings of
// refined nodes from the finest level up, then prolongations from the
// coarsest down
// the coarse levels of a frozen grid: those of at most COARSE_NODES nodes,
// whose view passes run in one block (-1: none)
constexpr long long COARSE_NODES = 1024;
int coarse_level(const mwdg_adj *a) {
  int lc = -1;
  while (lc + 1 < a->levels && ((long long)a->gM << (lc + 1)) * ((long long)a->gN << (lc + 1)) <= COARSE_NODES) lc++;
  return lc;
}

template <typename T>
void launch_views(const mwdg_adj *a, const Levels<T> &LV, const Par<T> *PL, T *F, T *Zf, cudaStream_t st) {
  if (!a->levels) return;
  const int L = a->levels - 1, lc = coarse_level(a);
  for (int l = L - 1; l > lc; l--)
    k_view_encode<T><<<blocks(PL[l].n), TPB, 0, st>>>(PL[l], F + loff(a, l), Zf + loff(a, l));
  if (std::min(lc, L - 1) >= 0) k_views_coarse<T, VP_ENCODE><<<1, CTPB, 0, st>>>(LV, F, Zf, std::min(lc, L - 1), 0);
  if (std::min(lc, L) >= 1) k_views_coarse<T, VP_PROLONG><<<1, CTPB, 0, st>>>(LV, F, Zf, 1, std::min(lc, L));
  for (int l = std::max(lc + 1, 1); l <= L; l++)
    k_view_prolong<T><<<blocks(PL[l].n), TPB, 0, st>>>(PL[l], F + loff(a, l), Zf + loff(a, l));
}

// the launch tables of one call: cells, update tiles, x and y faces of
// every level
template <typename T>
struct Tabs {
  std::vector<Par<T>> PL;
  Levels<T> cells, tiles, fxs, fys;
  unsigned nc = 0, nt = 0, nfx = 0, nfy = 0;
};

template <typename T>
void launch_update(const mwdg_adj *a, const Tabs<T> &TB, int stage, const T *F, const T *Zf, const T *Wst,
                   const T *W1, const double *dts, int s, T *Out, uint8_t *clip, cudaStream_t st) {
  if (a->levels)
    k_update<T, true><<<TB.nt, UT * UT, 0, st>>>(TB.tiles, stage, F, Zf, Wst, W1, dts, a->tt, s, Out, clip);
  else
    k_update<T, false><<<TB.nt, UT * UT, 0, st>>>(TB.tiles, stage, F, Zf, Wst, W1, dts, a->tt, s, Out, clip);
}

template <typename T>
void launch_limit(const mwdg_adj *a, const Tabs<T> &TB, const T *X, const T *z, T *Wst, T *F, T *Zf,
                  cudaStream_t st) {
  if (a->levels) k_limit<T, true><<<TB.nc, TPB, 0, st>>>(TB.cells, X, z, Wst, F, Zf);
  else k_limit<T, false><<<TB.nc, TPB, 0, st>>>(TB.cells, X, z, Wst, F, Zf);
  launch_views<T>(a, TB.cells, TB.PL.data(), F, Zf, st);
}

// friction, limit, stage 1 and limit of step s: the two stage inputs (Un, Ui)
// and their stored and flux views (on a frozen grid the views of every level)
template <typename T>
void recompute_stages(mwdg_adj *a, const Tabs<T> &TB, const T *U, const T *z, const T *nman, int s,
                      const double *dts, uint8_t *clip, cudaStream_t st) {
  const StageArrays<T> v = stage_arrays<T>(a, s);
  T *Un = v.Un, *Ui = v.Ui, *W1 = ptr<T>(a->W1), *F1 = v.F1, *Z1 = v.Z1;
  T *W2 = ptr<T>(a->W2), *F2 = v.F2, *Z2 = v.Z2;
  {
    Timed tm(a, MWDG_ADJ_KC_FRICTION, st);
    if (a->levels) k_friction<T, true><<<TB.nc, TPB, 0, st>>>(TB.cells, U, nman, dts, a->tt, s, Un);
    else k_friction<T, false><<<TB.nc, TPB, 0, st>>>(TB.cells, U, nman, dts, a->tt, s, Un);
  }
  {
    Timed tm(a, MWDG_ADJ_KC_LIMIT, st);
    launch_limit<T>(a, TB, Un, z, W1, F1, Z1, st);
  }
  {
    Timed tm(a, MWDG_ADJ_KC_UPDATE, st);
    launch_update<T>(a, TB, 1, F1, Z1, W1, nullptr, dts, s, Ui, clip, st);
  }
  Timed tm(a, MWDG_ADJ_KC_LIMIT, st);
  launch_limit<T>(a, TB, Ui, z, W2, F2, Z2, st);
}

// the forward sweep of one step s from tape slot s into slot s + 1
template <typename T>
void launch_step(mwdg_adj *a, const Tabs<T> &TB, const T *z, const T *nman, int s, bool cfl, double *dts,
                 cudaStream_t st) {
  const long long n = a->n;
  const T *U = ptr<T>(a->tape) + (long long)s * 9 * n;
  T *Unext = ptr<T>(a->tape) + (long long)(s + 1) * 9 * n;
  uint8_t *clip = a->clip + (long long)s * n;
  if (cfl) {
    Timed tm(a, MWDG_ADJ_KC_CFL, st);
    if (a->levels) k_cfl<T, true><<<TB.nc, TPB, 0, st>>>(TB.cells, U, a->tt, s, a->best);
    else k_cfl<T, false><<<TB.nc, TPB, 0, st>>>(TB.cells, U, a->tt, s, a->best);
    k_dt<<<1, 1, 0, st>>>(TB.PL[0].cfl, TB.PL[0].dt_max, a->best, dts, a->tt, s);
  }
  recompute_stages<T>(a, TB, U, z, nman, s, dts, clip, st);
  const StageArrays<T> v = stage_arrays<T>(a, s);
  Timed tm(a, MWDG_ADJ_KC_UPDATE, st);
  launch_update<T>(a, TB, 2, v.F2, v.Z2, ptr<T>(a->W2), ptr<T>(a->W1), dts, s, Unext, clip, st);
}

// per-level parameters (one entry on a uniform grid) and the launch tables
template <typename T>
Tabs<T> make_tabs(const mwdg_adj *a, int nknots, const double *kt, const double *kQ) {
  Tabs<T> TB;
  for (int l = 0; l < nlev(a); l++) TB.PL.push_back(level_par<T>(a, l, nknots, kt, kQ));
  TB.cells = make_levels(TB.PL, [](const Par<T> &P) { return blocks(P.n); }, TB.nc);
  TB.tiles = make_levels(TB.PL, [](const Par<T> &P) {
    return (long long)((P.nx + UT - 1) / UT) * ((P.ny + UT - 1) / UT); }, TB.nt);
  TB.fxs = make_levels(TB.PL, [](const Par<T> &P) { return blocks((long long)P.ny * (P.nx + 1)); }, TB.nfx);
  TB.fys = make_levels(TB.PL, [](const Par<T> &P) { return blocks((long long)(P.ny + 1) * P.nx); }, TB.nfy);
  return TB;
}

template <typename T>
std::vector<Par<T>> level_pars(const mwdg_adj *a, int nknots, const double *kt, const double *kQ) {
  std::vector<Par<T>> PL;
  for (int l = 0; l < nlev(a); l++) PL.push_back(level_par<T>(a, l, nknots, kt, kQ));
  return PL;
}

// a frozen grid's bed and Manning pyramids from the finest planes and raster
template <typename T>
void launch_pyramids(const mwdg_adj *a, const Par<T> *PL, const T *z, const T *nman, cudaStream_t st) {
  const int L = a->levels - 1;
  const long long nt = a->n, nf = a->nfin, oL = a->off[L];
  k_copy_planes<T><<<blocks(nf), TPB, 0, st>>>(3, nf, z, nf, ptr<T>(a->zp) + oL, nt, 0);
  k_copy_planes<T><<<blocks(nf), TPB, 0, st>>>(1, nf, nman, nf, ptr<T>(a->np) + oL, nt, 0);
  for (int l = L - 1; l >= 0; l--)
    k_pyramid_level<T><<<blocks(PL[l].n), TPB, 0, st>>>(PL[l], ptr<T>(a->zp) + a->off[l], ptr<T>(a->np) + a->off[l]);
}

// a frozen grid's tape slot 0: still water everywhere, the leaves' coefficients at their nodes
template <typename T>
void launch_scatter_state(const mwdg_adj *a, const T *U0, cudaStream_t st) {
  k_still<T><<<blocks(a->n), TPB, 0, st>>>(a->n, ptr<T>(a->tape));
  k_leaves_to_nodes<T><<<blocks(a->nl), TPB, 0, st>>>(a->nl, a->n, a->node, U0, ptr<T>(a->tape));
}

mwdg_status check_run(mwdg_adj *a, const void *U0, const void *z, const void *n, int32_t nknots, const double *kt,
                      const double *kQ, int32_t steps, const double *dts) {
  if (!a) return MWDG_ERR_ARG;
  if (!U0 || !z || !n || (!dts && steps > 0) || steps < 0) return fail(a, MWDG_ERR_ARG, "NULL pointer or steps < 0");
  if (steps > a->p.max_steps) return fail(a, MWDG_ERR_CAPACITY, "steps > max_steps");
  if (a->p.inflow_edge >= 0 && (nknots < 1 || !kt || !kQ))
    return fail(a, MWDG_ERR_ARG, "an inflow edge needs nknots >= 1 knots");
  return MWDG_OK;
}

template <typename T>
mwdg_status forward_t(mwdg_adj *a, const T *U0, const T *z, const T *nman, int32_t nknots, const double *kt,
                      const double *kQ, double t0, int32_t steps, int32_t fixed_dt, double *dts, T *U_out,
                      cudaStream_t st) {
  const Tabs<T> TB = make_tabs<T>(a, nknots, kt, kQ);
  const size_t bytes = (size_t)9 * a->n * sizeof(T);
  if (a->levels) {
    launch_pyramids<T>(a, TB.PL.data(), z, nman, st);
    z = ptr<T>(a->zp);
    nman = ptr<T>(a->np);
    launch_scatter_state<T>(a, U0, st);
  } else if (cudaMemcpyAsync(a->tape, U0, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    return cuda_check(a, "mwdg_adj_forward copy-in");
  }
  k_set_t0<<<1, 1, 0, st>>>(a->tt, t0);
  if (fixed_dt) k_times<<<1, 1, 0, st>>>(dts, steps, a->tt);
  for (int k = 0; k < steps; k++) launch_step<T>(a, TB, z, nman, k, !fixed_dt, dts, st);
  const T *UK = ptr<T>(a->tape) + (long long)steps * 9 * a->n;
  if (a->levels)
    k_nodes_to_leaves<T><<<blocks(a->nl), TPB, 0, st>>>(a->nl, a->n, a->node, UK, U_out);
  else if (cudaMemcpyAsync(U_out, UK, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return cuda_check(a, "mwdg_adj_forward copy-out");
  return cuda_check(a, "mwdg_adj_forward");
}

template <typename T>
mwdg_status backward_t(mwdg_adj *a, const T *U0, const T *z, const T *nman, int32_t nknots, const double *kt,
                       const double *kQ, double t0, int32_t steps, const double *dts_in, const T *gUK, T *gU0, T *gz,
                       T *gn, double *gQ, bool reuse, cudaStream_t st) {
  const Tabs<T> TB = make_tabs<T>(a, nknots, kt, kQ);
  const std::vector<Par<T>> &PL = TB.PL;
  const long long n = a->n;
  const bool fz = a->levels > 0;
  const int NL = nlev(a), L = NL - 1;
  const size_t bytes = (size_t)9 * n * sizeof(T);
  T *lU = ptr<T>(a->lU), *lX = ptr<T>(a->lX), *lW1 = ptr<T>(a->lW1);
  T *limx = ptr<T>(a->limx), *limy = ptr<T>(a->limy), *lXo = ptr<T>(a->lXo), *lnb = ptr<T>(a->lnb);
  T *gV = ptr<T>(a->gV);
  // the gradients of a frozen grid's level pyramids, folded to the finest
  // level at the end
  T *gzl = gz, *gnl = gn;
  if (fz) {
    launch_pyramids<T>(a, PL.data(), z, nman, st);
    z = ptr<T>(a->zp);
    nman = ptr<T>(a->np);
    gzl = ptr<T>(a->gzp);
    gnl = ptr<T>(a->gnp);
    if (cudaMemsetAsync(gzl, 0, (size_t)3 * n * sizeof(T), st) != cudaSuccess ||
        cudaMemsetAsync(gnl, 0, (size_t)n * sizeof(T), st) != cudaSuccess)
      return cuda_check(a, "mwdg_adj_backward clear");
  }
  // the tape: the run recomputed from its checkpoint U0 over the given steps,
  // unless the caller states that the last forward call left it in place
  if (steps > 0 && cudaMemcpyAsync(a->dtbuf, dts_in, (size_t)steps * sizeof(double), cudaMemcpyDeviceToDevice,
                                   st) != cudaSuccess)
    return cuda_check(a, "mwdg_adj_backward dts");
  if (!reuse) {
    if (fz)
      launch_scatter_state<T>(a, U0, st);
    else if (cudaMemcpyAsync(a->tape, U0, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return cuda_check(a, "mwdg_adj_backward copy-in");
    k_set_t0<<<1, 1, 0, st>>>(a->tt, t0);
    k_times<<<1, 1, 0, st>>>(a->dtbuf, steps, a->tt);
    for (int k = 0; k < steps; k++) launch_step<T>(a, TB, z, nman, k, false, a->dtbuf, st);
  }
  if (fz) {
    if (cudaMemsetAsync(lU, 0, bytes, st) != cudaSuccess) return cuda_check(a, "mwdg_adj_backward seed");
    k_leaves_to_nodes<T><<<blocks(a->nl), TPB, 0, st>>>(a->nl, n, a->node, gUK, lU);
  } else if (cudaMemcpyAsync(lU, gUK, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    return cuda_check(a, "mwdg_adj_backward seed");
  }
  const double *dts = a->dtbuf;
  for (int k = steps - 1; k >= 0; k--) {
    const T *U = ptr<T>(a->tape) + (long long)k * 9 * n;
    const T *Y2 = ptr<T>(a->tape) + (long long)(k + 1) * 9 * n;
    uint8_t *clip = a->clip + (long long)k * n;
    // the stage inputs of step k and their flux views: kept on the tape, or
    // recomputed (stage 1 then rewrites its clip bit with the same value and
    // keeps stage 2's from the tape run)
    if (!a->views) recompute_stages<T>(a, TB, U, z, nman, k, dts, clip, st);
    const StageArrays<T> v = stage_arrays<T>(a, k);
    const T *Un = v.Un, *Ui = v.Ui, *F1 = v.F1, *Z1 = v.Z1, *F2 = v.F2, *Z2 = v.Z2;
    for (int stage = 2; stage >= 1; stage--) {
      const T *X = stage == 2 ? Ui : Un;
      const T *Y = stage == 2 ? Y2 : Ui;
      const T *Wf = stage == 2 ? F2 : F1;
      const T *Zf = stage == 2 ? Z2 : Z1;
      const T *lY = stage == 2 ? lU : lX;
      {
        Timed tm(a, MWDG_ADJ_KC_REV_FACE, st);
        if (fz) {
          k_rev_face<T, true, true><<<TB.nfx, TPB, 0, st>>>(TB.fxs, stage, dts, a->tt, k, Wf, Zf, lY, Y, clip,
                                                            limx, a->lq);
          k_rev_face<T, false, true><<<TB.nfy, TPB, 0, st>>>(TB.fys, stage, dts, a->tt, k, Wf, Zf, lY, Y, clip,
                                                             limy, a->lq);
        } else {
          k_rev_face<T, true, false><<<TB.nfx, TPB, 0, st>>>(TB.fxs, stage, dts, a->tt, k, Wf, Zf, lY, Y, clip,
                                                             limx, a->lq);
          k_rev_face<T, false, false><<<TB.nfy, TPB, 0, st>>>(TB.fys, stage, dts, a->tt, k, Wf, Zf, lY, Y, clip,
                                                              limy, a->lq);
        }
      }
      if (PL[0].nknots > 0) {
        Timed tm(a, MWDG_ADJ_KC_REV_KNOTS, st);
        k_rev_knots<T><<<1, TPB, 0, st>>>(TB.cells, stage, dts, a->tt, k, a->lq, gQ);
      }
      {
        Timed tm(a, MWDG_ADJ_KC_REV_LIMIT, st);
        if (fz) {
          // the views in reverse: every node's view-plane cotangents, then
          // the prolongations (finest level up) and encodings (coarsest
          // down) transposed onto the leaves
          k_rev_view_gather<T><<<TB.nc, TPB, 0, st>>>(TB.cells, limx, limy, gV);
          const int lc = coarse_level(a);
          for (int l = L - 1; l > lc; l--) k_rev_prolong<T><<<blocks(PL[l].n), TPB, 0, st>>>(PL[l], gV + loff(a, l));
          if (std::min(lc, L - 1) >= 0)
            k_views_coarse<T, VP_REV_PROLONG><<<1, CTPB, 0, st>>>(TB.cells, gV, nullptr, std::min(lc, L - 1), 0);
          if (std::min(lc, L) >= 1)
            k_views_coarse<T, VP_REV_ENCODE><<<1, CTPB, 0, st>>>(TB.cells, gV, nullptr, 1, std::min(lc, L));
          for (int l = std::max(lc + 1, 1); l <= L; l++)
            k_rev_encode<T><<<blocks(PL[l].n), TPB, 0, st>>>(PL[l], gV + loff(a, l));
          k_rev_limit<T, true><<<TB.nc, TPB, 0, st>>>(TB.cells, stage, dts, k, X, z, lY, Y, clip, lW1, nullptr,
                                                      nullptr, gV, lXo, lnb, gzl);
        } else {
          k_rev_limit<T, false><<<TB.nc, TPB, 0, st>>>(TB.cells, stage, dts, k, X, z, lY, Y, clip, lW1, limx, limy,
                                                       nullptr, lXo, lnb, gzl);
        }
      }
      Timed tm(a, MWDG_ADJ_KC_REV_GATHER, st);
      if (fz) k_rev_gather<T, true><<<TB.nc, TPB, 0, st>>>(TB.cells, lXo, lnb, lX, gzl);
      else k_rev_gather<T, false><<<TB.nc, TPB, 0, st>>>(TB.cells, lXo, lnb, lX, gzl);
    }
    Timed tm(a, MWDG_ADJ_KC_REV_FRICTION, st);
    if (fz) k_rev_friction<T, true><<<TB.nc, TPB, 0, st>>>(TB.cells, U, nman, dts, a->tt, k, lX, lU, gnl);
    else k_rev_friction<T, false><<<TB.nc, TPB, 0, st>>>(TB.cells, U, nman, dts, a->tt, k, lX, lU, gnl);
  }
  if (fz) {
    k_nodes_to_leaves<T><<<blocks(a->nl), TPB, 0, st>>>(a->nl, n, a->node, lU, gU0);
    // the pyramids in reverse, from the coarsest level down; the finest
    // level's cotangents are the gradients of z and n
    for (int l = 1; l <= L; l++)
      k_pyramid_level_t<T><<<blocks(PL[l].n), TPB, 0, st>>>(PL[l], gzl + a->off[l], gnl + a->off[l]);
    const long long nf = a->nfin, oL = a->off[L];
    k_copy_planes<T><<<blocks(nf), TPB, 0, st>>>(3, nf, gzl + oL, n, gz, nf, 1);
    k_copy_planes<T><<<blocks(nf), TPB, 0, st>>>(1, nf, gnl + oL, n, gn, nf, 1);
  } else if (cudaMemcpyAsync(gU0, lU, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    return cuda_check(a, "mwdg_adj_backward copy-out");
  }
  return cuda_check(a, "mwdg_adj_backward");
}

// the old grid's state on every node of its levels (D, 9 x nodes) from its
// leaves' coefficients
template <typename T>
void launch_regrid_state(const mwdg_adj *f, const T *U_from, T *D, cudaStream_t st) {
  const int L = f->levels - 1;
  const std::vector<Par<T>> PL = level_pars<T>(f, 0, nullptr, nullptr);
  k_still<T><<<blocks(f->n), TPB, 0, st>>>(f->n, D);
  k_leaves_to_nodes<T><<<blocks(f->nl), TPB, 0, st>>>(f->nl, f->n, f->node, U_from, D);
  for (int l = 1; l <= L; l++) k_regrid_prolong<T><<<blocks(PL[l].n), TPB, 0, st>>>(PL[l], D + f->off[l]);
  for (int l = L - 1; l >= 0; l--) k_regrid_encode<T><<<blocks(PL[l].n), TPB, 0, st>>>(PL[l], D + f->off[l]);
}

template <typename T>
void launch_regrid(mwdg_adj *f, mwdg_adj *t, const T *U_from, T *U_to, cudaStream_t st) {
  T *D = ptr<T>(f->lXo);
  launch_regrid_state<T>(f, U_from, D, st);
  k_nodes_to_leaves<T><<<blocks(t->nl), TPB, 0, st>>>(t->nl, f->n, t->node, D, U_to);
}

template <typename T>
void launch_regrid_t(mwdg_adj *f, mwdg_adj *t, const T *U_from, const T *gU_to, T *gU_from, cudaStream_t st) {
  const int L = f->levels - 1;
  const std::vector<Par<T>> PL = level_pars<T>(f, 0, nullptr, nullptr);
  T *D = ptr<T>(f->lXo), *gD = ptr<T>(f->lX);
  launch_regrid_state<T>(f, U_from, D, st);
  cudaMemsetAsync(gD, 0, (size_t)9 * f->n * sizeof(T), st);
  k_leaves_to_nodes<T><<<blocks(t->nl), TPB, 0, st>>>(t->nl, f->n, t->node, gU_to, gD);
  for (int l = 1; l <= L; l++) k_regrid_encode_t<T><<<blocks(PL[l].n), TPB, 0, st>>>(PL[l], gD + f->off[l]);
  for (int l = L - 1; l >= 0; l--)
    k_regrid_prolong_t<T><<<blocks(PL[l].n), TPB, 0, st>>>(PL[l], D + f->off[l], gD + f->off[l]);
  k_nodes_to_leaves<T><<<blocks(f->nl), TPB, 0, st>>>(f->nl, f->n, f->node, gD, gU_from);
}

mwdg_status check_pair(mwdg_adj *f, mwdg_adj *t) {
  if (!f || !t) return MWDG_ERR_ARG;
  if (!f->levels || !t->levels) return fail(f, MWDG_ERR_ARG, "regridding needs two frozen-grid contexts");
  if (f->levels != t->levels || f->gM != t->gM || f->gN != t->gN) return fail(f, MWDG_ERR_DIMS, "grids differ in roots or levels");
  if (f->p.precision != t->p.precision) return fail(f, MWDG_ERR_ARG, "contexts differ in precision");
  return MWDG_OK;
}

mwdg_status check_params(const mwdg_adj_params *p) {
  if (p->nx < 1 || p->ny < 1 || (long long)p->nx * p->ny > (1LL << 28) || !(p->dx > 0.0) || p->max_steps < 1)
    return MWDG_ERR_DIMS;
  if (!(p->g > 0.0) || !(p->h_dry >= 0.0) || !(p->cfl > 0.0) || !(p->dt_max > 0.0) || p->rain_rate < 0.0)
    return MWDG_ERR_ARG;
  if (p->precision != MWDG_F64 && p->precision != MWDG_F32) return MWDG_ERR_ARG;
  for (int e = 0; e < 4; e++)
    if (p->bc[e] != MWDG_WALL && p->bc[e] != MWDG_OPEN) return MWDG_ERR_ARG;
  if (p->inflow_edge >= 4 || p->inflow_edge < -1) return MWDG_ERR_ARG;
  if (p->inflow_edge >= 0) {
    const int len = p->inflow_edge < 2 ? p->ny : p->nx;
    if (p->inflow_c0 < 0 || p->inflow_c1 < p->inflow_c0 || p->inflow_c1 >= len) return MWDG_ERR_ARG;
  }
  return MWDG_OK;
}

// the tape and work arrays of a context with a->n nodes, nfx and nfy faces
// (all levels) and nedge boundary entries; false when an allocation fails
bool allocate(mwdg_adj *a, long long nfx, long long nfy, long long nedge) {
  const mwdg_adj_params *p = &a->p;
  a->elem = p->precision == MWDG_F32 ? sizeof(float) : sizeof(double);
  const long long n = a->n, S = p->max_steps;
  const size_t E = a->elem;
  bool ok = true;
  auto alloc = [&](void **ptrp, long long count, size_t elem) {
    if (ok && cudaMalloc(ptrp, (size_t)count * elem) != cudaSuccess) ok = false;
  };
  alloc(&a->tape, (S + 1) * 9 * n, E);
  alloc((void **)&a->clip, S * n, 1);
  alloc((void **)&a->tt, S + 1, sizeof(double));
  alloc((void **)&a->dtbuf, S, sizeof(double));
  alloc((void **)&a->best, 1, sizeof(unsigned long long));
  a->views = p->tape_views != 0;
  const long long SV = a->views ? S : 1;   // copies of the stage arrays
  for (void **w : {&a->Un, &a->Ui, &a->F1, &a->F2}) alloc(w, SV * 9 * n, E);
  alloc(&a->Z1, SV * 3 * n, E);
  alloc(&a->Z2, SV * 3 * n, E);
  for (void **w : {&a->W1, &a->W2, &a->lU, &a->lX, &a->lW1, &a->lXo}) alloc(w, 9 * n, E);
  alloc(&a->lnb, 12 * n, E);
  alloc(&a->limx, 14 * nfx, E);
  alloc(&a->limy, 14 * nfy, E);
  alloc((void **)&a->lq, nedge, sizeof(double));
  if (ok) {
    const unsigned long long inf = 0x7ff0000000000000ull;
    ok = cudaMemcpy(a->best, &inf, sizeof inf, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(a->lq, 0, (size_t)nedge * sizeof(double)) == cudaSuccess &&
         cudaMemset(a->clip, 0, (size_t)(S * n)) == cudaSuccess;
  }
  if (!ok) cudaGetLastError();
  return ok;
}

}  // namespace

extern "C" {

mwdg_status mwdg_adj_params_default(mwdg_adj_params *p) {
  if (!p) return MWDG_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->g = 9.80665;
  p->h_dry = 1e-3;
  p->cfl = 0.33;
  p->dt_max = 1.0;
  p->limiter = 1;
  p->inflow_edge = -1;
  p->inflow_c0 = 0;
  p->inflow_c1 = -1;
  p->max_steps = 200;
  p->precision = MWDG_F64;
  p->tape_views = 0;
  return MWDG_OK;
}

mwdg_status mwdg_adj_create(const mwdg_adj_params *p, mwdg_adj **out) {
  if (!p || !out) return MWDG_ERR_ARG;
  *out = nullptr;
  const mwdg_status v = check_params(p);
  if (v != MWDG_OK) return v;
  mwdg_adj *a = new (std::nothrow) mwdg_adj;
  if (!a) return MWDG_ERR_CUDA;
  a->p = *p;
  a->n = a->nfin = (long long)p->nx * p->ny;
  const long long nfx = (long long)p->ny * (p->nx + 1), nfy = (long long)(p->ny + 1) * p->nx;
  if (!allocate(a, nfx, nfy, p->nx > p->ny ? p->nx : p->ny)) {
    free_all(a);
    delete a;
    return MWDG_ERR_CUDA;
  }
  *out = a;
  return MWDG_OK;
}

mwdg_status mwdg_adj_create_frozen(const mwdg_adj_params *p, int32_t M, int32_t N, int32_t L, int32_t mode,
                                   int64_t n_leaves, const int32_t *level, const int32_t *ii, const int32_t *jj,
                                   mwdg_adj **out) {
  if (!p || !out) return MWDG_ERR_ARG;
  *out = nullptr;
  if (M < 1 || N < 1 || L < 0 || L > MWDG_LMAX || ((long long)M << L) != p->nx || ((long long)N << L) != p->ny)
    return MWDG_ERR_DIMS;
  if (mode != MWDG_STATIC && mode != MWDG_ADAPTIVE) return MWDG_ERR_ARG;
  const mwdg_status v = check_params(p);
  if (v != MWDG_OK) return v;
  if (n_leaves < 1 || !level || !ii || !jj) return MWDG_ERR_ARG;
  // the levels' geometry and node kinds; the leaves must tile the domain
  std::vector<long long> off(L + 2), fxo(L + 2), fyo(L + 2), lqo(L + 2);
  for (int l = 0; l <= L; l++) {
    const long long nx = (long long)M << l, ny = (long long)N << l;
    off[l + 1] = off[l] + nx * ny;
    fxo[l + 1] = fxo[l] + ny * (nx + 1);
    fyo[l + 1] = fyo[l] + (ny + 1) * nx;
    lqo[l + 1] = lqo[l] + (nx > ny ? nx : ny);
  }
  const long long nt = off[L + 1];
  std::vector<uint8_t> kind((size_t)nt, K_BELOW);
  std::vector<long long> node((size_t)n_leaves);
  for (int64_t q = 0; q < n_leaves; q++) {
    const int l = level[q];
    if (l < 0 || l > L) return MWDG_ERR_ARG;
    const long long nx = (long long)M << l, ny = (long long)N << l;
    if (ii[q] < 0 || jj[q] < 0 || ii[q] >= nx || jj[q] >= ny) return MWDG_ERR_ARG;
    const long long k = off[l] + (long long)jj[q] * nx + ii[q];
    if (kind[(size_t)k] == K_LEAF) return MWDG_ERR_ARG;  // listed twice
    kind[(size_t)k] = K_LEAF;
    node[(size_t)q] = k;
  }
  // refined: a node with a leaf or a refined node among its children
  for (int l = L - 1; l >= 0; l--) {
    const long long nx = (long long)M << l, ny = (long long)N << l;
    for (long long j = 0; j < ny; j++)
      for (long long i = 0; i < nx; i++) {
        const long long k = off[l] + j * nx + i;
        bool sub = false;
        for (int c = 0; c < 4; c++) {
          const long long kc = off[l + 1] + (2 * j + (c >> 1)) * (2 * nx) + 2 * i + (c & 1);
          sub = sub || kind[(size_t)kc] != K_BELOW;
        }
        if (sub) {
          if (kind[(size_t)k] == K_LEAF) return MWDG_ERR_ARG;  // a leaf above another leaf
          kind[(size_t)k] = K_SIG;
        }
      }
  }
  // every root is a leaf or refined, every refined node's children leaves or
  // refined, so that each finest cell lies under exactly one leaf
  for (long long k = 0; k < off[1]; k++)
    if (kind[(size_t)k] == K_BELOW) return MWDG_ERR_ARG;
  for (int l = 0; l < L; l++) {
    const long long nx = (long long)M << l, ny = (long long)N << l;
    for (long long j = 0; j < ny; j++)
      for (long long i = 0; i < nx; i++) {
        if (kind[(size_t)(off[l] + j * nx + i)] != K_SIG) continue;
        for (int c = 0; c < 4; c++) {
          const long long kc = off[l + 1] + (2 * j + (c >> 1)) * (2 * nx) + 2 * i + (c & 1);
          if (kind[(size_t)kc] == K_BELOW) return MWDG_ERR_ARG;
        }
      }
  }
  mwdg_adj *a = new (std::nothrow) mwdg_adj;
  if (!a) return MWDG_ERR_CUDA;
  a->p = *p;
  a->levels = L + 1;
  a->mode = mode;
  a->gM = M;
  a->gN = N;
  a->off = off;
  a->fxo = fxo;
  a->fyo = fyo;
  a->lqo = lqo;
  a->nl = n_leaves;
  a->n = nt;
  a->nfin = (long long)p->nx * p->ny;
  const size_t E = p->precision == MWDG_F32 ? sizeof(float) : sizeof(double);
  bool ok = allocate(a, fxo[L + 1], fyo[L + 1], lqo[L + 1]);
  auto alloc = [&](void **ptrp, long long count, size_t elem) {
    if (ok && cudaMalloc(ptrp, (size_t)count * elem) != cudaSuccess) ok = false;
  };
  alloc((void **)&a->kind, nt, 1);
  alloc((void **)&a->node, n_leaves, sizeof(long long));
  alloc(&a->zp, 3 * nt, E);
  alloc(&a->np, nt, E);
  alloc(&a->gzp, 3 * nt, E);
  alloc(&a->gnp, nt, E);
  alloc(&a->gV, 12 * nt, E);
  ok = ok && cudaMemcpy(a->kind, kind.data(), (size_t)nt, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(a->node, node.data(), (size_t)n_leaves * sizeof(long long), cudaMemcpyHostToDevice) ==
           cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_all(a);
    delete a;
    return MWDG_ERR_CUDA;
  }
  *out = a;
  return MWDG_OK;
}

void mwdg_adj_destroy(mwdg_adj *a) {
  if (!a) return;
  cudaDeviceSynchronize();
  free_all(a);
  delete a;
}

const char *mwdg_adj_last_error(const mwdg_adj *a) { return a ? a->err.c_str() : ""; }

mwdg_status mwdg_adj_profile(mwdg_adj *a, int32_t max_launches) {
  if (!a || max_launches < 0) return MWDG_ERR_ARG;
  cudaDeviceSynchronize();
  free_events(a);
  if (max_launches == 0) return MWDG_OK;
  a->evs.resize((size_t)2 * max_launches, nullptr);
  a->ev_class.assign((size_t)max_launches, 0);
  for (auto &e : a->evs)
    if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
      free_events(a);
      return cuda_check(a, "mwdg_adj_profile");
    }
  return MWDG_OK;
}

mwdg_status mwdg_adj_kernel_times(mwdg_adj *a, double *ms, int64_t *count) {
  if (!a || !ms || !count) return MWDG_ERR_ARG;
  for (int c = 0; c < MWDG_ADJ_KC_COUNT; c++) {
    ms[c] = 0.0;
    count[c] = 0;
  }
  for (size_t q = 0; q + 1 < a->ev_used; q += 2) {
    float t = 0.0f;
    if (cudaEventSynchronize(a->evs[q + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, a->evs[q], a->evs[q + 1]) != cudaSuccess)
      return cuda_check(a, "mwdg_adj_kernel_times");
    ms[a->ev_class[q / 2]] += t;
    count[a->ev_class[q / 2]] += 1;
  }
  a->ev_used = 0;
  return MWDG_OK;
}

mwdg_status mwdg_adj_project(mwdg_adj *a, const double *vert, void *out, void *stream) {
  if (!a) return MWDG_ERR_ARG;
  if (!vert || !out) return fail(a, MWDG_ERR_ARG, "NULL pointer");
  const unsigned nb = blocks((long long)a->p.nx * a->p.ny);
  if (a->p.precision == MWDG_F32)
    k_project<float><<<nb, TPB, 0, (cudaStream_t)stream>>>(make_par<float>(a, 0, nullptr, nullptr), vert,
                                                            ptr<float>(out));
  else
    k_project<double><<<nb, TPB, 0, (cudaStream_t)stream>>>(make_par<double>(a, 0, nullptr, nullptr), vert,
                                                              ptr<double>(out));
  return cuda_check(a, "mwdg_adj_project");
}

mwdg_status mwdg_adj_project_transpose(mwdg_adj *a, const void *gp, void *gv, void *stream) {
  if (!a) return MWDG_ERR_ARG;
  if (!gp || !gv) return fail(a, MWDG_ERR_ARG, "NULL pointer");
  const unsigned nb = blocks((long long)(a->p.nx + 1) * (a->p.ny + 1));
  if (a->p.precision == MWDG_F32)
    k_project_t<float><<<nb, TPB, 0, (cudaStream_t)stream>>>(make_par<float>(a, 0, nullptr, nullptr),
                                                              static_cast<const float *>(gp), ptr<float>(gv));
  else
    k_project_t<double><<<nb, TPB, 0, (cudaStream_t)stream>>>(make_par<double>(a, 0, nullptr, nullptr),
                                                                static_cast<const double *>(gp), ptr<double>(gv));
  return cuda_check(a, "mwdg_adj_project_transpose");
}

mwdg_status mwdg_adj_regrid(mwdg_adj *from, mwdg_adj *to, const void *U_from, void *U_to, void *stream) {
  const mwdg_status s = check_pair(from, to);
  if (s != MWDG_OK) return s;
  if (!U_from || !U_to) return fail(from, MWDG_ERR_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  if (from->p.precision == MWDG_F32)
    launch_regrid<float>(from, to, static_cast<const float *>(U_from), ptr<float>(U_to), st);
  else
    launch_regrid<double>(from, to, static_cast<const double *>(U_from), ptr<double>(U_to), st);
  return cuda_check(from, "mwdg_adj_regrid");
}

mwdg_status mwdg_adj_regrid_transpose(mwdg_adj *from, mwdg_adj *to, const void *U_from, const void *gU_to,
                                      void *gU_from, void *stream) {
  const mwdg_status s = check_pair(from, to);
  if (s != MWDG_OK) return s;
  if (!U_from || !gU_to || !gU_from) return fail(from, MWDG_ERR_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  if (from->p.precision == MWDG_F32)
    launch_regrid_t<float>(from, to, static_cast<const float *>(U_from), static_cast<const float *>(gU_to),
                           ptr<float>(gU_from), st);
  else
    launch_regrid_t<double>(from, to, static_cast<const double *>(U_from), static_cast<const double *>(gU_to),
                            ptr<double>(gU_from), st);
  return cuda_check(from, "mwdg_adj_regrid_transpose");
}

mwdg_status mwdg_adj_forward(mwdg_adj *a, const void *U0, const void *z, const void *nman, int32_t nknots,
                             const double *kt, const double *kQ, double t0, int32_t steps, int32_t fixed_dt,
                             double *dts, void *U_out, void *stream) {
  mwdg_status s = check_run(a, U0, z, nman, nknots, kt, kQ, steps, dts);
  if (s != MWDG_OK) return s;
  if (!U_out) return fail(a, MWDG_ERR_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  a->tape_steps = steps;
  if (a->p.precision == MWDG_F32)
    return forward_t<float>(a, static_cast<const float *>(U0), static_cast<const float *>(z),
                            static_cast<const float *>(nman), nknots, kt, kQ, t0, steps, fixed_dt, dts,
                            ptr<float>(U_out), st);
  return forward_t<double>(a, static_cast<const double *>(U0), static_cast<const double *>(z),
                           static_cast<const double *>(nman), nknots, kt, kQ, t0, steps, fixed_dt, dts,
                           ptr<double>(U_out), st);
}

mwdg_status mwdg_adj_backward(mwdg_adj *a, const void *U0, const void *z, const void *nman, int32_t nknots,
                              const double *kt, const double *kQ, double t0, int32_t steps, const double *dts_in,
                              const void *gUK, void *gU0, void *gz, void *gn, double *gQ, int32_t reuse_tape,
                              void *stream) {
  mwdg_status s = check_run(a, U0, z, nman, nknots, kt, kQ, steps, dts_in);
  if (s != MWDG_OK) return s;
  const bool reuse = reuse_tape != 0;
  if (reuse && steps != a->tape_steps) return fail(a, MWDG_ERR_STATE, "the tape holds another number of steps");
  a->tape_steps = steps;
  if (!gUK || !gU0 || !gz || !gn || (a->p.inflow_edge >= 0 && !gQ)) return fail(a, MWDG_ERR_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  if (a->p.precision == MWDG_F32)
    return backward_t<float>(a, static_cast<const float *>(U0), static_cast<const float *>(z),
                             static_cast<const float *>(nman), nknots, kt, kQ, t0, steps, dts_in,
                             static_cast<const float *>(gUK), ptr<float>(gU0), ptr<float>(gz), ptr<float>(gn), gQ,
                             reuse, st);
  return backward_t<double>(a, static_cast<const double *>(U0), static_cast<const double *>(z),
                            static_cast<const double *>(nman), nknots, kt, kQ, t0, steps, dts_in,
                            static_cast<const double *>(gUK), ptr<double>(gU0), ptr<double>(gz), ptr<double>(gn), gQ,
                            reuse, st);
}

}  // extern "C"
