// Kernels of the DG2 / multiwavelet-MRA flood solver (arXiv 2107.02750) and
// their launchers, templated on the coefficient type.  Included once per
// precision (mwdg_f64.cu without FMA contraction, mwdg_f32.cu with it).
//
// Data layout: dense per-level pyramids, component-major (see
// mwdg_internal.h).  Active leaves are listed, level-major and row-major
// within a level, in p.leaves; leaf kernels run a fixed grid that strides
// over the device-side count, so a step needs no host synchronisation.
#pragma once
#include <cstdint>
#include <algorithm>
#include <type_traits>

#include "dg2_math.cuh"
#include "mwdg_internal.h"

namespace mwdg {

constexpr int TPB = 256;

// Storage of the first variable's three coefficients.  Depth form (FP64):
// (h0, h1x, h1y).  Free-surface form (FP32): (h0, eta1x, eta1y), the average
// as depth and the slopes of the free surface eta = h + z, so that a flat
// surface is stored with exactly zero slopes while rain and flux increments
// keep the precision of the depth.
template <typename T> struct Form { static constexpr bool eta = std::is_same<T, float>::value; };

// stored slopes -> depth slopes, and back, given the bed slopes
template <typename T>
__device__ __forceinline__ void slopes_to_h(T &s1, T &s2, T z1, T z2) {
  if (Form<T>::eta) {
    s1 = s1 - z1;
    s2 = s2 - z2;
  }
}
template <typename T>
__device__ __forceinline__ void slopes_from_h(T &s1, T &s2, T z1, T z2) {
  if (Form<T>::eta) {
    s1 = s1 + z1;
    s2 = s2 + z2;
  }
}

// Geo constants in the coefficient type (FP32: the single-precision copies)
template <typename T> __device__ __forceinline__ T geo_g(const Geo &g);
template <> __device__ __forceinline__ float geo_g<float>(const Geo &g) { return g.gf; }
template <> __device__ __forceinline__ double geo_g<double>(const Geo &g) { return g.g; }
template <typename T> __device__ __forceinline__ T geo_hd(const Geo &g);
template <> __device__ __forceinline__ float geo_hd<float>(const Geo &g) { return g.hdf; }
template <> __device__ __forceinline__ double geo_hd<double>(const Geo &g) { return g.hd; }
template <typename T> __device__ __forceinline__ T geo_dx(const Geo &g, int l);
template <> __device__ __forceinline__ float geo_dx<float>(const Geo &g, int l) { return g.dxlf[l]; }
template <> __device__ __forceinline__ double geo_dx<double>(const Geo &g, int l) { return g.dxl[l]; }

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

__device__ __forceinline__ void atomic_min_pos(unsigned long long *a, double x) {
  atomicMin(a, dbits(x));  // ordering of positive doubles equals that of their bits
}
__device__ __forceinline__ void atomic_max_pos(unsigned long long *a, double x) {
  atomicMax(a, dbits(x));
}

__device__ __forceinline__ void node_of(const Geo &g, long long k, int &l, int &i, int &j) {
  l = 0;
  while (l < g.L && k >= g.off[l + 1]) l++;
  const long long r = k - g.off[l];
  if (r < (1LL << 32)) {  // 32-bit division (levels of fewer than 2^32 nodes)
    const unsigned r32 = (unsigned)r, n = (unsigned)g.nxl[l];
    j = (int)(r32 / n);
    i = (int)(r32 - (unsigned)j * n);
  } else {
    j = (int)(r / g.nxl[l]);
    i = (int)(r - (long long)j * g.nxl[l]);
  }
}
__device__ __forceinline__ long long nid(const Geo &g, int l, int i, int j) {
  return g.off[l] + (long long)j * g.nxl[l] + i;
}
// flux-view record of a node: 12 values (9 coefficients, 3 bed) read with
// 16-byte vector loads
template <typename T>
__device__ __forceinline__ void load_rec(const T *FZ, long long k, T (&r)[12]);
template <>
__device__ __forceinline__ void load_rec<float>(const float *FZ, long long k, float (&r)[12]) {
  const float4 *q = reinterpret_cast<const float4 *>(FZ + 12 * k);
  float4 a = q[0], b = q[1], c = q[2];
  r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
  r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
  r[8] = c.x; r[9] = c.y; r[10] = c.z; r[11] = c.w;
}
template <>
__device__ __forceinline__ void load_rec<double>(const double *FZ, long long k, double (&r)[12]) {
  const double2 *q = reinterpret_cast<const double2 *>(FZ + 12 * k);
#pragma unroll
  for (int m = 0; m < 6; m++) {
    double2 a = q[m];
    r[2 * m] = a.x;
    r[2 * m + 1] = a.y;
  }
}
template <typename T>
__device__ __forceinline__ void store_rec(T *FZ, long long k, const T (&r)[12]);
template <>
__device__ __forceinline__ void store_rec<float>(float *FZ, long long k, const float (&r)[12]) {
  float4 *q = reinterpret_cast<float4 *>(FZ + 12 * k);
  q[0] = make_float4(r[0], r[1], r[2], r[3]);
  q[1] = make_float4(r[4], r[5], r[6], r[7]);
  q[2] = make_float4(r[8], r[9], r[10], r[11]);
}
template <>
__device__ __forceinline__ void store_rec<double>(double *FZ, long long k, const double (&r)[12]) {
  double2 *q = reinterpret_cast<double2 *>(FZ + 12 * k);
#pragma unroll
  for (int m = 0; m < 6; m++) q[m] = make_double2(r[2 * m], r[2 * m + 1]);
}

// active-list entries carry the leaf's level and indices
__device__ __forceinline__ long long pack_leaf(int l, int i, int j) {
  return ((long long)l << 56) | ((long long)j << 28) | (long long)i;
}
__device__ __forceinline__ long long unpack_leaf(const Geo &g, long long v, int &l, int &i, int &j) {
  l = (int)(v >> 56);
  j = (int)((v >> 28) & 0xFFFFFFFLL);
  i = (int)(v & 0xFFFFFFFLL);
  return nid(g, l, i, j);
}

// ---------------------------------------------------------------------------
// Set-up
// ---------------------------------------------------------------------------

// Eq. 8 (in FP64): interface-centre values are vertex means, average and
// slopes from them.  The printed four-vertex form of Eq. 8a has 1/2 where the
// E/W and N/S forms on the same line give 1/4; 1/4 is used.
template <typename T>
__global__ void k_project(const double *vert, int nx, int ny, T *c0, T *c1x, T *c1y) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= (long long)nx * ny) return;
  int j = (int)(k / nx), i = (int)(k - (long long)j * nx);
  const double s3 = 1.7320508075688772;
  double sw = vert[(long long)j * (nx + 1) + i], se = vert[(long long)j * (nx + 1) + i + 1];
  double nw = vert[(long long)(j + 1) * (nx + 1) + i], ne = vert[(long long)(j + 1) * (nx + 1) + i + 1];
  double zn = 0.5 * (nw + ne), zs = 0.5 * (sw + se);
  double ze = 0.5 * (ne + se), zw = 0.5 * (nw + sw);
  c0[k] = (T)(0.5 * (ze + zw));
  c1x[k] = (T)((ze - zw) / (2.0 * s3));
  c1y[k] = (T)((zn - zs) / (2.0 * s3));
}

// max |z0| on the finest level (normalisation of topography details)
template <typename T>
__global__ void k_zmax(Geo g, Ptrs<T> p) {
  long long n = (long long)g.nxl[g.L] * g.nyl[g.L];
  double m = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs((double)p.Z[g.off[g.L] + k]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomic_max_pos(&p.ctl->vmax[0], m);
}

// z pyramid level l from level l+1 (Eq. 9) and each node's normalised detail
template <typename T>
__global__ void k_encode_z(Geo g, Ptrs<T> p, int l) {
  long long n = (long long)g.nxl[l] * g.nyl[l];
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= n) return;
  int j = (int)(r / g.nxl[l]), i = (int)(r - (long long)j * g.nxl[l]);
  const long long P = g.P;
  T ch[4][3];
#pragma unroll
  for (int c = 0; c < 4; c++) {
    long long kc = nid(g, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
#pragma unroll
    for (int m = 0; m < 3; m++) ch[c][m] = p.Z[m * P + kc];
  }
  T sp[3];
  encode3(ch, sp);
  long long k = g.off[l] + r;
#pragma unroll
  for (int m = 0; m < 3; m++) p.Z[m * P + k] = sp[m];
  double norm = fmax(1.0, __longlong_as_double((long long)p.ctl->vmax[0]));
  p.DZ[k] = (double)detail_max3(ch) / norm;
}

// Manning n: coarser nodes hold the mean of their children
template <typename T>
__global__ void k_nm_level(Geo g, Ptrs<T> p, int l) {
  long long n = (long long)g.nxl[l] * g.nyl[l];
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= n) return;
  int j = (int)(r / g.nxl[l]), i = (int)(r - (long long)j * g.nxl[l]);
  T acc = T(0);
  for (int c = 0; c < 4; c++) acc = acc + p.NM[nid(g, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1))];
  p.NM[g.off[l] + r] = T(0.25) * acc;
}

// Finest-level initial state.  On entry the first three components hold the
// projected depth (is_eta = 0) or free surface (is_eta = 1).  With is_eta,
// wet elements (average free surface above the average bed) get h = eta - z,
// others are dry.  The free-surface form stores free-surface slopes.
// FV1 sees the bed as one level per element (Eq. 6): the pyramid keeps the
// averages (the multiwavelet average is the children's mean) and drops the
// slopes; HWFV1 (adaptive) thresholds Haar details of the piecewise-constant
// bed (Sect. 2.3) instead of the multiwavelet ones
template <typename T>
__global__ void k_fv1_bed(Geo g, Ptrs<T> p) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= g.P) return;
  const long long P = g.P;
  int l, i, j;
  node_of(g, k, l, i, j);
  if (g.scheme == MWDG_FV1 && g.mode == MWDG_ADAPTIVE && l < g.L) {
    T a[4];
#pragma unroll
    for (int c = 0; c < 4; c++) a[c] = p.Z[nid(g, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1))];
    const double norm = fmax(1.0, __longlong_as_double((long long)p.ctl->vmax[0]));
    p.DZ[k] = (double)haar_detail_max(a[0], a[1], a[2], a[3]) / norm;
  }
  p.Z[P + k] = T(0);
  p.Z[2 * P + k] = T(0);
}

template <typename T>
__global__ void k_initial_finest(Geo g, Ptrs<T> p, int is_eta) {
  const int L = g.L;
  long long n = (long long)g.nxl[L] * g.nyl[L];
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const long long P = g.P, k = g.off[L] + r;
  T *U = p.U;
  if (Form<T>::eta) {
    if (!is_eta) {
      for (int m = 1; m < 3; m++) U[m * P + k] = U[m * P + k] + p.Z[m * P + k];
    } else if (U[k] > p.Z[k]) {
      U[k] = U[k] - p.Z[k];
    } else {
      U[k] = T(0);
      for (int m = 1; m < 3; m++) U[m * P + k] = p.Z[m * P + k];
      for (int m = 3; m < 9; m++) U[m * P + k] = T(0);
    }
  } else if (is_eta) {
    if (U[k] > p.Z[k]) {
      for (int m = 0; m < 3; m++) U[m * P + k] = U[m * P + k] - p.Z[m * P + k];
    } else {
      for (int m = 0; m < 9; m++) U[m * P + k] = T(0);
    }
  }
  if (g.scheme != MWDG_DG2)  // FV1, ACC: averages only (Eq. 5); the bed slopes are zero
    for (int v = 0; v < 3; v++) U[(3 * v + 1) * P + k] = U[(3 * v + 2) * P + k] = T(0);
}

// dense Eq. 9 of `ncomp` components of X from level l+1 to level l; with a
// bed pyramid Zb the first variable is in storage form and is encoded as
// depth
template <typename T>
__global__ void k_encode_dense(Geo g, T *X, int ncomp, int l, const T *Zb) {
  long long n = (long long)g.nxl[l] * g.nyl[l];
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= n) return;
  int j = (int)(r / g.nxl[l]), i = (int)(r - (long long)j * g.nxl[l]);
  const long long P = g.P, k = g.off[l] + r;
  for (int v = 0; v < ncomp / 3; v++) {
    T ch[4][3], sp[3];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      long long kc = nid(g, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
#pragma unroll
      for (int m = 0; m < 3; m++) ch[c][m] = X[(3 * v + m) * P + kc];
      if (Zb && v == 0) slopes_to_h(ch[c][1], ch[c][2], Zb[P + kc], Zb[2 * P + kc]);
    }
    if (g.scheme == MWDG_FV1) {  // Haar: the average, no slopes
      sp[0] = haar_avg(ch[0][0], ch[1][0], ch[2][0], ch[3][0]);
      sp[1] = sp[2] = T(0);
    } else {
      encode3(ch, sp);
      if (Zb && v == 0) slopes_from_h(sp[1], sp[2], Zb[P + k], Zb[2 * P + k]);
    }
#pragma unroll
    for (int m = 0; m < 3; m++) X[(3 * v + m) * P + k] = sp[m];
  }
}

// static grid, free-surface initial state: the encoded free surface (held in
// Wn[0..2]) is split into depth per leaf with the wet/dry rule
template <typename T>
__global__ void k_eta_rule_leaves(Geo g, Ptrs<T> p) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= g.P || p.kind[k] != K_LEAF) return;
  const long long P = g.P;
  const T *E = p.Wn;
  if (E[k] > p.Z[k]) {
    p.U[k] = E[k] - p.Z[k];
    for (int m = 1; m < 3; m++)
      p.U[m * P + k] = Form<T>::eta ? E[m * P + k] : E[m * P + k] - p.Z[m * P + k];
  } else {
    p.U[k] = T(0);
    for (int m = 1; m < 3; m++) p.U[m * P + k] = Form<T>::eta ? p.Z[m * P + k] : T(0);
    for (int m = 3; m < 9; m++) p.U[m * P + k] = T(0);
  }
}

// static grid: significant topography details (Sect. 2.2)
template <typename T>
__global__ void k_static_flags(Geo g, Ptrs<T> p) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= g.P) return;
  p.flag[k] = (k < g.off[g.L]) ? (uint8_t)(p.DZ[k] >= g.eps) : (uint8_t)0;
}

// parent closure from level l to l-1: a flagged child flags its parent
static __global__ void k_closure(Geo g, uint8_t *flag, int l) {
  long long n = (long long)g.nxl[l] * g.nyl[l];
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= n) return;
  if (!flag[g.off[l] + r]) return;
  int j = (int)(r / g.nxl[l]), i = (int)(r - (long long)j * g.nxl[l]);
  flag[nid(g, l - 1, i >> 1, j >> 1)] = 1;
}

// 2:1 grading (Sect. 2.2.1, Fig. 2b): the face neighbours of a flagged node
// at level l >= 1 must exist, so their parents are flagged
template <typename T>
__global__ void k_grading(Geo g, Ptrs<T> p, int l) {
  long long n = (long long)g.nxl[l] * g.nyl[l];
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= n) return;
  if (!p.flag[g.off[l] + r]) return;
  int j = (int)(r / g.nxl[l]), i = (int)(r - (long long)j * g.nxl[l]);
  const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
  for (int f = 0; f < 4; f++) {
    int a = i + di[f], b = j + dj[f];
    if (a < 0 || b < 0 || a >= g.nxl[l] || b >= g.nyl[l]) continue;
    long long kp = nid(g, l - 1, a >> 1, b >> 1);
    if (!p.flag[kp]) {
      p.flag[kp] = 1;
      p.ctl->changed = 1;
    }
  }
}

// node kinds from flags (flags already closed under parents): refined,
// active leaf (parent refined or root, not refined itself) or below a leaf
template <typename T>
__global__ void k_kinds(Geo g, Ptrs<T> p, const uint8_t *flag) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= g.P) return;
  int l, i, j;
  node_of(g, k, l, i, j);
  int f = (l < g.L) ? flag[k] : 0;
  int parent = (l == 0) ? 1 : flag[nid(g, l - 1, i >> 1, j >> 1)];
  p.kind[k] = f ? K_SIG : (parent ? K_LEAF : K_BELOW);
}

template <typename T>
__global__ void k_all_finest(Geo g, Ptrs<T> p) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= g.P) return;
  p.kind[k] = (k >= g.off[g.L]) ? K_LEAF : K_SIG;
}

// ---------------------------------------------------------------------------
// Ballot / prefix-sum compaction of the active leaves (order preserved)
// ---------------------------------------------------------------------------
constexpr int CPT = 8;                 // nodes per thread
constexpr int CTILE = TPB * CPT;       // nodes per block

static __global__ void k_compact_count(long long P, const uint8_t *kind, int *blk) {
  long long base = (long long)blockIdx.x * CTILE;
  int c = 0;
  for (int q = 0; q < CPT; q++) {
    long long k = base + q * TPB + threadIdx.x;
    c += (k < P && kind[k] == K_LEAF);
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ int ws[TPB / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < TPB / 32; w++) s += ws[w];
    blk[blockIdx.x] = s;
  }
}

// exclusive scan of the per-block leaf counts in place (read through L2)
// and their total, by one block: each thread reads its run of up to SCAN_RUN
// consecutive counts at once, then one block-wide scan of the run sums
constexpr int SCAN_RUN = 16;
__device__ __forceinline__ void block_scan_counts(int nb, int *blk, int *total) {
  __shared__ int carry;
  __shared__ int ws[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int span = blockDim.x * SCAN_RUN;
  for (int base = 0; base < nb; base += span) {
    const int b0 = base + threadIdx.x * SCAN_RUN;
    int v[SCAN_RUN];
#pragma unroll
    for (int q = 0; q < SCAN_RUN; q++) v[q] = (b0 + q < nb) ? __ldcg(&blk[b0 + q]) : 0;
    int run = 0;
#pragma unroll
    for (int q = 0; q < SCAN_RUN; q++) run += v[q];
    int x = run;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      int w = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, w, o);
        if (threadIdx.x >= o) w += y;
      }
      ws[threadIdx.x] = w;
    }
    __syncthreads();
    const int warp_off = (threadIdx.x >> 5) ? ws[(threadIdx.x >> 5) - 1] : 0;
    const int incl = x + warp_off + carry;
    int e = incl - run;  // exclusive prefix of this run
#pragma unroll
    for (int q = 0; q < SCAN_RUN; q++)
      if (b0 + q < nb) {
        blk[b0 + q] = e;
        e += v[q];
      }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

static __global__ void k_compact_scan(int nb, int *blk, int *total) { block_scan_counts(nb, blk, total); }

// true in exactly one block, the last to get here; every block's global
// writes before this point are visible to that block's L2 reads afterwards
__device__ __forceinline__ bool last_block(unsigned int *ticket, unsigned nblk) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int v = atomicAdd(ticket, 1u);
    last = (v == nblk - 1);
    if (last) {
      *ticket = 0u;  // ready for the next launch
      __threadfence();
    }
  }
  __syncthreads();
  return last != 0;
}

// dt = min(C * min candidate, dt_max, t_end - t) and per-step resets (one thread)
__device__ __forceinline__ void begin_step(const Geo &g, Ctl *c, const int *nleaf) {
  double best = __longlong_as_double((long long)c->dtmin);
  double dt = g.dt_max;
  if (best < __longlong_as_double(0x7ff0000000000000LL)) dt = fmin(dt, g.cfl * best);
  if (c->dt_fixed > 0.0) dt = c->dt_fixed;  // a prescribed step (mwdg_dg2_step_dt)
  dt = fmin(dt, c->t_end - c->t);
  c->dt = dt > 0.0 ? dt : 0.0;
  c->dt_f = (float)c->dt;
  c->rain_on = (c->t < g.rain_t_end && g.rain_rate > 0.0) ? 1 : 0;
  c->rain_inc = c->rain_on ? g.rain_rate * c->dt : 0.0;
  c->rain_inc_f = (float)c->rain_inc;
  c->bnd[0] = 0.0;
  c->bnd[1] = 0.0;
  c->blocks_done = 0u;
  // the reductions that the last kernel of this step accumulates for the
  // next; a zero step changes nothing, so the current ones stay valid
  if (c->dt > 0.0) {
    c->updates += *nleaf;
    c->dtmin = 0x7ff0000000000000ULL;
    c->vmax[0] = c->vmax[1] = c->vmax[2] = 0ULL;
  }
}

// Face-neighbour code of a leaf, fixed for a step (the grid does not change
// between the stages): what the same-level view of the neighbour across the
// face is made from, and which node holds it.
//   NB_EDGE     domain boundary
//   NB_LEAF     a leaf at the same level (its record)
//   NB_REFINED  a refined node at the same level (MWDG2: its encoded record;
//               static grid: its two finer leaves)
//   NB_COARSER  below a coarser leaf: that leaf and the level difference
enum : int { NB_EDGE = 0, NB_LEAF = 1, NB_REFINED = 2, NB_COARSER = 3 };
__device__ __forceinline__ long long nb_code(int type, int d, long long k) {
  return ((long long)type << 62) | ((long long)d << 56) | k;
}
__device__ __forceinline__ int nb_type(long long c) { return (int)((unsigned long long)c >> 62); }
__device__ __forceinline__ int nb_depth(long long c) { return (int)((c >> 56) & 0xF); }
__device__ __forceinline__ long long nb_node(long long c) { return c & 0xFFFFFFFFFFFFFFLL; }

// the four codes of leaf (l, i, j) under the kinds `kind`; the first kinds
// are read together, then the walks up (coarser neighbours) follow
__device__ __forceinline__ void leaf_nb_codes(const Geo &g, const uint8_t *kind, int l, int i, int j,
                                              long long (&out)[4]) {
  long long kn[4];
  uint8_t kd[4];
  bool in[4];
#pragma unroll
  for (int f = 0; f < 4; f++) {
    const int a = i + (f == 0) - (f == 1), b = j + (f == 2) - (f == 3);
    in[f] = !(a < 0 || b < 0 || a >= g.nxl[l] || b >= g.nyl[l]);
    kn[f] = in[f] ? nid(g, l, a, b) : 0;
    kd[f] = in[f] ? kind[kn[f]] : (uint8_t)K_BELOW;
  }
#pragma unroll
  for (int f = 0; f < 4; f++) {
    if (!in[f]) { out[f] = nb_code(NB_EDGE, 0, 0); continue; }
    if (kd[f] == K_LEAF) { out[f] = nb_code(NB_LEAF, 0, kn[f]); continue; }
    if (kd[f] == K_SIG) { out[f] = nb_code(NB_REFINED, 0, kn[f]); continue; }
    int a = i + (f == 0) - (f == 1), b = j + (f == 2) - (f == 3), la = l, d = 0;
    long long ka = kn[f];
    while (la > 0 && kind[ka] == K_BELOW) {
      a >>= 1;
      b >>= 1;
      la--;
      d++;
      ka = nid(g, la, a, b);
    }
    out[f] = nb_code(NB_COARSER, d, ka);
  }
}

// a leaf's four neighbour codes (E, W, N, S) from the per-step table
__device__ __forceinline__ void load_nb_codes(const long long *nbr, long long q, long long (&c)[4]) {
  const longlong2 *src = reinterpret_cast<const longlong2 *>(nbr + 4 * q);
  const longlong2 a = src[0], b = src[1];
  c[0] = a.x; c[1] = a.y; c[2] = b.x; c[3] = b.y;
}

// Active leaf q of a uniform grid (the one level of an L = 0 hierarchy,
// every node a leaf, the active list in node order): its node, indices and
// four neighbour codes, the ones the list and the code pass hold for it,
// formed from q without reading them.
__device__ __forceinline__ long long uniform_leaf(const Geo &g, long long q, int &l, int &i, int &j,
                                                  long long (&c)[4]) {
  const int nx = g.nxl[0], ny = g.nyl[0];
  l = 0;
  j = (int)(q / nx);
  i = (int)(q - (long long)j * nx);
  c[0] = (i + 1 < nx) ? nb_code(NB_LEAF, 0, q + 1) : nb_code(NB_EDGE, 0, 0);
  c[1] = (i > 0) ? nb_code(NB_LEAF, 0, q - 1) : nb_code(NB_EDGE, 0, 0);
  c[2] = (j + 1 < ny) ? nb_code(NB_LEAF, 0, q + nx) : nb_code(NB_EDGE, 0, 0);
  c[3] = (j > 0) ? nb_code(NB_LEAF, 0, q - nx) : nb_code(NB_EDGE, 0, 0);
  return q;
}

// order-preserving scatter of the active leaves (each thread owns CPT
// consecutive nodes, read as one 8-byte word); with kind_out the kinds are
// also copied there
static_assert(CPT == 8, "one 8-byte word of kinds per thread");
// ctl == nullptr: blk holds each block's exclusive offset (k_compact_scan
// wrote it and the total).  ctl != nullptr: blk holds each block's raw leaf
// count (the decode's); every block sums the counts before its own, the
// block with the highest index writes the total to *nleaf before it takes
// its completion ticket, and with begin the last block to finish starts the
// step on the new leaves.
__device__ __forceinline__ void compact_scatter(const Geo &g, const uint8_t *kind, const int *blk, long long *leaves,
                                                uint8_t *kind_out, Ctl *ctl, int *nleaf, int begin, unsigned bid,
                                                unsigned nblk) {
  const long long P = g.P;
  const long long base = (long long)bid * CTILE + (long long)threadIdx.x * CPT;
  const bool full = base + CPT <= P;
  // the counts of the blocks before this one (their loads in flight with
  // the kinds')
  int before = 0;
  if (ctl)
    for (int r = threadIdx.x; r < (int)bid; r += TPB) before += blk[r];
  uint8_t kk[CPT];
  uint2 w8 = make_uint2(0u, 0u);
  if (full) {
    w8 = *reinterpret_cast<const uint2 *>(kind + base);
#pragma unroll
    for (int q = 0; q < CPT; q++) kk[q] = (uint8_t)(((q < 4) ? (w8.x >> (8 * q)) : (w8.y >> (8 * (q - 4)))) & 0xffu);
  } else {
#pragma unroll
    for (int q = 0; q < CPT; q++) kk[q] = (base + q < P) ? kind[base + q] : (uint8_t)K_BELOW;
  }
  int c = 0;
#pragma unroll
  for (int q = 0; q < CPT; q++) c += (kk[q] == K_LEAF);
  if (kind_out) {
    if (full) *reinterpret_cast<uint2 *>(kind_out + base) = w8;
    else
      for (int q = 0; q < CPT; q++)
        if (base + q < P) kind_out[base + q] = kk[q];
  }
  // block-wide exclusive scan of per-thread counts
  int x = c;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) >= o) x += y;
  }
  __shared__ int ws[TPB / 32];
  if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    int w = (threadIdx.x < TPB / 32) ? ws[threadIdx.x] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (threadIdx.x >= o) w += y;
    }
    if (threadIdx.x < TPB / 32) ws[threadIdx.x] = w;
  }
  __syncthreads();
  int off;
  if (ctl) {
    __shared__ int wb[TPB / 32];
    for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
    if ((threadIdx.x & 31) == 0) wb[threadIdx.x >> 5] = before;
    __syncthreads();
    off = 0;
#pragma unroll
    for (int w = 0; w < TPB / 32; w++) off += wb[w];
    if (bid == nblk - 1 && threadIdx.x == TPB - 1) *nleaf = off + ws[TPB / 32 - 1];
  } else {
    off = blk[bid];
  }
  int pos = off + x - c + ((threadIdx.x >> 5) ? ws[(threadIdx.x >> 5) - 1] : 0);
  for (int q = 0; q < CPT; q++) {
    if (kk[q] == K_LEAF) {
      int l, i, j;
      node_of(g, base + q, l, i, j);
      leaves[pos++] = pack_leaf(l, i, j);
    }
  }
  // the last block to finish sees the total and starts the step
  if (ctl && last_block(&ctl->ticket, nblk) && begin && threadIdx.x == 0) begin_step(g, ctl, nleaf);
}

static __global__ void k_compact_scatter(Geo g, const uint8_t *kind, const int *blk, long long *leaves,
                                         uint8_t *kind_out, Ctl *ctl, int *nleaf, int begin) {
  compact_scatter(g, kind, blk, leaves, kind_out, ctl, nleaf, begin, blockIdx.x, gridDim.x);
}

// the four face-neighbour codes of every active leaf (one thread per leaf)
static __global__ void k_leaf_codes(Geo g, const uint8_t *kind, const long long *leaves, const int *nleaf,
                                    long long *nbr) {
  const int n = *nleaf;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    int l, i, j;
    unpack_leaf(g, leaves[q], l, i, j);
    long long c4[4];
    leaf_nb_codes(g, kind, l, i, j, c4);
    longlong2 *dst = reinterpret_cast<longlong2 *>(nbr + 4LL * q);
    dst[0] = make_longlong2(c4[0], c4[1]);
    dst[1] = make_longlong2(c4[2], c4[3]);
  }
}

// ---------------------------------------------------------------------------
// Boundary forcing
// ---------------------------------------------------------------------------
__device__ __forceinline__ double inflow_Q(const Geo &g, const double *kt, const double *kQ, double t) {
  int n = g.nknots;
  if (n <= 0) return 0.0;
  if (t <= kt[0]) return kQ[0];
  if (t >= kt[n - 1]) return kQ[n - 1];
  int k = 0;
  while (k + 1 < n && !(t < kt[k + 1])) k++;
  double tk = kt[k], tk1 = kt[k + 1], Qk = kQ[k], Qk1 = kQ[k + 1];
  return Qk + (Qk1 - Qk) * (t - tk) / (tk1 - tk);
}

// unit discharge through the boundary face of a leaf (level l, index k along
// edge e): the hydrograph spread over the inflow cells times the overlap
__device__ __forceinline__ double inflow_q(const Geo &g, const double *kt, const double *kQ, int e, int l,
                                           int k, double t) {
  if (g.inflow_edge != e) return 0.0;
  int sh = g.L - l;
  long long a = (long long)k << sh, b = (long long)(k + 1) << sh;
  long long lo = a > g.inflow_c0 ? a : g.inflow_c0;
  long long hi = b < (long long)g.inflow_c1 + 1 ? b : (long long)g.inflow_c1 + 1;
  long long ov = hi - lo;
  if (ov <= 0) return 0.0;
  long long nin = (long long)g.inflow_c1 - g.inflow_c0 + 1;
  return inflow_Q(g, kt, kQ, t) * (double)ov / ((double)nin * g.dxl[l]);
}

// ---------------------------------------------------------------------------
// Step kernels (leaf-list, fixed grid striding over the device count)
// ---------------------------------------------------------------------------
#define FOR_LEAVES(p) FOR_LEAVES_B(p, blockIdx.x, gridDim.x)
// the same for block bid of nblk (a batched launch's member-local block)
#define FOR_LEAVES_B(p, bid, nblk)                                                 \
  const int _nl = *(p).nleaf;                                                      \
  for (int _q = (int)(bid) * blockDim.x + threadIdx.x; _q < _nl; _q += (int)(nblk) * blockDim.x)

// max |v0| over the leaves of h, qx, qy (normalisation of flow details)
template <typename T>
__global__ void k_leaf_maxabs(Geo g, Ptrs<T> p) {
  double m0 = 0, m1 = 0, m2 = 0;
  const long long P = g.P;
  FOR_LEAVES(p) {
    int l, i, j;
    long long k = unpack_leaf(g, p.leaves[_q], l, i, j);
    T h0 = p.U[k];
    m0 = fmax(m0, (double)tabs(h0));
    m1 = fmax(m1, (double)tabs(p.U[3 * P + k]));
    m2 = fmax(m2, (double)tabs(p.U[6 * P + k]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmax(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_pos(&p.ctl->vmax[0], m0);
    atomic_max_pos(&p.ctl->vmax[1], m1);
    atomic_max_pos(&p.ctl->vmax[2], m2);
  }
}

// forcing time of the inflow hydrograph, read only where a boundary face
// needs it: t (stage 1 and the CFL pass) or t + dt (stage 2)
struct ForceTime {
  const Ctl *c;
  bool plus_dt;
  __device__ __forceinline__ double operator()() const { return plus_dt ? c->t + c->dt : c->t; }
};

// dt and the rain depth of the step in the coefficient type
template <typename T> __device__ __forceinline__ T ctl_dt(const Ctl *c);
template <> __device__ __forceinline__ float ctl_dt<float>(const Ctl *c) { return c->dt_f; }
template <> __device__ __forceinline__ double ctl_dt<double>(const Ctl *c) { return c->dt; }
template <typename T> __device__ __forceinline__ T ctl_rain(const Ctl *c);
template <> __device__ __forceinline__ float ctl_rain<float>(const Ctl *c) { return c->rain_inc_f; }
template <> __device__ __forceinline__ double ctl_rain<double>(const Ctl *c) { return c->rain_inc; }
// dt > 0 without FP64 arithmetic (a non-negative double orders as its bits)
__device__ __forceinline__ bool ctl_stepping(const Ctl *c) { return __double_as_longlong(c->dt) > 0; }

// CFL candidate of one leaf (Courant number applied in k_begin_step):
// min over x and y of dx / (|u| + sqrt(g h)) when wet, and the inflow ghost
// states at the critical depth on inflow faces; +inf when there is none
template <typename T>
__device__ __forceinline__ T leaf_dt_candidate(const Geo &g, const Ptrs<T> &p, int l, int i, int j,
                                               T h0, T qx0, T qy0, ForceTime t) {
  const T gg = geo_g<T>(g), hd = geo_hd<T>(g);
  const T dxl = geo_dx<T>(g, l);
  T best = tinf<T>();
  if (g.scheme == MWDG_ACC) return (h0 > hd) ? dxl / tsqrt(gg * h0) : best;  // gravity waves only
  if (h0 > hd) {
    T u = qx0 / h0, v = qy0 / h0;
    T c = tsqrt(gg * h0);
    best = tmin(dxl / (tabs(u) + c), dxl / (tabs(v) + c));
  }
  if (g.inflow_edge >= 0) {
    for (int e = 0; e < 4; e++) {
      bool on = (e == 0 && i == 0) || (e == 1 && i == g.nxl[l] - 1) || (e == 2 && j == 0) ||
                (e == 3 && j == g.nyl[l] - 1);
      if (!on) continue;
      double q = inflow_q(g, p.knot_t, p.knot_Q, e, l, (e < 2) ? j : i, t());
      if (q > 0.0) {
        T qt = (T)q;
        T hc = tcbrt(qt * qt / gg);
        if (hc > hd) best = tmin(best, dxl / (qt / hc + tsqrt(gg * hc)));
      }
    }
  }
  return best;
}

template <typename T>
__device__ __forceinline__ void warp_min_to(unsigned long long *dst, T v) {
  for (int o = 16; o > 0; o >>= 1) v = tmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v < tinf<T>()) atomic_min_pos(dst, (double)v);
}

// CFL candidates over the leaves
template <typename T>
__global__ void k_leaf_dt(Geo g, Ptrs<T> p) {
  const long long P = g.P;
  const ForceTime t{p.ctl, false};
  T best = tinf<T>();
  FOR_LEAVES(p) {
    int l, i, j;
    long long k = unpack_leaf(g, p.leaves[_q], l, i, j);
    best = tmin(best, leaf_dt_candidate(g, p, l, i, j, p.U[k], p.U[3 * P + k], p.U[6 * P + k], t));
  }
  warp_min_to(&p.ctl->dtmin, best);
}

// ---------------------------------------------------------------------------
// Tiled multi-level MRA passes
// ---------------------------------------------------------------------------
// A block owns a 16 x 16 tile of nodes at a chunk's finest level ltop and
// the nodes above them at up to four coarser levels (8 x 8, 4 x 4, 2 x 2,
// 1).  It first stages in shared memory what each tile node brings from
// global memory (its kind, and a leaf's own coefficients) while the
// refined nodes of the finest tile level read their children, then runs
// the coarser levels from shared memory with a block barrier between them:
// a chunk of five levels is one launch with two memory round trips per
// block.  The coarsest levels (at most g.coarse_nodes nodes each) are run by
// the last block of the chunk below them to finish: each block takes a
// completion ticket after its writes and the block that draws the last one
// continues (no block waits on another).
constexpr int MT = 16;         // tile side at a chunk's finest level (one node per thread)
constexpr int MT_LEVELS = 5;   // levels per chunk: 16, 8, 4, 2, 1 nodes per side
static_assert(MT * MT == TPB, "one thread per node of a tile's finest level");

// first shared-memory slot of tile level s (levels stacked finest first)
// (the geometric sum MT^2 + (MT/2)^2 + ... of the s finer levels, in closed
// form: no recursion at run time)
__host__ __device__ constexpr int tbase(int s) {
  return (4 * MT * MT - ((4 * MT * MT) >> (2 * s))) / 3;
}
constexpr int MT_NODES = tbase(MT_LEVELS);  // 341 nodes in a full tile
static_assert(tbase(1) == 256 && tbase(2) == 320 && tbase(3) == 336 && tbase(4) == 340 && MT_NODES == 341,
              "tile levels of 16, 8, 4, 2 and 1 nodes a side");
static_assert(MT_NODES <= 2 * TPB, "two staged slots per thread");
constexpr uint8_t K_OUT = 0xff;             // slot outside its level

struct Tile { int ltop, nlev, bx, by; };

// resident blocks per SM asked of the latency-bound MRA kernels (FP32: at
// most 64 registers a thread; FP64 keeps its registers)
template <typename T> struct MraOcc { static constexpr int blocks = std::is_same<T, float>::value ? 4 : 1; };

// the tile of block bid of a launch over the tiles of level ltop
__device__ __forceinline__ Tile tile_of_block(const Geo &g, int ltop, int nlev, unsigned bid) {
  const int tiles_x = (g.nxl[ltop] + MT - 1) / MT;
  return Tile{ltop, nlev, (int)(bid % tiles_x), (int)(bid / tiles_x)};
}

// the coarsest levels fit one tile (run from shared memory by the last block)
__device__ __forceinline__ bool tail_is_tile(const Geo &g, int tail) {
  return tail + 1 <= MT_LEVELS && g.nxl[tail] <= MT && g.nyl[tail] <= MT;
}

// tile level s and index t within it of a slot
__device__ __forceinline__ void slot_st(int slot, int &s, int &t) {
  s = (slot >= tbase(1)) + (slot >= tbase(2)) + (slot >= tbase(3)) + (slot >= tbase(4));
  t = slot - ((s == 0) ? 0 : (s == 1) ? tbase(1) : (s == 2) ? tbase(2) : (s == 3) ? tbase(3) : tbase(4));
}

// grid node (level ltop - s) of node t of tile level s; false outside the level
__device__ __forceinline__ bool tile_coord(const Geo &g, const Tile &tl, int s, int t, int &i, int &j) {
  const int lg = 4 - s, l = tl.ltop - s;  // side = MT >> s = 2^lg
  static_assert(MT == 16, "tile side 2^4");
  i = (tl.bx << lg) + (t & ((1 << lg) - 1));
  j = (tl.by << lg) + (t >> lg);
  return i < g.nxl[l] && j < g.nyl[l];
}

// slot of child c (= cx + 2 cy) of node t of tile level s >= 1
__device__ __forceinline__ int child_slot(int s, int t, int c) {
  const int lg = 4 - s;  // side = 2^lg
  const int a = 2 * (t & ((1 << lg) - 1)) + (c & 1), b = 2 * (t >> lg) + (c >> 1);
  return tbase(s - 1) + (b << (lg + 1)) + a;
}

// the two slots a thread stages, with their grid node (-1: none)
__device__ __forceinline__ void staged_slots(const Geo &g, const Tile &tl, int sl[2], long long kk[2]) {
  const int n_slots = tbase(tl.nlev);
#pragma unroll
  for (int q = 0; q < 2; q++) {
    sl[q] = (int)threadIdx.x + q * TPB;
    kk[q] = -1;
    if (sl[q] < n_slots) {
      int s, t, i, j;
      slot_st(sl[q], s, t);
      if (tile_coord(g, tl, s, t, i, j)) kk[q] = nid(g, tl.ltop - s, i, j);
    }
  }
}

// load through L2 (CG: data written by other blocks of the same launch)
template <bool CG, typename X>
__device__ __forceinline__ X ldx(const X *a) {
  if (CG) return __ldcg(a);
  return *a;
}

// Significance of a flow detail: max |d| / max(1, max |v0|) >= eps, decided
// as an FP64 comparison in both precisions.  FP64: in that form (the
// oracle's order).  FP32: as (double) max |d| >= thr with thr = eps *
// max(1, max |v0|) formed in FP64 once per block; for a non-negative float
// that equals max |d| >= thr_f, thr_f the smallest float not below thr, so
// the comparison itself needs no FP64 unit.
template <typename T>
__device__ __forceinline__ bool detail_significant(T dm, double mx, float thr_f, double eps);
template <>
__device__ __forceinline__ bool detail_significant<double>(double dm, double mx, float, double eps) {
  return dm / fmax(1.0, mx) >= eps;
}
template <>
__device__ __forceinline__ bool detail_significant<float>(float dm, double, float thr_f, double) {
  return dm >= thr_f;
}
__device__ __forceinline__ float float_at_or_above(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, __int_as_float(0x7f800000));
  return f;
}
// a >= b for non-negative doubles, on their bits (integer unit)
__device__ __forceinline__ bool ge_nonneg(double a, double b) {
  return __double_as_longlong(a) >= __double_as_longlong(b);
}

// Eq. 9 encode of a refined node from its children's stored coefficients
// ch[v][c][m] and bed slopes zc[c]; the node's stored coefficients go to
// out; true when a normalised flow detail is significant
template <typename T>
__device__ __forceinline__ bool encode_sig(T (&ch)[3][4][3], const T (&zc)[4][2], T zp1, T zp2,
                                           const double (&mx)[3], const float (&thr)[3], double eps,
                                           bool fv1, T (&out)[9]) {
  bool sig = false;
  if (fv1) {  // HWFV1: Haar average and details of the child averages
#pragma unroll
    for (int v = 0; v < 3; v++) {
      out[3 * v] = haar_avg(ch[v][0][0], ch[v][1][0], ch[v][2][0], ch[v][3][0]);
      out[3 * v + 1] = out[3 * v + 2] = T(0);
      sig = sig | detail_significant<T>(haar_detail_max(ch[v][0][0], ch[v][1][0], ch[v][2][0], ch[v][3][0]),
                                         mx[v], thr[v], eps);
    }
    return sig;
  }
#pragma unroll
  for (int c = 0; c < 4; c++) slopes_to_h(ch[0][c][1], ch[0][c][2], zc[c][0], zc[c][1]);
#pragma unroll
  for (int v = 0; v < 3; v++) {
    T sp[3];
    encode3(ch[v], sp);
    if (v == 0) slopes_from_h(sp[1], sp[2], zp1, zp2);
#pragma unroll
    for (int m = 0; m < 3; m++) out[3 * v + m] = sp[m];
    sig = sig | detail_significant<T>(detail_max3(ch[v]), mx[v], thr[v], eps);
  }
  return sig;
}

// MWDG2 encode of one node of level l (Sect. 2.3): a refined node gets the
// scale coefficients of its children (Eq. 9) and is flagged when its largest
// normalised flow or topography detail reaches epsilon; other nodes carry no
// flow details, so only their topography detail counts.  SPEC: the
// children's coefficients are read together with the node's kind (one
// memory round trip; used on the small coarsest levels).
template <bool SPEC, bool FV1, typename T>
__device__ __forceinline__ void encode_flag_node(const Geo &g, const Ptrs<T> &p, int l, int i, int j) {
  const long long P = g.P, k = nid(g, l, i, j);
  const uint8_t kd = p.kind[k];
  bool sig = ge_nonneg(p.DZ[k], g.eps);
  T ch[3][4][3], zc[4][2];
  if (SPEC || kd == K_SIG) {
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const long long kc = nid(g, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
#pragma unroll
      for (int v = 0; v < 3; v++)
#pragma unroll
        for (int m = 0; m < 3; m++) ch[v][c][m] = ldx<SPEC>(&p.U[(3 * v + m) * P + kc]);
      zc[c][0] = p.Z[P + kc];
      zc[c][1] = p.Z[2 * P + kc];
    }
  }
  if (kd == K_SIG) {
    double mx[3];
    float thr[3];
#pragma unroll
    for (int v = 0; v < 3; v++) {
      mx[v] = __longlong_as_double((long long)p.ctl->vmax[v]);
      thr[v] = float_at_or_above(g.eps * fmax(1.0, mx[v]));
    }
    T out[9];
    sig = encode_sig(ch, zc, p.Z[P + k], p.Z[2 * P + k], mx, thr, g.eps, FV1, out) || sig;
#pragma unroll
    for (int m = 0; m < 9; m++) p.U[m * P + k] = out[m];
  }
  p.flag[k] = (uint8_t)sig;
}

// regularised flag of node (m, a, b): prediction (the node or one of its
// eight same-level neighbours is significant) or closure (a child is
// refined; the children's regularised flags are final by then)
template <bool CG, typename T>
__device__ __forceinline__ uint8_t regular_flag(const Geo &g, const Ptrs<T> &p, int m, int a, int b) {
  uint8_t f = 0;
#pragma unroll
  for (int bb = -1; bb <= 1; bb++)
#pragma unroll
    for (int aa = -1; aa <= 1; aa++) {
      const int x = a + aa, y = b + bb;
      if (x >= 0 && y >= 0 && x < g.nxl[m] && y < g.nyl[m]) f |= p.flag[nid(g, m, x, y)];
    }
  if (m + 1 < g.L)
#pragma unroll
    for (int c = 0; c < 4; c++) f |= ldx<CG>(&p.flag2[nid(g, m + 1, 2 * a + (c & 1), 2 * b + (c >> 1))]);
  return f;
}

// adaptation runs only while there is time left to step (steps queued
// beyond the end time are no-ops, as on the host side); the condition is
// the same in every block of a launch
#define ADAPT_LIVE(p) (!ge_nonneg((p).ctl->t, (p).ctl->t_end))

template <typename T>
struct SigStage {
  T u[MT_NODES][9];     // stored coefficients (leaves: own; refined: encoded)
  T z[MT_NODES][2];     // bed slopes (free-surface form)
  uint8_t kind[MT_NODES];
  uint8_t topo[MT_NODES];  // topography detail significant
  double mx[3];            // max |v0| of h, qx, qy (normalisation of the flow details)
  float thr[3];            // eps * max(1, mx), rounded up to a float
};

// encode + significance of one tile (CG: the children of its finest level
// were written by other blocks of this launch)
template <bool CG, bool FV1, typename T>
__device__ __forceinline__ void sig_tile(const Geo &g, const Ptrs<T> &p, const Tile &tl, SigStage<T> &sh) {
  const long long P = g.P;
  if (threadIdx.x < 3) {
    const double m = __longlong_as_double((long long)p.ctl->vmax[threadIdx.x]);
    sh.mx[threadIdx.x] = m;
    sh.thr[threadIdx.x] = float_at_or_above(g.eps * fmax(1.0, m));
  }
  int sl[2];
  long long kk[2];
  staged_slots(g, tl, sl, kk);
  uint8_t kd[2];
  bool tp[2];
  T zs[2][2];
#pragma unroll
  for (int q = 0; q < 2; q++) {
    kd[q] = K_OUT;
    tp[q] = false;
    zs[q][0] = zs[q][1] = T(0);
    if (kk[q] >= 0) {
      kd[q] = p.kind[kk[q]];
      tp[q] = ge_nonneg(p.DZ[kk[q]], g.eps);
      if (Form<T>::eta) {
        zs[q][0] = p.Z[P + kk[q]];
        zs[q][1] = p.Z[2 * P + kk[q]];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 2; q++)
    if (sl[q] < MT_NODES) {
      sh.kind[sl[q]] = kd[q];
      sh.topo[sl[q]] = tp[q];
      sh.z[sl[q]][0] = zs[q][0];
      sh.z[sl[q]][1] = zs[q][1];
      if (kd[q] == K_LEAF)
#pragma unroll
        for (int m = 0; m < 9; m++) sh.u[sl[q]][m] = p.U[m * P + kk[q]];
    }
  __syncthreads();
  double mx[3];
  float thr[3];
#pragma unroll
  for (int v = 0; v < 3; v++) {
    mx[v] = sh.mx[v];
    thr[v] = sh.thr[v];
  }
  // finest tile level: refined nodes read their children from global memory
  if (kk[0] >= 0) {
    bool sig = tp[0];
    if (kd[0] == K_SIG) {
      int s0, t0, i, j;
      slot_st(sl[0], s0, t0);
      tile_coord(g, tl, 0, t0, i, j);
      T ch[3][4][3], zc[4][2], out[9];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const long long kc = nid(g, tl.ltop + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
#pragma unroll
        for (int v = 0; v < 3; v++)
#pragma unroll
          for (int m = 0; m < 3; m++) ch[v][c][m] = ldx<CG>(&p.U[(3 * v + m) * P + kc]);
        zc[c][0] = p.Z[P + kc];
        zc[c][1] = p.Z[2 * P + kc];
      }
      sig = encode_sig(ch, zc, zs[0][0], zs[0][1], mx, thr, g.eps, FV1, out) || sig;
#pragma unroll
      for (int m = 0; m < 9; m++) {
        p.U[m * P + kk[0]] = out[m];
        sh.u[sl[0]][m] = out[m];
      }
    }
    p.flag[kk[0]] = (uint8_t)sig;
  }
  // coarser tile levels from shared memory
  for (int s = 1; s < tl.nlev; s++) {
    __syncthreads();
    const int side = MT >> s, t = threadIdx.x;
    if (t >= side * side) continue;
    const int slot = tbase(s) + t;
    const uint8_t k2 = sh.kind[slot];
    if (k2 == K_OUT) continue;
    int i, j;
    tile_coord(g, tl, s, t, i, j);
    const long long k = nid(g, tl.ltop - s, i, j);
    bool sig = sh.topo[slot] != 0;
    if (k2 == K_SIG) {
      T ch[3][4][3], zc[4][2], out[9];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const int cs = child_slot(s, t, c);
#pragma unroll
        for (int v = 0; v < 3; v++)
#pragma unroll
          for (int m = 0; m < 3; m++) ch[v][c][m] = sh.u[cs][3 * v + m];
        zc[c][0] = sh.z[cs][0];
        zc[c][1] = sh.z[cs][1];
      }
      sig = encode_sig(ch, zc, sh.z[slot][0], sh.z[slot][1], mx, thr, g.eps, FV1, out) || sig;
#pragma unroll
      for (int m = 0; m < 9; m++) {
        p.U[m * P + k] = out[m];
        sh.u[slot][m] = out[m];
      }
    }
    p.flag[k] = (uint8_t)sig;
  }
}

// encode + significance of the coarsest levels tail..0 by one block (the
// levels below are final)
template <bool FV1, typename T>
__device__ __forceinline__ void sig_tail(const Geo &g, const Ptrs<T> &p, int tail, SigStage<T> &sh) {
  if (tail_is_tile(g, tail)) {
    sig_tile<true, FV1>(g, p, Tile{tail, tail + 1, 0, 0}, sh);
    return;
  }
  for (int l = tail; l >= 0; l--) {
    const int n = g.nxl[l] * g.nyl[l];
    for (int r = threadIdx.x; r < n; r += blockDim.x) encode_flag_node<true, FV1>(g, p, l, r % g.nxl[l], r / g.nxl[l]);
    __syncthreads();
  }
}

// encode + significance flags: levels ltop..ltop-nlev+1 in tiles, then
// (tail >= 0) levels tail..0 in the last block
template <typename T, bool FV1>
__device__ __forceinline__ void mra_sig(const Geo &g, const Ptrs<T> &p, int ltop, int nlev, int tail, unsigned bid,
                                        unsigned nblk) {
  __shared__ SigStage<T> sh;
  if (!ADAPT_LIVE(p)) return;
  if (nlev > 0) sig_tile<false, FV1>(g, p, tile_of_block(g, ltop, nlev, bid), sh);
  if (tail < 0 || !last_block(&p.ctl->ticket, nblk)) return;
  sig_tail<FV1>(g, p, tail, sh);
}

template <typename T, bool FV1>
__global__ void __launch_bounds__(TPB, MraOcc<T>::blocks) k_mra_sig(Geo g, Ptrs<T> p, int ltop, int nlev, int tail) {
  mra_sig<T, FV1>(g, p, ltop, nlev, tail, blockIdx.x, gridDim.x);
}

struct RegStage {
  uint8_t pred[MT_NODES];  // prediction: a node of the 3 x 3 same-level neighbourhood is significant
  uint8_t f2[MT_NODES];    // regularised flag
};

// prediction flag of node (m, a, b)
template <typename T>
__device__ __forceinline__ uint8_t predicted(const Geo &g, const Ptrs<T> &p, int m, int a, int b) {
  const int nx = g.nxl[m], ny = g.nyl[m];
  const uint8_t *row = p.flag + nid(g, m, a, b);
  const bool w = a > 0, e = a + 1 < nx, s_ = b > 0, n_ = b + 1 < ny;
  uint8_t f = row[0];
  if (w) f |= row[-1];
  if (e) f |= row[1];
  if (s_) {
    const uint8_t *r = row - nx;
    f |= r[0];
    if (w) f |= r[-1];
    if (e) f |= r[1];
  }
  if (n_) {
    const uint8_t *r = row + nx;
    f |= r[0];
    if (w) f |= r[-1];
    if (e) f |= r[1];
  }
  return f;
}

// regularised flags of one tile: prediction, then closure bottom-up
template <bool CG, typename T>
__device__ __forceinline__ void reg_tile(const Geo &g, const Ptrs<T> &p, const Tile &tl, RegStage &sh) {
  int sl[2];
  long long kk[2];
  staged_slots(g, tl, sl, kk);
  uint8_t pr[2] = {0, 0};
#pragma unroll
  for (int q = 0; q < 2; q++)
    if (kk[q] >= 0) {
      int s, t, i, j;
      slot_st(sl[q], s, t);
      tile_coord(g, tl, s, t, i, j);
      pr[q] = predicted(g, p, tl.ltop - s, i, j);
    }
  uint8_t cl = 0;  // closure from the children of the finest tile level
  if (kk[0] >= 0 && tl.ltop + 1 < g.L) {
    int i, j;
    tile_coord(g, tl, 0, threadIdx.x, i, j);
#pragma unroll
    for (int c = 0; c < 4; c++) cl |= ldx<CG>(&p.flag2[nid(g, tl.ltop + 1, 2 * i + (c & 1), 2 * j + (c >> 1))]);
  }
#pragma unroll
  for (int q = 0; q < 2; q++)
    if (sl[q] < MT_NODES) sh.pred[sl[q]] = pr[q];
  if (kk[0] >= 0) {
    const uint8_t f = pr[0] | cl;
    p.flag2[kk[0]] = f;
    sh.f2[sl[0]] = f;
  }
  for (int s = 1; s < tl.nlev; s++) {
    __syncthreads();
    const int side = MT >> s, t = threadIdx.x;
    if (t >= side * side) continue;
    int i, j;
    if (!tile_coord(g, tl, s, t, i, j)) continue;
    const int slot = tbase(s) + t;
    uint8_t f = sh.pred[slot];
#pragma unroll
    for (int c = 0; c < 4; c++) f |= sh.f2[child_slot(s, t, c)];
    sh.f2[slot] = f;
    p.flag2[nid(g, tl.ltop - s, i, j)] = f;
  }
}

// regularised flags of the coarsest levels tail..0 by one block
template <typename T>
__device__ __forceinline__ void reg_tail(const Geo &g, const Ptrs<T> &p, int tail, RegStage &sh) {
  if (tail_is_tile(g, tail)) {
    reg_tile<true>(g, p, Tile{tail, tail + 1, 0, 0}, sh);
    return;
  }
  for (int l = tail; l >= 0; l--) {
    const int n = g.nxl[l] * g.nyl[l];
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const int i = r % g.nxl[l], j = r / g.nxl[l];
      p.flag2[nid(g, l, i, j)] = regular_flag<true>(g, p, l, i, j);
    }
    __syncthreads();
  }
}

// regularised flags, same chunking; the CFL minimum is reset here for the
// decode pass that follows
template <typename T>
__device__ __forceinline__ void mra_regularise(const Geo &g, const Ptrs<T> &p, int ltop, int nlev, int tail,
                                               unsigned bid, unsigned nblk) {
  __shared__ RegStage sh;
  if (ltop == g.L - 1 && bid == 0 && threadIdx.x == 0) p.ctl->dtmin = 0x7ff0000000000000ULL;
  if (!ADAPT_LIVE(p)) return;
  if (nlev > 0) reg_tile<false>(g, p, tile_of_block(g, ltop, nlev, bid), sh);
  if (tail < 0 || !last_block(&p.ctl->ticket, nblk)) return;
  reg_tail(g, p, tail, sh);
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_mra_regularise(Geo g, Ptrs<T> p, int ltop, int nlev, int tail) {
  mra_regularise<T>(g, p, ltop, nlev, tail, blockIdx.x, gridDim.x);
}

// The regularisation's coarsest levels tail..0, run by the first block of
// the decode when the regularise pass leaves them out.  Only nodes of levels
// up to tail + 1 read these flags (a node's kind depends on its own flag and
// its parent's), and the host defers only when all of them belong to that
// first block, which runs this before them; so the other blocks need nothing
// from here and the coarsest levels leave the critical path.  (The encode
// and significance tail stays in the last block of its own pass: run here,
// beside three decode blocks on one SM, its chain of five dependent levels
// took longer than the decode itself.)
template <typename T>
__device__ __noinline__ void coarse_flags(const Geo &g, const Ptrs<T> &p, int tail) {
  __shared__ RegStage sh;
  reg_tail(g, p, tail, sh);
  __syncthreads();
}

// New kinds from the regularised flags (refined; active leaf: parent
// refined or root, not refined itself; below a leaf), written to
// kind_new while kind keeps the old ones.  Eq. 10 for the new active set:
// every new leaf that was below an old leaf takes the prolongation of that
// leaf's plane (one level at a time, flow in depth form).  Each block counts
// its new leaves (the scatter turns the counts into offsets), and every new
// leaf contributes its CFL candidate for the coming step.
// The depth plane (s0, s1x, s1y) of a parent before it is prolonged to its
// children: its slopes scaled about the average so that no child's average
// is negative (the wet/dry treatment keeps depths non-negative; scaling
// limiter of Zhang & Shu 2010 at the children's centres), or dropped when
// the parent holds no water; unchanged when every child is non-negative.
template <typename T>
__device__ __forceinline__ void depth_plane_for_children(T &s0, T &s1x, T &s1y) {
  T m = tinf<T>();
#pragma unroll
  for (int c = 0; c < 4; c++) {
    T o[3];
    prolong3(s0, s1x, s1y, c, o);
    m = tmin(m, o[0]);
  }
  if (!(m < T(0))) return;
  if (s0 > T(0)) {
    const T th = s0 / (s0 - m);
    s1x = s1x * th;
    s1y = s1y * th;
  } else {
    s1x = T(0);
    s1y = T(0);
  }
}

// prolongation (Eq. 10) into new leaf k (level l, i, j) from the old leaf
// above it (flow in depth form, one level at a time; the depth plane kept
// non-negative at every level)
template <typename T>
__device__ __noinline__ void prolong_from_old_leaf(const Geo &g, const Ptrs<T> &p, long long k, int l, int i,
                                                   int j) {
  const long long P = g.P;
  // the old leaf above: the node itself was below a leaf, so start at its
  // parent; the next three ancestors' kinds are read together
  int d = 1;
  for (;;) {
    uint8_t kd[3];
#pragma unroll
    for (int q = 0; q < 3; q++) kd[q] = (l - d - q >= 0) ? p.kind[nid(g, l - d - q, i >> (d + q), j >> (d + q))]
                                                         : (uint8_t)K_LEAF;
    if (kd[0] != K_BELOW || l - d == 0) break;
    if (kd[1] != K_BELOW || l - d - 1 == 0) { d += 1; break; }
    if (kd[2] != K_BELOW || l - d - 2 == 0) { d += 2; break; }
    d += 3;
  }
  const long long ka = nid(g, l - d, i >> d, j >> d);
  T u[9];
#pragma unroll
  for (int m = 0; m < 9; m++) u[m] = p.U[m * P + ka];
  const T za1 = p.Z[P + ka], za2 = p.Z[2 * P + ka], zk1 = p.Z[P + k], zk2 = p.Z[2 * P + k];
  T out[9];
  for (int v = 0; v < 3; v++) {
    T sv[3] = {u[3 * v], u[3 * v + 1], u[3 * v + 2]};
    if (v == 0) slopes_to_h(sv[1], sv[2], za1, za2);
    for (int qq = d - 1; qq >= 0; qq--) {  // child at level l - qq: bits qq of i and j
      T o[3];
      if (v == 0) depth_plane_for_children(sv[0], sv[1], sv[2]);
      prolong3(sv[0], sv[1], sv[2], ((i >> qq) & 1) + 2 * ((j >> qq) & 1), o);
      if (v == 0) o[0] = tmax(o[0], T(0));  // rounding residue brought to zero depth
      sv[0] = o[0]; sv[1] = o[1]; sv[2] = o[2];
    }
    if (v == 0) slopes_from_h(sv[1], sv[2], zk1, zk2);
    out[3 * v] = sv[0]; out[3 * v + 1] = sv[1]; out[3 * v + 2] = sv[2];
  }
#pragma unroll
  for (int m = 0; m < 9; m++) p.U[m * P + k] = out[m];
}

// bytes q of an 8-byte word
__device__ __forceinline__ uint8_t byte_of(uint2 w, int q) {
  return (uint8_t)(((q < 4) ? (w.x >> (8 * q)) : (w.y >> (8 * (q - 4)))) & 0xffu);
}

// Each thread takes CPT consecutive nodes (the scatter's layout); when they
// lie in one row of one level (the common case) their flags and kinds are
// read as 8-byte words and their parents follow from the first node.
// ftail >= 0: the first block first runs the coarsest levels ftail..0 of
// the regularisation (coarse_flags).
template <typename T>
__device__ __forceinline__ void mra_decode(const Geo &g, const Ptrs<T> &p, int ftail, unsigned bid) {
  const long long P = g.P;
  if (ftail >= 0 && bid == 0 && ADAPT_LIVE(p)) coarse_flags<T>(g, p, ftail);
  const long long k0 = (long long)bid * CTILE + (long long)threadIdx.x * CPT;
  const ForceTime t{p.ctl, false};
  int cnt = 0;
  T best = tinf<T>();
  if (k0 < P) {
    int l, i0, j0;
    node_of(g, k0, l, i0, j0);
    uint8_t nk[CPT];
    unsigned leaf_mask = 0u, below_mask = 0u;
    const bool row = (k0 + CPT <= P) && (i0 + CPT <= g.nxl[l]);
    if (row) {
      const uint2 ko8 = *reinterpret_cast<const uint2 *>(p.kind + k0);
      const uint2 f8 = (l < g.L) ? *reinterpret_cast<const uint2 *>(p.flag2 + k0) : make_uint2(0u, 0u);
      // parents' flags, byte m for parent (i0 >> 1) + m (five when i0 is odd)
      unsigned long long fpw = 0x0101010101ULL;
      if (l > 0) {
        const long long kp = nid(g, l - 1, i0 >> 1, j0 >> 1);
        fpw = 0ULL;
#pragma unroll
        for (int m = 0; m <= CPT / 2; m++)
          if (m < CPT / 2 || (i0 & 1)) fpw |= (unsigned long long)p.flag2[kp + m] << (8 * m);
      }
#pragma unroll
      for (int q = 0; q < CPT; q++) {
        const uint8_t f = byte_of(f8, q);
        const uint8_t par = (uint8_t)((fpw >> (8 * ((q + (i0 & 1)) >> 1))) & 0xffULL);
        nk[q] = f ? K_SIG : (par ? K_LEAF : K_BELOW);
        if (nk[q] == K_LEAF) {
          leaf_mask |= 1u << q;
          if (byte_of(ko8, q) == K_BELOW) below_mask |= 1u << q;
        }
      }
      uint2 w = make_uint2(0u, 0u);
#pragma unroll
      for (int q = 0; q < CPT; q++) {
        if (q < 4) w.x |= (unsigned)nk[q] << (8 * q);
        else w.y |= (unsigned)nk[q] << (8 * (q - 4));
      }
      *reinterpret_cast<uint2 *>(p.kind_new + k0) = w;
      // prolongation into new leaves that were below an old leaf (rare)
      for (int q = 0; q < CPT; q++)
        if ((below_mask >> q) & 1u) prolong_from_old_leaf(g, p, k0 + q, l, i0 + q, j0);
      // CFL candidates of the new leaves
      T h[CPT], qx[CPT], qy[CPT];
#pragma unroll
      for (int q = 0; q < CPT; q++)
        if ((leaf_mask >> q) & 1u) {
          h[q] = p.U[k0 + q];
          qx[q] = p.U[3 * P + k0 + q];
          qy[q] = p.U[6 * P + k0 + q];
        }
#pragma unroll
      for (int q = 0; q < CPT; q++)
        if ((leaf_mask >> q) & 1u) best = tmin(best, leaf_dt_candidate(g, p, l, i0 + q, j0, h[q], qx[q], qy[q], t));
      cnt = __popc(leaf_mask);
    } else {
      // nodes across a row or level boundary, or the end of the pyramid
      for (int q = 0; q < CPT; q++) {
        const long long k = k0 + q;
        if (k >= P) break;
        int lq, i, j;
        node_of(g, k, lq, i, j);
        const int f = (lq < g.L) ? p.flag2[k] : 0;
        const int par = (lq == 0) ? 1 : p.flag2[nid(g, lq - 1, i >> 1, j >> 1)];
        const uint8_t n = f ? K_SIG : (par ? K_LEAF : K_BELOW);
        p.kind_new[k] = n;
        if (n != K_LEAF) continue;
        cnt++;
        if (p.kind[k] == K_BELOW) prolong_from_old_leaf(g, p, k, lq, i, j);
        best = tmin(best, leaf_dt_candidate(g, p, lq, i, j, p.U[k], p.U[3 * P + k], p.U[6 * P + k], t));
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    best = tmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  }
  __shared__ int ws[TPB / 32];
  __shared__ T wb[TPB / 32];
  if ((threadIdx.x & 31) == 0) {
    ws[threadIdx.x >> 5] = cnt;
    wb[threadIdx.x >> 5] = best;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int sum = 0;
    T b = wb[0];
    for (int w = 0; w < TPB / 32; w++) {
      sum += ws[w];
      b = tmin(b, wb[w]);
    }
    p.blk[bid] = sum;
    if (b < tinf<T>()) atomic_min_pos(&p.ctl->dtmin, (double)b);  // one FP64 conversion per block
  }
}

template <typename T>
__global__ void __launch_bounds__(TPB, MraOcc<T>::blocks) k_mra_decode(Geo g, Ptrs<T> p, int ftail) {
  mra_decode<T>(g, p, ftail, blockIdx.x);
}

static __global__ void k_begin_step(Geo g, Ctl *c, const int *nleaf) { begin_step(g, c, nleaf); }

// end of a step: mass budget, time and step count (run once, by the last
// block of the stage-2 update to finish)
// (euler: one stage, Eq. 7, whose boundary fluxes are in bnd[0])
__device__ __forceinline__ void end_step(const Geo &g, Ctl *c, bool euler) {
  double dt = c->dt;
  if (!(dt > 0.0)) return;
  double b0 = atomicAdd(&c->bnd[0], 0.0), b1 = atomicAdd(&c->bnd[1], 0.0);
  double net = euler ? dt * b0 : 0.5 * dt * (b0 + b1);
  if (net >= 0.0) c->v_out += net;
  else c->v_in += -net;
  if (c->t < g.rain_t_end && g.rain_rate > 0.0) c->v_rain += g.rain_rate * dt * g.area;
  c->t = c->t + dt;
  c->steps += 1;
}

// Split implicit friction (Sect. 2.1.1): the factor of the linearised
// backward Euler step of dq/dt = -g n^2 |u| q / h^(4/3), applied to the
// average and slope coefficients of the discharges (rain has been added to
// the depth first); dry leaves lose their discharge.
template <typename T>
__device__ __forceinline__ T friction_factor(T h0, T qx0, T qy0, T nm, T dt, T gg) {
  T u = qx0 / h0, v = qy0 / h0;
  T sp = tsqrt(u * u + v * v);
  T den = T(1) + dt * gg * nm * nm * sp / (h0 * tcbrt(h0));
  return T(1) / den;
}

// Partial-wet test of a leaf's stage input w (after rain and friction in
// stage 1) with bed planes zp: a leaf whose average, any interface depth of
// its plane, or any interface depth under a flat free surface h0 + z0 is not
// wetter than h_dry drops to first order, stored as a flat free surface
// over its planar bed (ws) and seen by the fluxes as flat depth over a flat
// bed (wf, ze).  Returns false, with ws = w and ze = zp, for a leaf that is
// not reduced.
template <typename T>
__device__ __forceinline__ bool limit_reduced(const Geo &g, const T (&w)[9], const T (&zp)[3], T (&ws)[9],
                                              T (&wf)[9], T (&ze)[3]) {
  const T hd = geo_hd<T>(g);
  const T h0 = w[0];
  const T eta0 = h0 + zp[0];
  T h1x = w[1], h1y = w[2];
  slopes_to_h(h1x, h1y, zp[1], zp[2]);
  bool reduced = !(h0 > hd);
#pragma unroll
  for (int f = 0; f < 4; f++) {
    if (!(face_value(h0, h1x, h1y, f) > hd)) reduced = true;
    if (!(eta0 - face_value(zp[0], zp[1], zp[2], f) > hd)) reduced = true;
  }
#pragma unroll
  for (int m = 0; m < 9; m++) ws[m] = w[m];
  if (!reduced) {
    ze[0] = zp[0]; ze[1] = zp[1]; ze[2] = zp[2];
    return false;
  }
  // stored: flat free surface over the planar bed; flux view: flat depth
  // over a flat bed (the same numbers in the free-surface form)
  if (Form<T>::eta) {
    ws[1] = T(0); ws[2] = T(0);
  } else {
    ws[1] = -zp[1]; ws[2] = -zp[2];
  }
  ws[4] = ws[5] = ws[7] = ws[8] = T(0);
#pragma unroll
  for (int m = 0; m < 9; m++) wf[m] = ws[m];
  wf[1] = T(0); wf[2] = T(0);
  ze[0] = zp[0]; ze[1] = T(0); ze[2] = T(0);
  return true;
}

// Minmod of a leaf that is not reduced, per direction against its same-level
// leaf neighbours (E, W, N, S: has[d], their depth averages nh (after rain),
// discharge averages nq (after friction) and bed averages nzb), on the
// interface offsets sqrt3 v1: two-argument minmod where only one neighbour
// exists; qx and qy always (a dry neighbour has zero discharge), eta where
// the leaf and its neighbours are wet.  ws holds w on entry and the limited
// stored view on return.
template <typename T>
__device__ __forceinline__ void limit_minmod(const Geo &g, const T (&w)[9], const T (&zp)[3], const bool (&has)[4],
                                             const T (&nh)[4], const T (&nq)[4][2], const T (&nzb)[4], T (&ws)[9]) {
  const T hd = geo_hd<T>(g), s3 = s3v<T>();
#pragma unroll
  for (int dir = 0; dir < 2; dir++) {
    const int dA = 2 * dir, dB = 2 * dir + 1;  // E/W, then N/S
    const bool hasA = has[dA], hasB = has[dB];
    if (!hasA && !hasB) continue;
    const T hC = w[0], hA = nh[dA], hB = nh[dB];
    const bool wet = (hC > hd) && (!hasA || hA > hd) && (!hasB || hB > hd);
    const int cs = 1 + dir;
#pragma unroll
    for (int v = 0; v < 3; v++) {
      if (v == 0 && !wet) continue;
      T a0, aC, aB, slope;
      const T zs = zp[cs];
      if (v == 0) {
        aC = hC + zp[0];
        a0 = hA + nzb[dA];
        aB = hB + nzb[dB];
        slope = Form<T>::eta ? w[cs] : w[cs] + zs;
      } else {
        aC = w[3 * v];
        a0 = nq[dA][v - 1];
        aB = nq[dB][v - 1];
        slope = w[3 * v + cs];
      }
      T a = s3 * slope, mm;
      if (hasA && hasB) mm = minmod3(a, a0 - aC, aC - aB);
      else if (hasA) mm = minmod2(a, a0 - aC);
      else mm = minmod2(a, aC - aB);
      if (mm != a) {
        T ns = mm / s3;
        if (v == 0) ws[cs] = Form<T>::eta ? ns : ns - zs;
        else ws[3 * v + cs] = ns;
      }
    }
  }
}

// Stage-input limiting of each leaf, giving the stored view Wst (used by
// the RK2 combination) and the flux view F with its bed planes Ze.
// Partially wet leaves (average, any interface depth of the plane, or any
// interface depth under a flat free surface h0 + z0, not wetter than h_dry:
// water shallower than the leaf's own bed relief) drop to first order: stored as a flat free surface over the planar bed,
// seen by the fluxes as flat depth over a flat bed.  Other leaves get the
// minmod limiter per direction against their same-level leaf neighbours
// (two-argument minmod where only one exists): on qx and qy always (a dry
// neighbour has zero discharge), on eta where the leaf and its neighbours
// are wet.
// With FRIC (stage 1), the stage input is U after rain and friction, which
// are applied here to the leaf and, for the limiter, to its neighbours'
// averages (both are pointwise, so every leaf sees the same values).
// CODES (the first kernel after an adaptation): the leaf's four neighbour
// codes are computed here from the kinds and stored for the later kernels
// FP32: at most 64 registers a thread (four resident blocks per SM)
template <typename T> struct LimOcc { static constexpr int blocks = std::is_same<T, float>::value ? 4 : 1; };
// UNI: a uniform grid (uniform_leaf instead of the active list and codes)
template <typename T, bool FRIC, bool FV1, bool CODES, bool UNI>
__device__ __forceinline__ void leaf_limit(const Geo &g, const Ptrs<T> &p, const T *X, T *Wst, unsigned bid,
                                           unsigned nblk) {
  const long long P = g.P;
  const T hd = geo_hd<T>(g), s3 = s3v<T>(), gg = geo_g<T>(g);
  const T dt = ctl_dt<T>(p.ctl);
  const bool rain = FRIC && p.ctl->rain_on;
  const T rinc = ctl_rain<T>(p.ctl);
  FOR_LEAVES_B(p, bid, nblk) {
    int l, i, j;
    long long code[4];
    const long long k = UNI ? uniform_leaf(g, _q, l, i, j, code) : unpack_leaf(g, p.leaves[_q], l, i, j);
    if (CODES) {
      leaf_nb_codes(g, p.kind, l, i, j, code);
      longlong2 *dst = reinterpret_cast<longlong2 *>(p.nbr + 4LL * _q);
      dst[0] = make_longlong2(code[0], code[1]);
      dst[1] = make_longlong2(code[2], code[3]);
    }
    T w[9], zp[3];
#pragma unroll
    for (int m = 0; m < 9; m++) w[m] = X[m * P + k];
#pragma unroll
    for (int m = 0; m < 3; m++) zp[m] = p.Z[m * P + k];
    if (FRIC) {
      if (rain) w[0] = w[0] + rinc;
      if (w[0] > hd) {
        const T f = friction_factor(w[0], w[3], w[6], p.NM[k], dt, gg);
#pragma unroll
        for (int m = 3; m < 9; m++) w[m] = w[m] * f;
      } else {
#pragma unroll
        for (int m = 3; m < 9; m++) w[m] = T(0);
      }
    }
    if (FV1) {  // first order: nothing to limit
      T rec[12];
#pragma unroll
      for (int m = 0; m < 9; m++) {
        Wst[m * P + k] = w[m];
        rec[m] = w[m];
      }
#pragma unroll
      for (int m = 0; m < 3; m++) rec[9 + m] = zp[m];
      store_rec(p.FZ, k, rec);
      continue;
    }
    T ws[9], wf[9], ze[3];
    if (!limit_reduced(g, w, zp, ws, wf, ze)) {
      if (g.limiter) {
        // same-level leaf neighbours from the step's neighbour codes: the
        // averages (and Manning n) of all four read together (a missing
        // neighbour reads the leaf's own, unused)
        if (!CODES && !UNI) load_nb_codes(p.nbr, _q, code);
        bool has[4];
        T nh[4], nq[4][2], nzb[4], nmn[4];
#pragma unroll
        for (int d = 0; d < 4; d++) {
          has[d] = nb_type(code[d]) == NB_LEAF;
          const long long kn = has[d] ? nb_node(code[d]) : k;
          nh[d] = X[kn];
          nq[d][0] = X[3 * P + kn];
          nq[d][1] = X[6 * P + kn];
          nzb[d] = p.Z[kn];
          nmn[d] = FRIC ? p.NM[kn] : T(0);
        }
        // stage 1: the neighbours' averages after rain and friction (both
        // pointwise, so every leaf sees the values their own threads form)
        if (FRIC) {
#pragma unroll
          for (int d = 0; d < 4; d++) {
            if (!has[d]) continue;
            if (rain) nh[d] = nh[d] + rinc;
            if (nh[d] > hd) {
              const T f = friction_factor(nh[d], nq[d][0], nq[d][1], nmn[d], dt, gg);
              nq[d][0] = nq[d][0] * f;
              nq[d][1] = nq[d][1] * f;
            } else {
              nq[d][0] = nq[d][1] = T(0);
            }
          }
        }
        limit_minmod(g, w, zp, has, nh, nq, nzb, ws);
      }
#pragma unroll
      for (int m = 0; m < 9; m++) wf[m] = ws[m];
    }
#pragma unroll
    for (int m = 0; m < 9; m++) Wst[m * P + k] = ws[m];
    T rec[12];
#pragma unroll
    for (int m = 0; m < 9; m++) rec[m] = wf[m];
#pragma unroll
    for (int m = 0; m < 3; m++) rec[9 + m] = ze[m];
    store_rec(p.FZ, k, rec);
  }
}

template <typename T, bool FRIC, bool FV1, bool CODES, bool UNI>
__global__ void __launch_bounds__(TPB, LimOcc<T>::blocks) k_leaf_limit(Geo g, Ptrs<T> p, const T *X, T *Wst) {
  leaf_limit<T, FRIC, FV1, CODES, UNI>(g, p, X, Wst, blockIdx.x, gridDim.x);
}

// local encoding (Eq. 9) of the flux view and its beds onto a refined node
// (MWDG2 interfaces, Sect. 2.3) from its children's records rc[c]
template <typename T>
__device__ __forceinline__ void encode_view_rec(const T (&rc)[4][12], T (&rec)[12], bool fv1) {
  if (fv1) {  // HWFV1: averages of the children (Haar), no slopes
#pragma unroll
    for (int q = 0; q < 4; q++) {
      rec[3 * q] = haar_avg(rc[0][3 * q], rc[1][3 * q], rc[2][3 * q], rc[3][3 * q]);
      rec[3 * q + 1] = rec[3 * q + 2] = T(0);
    }
    return;
  }
  T zc[4][3], zpar[3];
#pragma unroll
  for (int c = 0; c < 4; c++)
#pragma unroll
    for (int m = 0; m < 3; m++) zc[c][m] = rc[c][9 + m];
  encode3(zc, zpar);
#pragma unroll
  for (int m = 0; m < 3; m++) rec[9 + m] = zpar[m];
#pragma unroll
  for (int v = 0; v < 3; v++) {
    T ch[4][3], sp[3];
#pragma unroll
    for (int c = 0; c < 4; c++) {
#pragma unroll
      for (int m = 0; m < 3; m++) ch[c][m] = rc[c][3 * v + m];
      if (v == 0) slopes_to_h(ch[c][1], ch[c][2], zc[c][1], zc[c][2]);
    }
    encode3(ch, sp);
    if (v == 0) slopes_from_h(sp[1], sp[2], zpar[1], zpar[2]);
#pragma unroll
    for (int m = 0; m < 3; m++) rec[3 * v + m] = sp[m];
  }
}

// one node, records read through L2 together with its kind (coarsest
// levels that do not fit one tile)
template <bool FV1, typename T>
__device__ __forceinline__ void encode_view_node(const Geo &g, const Ptrs<T> &p, int l, int i, int j) {
  const long long k = nid(g, l, i, j);
  const uint8_t kd = p.kind[k];
  T rc[4][12], rec[12];
#pragma unroll
  for (int c = 0; c < 4; c++) {
    const long long kc = nid(g, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
#pragma unroll
    for (int m = 0; m < 12; m++) rc[c][m] = __ldcg(&p.FZ[12 * kc + m]);
  }
  if (kd != K_SIG) return;
  encode_view_rec(rc, rec, FV1);
  store_rec(p.FZ, k, rec);
}

template <typename T>
struct ViewStage {
  T r[MT_NODES][12];  // flux-view records (leaves: own; refined: encoded)
  uint8_t kind[MT_NODES];
};

template <bool CG, bool FV1, typename T>
__device__ __forceinline__ void view_tile(const Geo &g, const Ptrs<T> &p, const Tile &tl, ViewStage<T> &sh) {
  int sl[2];
  long long kk[2];
  staged_slots(g, tl, sl, kk);
  uint8_t kd[2];
#pragma unroll
  for (int q = 0; q < 2; q++) kd[q] = (kk[q] >= 0) ? p.kind[kk[q]] : K_OUT;
#pragma unroll
  for (int q = 0; q < 2; q++)
    if (sl[q] < MT_NODES) {
      sh.kind[sl[q]] = kd[q];
      if (kd[q] == K_LEAF) {
        T r[12];
        load_rec(p.FZ, kk[q], r);
#pragma unroll
        for (int m = 0; m < 12; m++) sh.r[sl[q]][m] = r[m];
      }
    }
  if (kd[0] == K_SIG) {
    int i, j;
    tile_coord(g, tl, 0, threadIdx.x, i, j);
    T rc[4][12], rec[12];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const long long kc = nid(g, tl.ltop + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
      if (CG) {
#pragma unroll
        for (int m = 0; m < 12; m++) rc[c][m] = __ldcg(&p.FZ[12 * kc + m]);
      } else {
        load_rec(p.FZ, kc, rc[c]);
      }
    }
    encode_view_rec(rc, rec, FV1);
    store_rec(p.FZ, kk[0], rec);
#pragma unroll
    for (int m = 0; m < 12; m++) sh.r[sl[0]][m] = rec[m];
  }
  for (int s = 1; s < tl.nlev; s++) {
    __syncthreads();
    const int side = MT >> s, t = threadIdx.x;
    if (t >= side * side) continue;
    const int slot = tbase(s) + t;
    if (sh.kind[slot] != K_SIG) continue;
    int i, j;
    tile_coord(g, tl, s, t, i, j);
    T rc[4][12], rec[12];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const int cs = child_slot(s, t, c);
#pragma unroll
      for (int m = 0; m < 12; m++) rc[c][m] = sh.r[cs][m];
    }
    encode_view_rec(rc, rec, FV1);
    store_rec(p.FZ, nid(g, tl.ltop - s, i, j), rec);
#pragma unroll
    for (int m = 0; m < 12; m++) sh.r[slot][m] = rec[m];
  }
}

// flux-view encode of the refined nodes, chunked as the MRA passes (FP32:
// seven resident blocks per SM, 32 registers a thread, so that the 1024
// tiles of a 512 x 512 level run in one wave; FP64 keeps its registers)
template <typename T> struct ViewOcc { static constexpr int blocks = std::is_same<T, float>::value ? 7 : 1; };
template <typename T, bool FV1>
__device__ __forceinline__ void view_tiles(const Geo &g, const Ptrs<T> &p, int ltop, int nlev, int tail, unsigned bid,
                                           unsigned nblk) {
  __shared__ ViewStage<T> sh;
  if (nlev > 0) view_tile<false, FV1>(g, p, tile_of_block(g, ltop, nlev, bid), sh);
  if (tail < 0 || !last_block(&p.ctl->ticket, nblk)) return;
  if (tail_is_tile(g, tail)) {
    view_tile<true, FV1>(g, p, Tile{tail, tail + 1, 0, 0}, sh);
    return;
  }
  for (int l = tail; l >= 0; l--) {
    const int n = g.nxl[l] * g.nyl[l];
    for (int r = threadIdx.x; r < n; r += blockDim.x) encode_view_node<FV1>(g, p, l, r % g.nxl[l], r / g.nxl[l]);
    __syncthreads();
  }
}

template <typename T, bool FV1>
__global__ void __launch_bounds__(TPB, ViewOcc<T>::blocks) k_view_tiles(Geo g, Ptrs<T> p, int ltop, int nlev, int tail) {
  view_tiles<T, FV1>(g, p, ltop, nlev, tail, blockIdx.x, gridDim.x);
}

// Flux-view encode of the coarsest levels tail..0, run by the first block of
// a stage update when the view pass leaves them out.  A leaf reads encoded
// views of its own level only; the leaves of levels up to tail come first
// in the leaf list (node order, coarsest level first) and are at most as
// many as the nodes of level tail, which the host defers only when they fit
// the first block's first pass over the list.  So they are updated by that
// block, after this, and no other block reads what it writes.
template <typename T>
__device__ __noinline__ void coarse_views(const Geo &g, const Ptrs<T> &p, int tail) {
  const bool fv1 = g.scheme == MWDG_FV1;
  for (int l = tail; l >= 0; l--) {
    const int n = g.nxl[l] * g.nyl[l];
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      if (fv1) encode_view_node<true>(g, p, l, r % g.nxl[l], r / g.nxl[l]);
      else encode_view_node<false>(g, p, l, r % g.nxl[l], r / g.nxl[l]);
    }
    __syncthreads();
  }
}

// interface-centre limit of the first variable of a flux-view plane: the
// depth (depth form) or the free surface (free-surface form)
template <typename T>
__device__ __forceinline__ T first_face(T c0, T c1, T c2, T ze0, int f) {
  return Form<T>::eta ? face_value(c0 + ze0, c1, c2, f) : face_value(c0, c1, c2, f);
}

// limit (first variable, qx, qy, z) of the same-level view of the neighbour
// across face f of leaf (l, i, j), from the leaf's neighbour code: the
// leaf's or encoded node's record, the prolongation of the covering
// coarser leaf's record down to the neighbour node, or on a static grid's
// coarse side the mean of the two finer leaves' interface limits
template <typename T>
__device__ void nbr_view_code(const Geo &g, const Ptrs<T> &p, int l, int i, int j, int f, long long code,
                              T out[4]) {
  const int a = i + (f == 0) - (f == 1), b = j + (f == 2) - (f == 3);
  const int fo = f ^ 1;
  const int type = nb_type(code);
  const long long k = nb_node(code);
  if (type == NB_REFINED && g.mode == MWDG_STATIC) {
    int c1, c2;
    if (f == 0) { c1 = 0; c2 = 2; }
    else if (f == 1) { c1 = 1; c2 = 3; }
    else if (f == 2) { c1 = 0; c2 = 1; }
    else { c1 = 2; c2 = 3; }
    long long k1 = nid(g, l + 1, 2 * a + (c1 & 1), 2 * b + (c1 >> 1));
    long long k2 = nid(g, l + 1, 2 * a + (c2 & 1), 2 * b + (c2 >> 1));
    T r1[12], r2[12];
    load_rec(p.FZ, k1, r1);
    load_rec(p.FZ, k2, r2);
    out[0] = T(0.5) * (first_face(r1[0], r1[1], r1[2], r1[9], fo) + first_face(r2[0], r2[1], r2[2], r2[9], fo));
    for (int v = 1; v < 3; v++)
      out[v] = T(0.5) * (face_value(r1[3 * v], r1[3 * v + 1], r1[3 * v + 2], fo) +
                         face_value(r2[3 * v], r2[3 * v + 1], r2[3 * v + 2], fo));
    out[3] = T(0.5) * (face_value(r1[9], r1[10], r1[11], fo) + face_value(r2[9], r2[10], r2[11], fo));
    return;
  }
  T r[12];
  load_rec(p.FZ, k, r);
  if (type == NB_COARSER) {
    // prolongation of the coarser leaf's plane down to the neighbour node,
    // one level at a time (child of level l - q: bits q of a and b)
    const int d = nb_depth(code);
    for (int v = 3; v >= 0; v--) {
      T sv[3] = {r[3 * v], r[3 * v + 1], r[3 * v + 2]};
      if (v == 0) slopes_to_h(sv[1], sv[2], r[10], r[11]);
      for (int q = d - 1; q >= 0; q--) {
        T o[3];
        prolong3(sv[0], sv[1], sv[2], ((a >> q) & 1) + 2 * ((b >> q) & 1), o);
        sv[0] = o[0]; sv[1] = o[1]; sv[2] = o[2];
      }
      out[v] = face_value(sv[0], sv[1], sv[2], fo);
    }
    if (Form<T>::eta) out[0] = out[0] + out[3];  // depth + bed = free surface
    return;
  }
  out[0] = first_face(r[0], r[1], r[2], r[9], fo);
  for (int v = 1; v < 3; v++) out[v] = face_value(r[3 * v], r[3 * v + 1], r[3 * v + 2], fo);
  out[3] = face_value(r[9], r[10], r[11], fo);
}

// the averages (depth, qx, qy) of the same view, evaluated only where the
// neighbour is the donor of an interface's outflow limit: the leaf's or
// encoded node's own, the prolonged plane's, or on a static grid's coarse
// side the mean of the two finer leaves'
template <typename T>
__device__ __forceinline__ void nbr_avg_code(const Geo &g, const Ptrs<T> &p, int l, int i, int j, int f,
                                             long long code, T avg[3]) {
  const int a = i + (f == 0) - (f == 1), b = j + (f == 2) - (f == 3);
  const int type = nb_type(code);
  const long long k = nb_node(code);
  if (type == NB_REFINED && g.mode == MWDG_STATIC) {
    int c1, c2;
    if (f == 0) { c1 = 0; c2 = 2; }
    else if (f == 1) { c1 = 1; c2 = 3; }
    else if (f == 2) { c1 = 0; c2 = 1; }
    else { c1 = 2; c2 = 3; }
    const long long k1 = nid(g, l + 1, 2 * a + (c1 & 1), 2 * b + (c1 >> 1));
    const long long k2 = nid(g, l + 1, 2 * a + (c2 & 1), 2 * b + (c2 >> 1));
    for (int v = 0; v < 3; v++) avg[v] = T(0.5) * (p.FZ[12 * k1 + 3 * v] + p.FZ[12 * k2 + 3 * v]);
    return;
  }
  if (type == NB_COARSER) {
    T r[12];
    load_rec(p.FZ, k, r);
    const int d = nb_depth(code);
    for (int v = 0; v < 3; v++) {
      T sv[3] = {r[3 * v], r[3 * v + 1], r[3 * v + 2]};
      if (v == 0) slopes_to_h(sv[1], sv[2], r[10], r[11]);
      for (int q = d - 1; q >= 0; q--) {
        T o[3];
        prolong3(sv[0], sv[1], sv[2], ((a >> q) & 1) + 2 * ((b >> q) & 1), o);
        sv[0] = o[0]; sv[1] = o[1]; sv[2] = o[2];
      }
      avg[v] = sv[0];
    }
    return;
  }
  for (int v = 0; v < 3; v++) avg[v] = p.FZ[12 * k + 3 * v];
}

// Interface f of a leaf: its own limit, the neighbour's (same-level view or
// boundary ghost), both revised, and the HLL flux in (h, qx, qy) order.
template <typename T>
struct FaceOut {
  T F0, F1, F2;       // numerical flux
  T hs, us, vs, zr;   // own revised limit
  T bout;             // outward boundary mass flux (m^3/s), 0 inside
};

// given the neighbour's view limit and averages nb (inside) or a boundary
// (ghost); with dt > 0 the flux carries the outflow limit of a forward-Euler
// stage of length dt (the donor is this leaf or, inside, the neighbour's
// view; a boundary ghost is never a limited donor)
template <typename T, class NbAvg>
__device__ __forceinline__ FaceOut<T> face_flux_nb(const Geo &g, const Ptrs<T> &p, int l, int i, int j,
                                                   const T (&w)[9], const T (&zc)[3], int f, ForceTime tf,
                                                   bool inside, T (&nb)[4], T dt, const NbAvg &nbavg) {
  const T gg = geo_g<T>(g), hd = geo_hd<T>(g);
  T own[4];
  own[0] = first_face(w[0], w[1], w[2], zc[0], f);
  own[1] = face_value(w[3], w[4], w[5], f);
  own[2] = face_value(w[6], w[7], w[8], f);
  own[3] = face_value(zc[0], zc[1], zc[2], f);
  if (!inside) {
    // ghost: wall mirror, open copy, or critical-depth inflow
    const int e = (f == 0) ? 1 : (f == 1) ? 0 : (f == 2) ? 3 : 2;
    double q = inflow_q(g, p.knot_t, p.knot_Q, e, l, (e < 2) ? j : i, tf());
    nb[3] = own[3];
    if (q > 0.0) {
      T qt = (T)q;
      T hc = tcbrt(qt * qt / gg);
      T hown = Form<T>::eta ? own[0] - own[3] : own[0];
      T hg = tmax(hown, hc);
      nb[0] = Form<T>::eta ? hg + own[3] : hg;
      T qn = (e == 0 || e == 2) ? qt : -qt;
      if (e < 2) { nb[1] = qn; nb[2] = T(0); }
      else { nb[1] = T(0); nb[2] = qn; }
    } else if (g.bc[e] == MWDG_OPEN) {
      nb[0] = own[0]; nb[1] = own[1]; nb[2] = own[2];
    } else {
      nb[0] = own[0];
      if (e < 2) { nb[1] = -own[1]; nb[2] = own[2]; }
      else { nb[1] = own[1]; nb[2] = -own[2]; }
    }
  }
  const T zf = tmax(own[3], nb[3]);
  Side<T> so, sn;
  if (Form<T>::eta) {
    so = revise_eta(own[0], own[1], own[2], own[3], zf, hd);
    sn = revise_eta(nb[0], nb[1], nb[2], nb[3], zf, hd);
  } else {
    so = revise_h(own[0], own[1], own[2], own[3], zf, hd);
    sn = revise_h(nb[0], nb[1], nb[2], nb[3], zf, hd);
  }
  FaceOut<T> o;
  o.hs = so.hs; o.us = so.u; o.vs = so.v; o.zr = so.zr;
  T F3[3];
  if (f == 0) {
    hll(so.hs, so.u, so.v, sn.hs, sn.u, sn.v, gg, hd, F3);
    o.F0 = F3[0]; o.F1 = F3[1]; o.F2 = F3[2];
  } else if (f == 1) {
    hll(sn.hs, sn.u, sn.v, so.hs, so.u, so.v, gg, hd, F3);
    o.F0 = F3[0]; o.F1 = F3[1]; o.F2 = F3[2];
  } else if (f == 2) {
    hll(so.hs, so.v, so.u, sn.hs, sn.v, sn.u, gg, hd, F3);
    o.F0 = F3[0]; o.F1 = F3[2]; o.F2 = F3[1];
  } else {
    hll(sn.hs, sn.v, sn.u, so.hs, so.v, so.u, gg, hd, F3);
    o.F0 = F3[0]; o.F1 = F3[2]; o.F2 = F3[1];
  }
  if (dt > T(0) && o.F0 != T(0)) {
    const bool own_first = (f == 0 || f == 2);
    const bool from_own = own_first ? (o.F0 > T(0)) : (o.F0 < T(0));
    const bool xf = f < 2;
    const T dxl = geo_dx<T>(g, l);
    if (from_own)
      drain_limit(o.F0, o.F1, o.F2, w[0], xf ? w[3] : w[6], xf ? w[6] : w[3], gg, hd, dxl, dt);
    else if (inside) {
      T av[3];
      nbavg(av);
      drain_limit(o.F0, o.F1, o.F2, av[0], xf ? av[1] : av[2], xf ? av[2] : av[1], gg, hd, dxl, dt);
    }
  }
  o.bout = T(0);
  if (!inside) o.bout = ((f == 0 || f == 2) ? o.F0 : -o.F0) * geo_dx<T>(g, l);
  return o;
}

// Reflux rule on static grids (MWDG_IFACE_REFLUX): on the coarse side of a
// face whose neighbour is refined, the flux is the mean of the two fine
// leaves' own fluxes through their halves of the face, computed with the
// same operands and operations as theirs, so the mass leaving one side
// enters the other.  The grid is graded, so both fine leaves lie one level
// below this leaf (node k) and see it through a one-level prolongation of
// its flux-view record; the three records are read together.
template <typename T>
__device__ __forceinline__ void reflux_face(const Geo &g, const Ptrs<T> &p, int l, int i, int j, long long k, int f,
                                         ForceTime tf, T dt, T &F0, T &F1, T &F2) {
  const int a = i + (f == 0) - (f == 1), b = j + (f == 2) - (f == 3);
  int c1, c2;
  if (f == 0) { c1 = 0; c2 = 2; }
  else if (f == 1) { c1 = 1; c2 = 3; }
  else if (f == 2) { c1 = 0; c2 = 1; }
  else { c1 = 2; c2 = 3; }
  const int fo = f ^ 1;  // the fine leaves' face towards this leaf
  int ic[2], jc[2];
  T rc[12], r[2][12];
#pragma unroll
  for (int q = 0; q < 2; q++) {
    const int cq = q ? c2 : c1;
    ic[q] = 2 * a + (cq & 1);
    jc[q] = 2 * b + (cq >> 1);
    load_rec(p.FZ, nid(g, l + 1, ic[q], jc[q]), r[q]);
  }
  load_rec(p.FZ, k, rc);
  T G[2][3];
#pragma unroll
  for (int q = 0; q < 2; q++) {
    // the node across the fine leaf's face, at its level, lies under this
    // leaf: its child index in the prolongation
    const int an = ic[q] + (fo == 0) - (fo == 1), bn = jc[q] + (fo == 2) - (fo == 3);
    const int path = (an & 1) + 2 * (bn & 1);
    T nb[4], av[3];
    // beds (v = 3) first, then the flow planes in depth form
    for (int v = 3; v >= 0; v--) {
      T sv[3] = {rc[3 * v], rc[3 * v + 1], rc[3 * v + 2]};
      if (v == 0) slopes_to_h(sv[1], sv[2], rc[10], rc[11]);
      T o[3];
      prolong3(sv[0], sv[1], sv[2], path, o);
      nb[v] = face_value(o[0], o[1], o[2], f);
      if (v < 3) av[v] = o[0];
    }
    if (Form<T>::eta) nb[0] = nb[0] + nb[3];  // depth + bed = free surface
    T w[9], zc[3];
#pragma unroll
    for (int m = 0; m < 9; m++) w[m] = r[q][m];
#pragma unroll
    for (int m = 0; m < 3; m++) zc[m] = r[q][9 + m];
    const FaceOut<T> o = face_flux_nb(g, p, l + 1, ic[q], jc[q], w, zc, fo, tf, true, nb, dt, [&](T x[3]) {
      x[0] = av[0]; x[1] = av[1]; x[2] = av[2];
    });
    G[q][0] = o.F0; G[q][1] = o.F1; G[q][2] = o.F2;
  }
  F0 = T(0.5) * (G[0][0] + G[1][0]);
  F1 = T(0.5) * (G[0][1] + G[1][1]);
  F2 = T(0.5) * (G[0][2] + G[1][2]);
}

// The operator and update of variable v (0 h, 1 qx, 2 qy) of one leaf:
// L0 from the flux difference and the bed source with the revised
// interface beds, the slopes from the two-point interface rule with the bed
// source S1 = -(2 sqrt3 g / dx) h1 (h1 + z1) that cancels its hydrostatic
// error at rest, then Eq. 4a (STAGE 1) or Eq. 4b (STAGE 2).  Each
// direction's share is formed as soon as its two interfaces are known.
// physical flux component v of a revised limit (hs, us, vs): across an x
// face (F) or a y face (G)
template <typename T>
__device__ __forceinline__ T phys_flux(bool xdir, int v, T hs, T us, T vs, T gg) {
  if (xdir) {
    const T q = hs * us;
    return v == 0 ? q : (v == 1 ? q * us + T(0.5) * gg * hs * hs : q * vs);
  }
  const T r = hs * vs;
  return v == 0 ? r : (v == 1 ? r * us : r * vs + T(0.5) * gg * hs * hs);
}

// One direction's share of the operator, formed as soon as its two faces are
// known (so the four faces' fluxes and revised limits need not stay live):
// per variable the flux difference (F+ - F-) and the slope sum
// ((F+ + F-) - P+) - P- with P the physical flux of the own revised limits;
// and the bed-source factors (hs+ + hs-), (zr+ - zr-).
template <typename T>
struct DirTerms {
  T d[3], s[3], hsum, zdif;
};

template <typename T>
__device__ __forceinline__ void dir_terms(bool xdir, const FaceOut<T> &a, const FaceOut<T> &b, T gg, DirTerms<T> &o) {
  const T Fa[3] = {a.F0, a.F1, a.F2}, Fb[3] = {b.F0, b.F1, b.F2};
#pragma unroll
  for (int v = 0; v < 3; v++) {
    o.d[v] = Fa[v] - Fb[v];
    o.s[v] = Fa[v] + Fb[v] - phys_flux(xdir, v, a.hs, a.us, a.vs, gg) - phys_flux(xdir, v, b.hs, b.us, b.vs, gg);
  }
  o.hsum = a.hs + b.hs;
  o.zdif = a.zr - b.zr;
}

// the update of variable v from the two directions' terms
template <typename T, int STAGE>
__device__ __forceinline__ void finish_var_dir(const Geo &g, int v, long long k, int l, const T (&w)[9],
                                               const T (&zc)[3], const DirTerms<T> &X, const DirTerms<T> &Y, T dt,
                                               const T *Wst, const T *Wcomb, T &o0, T &o1, T &o2) {
  const long long P = g.P;
  const T gg = geo_g<T>(g), s3 = s3v<T>();
  const T dxl = geo_dx<T>(g, l);
  T h1x, h1y, e1x, e1y;
  if (Form<T>::eta) {
    e1x = w[1]; e1y = w[2];
    h1x = w[1] - zc[1]; h1y = w[2] - zc[2];
  } else {
    h1x = w[1]; h1y = w[2];
    e1x = w[1] + zc[1]; e1y = w[2] + zc[2];
  }
  T L0 = -(X.d[v]) / dxl - (Y.d[v]) / dxl;
  if (v == 1) L0 = L0 + -gg * T(0.5) * X.hsum * X.zdif / dxl;
  if (v == 2) L0 = L0 + -gg * T(0.5) * Y.hsum * Y.zdif / dxl;
  T L1x = -(s3 / dxl) * X.s[v];
  T L1y = -(s3 / dxl) * Y.s[v];
  if (v == 1) L1x = L1x + -(T(2) * s3 * gg / dxl) * h1x * e1x;
  if (v == 2) L1y = L1y + -(T(2) * s3 * gg / dxl) * h1y * e1y;
  if (STAGE == 3) L1x = L1y = T(0);  // FV1 (its only stage): L0 only (Sect. 2.1.2)
  const long long b0 = (long long)(3 * v) * P + k;
  if (STAGE == 1 || STAGE == 3) {
    o0 = Wst[b0] + dt * L0;
    o1 = Wst[b0 + P] + dt * L1x;
    o2 = Wst[b0 + 2 * P] + dt * L1y;
  } else {
    o0 = T(0.5) * (Wcomb[b0] + Wst[b0] + dt * L0);
    o1 = T(0.5) * (Wcomb[b0 + P] + Wst[b0 + P] + dt * L1x);
    o2 = T(0.5) * (Wcomb[b0 + 2 * P] + Wst[b0 + 2 * P] + dt * L1y);
  }
}

// the same with the stored views given as values: ws (this stage's input)
// and wc (stage 2: the stage-1 input), variable v's three coefficients
template <typename T, int STAGE>
__device__ __forceinline__ void finish_var_vals(const Geo &g, int v, int l, const T (&w)[9], const T (&zc)[3],
                                                const DirTerms<T> &X, const DirTerms<T> &Y, T dt, const T *ws,
                                                const T *wc, T &o0, T &o1, T &o2) {
  const T gg = geo_g<T>(g), s3 = s3v<T>();
  const T dxl = geo_dx<T>(g, l);
  T h1x, h1y, e1x, e1y;
  if (Form<T>::eta) {
    e1x = w[1]; e1y = w[2];
    h1x = w[1] - zc[1]; h1y = w[2] - zc[2];
  } else {
    h1x = w[1]; h1y = w[2];
    e1x = w[1] + zc[1]; e1y = w[2] + zc[2];
  }
  T L0 = -(X.d[v]) / dxl - (Y.d[v]) / dxl;
  if (v == 1) L0 = L0 + -gg * T(0.5) * X.hsum * X.zdif / dxl;
  if (v == 2) L0 = L0 + -gg * T(0.5) * Y.hsum * Y.zdif / dxl;
  T L1x = -(s3 / dxl) * X.s[v];
  T L1y = -(s3 / dxl) * Y.s[v];
  if (v == 1) L1x = L1x + -(T(2) * s3 * gg / dxl) * h1x * e1x;
  if (v == 2) L1y = L1y + -(T(2) * s3 * gg / dxl) * h1y * e1y;
  if (STAGE == 1) {
    o0 = ws[0] + dt * L0;
    o1 = ws[1] + dt * L1x;
    o2 = ws[2] + dt * L1y;
  } else {
    o0 = T(0.5) * (wc[0] + ws[0] + dt * L0);
    o1 = T(0.5) * (wc[1] + ws[1] + dt * L1x);
    o2 = T(0.5) * (wc[2] + ws[2] + dt * L1y);
  }
}

// positivity clip (h, counted) and dry reset of variable v given the
// leaf's updated depth average h0n
template <typename T>
__device__ __forceinline__ void post_var(const Geo &g, const Ptrs<T> &p, int v, long long k, int l, T h0n,
                                         T &o0, T &o1, T &o2, unsigned long long &ncl, double &csum,
                                         bool &bad) {
  const long long P = g.P;
  const T h0c = (h0n < T(0)) ? T(0) : h0n;
  const bool dry = !(h0c > geo_hd<T>(g));
  if (v == 0) {
    if (h0n < T(0)) {
      ncl++;
      csum += -(double)h0n * (g.dxl[l] * g.dxl[l]);
      o0 = T(0);
    }
    if (dry) {  // flat zero depth (free-surface slopes = bed slopes)
      o1 = Form<T>::eta ? p.Z[P + k] : T(0);
      o2 = Form<T>::eta ? p.Z[2 * P + k] : T(0);
    }
  } else if (dry) {
    o0 = o1 = o2 = T(0);
  }
  if (!isfinite(o0) || !isfinite(o1) || !isfinite(o2)) bad = true;
}

template <typename T>
__device__ __forceinline__ void store_var(long long P, int v, long long k, T *Out, T o0, T o1, T o2) {
  const long long b0 = (long long)(3 * v) * P + k;
  Out[b0] = o0;
  Out[b0 + P] = o1;
  Out[b0 + 2 * P] = o2;
}

// what the next step needs from the new state: max |v0| (adaptive) or the
// CFL candidate (fixed grids)
template <typename T>
__device__ __forceinline__ void next_step_reduce(const Geo &g, const Ptrs<T> &p, int l, int i, int j, T h0,
                                                 T qx0, T qy0, ForceTime tf, T &m0, T &m1, T &m2, T &best) {
  if (g.mode == MWDG_ADAPTIVE) {
    m0 = tmax(m0, tabs(h0));
    m1 = tmax(m1, tabs(qx0));
    m2 = tmax(m2, tabs(qy0));
  } else {
    best = tmin(best, leaf_dt_candidate(g, p, l, i, j, h0, qx0, qy0, tf));
  }
}

// The end of a stage update, per block: the non-finite flag, the block sums
// of the boundary fluxes (coefficient type, one FP64 atomic per block) and
// of the clips (FP64 where they occur), and in stage 2 the reductions the
// next step needs (max |v0| on adaptive grids, the CFL candidate on fixed
// ones); the last of the nblocks blocks to finish closes the step (no
// waiting: each block takes a ticket after its own atomics are visible).
template <typename T, int STAGE, int NT>
__device__ __forceinline__ void update_epilogue(const Geo &g, const Ptrs<T> &p, T bsum, double csum,
                                                unsigned long long ncl, bool bad, T m0, T m1, T m2, T best,
                                                unsigned int nblocks) {
  if (bad) p.ctl->nonfinite = 1;
  // block sums in the coefficient type, one FP64 conversion and atomic per
  // block; clip volumes (rare) in FP64 where they occur
  for (int o = 16; o > 0; o >>= 1) {
    bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
    ncl += __shfl_xor_sync(0xffffffffu, ncl, o);
  }
  if (__any_sync(0xffffffffu, ncl != 0ULL)) {
    for (int o = 16; o > 0; o >>= 1) csum += __shfl_xor_sync(0xffffffffu, csum, o);
    if ((threadIdx.x & 31) == 0 && ncl) {
      atomicAdd(&p.ctl->n_clip, ncl);
      atomicAdd(&p.ctl->v_clip, csum);
    }
  }
  if (STAGE >= 2 && g.mode == MWDG_ADAPTIVE)
    for (int o = 16; o > 0; o >>= 1) {
      m0 = tmax(m0, __shfl_xor_sync(0xffffffffu, m0, o));
      m1 = tmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
      m2 = tmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
  if (STAGE >= 2 && g.mode != MWDG_ADAPTIVE)
    for (int o = 16; o > 0; o >>= 1) best = tmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  __shared__ T red[5][NT / 32];
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][wid] = bsum;
    red[1][wid] = m0;
    red[2][wid] = m1;
    red[3][wid] = m2;
    red[4][wid] = best;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T b = red[0][0], r0 = red[1][0], r1 = red[2][0], r2 = red[3][0], r3 = red[4][0];
    for (int w = 1; w < NT / 32; w++) {
      b += red[0][w];
      r0 = tmax(r0, red[1][w]);
      r1 = tmax(r1, red[2][w]);
      r2 = tmax(r2, red[3][w]);
      r3 = tmin(r3, red[4][w]);
    }
    if (b != T(0)) atomicAdd(&p.ctl->bnd[STAGE == 2 ? 1 : 0], (double)b);
    if (STAGE >= 2) {
      if (g.mode == MWDG_ADAPTIVE) {
        atomic_max_pos(&p.ctl->vmax[0], (double)r0);
        atomic_max_pos(&p.ctl->vmax[1], (double)r1);
        atomic_max_pos(&p.ctl->vmax[2], (double)r2);
      } else if (r3 < tinf<T>()) {
        atomic_min_pos(&p.ctl->dtmin, (double)r3);
      }
    }
  }
  if (STAGE >= 2) {
    // the last block to finish closes the step (no waiting: each block takes
    // a ticket after its own atomics are visible)
    if (threadIdx.x == 0) __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) last = (atomicAdd(&p.ctl->blocks_done, 1u) == nblocks - 1);
    __syncthreads();
    if (last && threadIdx.x == 0) {
      __threadfence();
      end_step(g, p.ctl, STAGE == 3);
    }
  }
}

// One RK2 stage on every leaf (Eq. 4a for STAGE 1, Eq. 4b for STAGE 2; STAGE
// 3 is FV1's single forward-Euler stage, Eq. 7, which also ends the step):
// the DG2 operator L = [L0, L1x, L1y] from the flux view (interface fluxes
// of the revised limits by HLL, bed source with the revised interface beds,
// two-point interface rule for the slope volume integrals with the bed
// source S1 = -(2 sqrt3 g / dx) h1 (h1 + z1) that cancels its hydrostatic
// error at rest), then the update, the positivity clip and the dry reset.
// One thread per leaf: the four neighbours' kinds are read together, then
// their views, then the four interfaces and the three variables.
//
// resident blocks per SM asked of the update (FP32: at most 64 registers a
// thread, four blocks; FP64 keeps its registers)
template <typename T> struct UpdOcc { static constexpr int blocks = std::is_same<T, float>::value ? 4 : 1; };
// with the reflux rule inlined, one block fewer (FP32: 80 registers a thread)
template <typename T, bool REFLUX> struct UpdOccR {
  static constexpr int blocks = (REFLUX && UpdOcc<T>::blocks > 1) ? UpdOcc<T>::blocks - 1 : UpdOcc<T>::blocks;
};

// REFLUX: compiled with the reflux interface rule (static grids only).
// VIEWS (adaptive grids): with vtail >= 0 the first block first encodes the
// coarsest levels vtail..0 of the flux views (coarse_views); the other
// instantiations do not contain the call.
// UNI: a uniform grid (uniform_leaf instead of the active list and codes)
template <typename T, int STAGE, bool REFLUX, bool VIEWS, bool UNI>
__device__ __forceinline__ void leaf_update(const Geo &g, const Ptrs<T> &p, const T *Wst, const T *Wcomb, T *Out,
                                            int vtail, unsigned bid, unsigned nblk) {
  const long long P = g.P;
  if (!ctl_stepping(p.ctl)) return;  // a zero step changes nothing (end_step ignores it too)
  if (VIEWS && vtail >= 0 && bid == 0) coarse_views<T>(g, p, vtail);
  const T dt = ctl_dt<T>(p.ctl), gg = geo_g<T>(g), hd = geo_hd<T>(g), s3 = s3v<T>();
  const ForceTime tf{p.ctl, STAGE == 2};
  T bsum = T(0);  // per-thread sum of a few boundary fluxes; FP64 from the block sum on
  double csum = 0.0;
  unsigned long long ncl = 0;
  bool bad = false;
  // stage 2 also reduces, over the new state, what the next step needs:
  // max |v0| (adaptive: the next encode's normalisation) or the CFL
  // candidate (fixed grids: the next time step)
  T m0 = T(0), m1 = T(0), m2 = T(0);
  T best = tinf<T>();
  const int nl = *p.nleaf;
  // one thread per leaf: the four interfaces, then the three variables
  for (long long q = bid * (long long)blockDim.x + threadIdx.x; q < nl; q += (long long)nblk * blockDim.x) {
    int l, i, j;
    long long code[4];
    const long long k = UNI ? uniform_leaf(g, q, l, i, j, code) : unpack_leaf(g, p.leaves[q], l, i, j);
    T w[9], zc[3];
    {
      T r[12];
      load_rec(p.FZ, k, r);
#pragma unroll
      for (int m = 0; m < 9; m++) w[m] = r[m];
#pragma unroll
      for (int m = 0; m < 3; m++) zc[m] = r[9 + m];
    }
    // the four neighbours' views from the step's neighbour codes, all
    // loads in flight together
    if (!UNI) load_nb_codes(p.nbr, q, code);
    bool in[4];
    T nb[4][4];
#pragma unroll
    for (int d = 0; d < 4; d++) {
      in[d] = nb_type(code[d]) != NB_EDGE;
      if (in[d]) nbr_view_code(g, p, l, i, j, d, code[d], nb[d]);
    }
    // the interfaces in the order E, W, N, S; each direction's terms are
    // formed as soon as its two faces are known
    DirTerms<T> dx_, dy_;
#pragma unroll
    for (int dir = 0; dir < 2; dir++) {
      FaceOut<T> fa = face_flux_nb(g, p, l, i, j, w, zc, 2 * dir, tf, in[2 * dir], nb[2 * dir], dt,
                                   [&](T av[3]) { nbr_avg_code(g, p, l, i, j, 2 * dir, code[2 * dir], av); });
      // (only across a refined neighbour: its code says so without a load)
      if (REFLUX && nb_type(code[2 * dir]) == NB_REFINED) reflux_face(g, p, l, i, j, k, 2 * dir, tf, dt, fa.F0, fa.F1, fa.F2);
      bsum += fa.bout;
      FaceOut<T> fb = face_flux_nb(g, p, l, i, j, w, zc, 2 * dir + 1, tf, in[2 * dir + 1], nb[2 * dir + 1], dt,
                                   [&](T av[3]) { nbr_avg_code(g, p, l, i, j, 2 * dir + 1, code[2 * dir + 1], av); });
      if (REFLUX && nb_type(code[2 * dir + 1]) == NB_REFINED)
        reflux_face(g, p, l, i, j, k, 2 * dir + 1, tf, dt, fb.F0, fb.F1, fb.F2);
      bsum += fb.bout;
      dir_terms(dir == 0, fa, fb, gg, dir == 0 ? dx_ : dy_);
    }
    T o[3][3];
#pragma unroll
    for (int v = 0; v < 3; v++)
      finish_var_dir<T, STAGE>(g, v, k, l, w, zc, dx_, dy_, dt, Wst, Wcomb, o[v][0], o[v][1], o[v][2]);
    const T h0n = o[0][0];
#pragma unroll
    for (int v = 0; v < 3; v++) {
      post_var<T>(g, p, v, k, l, h0n, o[v][0], o[v][1], o[v][2], ncl, csum, bad);
      store_var(P, v, k, Out, o[v][0], o[v][1], o[v][2]);
    }
    if (STAGE >= 2) next_step_reduce<T>(g, p, l, i, j, o[0][0], o[1][0], o[2][0], tf, m0, m1, m2, best);
  }
  update_epilogue<T, STAGE, TPB>(g, p, bsum, csum, ncl, bad, m0, m1, m2, best, nblk);
}

template <typename T, int STAGE, bool REFLUX, bool VIEWS, bool UNI>
__global__ void __launch_bounds__(TPB, UpdOccR<T, REFLUX>::blocks) k_leaf_update(Geo g, Ptrs<T> p, const T *Wst, const T *Wcomb, T *Out,
                                                                      int vtail) {
  leaf_update<T, STAGE, REFLUX, VIEWS, UNI>(g, p, Wst, Wcomb, Out, vtail, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Uniform grids: one fused kernel per RK2 stage
// ---------------------------------------------------------------------------
// A block takes a tile of UniTile<T>::X x UniTile<T>::Y cells, one thread per
// cell.  It reads the stage input and the bed planes (stage 1: and Manning
// n) of the tile and a two-cell halo from HBM once into shared memory, and
// (stage 1) applies the step's rain and friction there; it limits the tile
// and its one-cell ring (the ring's limiter reads the second ring); then each
// thread forms its cell's four interfaces from the flux views in shared
// memory (revision, HLL, outflow limit) and updates the cell (Eq. 4a or 4b).
// Nothing between the limiter and the update goes through HBM: stage 1
// writes U_int and the stored view of the stage-1 input (which stage 2's
// Eq. 4b combines), stage 2 writes U^{n+1}.  The arithmetic is that of the
// leaf kernels (the same functions in the same order), so the results are
// the same bit for bit.  Halo cells are read again by the neighbouring
// tiles, through L2.
template <typename T> struct UniTile;
template <> struct UniTile<float> { static constexpr int X = 32, Y = 8, OCC = 3; };
template <> struct UniTile<double> { static constexpr int X = 16, Y = 8, OCC = 2; };

// the q-th cell of a tile's limited region ((TX + 2) x (TY + 2) cells,
// coordinates from the ring's south-west corner): the tile's own cells
// first (q < TX TY, so that thread q holds its own cell's stored view), then
// the ring's north and south rows and its west and east columns
template <int TX, int TY>
__device__ __forceinline__ void uni_limited_cell(int q, int &lx, int &ly) {
  constexpr int LX = TX + 2;
  if (q < TX * TY) {
    lx = 1 + q % TX;
    ly = 1 + q / TX;
    return;
  }
  q -= TX * TY;
  if (q < 2 * LX) {
    lx = q % LX;
    ly = (q < LX) ? TY + 1 : 0;
    return;
  }
  q -= 2 * LX;
  lx = (q < TY) ? 0 : LX - 1;
  ly = 1 + q % TY;
}

template <typename T, int STAGE>
__global__ void __launch_bounds__(UniTile<T>::X * UniTile<T>::Y, UniTile<T>::OCC)
    k_uni_stage(Geo g, Ptrs<T> p, const T *X, T *Wst_out, const T *Wcomb, T *Out) {
  constexpr int TX = UniTile<T>::X, TY = UniTile<T>::Y, NT = TX * TY;
  constexpr int RX = TX + 4, NR = RX * (TY + 4);   // loaded region: tile and two-cell halo
  constexpr int LX = TX + 2, NL = LX * (TY + 2);   // limited region: tile and its ring
  __shared__ T sR[12][NR];   // stage input (9; stage 1 after rain and friction) and bed planes (3)
  __shared__ T sF[12][NL];   // flux views (9) and their bed planes (3)
  __shared__ T sW[STAGE == 2 ? 9 : 1][STAGE == 2 ? NT : 1];  // stage 2: the tile's stage-1 stored view
  if (!ctl_stepping(p.ctl)) return;  // a zero step changes nothing
  const long long P = g.P;
  const int nx = g.nxl[0], ny = g.nyl[0];
  const int tiles_x = (nx + TX - 1) / TX, tiles = tiles_x * ((ny + TY - 1) / TY);
  const T dt = ctl_dt<T>(p.ctl), gg = geo_g<T>(g), hd = geo_hd<T>(g);
  const bool rain = STAGE == 1 && p.ctl->rain_on;
  const T rinc = ctl_rain<T>(p.ctl);
  const ForceTime tf{p.ctl, STAGE == 2};
  T bsum = T(0);
  double csum = 0.0;
  unsigned long long ncl = 0;
  bool bad = false;
  T m0 = T(0), m1 = T(0), m2 = T(0);
  T best = tinf<T>();
  // the block strides over the tiles (so that the step's per-block reductions
  // and completion ticket stay few)
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int i0 = (tile % tiles_x) * TX, j0 = (tile / tiles_x) * TY;
    // 1. the region from HBM (rows of RX consecutive cells per coefficient)
    for (int r = threadIdx.x; r < NR; r += NT) {
      const int i = i0 - 2 + r % RX, j = j0 - 2 + r / RX;
      if (i < 0 || j < 0 || i >= nx || j >= ny) continue;
      const long long k = (long long)j * nx + i;
      T w[9];
#pragma unroll
      for (int m = 0; m < 9; m++) w[m] = X[m * P + k];
#pragma unroll
      for (int m = 0; m < 3; m++) sR[9 + m][r] = p.Z[m * P + k];
      if (STAGE == 1) {
        if (rain) w[0] = w[0] + rinc;
        if (w[0] > hd) {
          const T f = friction_factor(w[0], w[3], w[6], p.NM[k], dt, gg);
#pragma unroll
          for (int m = 3; m < 9; m++) w[m] = w[m] * f;
        } else {
#pragma unroll
          for (int m = 3; m < 9; m++) w[m] = T(0);
        }
      }
#pragma unroll
      for (int m = 0; m < 9; m++) sR[m][r] = w[m];
    }
    if (STAGE == 2) {
      const int i = i0 + threadIdx.x % TX, j = j0 + threadIdx.x / TX;
      if (i < nx && j < ny) {
        const long long k = (long long)j * nx + i;
#pragma unroll
        for (int m = 0; m < 9; m++) sW[m][threadIdx.x] = Wcomb[m * P + k];
      }
    }
    __syncthreads();
    // 2. limiting of the tile and its ring into flux views; each thread keeps
    // its own cell's stored view
    T ws_own[9];
    for (int q = threadIdx.x; q < NL; q += NT) {
      int lx, ly;
      uni_limited_cell<TX, TY>(q, lx, ly);
      const int i = i0 - 1 + lx, j = j0 - 1 + ly;
      if (i < 0 || j < 0 || i >= nx || j >= ny) continue;
      const int r = (ly + 1) * RX + (lx + 1);
      T w[9], zp[3];
#pragma unroll
      for (int m = 0; m < 9; m++) w[m] = sR[m][r];
#pragma unroll
      for (int m = 0; m < 3; m++) zp[m] = sR[9 + m][r];
      T ws[9], wf[9], ze[3];
      if (!limit_reduced(g, w, zp, ws, wf, ze)) {
        if (g.limiter) {
          const bool has[4] = {i + 1 < nx, i > 0, j + 1 < ny, j > 0};
          const int rn[4] = {r + 1, r - 1, r + RX, r - RX};
          T nh[4], nq[4][2], nzb[4];
#pragma unroll
          for (int d = 0; d < 4; d++) {
            const int rr = has[d] ? rn[d] : r;
            nh[d] = sR[0][rr];
            nq[d][0] = sR[3][rr];
            nq[d][1] = sR[6][rr];
            nzb[d] = sR[9][rr];
          }
          limit_minmod(g, w, zp, has, nh, nq, nzb, ws);
        }
#pragma unroll
        for (int m = 0; m < 9; m++) wf[m] = ws[m];
      }
      const int li = ly * LX + lx;
#pragma unroll
      for (int m = 0; m < 9; m++) sF[m][li] = wf[m];
#pragma unroll
      for (int m = 0; m < 3; m++) sF[9 + m][li] = ze[m];
      if (q < NT) {
#pragma unroll
        for (int m = 0; m < 9; m++) ws_own[m] = ws[m];
        if (STAGE == 1) {
          const long long k = (long long)j * nx + i;
#pragma unroll
          for (int m = 0; m < 9; m++) Wst_out[m * P + k] = ws[m];
        }
      }
    }
    __syncthreads();
    // 3. the cell's interfaces and its update
    const int i = i0 + threadIdx.x % TX, j = j0 + threadIdx.x / TX;
    if (i < nx && j < ny) {
      const long long k = (long long)j * nx + i;
      const int li = (1 + threadIdx.x / TX) * LX + 1 + threadIdx.x % TX;
      T w[9], zc[3];
#pragma unroll
      for (int m = 0; m < 9; m++) w[m] = sF[m][li];
#pragma unroll
      for (int m = 0; m < 3; m++) zc[m] = sF[9 + m][li];
      const bool in[4] = {i + 1 < nx, i > 0, j + 1 < ny, j > 0};
      const int ln[4] = {li + 1, li - 1, li + LX, li - LX};
      T nb[4][4];
#pragma unroll
      for (int d = 0; d < 4; d++) {
        if (!in[d]) continue;
        const int fo = d ^ 1, q = ln[d];
        nb[d][0] = first_face(sF[0][q], sF[1][q], sF[2][q], sF[9][q], fo);
#pragma unroll
        for (int v = 1; v < 3; v++) nb[d][v] = face_value(sF[3 * v][q], sF[3 * v + 1][q], sF[3 * v + 2][q], fo);
        nb[d][3] = face_value(sF[9][q], sF[10][q], sF[11][q], fo);
      }
      DirTerms<T> dx_, dy_;
#pragma unroll
      for (int dir = 0; dir < 2; dir++) {
        const int fa_ = 2 * dir, fb_ = 2 * dir + 1;
        FaceOut<T> fa = face_flux_nb(g, p, 0, i, j, w, zc, fa_, tf, in[fa_], nb[fa_], dt, [&](T av[3]) {
          av[0] = sF[0][ln[fa_]]; av[1] = sF[3][ln[fa_]]; av[2] = sF[6][ln[fa_]];
        });
        bsum += fa.bout;
        FaceOut<T> fb = face_flux_nb(g, p, 0, i, j, w, zc, fb_, tf, in[fb_], nb[fb_], dt, [&](T av[3]) {
          av[0] = sF[0][ln[fb_]]; av[1] = sF[3][ln[fb_]]; av[2] = sF[6][ln[fb_]];
        });
        bsum += fb.bout;
        dir_terms(dir == 0, fa, fb, gg, dir == 0 ? dx_ : dy_);
      }
      T o[3][3];
#pragma unroll
      for (int v = 0; v < 3; v++) {
        T wc[3] = {T(0), T(0), T(0)};
        if (STAGE == 2) {
          wc[0] = sW[3 * v][threadIdx.x];
          wc[1] = sW[3 * v + 1][threadIdx.x];
          wc[2] = sW[3 * v + 2][threadIdx.x];
        }
        finish_var_vals<T, STAGE>(g, v, 0, w, zc, dx_, dy_, dt, ws_own + 3 * v, wc, o[v][0], o[v][1], o[v][2]);
      }
      const T h0n = o[0][0];
#pragma unroll
      for (int v = 0; v < 3; v++) {
        post_var<T>(g, p, v, k, 0, h0n, o[v][0], o[v][1], o[v][2], ncl, csum, bad);
        store_var(P, v, k, Out, o[v][0], o[v][1], o[v][2]);
      }
      if (STAGE == 2) next_step_reduce<T>(g, p, 0, i, j, o[0][0], o[1][0], o[2][0], tf, m0, m1, m2, best);
    }
    __syncthreads();  // the shared arrays are refilled by the next tile
  }
  update_epilogue<T, STAGE, NT>(g, p, bsum, csum, ncl, bad, m0, m1, m2, best, gridDim.x);
}

// ---------------------------------------------------------------------------
// ACC: the local inertial solver (Sect. 2.1.3)
// ---------------------------------------------------------------------------
// Depth and bed piecewise constant; a discharge per interface from the
// momentum equation without convective acceleration with the Manning
// resistance taken semi-implicitly (the scheme of Bates et al. 2010, which
// the paper cites):
//   q' = (q - g h_f dt (eta_b - eta_a) / d) / (1 + g dt n_f^2 |q| / h_f^{7/3}),
// h_f = max(eta_a, eta_b) - max(z_a, z_b) (no flow where h_f <= h_dry), n_f the
// mean Manning n, d the distance between the cell centres.  Each leaf holds
// the discharges of its four faces (E, W, N, S; m^2/s towards +x / +y): a
// face between two leaves of one level is computed by both with the same
// operands; on graded static grids each finer leaf computes its half of a
// face with the coarser leaf, and the coarser leaf sums the halves
// (Sect. 2.2.1).  Old discharges are read from Wi, new ones written to Ui;
// the continuity pass copies them back.  Open faces carry the discharge of
// the leaf's opposite face, inflow faces the hydrograph.
template <typename T>
__device__ __forceinline__ T acc_face_q(T q0, T ha, T za, T hb, T zb, T d, T nf, T dt, T gg, T hd) {
  const T ea = ha + za, eb = hb + zb;
  const T hf = tmax(ea, eb) - tmax(za, zb);
  if (!(hf > hd)) return T(0);
  const T num = q0 - gg * hf * dt * (eb - ea) / d;
  const T den = T(1) + gg * dt * nf * nf * tabs(q0) / (hf * hf * tcbrt(hf));
  return num / den;
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_acc_q(Geo g, Ptrs<T> p) {
  if (!ctl_stepping(p.ctl)) return;
  const long long P = g.P;
  const T dt = ctl_dt<T>(p.ctl), gg = geo_g<T>(g), hd = geo_hd<T>(g);
  const ForceTime tf{p.ctl, false};
  FOR_LEAVES(p) {
    int l, i, j;
    const long long k = unpack_leaf(g, p.leaves[_q], l, i, j);
    long long code[4];
    load_nb_codes(p.nbr, _q, code);
    const T h = p.U[k], z = p.Z[k], nm = p.NM[k], dxl = geo_dx<T>(g, l);
#pragma unroll
    for (int f = 0; f < 4; f++) {
      const T q0 = p.Wi[f * P + k];
      T qn = T(0);
      const int type = nb_type(code[f]);
      if (type == NB_EDGE) {
        const int e = (f == 0) ? 1 : (f == 1) ? 0 : (f == 2) ? 3 : 2;
        const double qin = inflow_q(g, p.knot_t, p.knot_Q, e, l, (e < 2) ? j : i, tf());
        if (qin > 0.0) qn = (e == 0 || e == 2) ? (T)qin : -(T)qin;
        else if (g.bc[e] == MWDG_OPEN) qn = p.Wi[(f ^ 1) * P + k];
      } else if (type != NB_REFINED) {
        const long long kb = nb_node(code[f]);
        const int lb = l - nb_depth(code[f]);
        const T hb = p.U[kb], zb = p.Z[kb], nb = p.NM[kb];
        const T d = T(0.5) * (dxl + geo_dx<T>(g, lb));
        if (f == 0 || f == 2) qn = acc_face_q(q0, h, z, hb, zb, d, T(0.5) * (nm + nb), dt, gg, hd);
        else qn = acc_face_q(q0, hb, zb, h, z, d, T(0.5) * (nb + nm), dt, gg, hd);
      }
      p.Ui[f * P + k] = qn;
    }
  }
}

// continuity (rain as a source, clip of negative depth), read-out discharges,
// the next CFL candidate, and the end of the step in the last block
template <typename T>
__global__ void __launch_bounds__(TPB) k_acc_h(Geo g, Ptrs<T> p) {
  if (!ctl_stepping(p.ctl)) return;
  const long long P = g.P;
  const T dt = ctl_dt<T>(p.ctl), gg = geo_g<T>(g), hd = geo_hd<T>(g);
  const bool rain = p.ctl->rain_on;
  const T rinc = ctl_rain<T>(p.ctl);
  T bsum = T(0), best = tinf<T>();
  double csum = 0.0;
  unsigned long long ncl = 0;
  bool bad = false;
  FOR_LEAVES(p) {
    int l, i, j;
    const long long k = unpack_leaf(g, p.leaves[_q], l, i, j);
    long long code[4];
    load_nb_codes(p.nbr, _q, code);
    const T dxl = geo_dx<T>(g, l);
    T F[4], qs[4];
#pragma unroll
    for (int f = 0; f < 4; f++) {
      qs[f] = p.Ui[f * P + k];
      F[f] = qs[f] * dxl;
      const int type = nb_type(code[f]);
      if (type == NB_REFINED) {
        const int a = i + (f == 0) - (f == 1), b = j + (f == 2) - (f == 3);
        int c1, c2;
        if (f == 0) { c1 = 0; c2 = 2; }
        else if (f == 1) { c1 = 1; c2 = 3; }
        else if (f == 2) { c1 = 0; c2 = 1; }
        else { c1 = 2; c2 = 3; }
        const T q1 = p.Ui[(f ^ 1) * P + nid(g, l + 1, 2 * a + (c1 & 1), 2 * b + (c1 >> 1))];
        const T q2 = p.Ui[(f ^ 1) * P + nid(g, l + 1, 2 * a + (c2 & 1), 2 * b + (c2 >> 1))];
        const T dxf = geo_dx<T>(g, l + 1);
        F[f] = q1 * dxf + q2 * dxf;
        qs[f] = T(0.5) * (q1 + q2);
      }
      if (type == NB_EDGE) bsum += (f == 0 || f == 2) ? F[f] : -F[f];
    }
    T h = p.U[k];
    if (rain) h = h + rinc;
    h = h + dt * ((F[1] - F[0]) + (F[3] - F[2])) / (dxl * dxl);
    if (h < T(0)) {
      ncl++;
      csum += -(double)h * (g.dxl[l] * g.dxl[l]);
      h = T(0);
    }
    if (!isfinite(h)) bad = true;
    p.U[k] = h;
    p.U[3 * P + k] = T(0.5) * (qs[0] + qs[1]);
    p.U[6 * P + k] = T(0.5) * (qs[2] + qs[3]);
#pragma unroll
    for (int f = 0; f < 4; f++) p.Wi[f * P + k] = qs[f];
    if (h > hd) best = tmin(best, dxl / tsqrt(gg * h));
  }
  if (bad) p.ctl->nonfinite = 1;
  for (int o = 16; o > 0; o >>= 1) {
    bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
    best = tmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    ncl += __shfl_xor_sync(0xffffffffu, ncl, o);
  }
  if (__any_sync(0xffffffffu, ncl != 0ULL)) {
    for (int o = 16; o > 0; o >>= 1) csum += __shfl_xor_sync(0xffffffffu, csum, o);
    if ((threadIdx.x & 31) == 0 && ncl) {
      atomicAdd(&p.ctl->n_clip, ncl);
      atomicAdd(&p.ctl->v_clip, csum);
    }
  }
  __shared__ T red[2][TPB / 32];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = bsum;
    red[1][threadIdx.x >> 5] = best;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T b = red[0][0], m = red[1][0];
    for (int w = 1; w < TPB / 32; w++) {
      b += red[0][w];
      m = tmin(m, red[1][w]);
    }
    if (b != T(0)) atomicAdd(&p.ctl->bnd[0], (double)b);
    if (m < tinf<T>()) atomic_min_pos(&p.ctl->dtmin, (double)m);
    __threadfence();
  }
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) last = (atomicAdd(&p.ctl->blocks_done, 1u) == gridDim.x - 1);
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    end_step(g, p.ctl, true);
  }
}

// ---------------------------------------------------------------------------
// Read-back
// ---------------------------------------------------------------------------
// h, u, v of finest cell (I, J): the plane of the active leaf covering it
// evaluated at the cell centre (FP64); velocities q/h where h > h_dry, else 0
template <typename T>
__device__ __forceinline__ void finest_values(const Geo &g, const Ptrs<T> &p, int I, int J, double (&out)[3]) {
  const int L = g.L;
  int l = L, a = I, b = J;
  long long k = nid(g, l, a, b);
  while (l > 0 && p.kind[k] != K_LEAF) {
    a >>= 1; b >>= 1; l--;
    k = nid(g, l, a, b);
  }
  const int w = 1 << (L - l);
  const double s3 = 1.7320508075688772;
  double xi = ((double)(I - a * w) + 0.5) / (double)w - 0.5;
  double et = ((double)(J - b * w) + 0.5) / (double)w - 0.5;
  const long long P = g.P;
  double val[3];
  for (int q = 0; q < 3; q++) {
    double c0 = (double)p.U[3 * q * P + k], c1 = (double)p.U[(3 * q + 1) * P + k],
           c2 = (double)p.U[(3 * q + 2) * P + k];
    if (Form<T>::eta && q == 0) {
      c1 -= (double)p.Z[P + k]; c2 -= (double)p.Z[2 * P + k];
    }
    val[q] = c0 + 2.0 * s3 * xi * c1 + 2.0 * s3 * et * c2;
  }
  out[0] = val[0];
  out[1] = out[2] = 0.0;
  if (val[0] > g.hd) {
    out[1] = val[1] / val[0];
    out[2] = val[2] / val[0];
  }
}

template <typename T>
__global__ void k_fields(Geo g, Ptrs<T> p, double *h, double *u, double *v) {
  const int L = g.L;
  long long n = (long long)g.nxl[L] * g.nyl[L];
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= n) return;
  int J = (int)(r / g.nxl[L]), I = (int)(r - (long long)J * g.nxl[L]);
  double o[3];
  finest_values(g, p, I, J, o);
  if (h) h[r] = o[0];
  if (u) u[r] = o[1];
  if (v) v[r] = o[2];
}

// the same at n gauge cells (ij: i, j pairs) into out (h, u, v blocks of n)
template <typename T>
__global__ void k_gauges(Geo g, Ptrs<T> p, const int32_t *ij, int n, double *out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  double o[3];
  finest_values(g, p, ij[2 * q], ij[2 * q + 1], o);
  out[q] = o[0];
  out[n + q] = o[1];
  out[2 * n + q] = o[2];
}

template <typename T>
__global__ void k_read_active(Geo g, Ptrs<T> p, int32_t *lev, int32_t *ii, int32_t *jj, double *coef) {
  const int n = *p.nleaf;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int l, i, j;
  long long k = unpack_leaf(g, p.leaves[q], l, i, j);
  if (lev) lev[q] = l;
  if (ii) ii[q] = i;
  if (jj) jj[q] = j;
  if (coef) {
    const long long P = g.P;
    for (int m = 0; m < 9; m++) {
      double c = (double)p.U[m * P + k];
      if (Form<T>::eta && (m == 1 || m == 2)) c -= (double)p.Z[m * P + k];
      coef[9 * (long long)q + m] = c;
    }
  }
}

// volume: per-block partial sums in a fixed order, then one block sums the
// partials in a fixed order (deterministic FP64)
template <typename T>
__global__ void k_volume_part(Geo g, Ptrs<T> p) {
  const int n = *p.nleaf;
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    int l, i, j;
    long long k = unpack_leaf(g, p.leaves[q], l, i, j);
    double h0 = (double)p.U[k];
    acc += h0 * (g.dxl[l] * g.dxl[l]);
  }
  __shared__ double sh[TPB];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) p.part[blockIdx.x] = sh[0];
}

static __global__ void k_volume_final(const double *part, int nb, Ctl *c) {
  __shared__ double sh[TPB];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += TPB) acc += part[b];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) c->volume = sh[0];
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
inline unsigned nblk(long long n) { return (unsigned)((n + TPB - 1) / TPB); }
inline long long lvl(const Geo &g, int l) { return (long long)g.nxl[l] * g.nyl[l]; }

#define MARK(c) \
  do {          \
    if (mark) mark(mark_arg, (c)); \
  } while (0)

template <typename T>
int Launch<T>::project(const Geo &g, const Ptrs<T> &, const double *vert, T *c0, T *c1x, T *c1y,
                       cudaStream_t st) {
  const int L = g.L;
  k_project<T><<<nblk(lvl(g, L)), TPB, 0, st>>>(vert, g.nxl[L], g.nyl[L], c0, c1x, c1y);
  return 1;
}

template <typename T>
int Launch<T>::load_dem_pyramid(const Geo &g, const Ptrs<T> &p, cudaStream_t st) {
  int n = 0;
  k_zmax<T><<<152 * 4, TPB, 0, st>>>(g, p);
  n++;
  for (int l = g.L - 1; l >= 0; l--, n++) k_encode_z<T><<<nblk(lvl(g, l)), TPB, 0, st>>>(g, p, l);
  if (g.scheme != MWDG_DG2) {
    k_fv1_bed<T><<<nblk(g.P), TPB, 0, st>>>(g, p);
    n++;
  }
  return n;
}

template <typename T>
int Launch<T>::roughness_pyramid(const Geo &g, const Ptrs<T> &p, cudaStream_t st) {
  int n = 0;
  for (int l = g.L - 1; l >= 0; l--, n++) k_nm_level<T><<<nblk(lvl(g, l)), TPB, 0, st>>>(g, p, l);
  return n;
}

template <typename T>
int Launch<T>::initial_finest(const Geo &g, const Ptrs<T> &p, int is_eta, cudaStream_t st) {
  k_initial_finest<T><<<nblk(lvl(g, g.L)), TPB, 0, st>>>(g, p, is_eta);
  return 1;
}

template <typename T>
int Launch<T>::encode_dense_U(const Geo &g, const Ptrs<T> &p, cudaStream_t st) {
  int n = 0;
  for (int l = g.L - 1; l >= 0; l--, n++) k_encode_dense<T><<<nblk(lvl(g, l)), TPB, 0, st>>>(g, p.U, 9, l, p.Z);
  return n;
}

template <typename T>
int Launch<T>::eta_rule_leaves(const Geo &g, const Ptrs<T> &p, cudaStream_t st) {
  int n = 0;
  for (int l = g.L - 1; l >= 0; l--, n++) k_encode_dense<T><<<nblk(lvl(g, l)), TPB, 0, st>>>(g, p.Wn, 3, l, (const T *)nullptr);
  k_eta_rule_leaves<T><<<nblk(g.P), TPB, 0, st>>>(g, p);
  return n + 1;
}

template <typename T>
int Launch<T>::static_flags(const Geo &g, const Ptrs<T> &p, cudaStream_t st) {
  k_static_flags<T><<<nblk(g.P), TPB, 0, st>>>(g, p);
  return 1;
}

template <typename T>
int Launch<T>::closure(const Geo &g, uint8_t *flag, cudaStream_t st) {
  int n = 0;
  for (int l = g.L - 1; l >= 1; l--, n++) k_closure<<<nblk(lvl(g, l)), TPB, 0, st>>>(g, flag, l);
  return n;
}

template <typename T>
int Launch<T>::grading_sweep(const Geo &g, const Ptrs<T> &p, cudaStream_t st) {
  int n = 0;
  for (int l = g.L - 1; l >= 1; l--, n++) k_grading<T><<<nblk(lvl(g, l)), TPB, 0, st>>>(g, p, l);
  return n + closure(g, p.flag, st);
}

template <typename T>
int Launch<T>::kinds(const Geo &g, const Ptrs<T> &p, const uint8_t *flag, cudaStream_t st) {
  k_kinds<T><<<nblk(g.P), TPB, 0, st>>>(g, p, flag);
  return 1;
}

template <typename T>
int Launch<T>::all_finest(const Geo &g, const Ptrs<T> &p, cudaStream_t st) {
  k_all_finest<T><<<nblk(g.P), TPB, 0, st>>>(g, p);
  return 1;
}

template <typename T>
int Launch<T>::compact(const Geo &g, const Ptrs<T> &p, cudaStream_t st) {
  const int nb = (int)((g.P + CTILE - 1) / CTILE);
  k_compact_count<<<nb, TPB, 0, st>>>(g.P, p.kind, p.blk);
  k_compact_scan<<<1, 1024, 0, st>>>(nb, p.blk, p.nleaf);
  k_compact_scatter<<<nb, TPB, 0, st>>>(g, p.kind, p.blk, p.leaves, nullptr, nullptr, nullptr, 0);
  k_leaf_codes<<<(int)std::min<long long>(nblk(g.P), 152 * 8), TPB, 0, st>>>(g, p.kind, p.leaves, p.nleaf, p.nbr);
  return 4;
}

// levels 0..coarse_top run in one block (each has at most g.coarse_nodes
// nodes; -1: none)
inline int coarse_top(const Geo &g) {
  int lc = -1;
  while (lc + 1 < g.L && lvl(g, lc + 1) <= g.coarse_nodes) lc++;
  return lc;
}

// chunks of the tiled MRA passes, finest first: f(ltop, nlev, tail, blocks)
template <class F>
int for_chunks(const Geo &g, F &&f) {
  if (g.L < 1) return 0;
  const int lc = coarse_top(g);
  int l = g.L - 1, n = 0;
  if (l <= lc) {
    f(l, 0, lc, 1);
    return 1;
  }
  while (l > lc) {
    const int nlev = std::min(MT_LEVELS, l - lc);
    const int tail = (l - nlev == lc) ? lc : -1;
    const int blocks = ((g.nxl[l] + MT - 1) / MT) * ((g.nyl[l] + MT - 1) / MT);
    f(l, nlev, tail, blocks);
    l -= nlev;
    n++;
  }
  return n;
}

template <typename T>
int Launch<T>::adapt(const Geo &g, const Ptrs<T> &p, int encode_only, int with_maxabs, cudaStream_t st,
                     void (*mark)(void *, int), void *mark_arg, int begin, const Fork *fk) {
  int n = 0;
  const int grid = (int)std::min<long long>(nblk(g.P), 152 * 8);
  if (with_maxabs) {
    MARK(KC_ENCODE);
    k_leaf_maxabs<T><<<grid, TPB, 0, st>>>(g, p);
    n++;
  }
  // the coarsest levels of the regularisation move to the decode's first
  // block when every node that reads them (levels up to lc + 1) is its own
  const int lc = coarse_top(g);
  const bool defer = !encode_only && lc >= 0 && lc < g.L - 1 && g.off[lc + 2] <= CTILE;
  // with the regularisation's coarsest levels deferred, the encode's
  // coarsest levels (the last chunk's tail) run as one block on the fork,
  // beside the regularisation's tiles, which read only finer levels; the
  // decode, whose first block reads both, waits for the join
  const bool forked = fk && defer;
  // bottom-up encode + significance
  n += for_chunks(g, [&](int ltop, int nlev, int tail, int blocks) {
    MARK(KC_ENCODE);
    const int t = (forked && nlev > 0) ? -1 : tail;
    if (g.scheme == MWDG_FV1) k_mra_sig<T, true><<<blocks, TPB, 0, st>>>(g, p, ltop, nlev, t);
    else k_mra_sig<T, false><<<blocks, TPB, 0, st>>>(g, p, ltop, nlev, t);
    if (t != tail) {
      cudaEventRecord(fk->fork, st);
      cudaStreamWaitEvent(fk->aux, fk->fork, 0);
      if (g.scheme == MWDG_FV1) k_mra_sig<T, true><<<1, TPB, 0, fk->aux>>>(g, p, ltop, 0, tail);
      else k_mra_sig<T, false><<<1, TPB, 0, fk->aux>>>(g, p, ltop, 0, tail);
      cudaEventRecord(fk->join, fk->aux);
      n++;
    }
  });
  if (encode_only) return n;
  // prediction + closure
  n += for_chunks(g, [&](int ltop, int nlev, int tail, int blocks) {
    MARK(KC_FLAGS);
    if (defer) tail = -1;
    k_mra_regularise<T><<<blocks, TPB, 0, st>>>(g, p, ltop, nlev, tail);
  });
  if (forked) cudaStreamWaitEvent(st, fk->join, 0);
  // new kinds, decode, counts and offsets; then the scatter, which also
  // makes the new kinds current
  MARK(KC_DECODE);
  const int nb = (int)((g.P + CTILE - 1) / CTILE);
  k_mra_decode<T><<<nb, TPB, 0, st>>>(g, p, defer ? lc : -1);
  MARK(KC_COMPACT);
  k_compact_scatter<<<nb, TPB, 0, st>>>(g, p.kind_new, p.blk, p.leaves, p.kind, p.ctl, p.nleaf, begin);
  // (the neighbour codes of the new leaves: the stage-1 limiter of the step,
  // or a pass of their own when the adaptation is not followed by a step)
  if (!begin) {
    MARK(KC_COMPACT);
    k_leaf_codes<<<(int)std::min<long long>(nblk(g.P), 152 * 8), TPB, 0, st>>>(g, p.kind_new, p.leaves,
                                                                               p.nleaf, p.nbr);
    n++;
  }
  return n + 2;
}

template <typename T>
int Launch<T>::prime(const Geo &g, const Ptrs<T> &p, int grid_leaves, cudaStream_t st) {
  k_leaf_maxabs<T><<<grid_leaves, TPB, 0, st>>>(g, p);
  k_leaf_dt<T><<<grid_leaves, TPB, 0, st>>>(g, p);
  return 2;
}

template <typename T>
int Launch<T>::dt_only(const Geo &g, const Ptrs<T> &p, int grid_leaves, cudaStream_t st) {
  k_leaf_dt<T><<<grid_leaves, TPB, 0, st>>>(g, p);
  return 1;
}

template <typename T>
int Launch<T>::step(const Geo &g, const Ptrs<T> &p, int grid_leaves, cudaStream_t st,
                    void (*mark)(void *, int), void *mark_arg, int begun) {
  int n = 0;
  const bool view = (g.mode == MWDG_ADAPTIVE);
  if (!begun) {
    MARK(KC_CONTROL);
    k_begin_step<<<1, 1, 0, st>>>(g, p.ctl, p.nleaf);
    n++;
  }
  if (g.scheme == MWDG_ACC) {  // local inertial: discharges, then continuity
    MARK(KC_UPDATE1);
    k_acc_q<T><<<grid_leaves, TPB, 0, st>>>(g, p);
    MARK(KC_UPDATE2);
    k_acc_h<T><<<grid_leaves, TPB, 0, st>>>(g, p);
    MARK(-1);
    return n + 2;
  }
  const int stages = (g.scheme == MWDG_FV1) ? 1 : 2;  // FV1: forward Euler (Eq. 7)
  // the coarsest levels of the flux views move to the update's first block
  // when the coarse leaves fit its first pass (at most lvl(lc) of them)
  const int lc = coarse_top(g);
  const int vtail = (view && lc >= 0 && lc < g.L - 1 && lvl(g, lc) <= TPB) ? lc : -1;
  // uniform grids: leaf and neighbours from the thread index (no list or
  // code reads)
  const bool uni = (g.mode == MWDG_UNIFORM);
  if (uni && stages == 2) {
    // DG2 on a uniform grid: one fused kernel per stage
    const long long tiles = (long long)((g.nxl[0] + UniTile<T>::X - 1) / UniTile<T>::X) *
                            ((g.nyl[0] + UniTile<T>::Y - 1) / UniTile<T>::Y);
    // one resident wave of blocks, each striding over the tiles
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<long long>(tiles, (long long)std::max(sms, 1) * UniTile<T>::OCC);
    const int nt = UniTile<T>::X * UniTile<T>::Y;
    MARK(KC_UPDATE1);
    k_uni_stage<T, 1><<<grid, nt, 0, st>>>(g, p, p.U, p.Wn, nullptr, p.Ui);
    MARK(KC_UPDATE2);
    k_uni_stage<T, 2><<<grid, nt, 0, st>>>(g, p, p.Ui, nullptr, p.Wn, p.U);
    MARK(-1);
    return n + 2;
  }
  for (int stage = 1; stage <= stages; stage++) {
    MARK(KC_LIMIT);
    const bool codes = (stage == 1 && begun);  // the step follows an adaptation
    if (stages == 1) {
      if (codes) k_leaf_limit<T, true, true, true, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.U, p.Wn);
      else if (uni) k_leaf_limit<T, true, true, false, true><<<grid_leaves, TPB, 0, st>>>(g, p, p.U, p.Wn);
      else k_leaf_limit<T, true, true, false, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.U, p.Wn);
    } else if (stage == 1) {
      if (codes) k_leaf_limit<T, true, false, true, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.U, p.Wn);
      else if (uni) k_leaf_limit<T, true, false, false, true><<<grid_leaves, TPB, 0, st>>>(g, p, p.U, p.Wn);
      else k_leaf_limit<T, true, false, false, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.U, p.Wn);
    } else {
      if (uni) k_leaf_limit<T, false, false, false, true><<<grid_leaves, TPB, 0, st>>>(g, p, p.Ui, p.Wi);
      else k_leaf_limit<T, false, false, false, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.Ui, p.Wi);
    }
    n++;
    if (view)
      n += for_chunks(g, [&](int ltop, int nlev, int tail, int blocks) {
        MARK(KC_VIEW);
        if (vtail >= 0) tail = -1;
        if (g.scheme == MWDG_FV1) k_view_tiles<T, true><<<blocks, TPB, 0, st>>>(g, p, ltop, nlev, tail);
        else k_view_tiles<T, false><<<blocks, TPB, 0, st>>>(g, p, ltop, nlev, tail);
      });
    const bool reflux = (g.mode == MWDG_STATIC && g.iface == MWDG_IFACE_REFLUX);
    if (stages == 1) {
      MARK(KC_UPDATE2);
      if (reflux) k_leaf_update<T, 3, true, false, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wn, nullptr, p.U, -1);
      else if (view) k_leaf_update<T, 3, false, true, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wn, nullptr, p.U, vtail);
      else if (uni) k_leaf_update<T, 3, false, false, true><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wn, nullptr, p.U, -1);
      else k_leaf_update<T, 3, false, false, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wn, nullptr, p.U, -1);
    } else if (stage == 1) {
      MARK(KC_UPDATE1);
      if (reflux) k_leaf_update<T, 1, true, false, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wn, nullptr, p.Ui, -1);
      else if (view) k_leaf_update<T, 1, false, true, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wn, nullptr, p.Ui, vtail);
      else if (uni) k_leaf_update<T, 1, false, false, true><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wn, nullptr, p.Ui, -1);
      else k_leaf_update<T, 1, false, false, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wn, nullptr, p.Ui, -1);
    } else {
      MARK(KC_UPDATE2);
      if (reflux) k_leaf_update<T, 2, true, false, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wi, p.Wn, p.U, -1);
      else if (view) k_leaf_update<T, 2, false, true, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wi, p.Wn, p.U, vtail);
      else if (uni) k_leaf_update<T, 2, false, false, true><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wi, p.Wn, p.U, -1);
      else k_leaf_update<T, 2, false, false, false><<<grid_leaves, TPB, 0, st>>>(g, p, p.Wi, p.Wn, p.U, -1);
    }
    n++;
  }
  MARK(-1);
  return n;
}

template <typename T>
int Launch<T>::fields(const Geo &g, const Ptrs<T> &p, double *h, double *u, double *v, cudaStream_t st) {
  k_fields<T><<<nblk(lvl(g, g.L)), TPB, 0, st>>>(g, p, h, u, v);
  return 1;
}

template <typename T>
int Launch<T>::gauges(const Geo &g, const Ptrs<T> &p, const int32_t *ij, int n, double *out, cudaStream_t st) {
  if (n <= 0) return 0;
  k_gauges<T><<<(n + TPB - 1) / TPB, TPB, 0, st>>>(g, p, ij, n, out);
  return 1;
}

template <typename T>
int Launch<T>::read_active(const Geo &g, const Ptrs<T> &p, int32_t *lev, int32_t *i, int32_t *j,
                           double *coef, cudaStream_t st) {
  k_read_active<T><<<nblk(g.P), TPB, 0, st>>>(g, p, lev, i, j, coef);
  return 1;
}

template <typename T>
int Launch<T>::volume(const Geo &g, const Ptrs<T> &p, int grid_leaves, cudaStream_t st) {
  k_volume_part<T><<<grid_leaves, TPB, 0, st>>>(g, p);
  k_volume_final<<<1, TPB, 0, st>>>(p.part, grid_leaves, p.ctl);
  return 2;
}

// ---------------------------------------------------------------------------
// Batched ensemble steps: the kernels of an adaptive DG2 step, each launched
// once over the blocks of all members (a work list of (member, block)).
// ---------------------------------------------------------------------------
// the member of this block (its record copied to shared memory) and the
// block's index within the member's range
template <typename T>
__device__ __forceinline__ unsigned batch_member(const BMember<T> *tab, const BStarts &bs, BMember<T> &m) {
  __shared__ int mi;
  if (threadIdx.x == 0) {
    int lo = 0, hi = bs.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (bs.s[mid] <= blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    mi = lo;
  }
  __syncthreads();
  constexpr int W = (int)(sizeof(BMember<T>) / sizeof(unsigned));
  const unsigned *src = reinterpret_cast<const unsigned *>(tab + mi);
  unsigned *dst = reinterpret_cast<unsigned *>(&m);
  for (int w = threadIdx.x; w < W; w += blockDim.x) dst[w] = src[w];
  __syncthreads();
  return blockIdx.x - m.bstart;
}

template <typename T>
__global__ void __launch_bounds__(TPB, MraOcc<T>::blocks) kb_sig(const BMember<T> *tab, const BStarts bs) {
  __shared__ BMember<T> m;
  const unsigned b = batch_member(tab, bs, m);
  mra_sig<T, false>(m.g, m.p, m.a[0], m.a[1], m.a[2], b, m.nblk);
}

template <typename T>
__global__ void __launch_bounds__(TPB) kb_reg(const BMember<T> *tab, const BStarts bs) {
  __shared__ BMember<T> m;
  const unsigned b = batch_member(tab, bs, m);
  mra_regularise<T>(m.g, m.p, m.a[0], m.a[1], m.a[2], b, m.nblk);
}

template <typename T>
__global__ void __launch_bounds__(TPB, MraOcc<T>::blocks) kb_decode(const BMember<T> *tab, const BStarts bs) {
  __shared__ BMember<T> m;
  const unsigned b = batch_member(tab, bs, m);
  mra_decode<T>(m.g, m.p, m.a[0], b);
}

template <typename T>
__global__ void __launch_bounds__(TPB) kb_scatter(const BMember<T> *tab, const BStarts bs) {
  __shared__ BMember<T> m;
  const unsigned b = batch_member(tab, bs, m);
  compact_scatter(m.g, m.p.kind_new, m.p.blk, m.p.leaves, m.p.kind, m.p.ctl, m.p.nleaf, 1, b, m.nblk);
}

template <typename T, int STAGE>
__global__ void __launch_bounds__(TPB, LimOcc<T>::blocks) kb_limit(const BMember<T> *tab, const BStarts bs) {
  __shared__ BMember<T> m;
  const unsigned b = batch_member(tab, bs, m);
  if (STAGE == 1) leaf_limit<T, true, false, true, false>(m.g, m.p, m.p.U, m.p.Wn, b, m.nblk);
  else leaf_limit<T, false, false, false, false>(m.g, m.p, m.p.Ui, m.p.Wi, b, m.nblk);
}

template <typename T>
__global__ void __launch_bounds__(TPB, ViewOcc<T>::blocks) kb_view(const BMember<T> *tab, const BStarts bs) {
  __shared__ BMember<T> m;
  const unsigned b = batch_member(tab, bs, m);
  view_tiles<T, false>(m.g, m.p, m.a[0], m.a[1], m.a[2], b, m.nblk);
}

template <typename T, int STAGE>
__global__ void __launch_bounds__(TPB, UpdOcc<T>::blocks) kb_update(const BMember<T> *tab, const BStarts bs) {
  __shared__ BMember<T> m;
  const unsigned b = batch_member(tab, bs, m);
  if (STAGE == 1) leaf_update<T, 1, false, true, false>(m.g, m.p, m.p.Wn, nullptr, m.p.Ui, m.a[3], b, m.nblk);
  else leaf_update<T, 2, false, true, false>(m.g, m.p, m.p.Wi, m.p.Wn, m.p.U, m.a[3], b, m.nblk);
}

// The launches of Launch<T>::adapt (begin = 1) and Launch<T>::step
// (begun = 1) for every member, in their order and with their arguments:
// encode and regularisation per chunk, decode, scatter (which starts the
// step), then per stage the limiter, the flux views per chunk and the
// update.  A member takes part in the j-th chunk launch of a pass when it
// has that many chunks.
template <typename T>
bool Launch<T>::batch_plan(int n, const Geo *const *g, const Ptrs<T> *const *p, const int *grid_leaves,
                           std::vector<BatchLaunch> &plan) {
  struct Ch { int ltop, nlev, tail, blocks; };
  std::vector<std::vector<Ch>> sig(n), reg(n), view(n);
  std::vector<int> ftail(n), vtail(n), nb(n);
  size_t ns = 0, nr = 0, nv = 0;
  for (int m = 0; m < n; m++) {
    const Geo &G = *g[m];
    const int lc = coarse_top(G);
    const bool defer = lc >= 0 && lc < G.L - 1 && G.off[lc + 2] <= CTILE;
    for_chunks(G, [&](int ltop, int nlev, int tail, int blocks) { sig[m].push_back({ltop, nlev, tail, blocks}); });
    for_chunks(G, [&](int ltop, int nlev, int tail, int blocks) {
      reg[m].push_back({ltop, nlev, defer ? -1 : tail, blocks});
    });
    ftail[m] = defer ? lc : -1;
    nb[m] = (int)((G.P + CTILE - 1) / CTILE);
    vtail[m] = (lc >= 0 && lc < G.L - 1 && lvl(G, lc) <= TPB) ? lc : -1;
    for_chunks(G, [&](int ltop, int nlev, int tail, int blocks) {
      view[m].push_back({ltop, nlev, vtail[m] >= 0 ? -1 : tail, blocks});
    });
    ns = std::max(ns, sig[m].size());
    nr = std::max(nr, reg[m].size());
    nv = std::max(nv, view[m].size());
  }
  bool ok = true;
  // one launch: the members for which rec(m, r) fills a record
  auto add = [&](int kind, auto &&rec) {
    if (!ok) return;
    std::vector<BMember<T>> recs;
    BatchLaunch bl{};
    bl.kind = kind;
    unsigned b = 0;
    for (int m = 0; m < n; m++) {
      BMember<T> r{};
      r.g = *g[m];
      r.p = *p[m];
      r.a[0] = r.a[1] = r.a[2] = r.a[3] = -1;
      if (!rec(m, r) || r.nblk == 0) continue;
      r.bstart = b;
      bl.bs.s[recs.size()] = b;
      b += r.nblk;
      recs.push_back(r);
    }
    if (recs.empty()) return;
    bl.bs.n = (int)recs.size();
    bl.bs.s[bl.bs.n] = b;
    if (cudaMalloc(&bl.tab, recs.size() * sizeof(BMember<T>)) != cudaSuccess) {
      ok = false;
      return;
    }
    plan.push_back(bl);
    ok = cudaMemcpy(bl.tab, recs.data(), recs.size() * sizeof(BMember<T>), cudaMemcpyHostToDevice) == cudaSuccess;
  };
  auto chunk = [&](const std::vector<std::vector<Ch>> &c, size_t j) {
    return [&c, j](int m, BMember<T> &r) {
      if (j >= c[m].size()) return false;
      r.a[0] = c[m][j].ltop;
      r.a[1] = c[m][j].nlev;
      r.a[2] = c[m][j].tail;
      r.nblk = (unsigned)c[m][j].blocks;
      return true;
    };
  };
  auto leaves = [&](int m, BMember<T> &r) {
    r.a[3] = vtail[m];
    r.nblk = (unsigned)grid_leaves[m];
    return true;
  };
  for (size_t j = 0; j < ns; j++) add(BK_SIG, chunk(sig, j));
  for (size_t j = 0; j < nr; j++) add(BK_REG, chunk(reg, j));
  add(BK_DECODE, [&](int m, BMember<T> &r) {
    r.a[0] = ftail[m];
    r.nblk = (unsigned)nb[m];
    return true;
  });
  add(BK_SCATTER, [&](int m, BMember<T> &r) {
    r.nblk = (unsigned)nb[m];
    return true;
  });
  add(BK_LIMIT1, leaves);
  for (size_t j = 0; j < nv; j++) add(BK_VIEW, chunk(view, j));
  add(BK_UPD1, leaves);
  add(BK_LIMIT2, leaves);
  for (size_t j = 0; j < nv; j++) add(BK_VIEW, chunk(view, j));
  add(BK_UPD2, leaves);
  return ok;
}

template <typename T>
int Launch<T>::batch_step(const std::vector<BatchLaunch> &plan, cudaStream_t st) {
  for (const BatchLaunch &b : plan) {
    const BMember<T> *tab = static_cast<const BMember<T> *>(b.tab);
    const unsigned nbk = b.bs.s[b.bs.n];
    switch (b.kind) {
      case BK_SIG: kb_sig<T><<<nbk, TPB, 0, st>>>(tab, b.bs); break;
      case BK_REG: kb_reg<T><<<nbk, TPB, 0, st>>>(tab, b.bs); break;
      case BK_DECODE: kb_decode<T><<<nbk, TPB, 0, st>>>(tab, b.bs); break;
      case BK_SCATTER: kb_scatter<T><<<nbk, TPB, 0, st>>>(tab, b.bs); break;
      case BK_LIMIT1: kb_limit<T, 1><<<nbk, TPB, 0, st>>>(tab, b.bs); break;
      case BK_VIEW: kb_view<T><<<nbk, TPB, 0, st>>>(tab, b.bs); break;
      case BK_UPD1: kb_update<T, 1><<<nbk, TPB, 0, st>>>(tab, b.bs); break;
      case BK_LIMIT2: kb_limit<T, 2><<<nbk, TPB, 0, st>>>(tab, b.bs); break;
      default: kb_update<T, 2><<<nbk, TPB, 0, st>>>(tab, b.bs); break;
    }
  }
  return (int)plan.size();
}

#undef MARK

}  // namespace mwdg
