// Discrete adjoint of the uniform-grid DG2 step (include/mwdg_adjoint.h).
//
// The forward sweep is the DG2 step of Sect. 2.1.1 (Eq. 1-4) on a dense
// uniform grid, FP64, compiled without FMA contraction and written in the
// operation order of the step in mwdg_kernels.cuh, so that it rounds the
// same way.  The reverse sweep differentiates that step by hand, kernel by
// kernel, with every branch replayed from the recomputed forward values:
//
//   forward per step   friction -> limit(Un) -> update stage 1 -> limit(Ui)
//                      -> update stage 2 (+ the CFL dt when not given)
//   reverse per step   recompute friction, limit, stage 1, limit; then for
//                      stage 2 and stage 1 in turn:
//                        rev_cell   post-stage clip/dry masks, RK2 weights,
//                                   operator terms local to a cell (flux
//                                   weights, physical fluxes of the own
//                                   revised limits, bed-slope sources)
//                        rev_face   per interface: HLL and the two
//                                   revisions, the interface bed max,
//                                   boundary ghosts (and the hydrograph)
//                        rev_limit  face-limit transpose and the limiter
//                                   (partial-wet reduction, minmod picks)
//                        rev_gather neighbour terms of the limiter
//                      then friction.
//
// Every cotangent is gathered by the thread that owns it (a cell or a
// face) from buffers written by the kernel before: no atomics, so a run is
// deterministic.  The tape holds the state at the start of each step and
// the clip flags of each stage; nothing else is stored.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include <cuda_runtime.h>

#include "dg2_math.cuh"
#include "mwdg_adjoint.h"

namespace mwdg {
namespace adj {

constexpr int TPB = 256;
constexpr double TIE_REL = 1e-10;

// parameters passed to the kernels by value
struct Par {
  int nx, ny;
  long long n;
  double dx, g, hd, cfl, dt_max;
  int limiter;
  int bc[4];
  int inflow_edge, c0, c1, nknots;
  double rain_rate, rain_t_end;
  const double *kt, *kQ;
};

__device__ __forceinline__ double S3() { return s3v<double>(); }

// ---------------------------------------------------------------------------
// hydrograph
// ---------------------------------------------------------------------------
// Q(t), piecewise linear over the knots and constant outside them; k0, k1
// and r give its weights: Q = (1 - r) Q[k0] + r Q[k1] in the derivative.
__device__ double hydro(const Par &P, double t, int &k0, int &k1, double &r) {
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

// unit discharge through the boundary face of cell `along` on edge e
__device__ double inflow_unit(const Par &P, int e, int along, double t) {
  if (P.inflow_edge != e || P.nknots < 1 || along < P.c0 || along > P.c1) return 0.0;
  int k0, k1;
  double r;
  const double Q = hydro(P, t, k0, k1, r);
  return Q * 1.0 / ((double)(P.c1 - P.c0 + 1) * P.dx);
}

// ---------------------------------------------------------------------------
// per-cell pieces shared by the sweeps
// ---------------------------------------------------------------------------
struct Lim {
  double h, qx, qy, z;
};

__device__ __forceinline__ Lim cell_lim(const double *W, const double *Z, long long n, long long k, int f) {
  Lim L;
  L.h = face_value(W[k], W[n + k], W[2 * n + k], f);
  L.qx = face_value(W[3 * n + k], W[4 * n + k], W[5 * n + k], f);
  L.qy = face_value(W[6 * n + k], W[7 * n + k], W[8 * n + k], f);
  L.z = face_value(Z[k], Z[n + k], Z[2 * n + k], f);
  return L;
}

// edge of the domain that face f of a boundary cell lies on, and the index
// along that edge
__device__ __forceinline__ int edge_of(int f) { return f == 0 ? 1 : f == 1 ? 0 : f == 2 ? 3 : 2; }

// ghost limit across a boundary face: inflow at the critical depth carrying
// the hydrograph, open (copy) or wall (mirror the normal discharge)
__device__ Lim ghost(const Par &P, int e, int along, const Lim &o, double t) {
  Lim gl;
  gl.z = o.z;
  const double q = inflow_unit(P, e, along, t);
  if (q > 0.0) {
    const double hc = newton_cbrt(q * q / P.g);
    gl.h = fmax(o.h, hc);
    const double qn = (e == 0 || e == 2) ? q : -q;
    if (e < 2) { gl.qx = qn; gl.qy = 0.0; }
    else { gl.qx = 0.0; gl.qy = qn; }
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

// the limits on the other side of face f of cell (i, j): the neighbour's
// flux view, or the ghost on the boundary
__device__ Lim other_side(const Par &P, const double *W, const double *Z, int i, int j, int f, const Lim &own,
                          double t, bool &inside) {
  const int di = f == 0 ? 1 : f == 1 ? -1 : 0, dj = f == 2 ? 1 : f == 3 ? -1 : 0;
  const int a = i + di, b = j + dj;
  inside = a >= 0 && b >= 0 && a < P.nx && b < P.ny;
  if (inside) return cell_lim(W, Z, P.n, (long long)b * P.nx + a, f ^ 1);
  const int e = edge_of(f);
  return ghost(P, e, e < 2 ? j : i, own, t);
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
__device__ void limit_cell(const Par &P, const double *X, const double *Z, int i, int j, double w_st[9],
                           double w_fx[9], double ze[3], LimRec &r) {
  const long long n = P.n, k = (long long)j * P.nx + i;
  const double hd = P.hd, s3 = S3();
#pragma unroll
  for (int m = 0; m < 9; m++) w_st[m] = X[m * n + k];
#pragma unroll
  for (int m = 0; m < 3; m++) ze[m] = Z[m * n + k];
  r.red = false;
#pragma unroll
  for (int d = 0; d < 2; d++)
#pragma unroll
    for (int v = 0; v < 3; v++) r.sel[d][v] = 0;
  const double h0 = w_st[0];
  const double eta0 = h0 + ze[0];
  bool red = !(h0 > hd);
#pragma unroll
  for (int f = 0; f < 4; f++) {
    if (!(face_value(w_st[0], w_st[1], w_st[2], f) > hd)) red = true;
    if (!(eta0 - face_value(ze[0], ze[1], ze[2], f) > hd)) red = true;
  }
  if (red) {
    r.red = true;
    w_st[1] = -ze[1]; w_st[2] = -ze[2];
    w_st[4] = 0.0; w_st[5] = 0.0;
    w_st[7] = 0.0; w_st[8] = 0.0;
#pragma unroll
    for (int m = 0; m < 9; m++) w_fx[m] = w_st[m];
    w_fx[1] = 0.0; w_fx[2] = 0.0;
    ze[1] = 0.0; ze[2] = 0.0;
    return;
  }
  if (P.limiter) {
    for (int d = 0; d < 2; d++) {
      const int ia = i + (d == 0), ja = j + (d == 1), ib = i - (d == 0), jb = j - (d == 1);
      const bool hasA = ia < P.nx && ja < P.ny, hasB = ib >= 0 && jb >= 0;
      if (!hasA && !hasB) continue;
      const long long ka = hasA ? (long long)ja * P.nx + ia : k, kb = hasB ? (long long)jb * P.nx + ib : k;
      const double hC = X[k], hA = X[ka], hB = X[kb];
      const bool wet = (hC > hd) && (!hasA || hA > hd) && (!hasB || hB > hd);
      const int cs = 1 + d;
      for (int v = 0; v < 3; v++) {
        if (v == 0 && !wet) continue;
        const double zs = Z[cs * n + k];
        double aC, a0, aB, slope;
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
        const double a = s3 * slope;
        const double d1 = a0 - aC, d2 = aC - aB;
        double mm;
        bool same;
        if (hasA && hasB) {
          same = (a > 0.0 && d1 > 0.0 && d2 > 0.0) || (a < 0.0 && d1 < 0.0 && d2 < 0.0);
          mm = minmod3(a, d1, d2);
        } else {
          const double o = hasA ? d1 : d2;
          same = (a > 0.0 && o > 0.0) || (a < 0.0 && o < 0.0);
          mm = minmod2(a, o);
        }
        if (mm != a) {
          const double ns = mm / s3;
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

// flux through face f of a cell with own limits o and other side b (already
// the ghost on the boundary); own revised limits in so
__device__ __forceinline__ void face_flux(const Par &P, const Lim &o, const Lim &b, int f, double F[3],
                                          Side<double> &so) {
  const double zf = fmax(o.z, b.z);
  so = revise_h(o.h, o.qx, o.qy, o.z, zf, P.hd);
  const Side<double> sb = revise_h(b.h, b.qx, b.qy, b.z, zf, P.hd);
  double H[3];
  if (f == 0) {
    hll(so.hs, so.u, so.v, sb.hs, sb.u, sb.v, P.g, P.hd, H);
    F[0] = H[0]; F[1] = H[1]; F[2] = H[2];
  } else if (f == 1) {
    hll(sb.hs, sb.u, sb.v, so.hs, so.u, so.v, P.g, P.hd, H);
    F[0] = H[0]; F[1] = H[1]; F[2] = H[2];
  } else if (f == 2) {
    hll(so.hs, so.v, so.u, sb.hs, sb.v, sb.u, P.g, P.hd, H);
    F[0] = H[0]; F[1] = H[2]; F[2] = H[1];
  } else {
    hll(sb.hs, sb.v, sb.u, so.hs, so.v, so.u, P.g, P.hd, H);
    F[0] = H[0]; F[1] = H[2]; F[2] = H[1];
  }
}

__device__ __forceinline__ bool cell_of(const Par &P, long long &k, int &i, int &j) {
  k = (long long)blockIdx.x * TPB + threadIdx.x;
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
__global__ void __launch_bounds__(TPB) k_cfl(Par P, const double *U, const double *tt, int step,
                                             unsigned long long *best) {
  __shared__ double sh[TPB];
  long long k;
  int i, j;
  double c = tinf<double>();
  if (cell_of(P, k, i, j)) {
    const long long n = P.n;
    const double h0 = U[k], dx = P.dx, g = P.g;
    if (h0 > P.hd) {
      const double u = U[3 * n + k] / h0, v = U[6 * n + k] / h0;
      const double cc = sqrt(g * h0);
      c = fmin(c, fmin(dx / (fabs(u) + cc), dx / (fabs(v) + cc)));
    }
    for (int e = 0; e < 4; e++) {
      const bool on = (e == 0 && i == 0) || (e == 1 && i == P.nx - 1) || (e == 2 && j == 0) ||
                      (e == 3 && j == P.ny - 1);
      if (!on) continue;
      const double q = inflow_unit(P, e, e < 2 ? j : i, tt[step]);
      if (q > 0.0) {
        const double hc = newton_cbrt(q * q / g);
        if (hc > P.hd) c = fmin(c, dx / (q / hc + sqrt(g * hc)));
      }
    }
  }
  sh[threadIdx.x] = c;
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0 && sh[0] < tinf<double>())
    atomicMin(best, (unsigned long long)__double_as_longlong(sh[0]));
}

__global__ void k_dt(Par P, unsigned long long *best, double *dts, double *tt, int step) {
  const double b = __longlong_as_double((long long)*best);
  double dt = P.dt_max;
  if (b < tinf<double>()) dt = fmin(dt, P.cfl * b);
  dts[step] = dt;
  tt[step + 1] = tt[step] + dt;
  *best = (unsigned long long)__double_as_longlong(tinf<double>());
}

// rain depth of the step, then split implicit Manning friction
__global__ void __launch_bounds__(TPB) k_friction(Par P, const double *U, const double *nman, const double *dts,
                                                  const double *tt, int step, double *Un) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long n = P.n;
  const double dt = dts[step], t = tt[step], g = P.g;
  const double rain = (t < P.rain_t_end) ? P.rain_rate : 0.0;
  double w[9];
#pragma unroll
  for (int m = 0; m < 9; m++) w[m] = U[m * n + k];
  if (rain > 0.0) w[0] = w[0] + rain * dt;
  const double h0 = w[0];
  if (h0 > P.hd) {
    const double u = w[3] / h0, v = w[6] / h0;
    const double sp = sqrt(u * u + v * v);
    const double nm = nman[k];
    const double den = 1.0 + dt * g * nm * nm * sp / (h0 * newton_cbrt(h0));
    const double f = 1.0 / den;
#pragma unroll
    for (int m = 3; m < 9; m++) w[m] = w[m] * f;
  } else {
#pragma unroll
    for (int m = 3; m < 9; m++) w[m] = 0.0;
  }
#pragma unroll
  for (int m = 0; m < 9; m++) Un[m * n + k] = w[m];
}

__global__ void __launch_bounds__(TPB) k_limit(Par P, const double *X, const double *Z, double *Wst, double *Wfx,
                                               double *Zfx) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long n = P.n;
  double ws[9], wf[9], ze[3];
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

// One RK2 stage (Eq. 4a for stage 1, Eq. 4b for stage 2): the DG2 operator
// of the cell from its four face fluxes, the stage combination and the
// positivity clip; the clip is recorded in bit (stage - 1) of clip[k].
__global__ void __launch_bounds__(TPB) k_update(Par P, int stage, const double *Wfx, const double *Zfx,
                                                const double *Wst, const double *W1, const double *dts,
                                                const double *tt, int step, double *Out, uint8_t *clip) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long n = P.n;
  const double dt = dts[step];
  const double t = stage == 1 ? tt[step] : tt[step] + dt;
  const double g = P.g, s3 = S3(), dxl = P.dx;
  double Fh[4][3], hs[4], us[4], vs[4], zr[4];
  for (int f = 0; f < 4; f++) {
    const Lim o = cell_lim(Wfx, Zfx, n, k, f);
    bool inside;
    const Lim b = other_side(P, Wfx, Zfx, i, j, f, o, t, inside);
    Side<double> so;
    face_flux(P, o, b, f, Fh[f], so);
    hs[f] = so.hs; us[f] = so.u; vs[f] = so.v; zr[f] = so.zr;
  }
  double Fx[2][3], Gy[2][3];
#pragma unroll
  for (int a = 0; a < 2; a++) {
    int f = a;
    const double q = hs[f] * us[f];
    Fx[a][0] = q;
    Fx[a][1] = q * us[f] + 0.5 * g * hs[f] * hs[f];
    Fx[a][2] = q * vs[f];
    f = 2 + a;
    const double r = hs[f] * vs[f];
    Gy[a][0] = r;
    Gy[a][1] = r * us[f];
    Gy[a][2] = r * vs[f] + 0.5 * g * hs[f] * hs[f];
  }
  const double w1 = Wfx[n + k], w2 = Wfx[2 * n + k], zc1 = Zfx[n + k], zc2 = Zfx[2 * n + k];
  double o[9];
#pragma unroll
  for (int v = 0; v < 3; v++) {
    double L0 = -(Fh[0][v] - Fh[1][v]) / dxl - (Fh[2][v] - Fh[3][v]) / dxl;
    if (v == 1) L0 = L0 + -g * 0.5 * (hs[0] + hs[1]) * (zr[0] - zr[1]) / dxl;
    if (v == 2) L0 = L0 + -g * 0.5 * (hs[2] + hs[3]) * (zr[2] - zr[3]) / dxl;
    double L1x = -(s3 / dxl) * (Fh[0][v] + Fh[1][v] - Fx[0][v] - Fx[1][v]);
    double L1y = -(s3 / dxl) * (Fh[2][v] + Fh[3][v] - Gy[0][v] - Gy[1][v]);
    if (v == 1) L1x = L1x + -(2.0 * s3 * g / dxl) * w1 * (w1 + zc1);
    if (v == 2) L1y = L1y + -(2.0 * s3 * g / dxl) * w2 * (w2 + zc2);
    const double Lo[3] = {L0, L1x, L1y};
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const int m = 3 * v + c;
      if (stage == 1) o[m] = Wst[m * n + k] + dt * Lo[c];
      else o[m] = 0.5 * (W1[m * n + k] + Wst[m * n + k] + dt * Lo[c]);
    }
  }
  // this stage's bit is written, the other stage's kept (a recomputed stage 1
  // must not erase the recorded stage-2 bit)
  const uint8_t mine = (uint8_t)(1u << (stage - 1));
  uint8_t bits = (uint8_t)(clip[k] & ~mine);
  if (o[0] < 0.0) {
    o[0] = 0.0;
    bits |= mine;
  }
  if (!(o[0] > P.hd)) {
#pragma unroll
    for (int m = 1; m < 9; m++) o[m] = 0.0;
  }
  clip[k] = bits;
#pragma unroll
  for (int m = 0; m < 9; m++) Out[m * n + k] = o[m];
}

// Eq. 8: vertex raster -> planes
__global__ void __launch_bounds__(TPB) k_project(Par P, const double *vert, double *out) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long w = P.nx + 1;
  const double s3 = S3();
  const double sw = vert[j * w + i], se = vert[j * w + i + 1];
  const double nw = vert[(j + 1) * w + i], ne = vert[(j + 1) * w + i + 1];
  const double zn = 0.5 * (nw + ne), zs = 0.5 * (sw + se);
  const double zE = 0.5 * (ne + se), zW = 0.5 * (nw + sw);
  out[k] = 0.5 * (zE + zW);
  out[P.n + k] = (zE - zW) / (2.0 * s3);
  out[2 * P.n + k] = (zn - zs) / (2.0 * s3);
}

// transpose of k_project: each vertex gathers from the up to four cells
// that touch it
__global__ void __launch_bounds__(TPB) k_project_t(Par P, const double *gp, double *gv) {
  const long long w = P.nx + 1;
  const long long v = (long long)blockIdx.x * TPB + threadIdx.x;
  if (v >= w * (P.ny + 1)) return;
  const int j = (int)(v / w), i = (int)(v - (long long)j * w);
  const double s3 = S3();
  double acc = 0.0;
  for (int cj = j - 1; cj <= j; cj++)
    for (int ci = i - 1; ci <= i; ci++) {
      if (ci < 0 || cj < 0 || ci >= P.nx || cj >= P.ny) continue;
      const long long k = (long long)cj * P.nx + ci;
      const double sx = ci == i ? -1.0 : 1.0;   // west or east column of the cell
      const double sy = cj == j ? -1.0 : 1.0;   // south or north row
      // c0 = (sw + se + nw + ne) / 4; c1x = (ne + se - nw - sw) / (4 s3);
      // c1y = (nw + ne - sw - se) / (4 s3), each 0.5 * 0.5 exactly as k_project
      acc += 0.25 * gp[k] + sx * gp[P.n + k] / (4.0 * s3) + sy * gp[2 * P.n + k] / (4.0 * s3);
    }
  gv[v] = acc;
}

// ---------------------------------------------------------------------------
// reverse sweep
// ---------------------------------------------------------------------------
// Cotangents of the own revised limits and fluxes of one cell's operator.
// Buffers: cF (4 faces x 3) the flux cotangent this cell contributes to
// each face, cR (4 x 4) the cotangents of its own revised (hs, u, v, zr) per
// face, cD (4) direct cotangents of (w1x of h, w1y of h, z1x, z1y) of the
// flux view from the bed-slope sources.  lWs receives the cotangent of the
// stage's stored view; lW1 carries stage 2's share of the stage-1 view.
__global__ void __launch_bounds__(TPB) k_rev_cell(Par P, int stage, const double *lY, const double *Y,
                                                  const uint8_t *clip, const double *dts, const double *tt,
                                                  int step, const double *Wfx, const double *Zfx, double *lWs,
                                                  double *lW1, double *cF, double *cR, double *cD) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long n = P.n;
  const double dt = dts[step];
  const double t = stage == 1 ? tt[step] : tt[step] + dt;
  const double g = P.g, s3 = S3(), dx = P.dx;
  const bool clipped = (clip[k] >> (stage - 1)) & 1u;
  const bool dry = !(Y[k] > P.hd);
  double lL[9];
#pragma unroll
  for (int m = 0; m < 9; m++) {
    double lo = lY[m * n + k];
    if ((m == 0 && clipped) || (m > 0 && dry)) lo = 0.0;
    if (stage == 2) {
      lWs[m * n + k] = 0.5 * lo;
      lW1[m * n + k] = 0.5 * lo;
      lL[m] = 0.5 * dt * lo;
    } else {
      lWs[m * n + k] = lo + lW1[m * n + k];
      lL[m] = dt * lo;
    }
  }
  // forward values of the own revised limits
  double hs[4], us[4], vs[4], zr[4];
  for (int f = 0; f < 4; f++) {
    const Lim o = cell_lim(Wfx, Zfx, n, k, f);
    bool inside;
    const Lim b = other_side(P, Wfx, Zfx, i, j, f, o, t, inside);
    const double zf = fmax(o.z, b.z);
    const Side<double> so = revise_h(o.h, o.qx, o.qy, o.z, zf, P.hd);
    hs[f] = so.hs; us[f] = so.u; vs[f] = so.v; zr[f] = so.zr;
  }
  double lF[4][3] = {}, lH[4] = {}, lU[4] = {}, lV[4] = {}, lZ[4] = {}, lFx[2][3] = {}, lGy[2][3] = {};
  double lD[4] = {};
  const double kx = -(s3 / dx);
  const double w1 = Wfx[n + k], w2 = Wfx[2 * n + k], zc1 = Zfx[n + k], zc2 = Zfx[2 * n + k];
#pragma unroll
  for (int v = 0; v < 3; v++) {
    const double l0 = lL[3 * v], lx = lL[3 * v + 1], ly = lL[3 * v + 2];
    lF[0][v] += -l0 / dx;
    lF[1][v] += l0 / dx;
    lF[2][v] += -l0 / dx;
    lF[3][v] += l0 / dx;
    lF[0][v] += kx * lx;
    lF[1][v] += kx * lx;
    lFx[0][v] -= kx * lx;
    lFx[1][v] -= kx * lx;
    lF[2][v] += kx * ly;
    lF[3][v] += kx * ly;
    lGy[0][v] -= kx * ly;
    lGy[1][v] -= kx * ly;
    const double c = -g * 0.5 / dx, c2 = -(2.0 * s3 * g / dx);
    if (v == 1) {
      lH[0] += l0 * c * (zr[0] - zr[1]);
      lH[1] += l0 * c * (zr[0] - zr[1]);
      lZ[0] += l0 * c * (hs[0] + hs[1]);
      lZ[1] -= l0 * c * (hs[0] + hs[1]);
      lD[0] += lx * c2 * (2.0 * w1 + zc1);
      lD[2] += lx * c2 * w1;
    }
    if (v == 2) {
      lH[2] += l0 * c * (zr[2] - zr[3]);
      lH[3] += l0 * c * (zr[2] - zr[3]);
      lZ[2] += l0 * c * (hs[2] + hs[3]);
      lZ[3] -= l0 * c * (hs[2] + hs[3]);
      lD[1] += ly * c2 * (2.0 * w2 + zc2);
      lD[3] += ly * c2 * w2;
    }
  }
#pragma unroll
  for (int a = 0; a < 2; a++) {
    int f = a;
    const double q = hs[f] * us[f];
    const double lq = lFx[a][0] + lFx[a][1] * us[f] + lFx[a][2] * vs[f];
    lU[f] += lFx[a][1] * q;
    lV[f] += lFx[a][2] * q;
    lH[f] += lFx[a][1] * g * hs[f];
    lH[f] += lq * us[f];
    lU[f] += lq * hs[f];
    f = 2 + a;
    const double r = hs[f] * vs[f];
    const double lr = lGy[a][0] + lGy[a][1] * us[f] + lGy[a][2] * vs[f];
    lU[f] += lGy[a][1] * r;
    lV[f] += lGy[a][2] * r;
    lH[f] += lGy[a][2] * g * hs[f];
    lH[f] += lr * vs[f];
    lV[f] += lr * hs[f];
  }
#pragma unroll
  for (int f = 0; f < 4; f++) {
#pragma unroll
    for (int v = 0; v < 3; v++) cF[(f * 3 + v) * n + k] = lF[f][v];
    cR[(f * 4 + 0) * n + k] = lH[f];
    cR[(f * 4 + 1) * n + k] = lU[f];
    cR[(f * 4 + 2) * n + k] = lV[f];
    cR[(f * 4 + 3) * n + k] = lZ[f];
  }
#pragma unroll
  for (int q = 0; q < 4; q++) cD[q * n + k] = lD[q];
}

// reverse of hll(): cotangents of (hL, unL, utL, hR, unR, utR) from those of F
__device__ void hll_rev(double hL, double unL, double utL, double hR, double unR, double utR, double g,
                        double hd, const double lF[3], double l[6]) {
#pragma unroll
  for (int q = 0; q < 6; q++) l[q] = 0.0;
  const bool dryL = !(hL > hd), dryR = !(hR > hd);
  if (dryL && dryR) return;
  const double cL = sqrt(g * hL), cR = sqrt(g * hR);
  double sL, sR;
  bool selA = false, selB = false;  // wet pair: sL from unL - cL, sR from unR + cR
  double us = 0.0, cs = 0.0;
  if (dryL) {
    sL = unR - 2.0 * cR;
    sR = unR + cR;
  } else if (dryR) {
    sL = unL - cL;
    sR = unL + 2.0 * cL;
  } else {
    us = 0.5 * (unL + unR) + cL - cR;
    cs = 0.5 * (cL + cR) + 0.25 * (unL - unR);
    const double a1 = unL - cL, a2 = us - cs, b1 = unR + cR, b2 = us + cs;
    selA = a1 <= a2;
    selB = b1 >= b2;
    sL = selA ? a1 : a2;
    sR = selB ? b1 : b2;
  }
  const double qL = hL * unL, qR = hR * unR;
  double lqL = 0.0, lqR = 0.0, lhL = 0.0, lhR = 0.0, lunL = 0.0, lunR = 0.0, lutL = 0.0, lutR = 0.0;
  double lsL = 0.0, lsR = 0.0;
  double lFL[3] = {0.0, 0.0, 0.0}, lFR[3] = {0.0, 0.0, 0.0};
  if (sL >= 0.0) {
    lFL[0] = lF[0]; lFL[1] = lF[1]; lFL[2] = lF[2];
  } else if (sR <= 0.0) {
    lFR[0] = lF[0]; lFR[1] = lF[1]; lFR[2] = lF[2];
  } else {
    const double FL[3] = {qL, qL * unL + 0.5 * g * hL * hL, qL * utL};
    const double FR[3] = {qR, qR * unR + 0.5 * g * hR * hR, qR * utR};
    const double UL[3] = {hL, qL, hL * utL}, UR[3] = {hR, qR, hR * utR};
    const double den = sR - sL;
    double lden = 0.0, lUL[3], lUR[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const double N = sR * FL[c] - sL * FR[c] + sL * sR * (UR[c] - UL[c]);
      const double lN = lF[c] / den;
      lden -= lF[c] * (N / den) / den;
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
  double lcL = 0.0, lcR = 0.0;
  if (dryL) {
    lunR += lsL + lsR;
    lcR += -2.0 * lsL + lsR;
  } else if (dryR) {
    lunL += lsL + lsR;
    lcL += -lsL + 2.0 * lsR;
  } else {
    double lus = 0.0, lcs = 0.0;
    if (selA) { lunL += lsL; lcL -= lsL; }
    else { lus += lsL; lcs -= lsL; }
    if (selB) { lunR += lsR; lcR += lsR; }
    else { lus += lsR; lcs += lsR; }
    lunL += 0.5 * lus;
    lunR += 0.5 * lus;
    lcL += lus;
    lcR -= lus;
    lcL += 0.5 * lcs;
    lcR += 0.5 * lcs;
    lunL += 0.25 * lcs;
    lunR -= 0.25 * lcs;
  }
  if (!dryL) lhL += lcL * g / (2.0 * cL);
  if (!dryR) lhR += lcR * g / (2.0 * cR);
  l[0] = lhL; l[1] = lunL; l[2] = lutL;
  l[3] = lhR; l[4] = lunR; l[5] = lutR;
}

// reverse of revise_h(): cotangents of the limit (h, qx, qy, z) and of the
// interface bed zf from those of (hs, u, v, zr)
__device__ __forceinline__ void revise_rev(const Lim &s, double zf, double hd, double lhs, double lu, double lv,
                                           double lzr, double out[4], double &lzf) {
  const double eta = s.h + s.z;
  const double d = eta - zf;
  double leta = 0.0, ld = 0.0;
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
  out[1] = 0.0;
  out[2] = 0.0;
  if (s.h > hd) {
    out[1] = lu / s.h;
    out[2] = lv / s.h;
    out[0] -= (lu * s.qx + lv * s.qy) / (s.h * s.h);
  }
}

// split of the cotangent of max(zL, zR)
__device__ __forceinline__ void tiemax_rev(double zL, double zR, double lzf, double &lL, double &lR) {
  const double scale = fmax(1.0, fmax(fabs(zL), fabs(zR)));
  if (fabs(zL - zR) <= TIE_REL * scale) {
    lL += 0.5 * lzf;
    lR += 0.5 * lzf;
  } else if (zL > zR) {
    lL += lzf;
  } else {
    lR += lzf;
  }
}

// reverse of ghost(): fold the ghost's cotangents into the own limit; the
// hydrograph's share (per unit of Q(t)) is returned
__device__ double ghost_rev(const Par &P, int e, int along, const Lim &o, double t, const double lg[4],
                            double lo[4]) {
  lo[3] += lg[3];
  const double q = inflow_unit(P, e, along, t);
  if (q > 0.0) {
    const double x = q * q / P.g;
    const double hc = newton_cbrt(x);
    double lq = 0.0;
    if (o.h >= hc) lo[0] += lg[0];
    else lq += lg[0] / (3.0 * hc * hc) * (2.0 * q / P.g);
    const double sg = (e == 0 || e == 2) ? 1.0 : -1.0;
    lq += sg * (e < 2 ? lg[1] : lg[2]);
    return lq * 1.0 / ((double)(P.c1 - P.c0 + 1) * P.dx);
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

// Per interface: the flux cotangent from both cells, HLL and the two
// revisions in reverse, the interface bed split, the ghost folded into the
// boundary cell.  Output per face: the cotangents of the low side's limit
// (slots 0-3: h, qx, qy, z) and the high side's (slots 4-7); `lq`, per
// boundary cell of the inflow edge, the cotangent of Q(t).
template <bool XF>
__global__ void __launch_bounds__(TPB) k_rev_face(Par P, int stage, const double *dts, const double *tt, int step,
                                                  const double *Wfx, const double *Zfx, const double *cF,
                                                  const double *cR, double *lim, double *lq) {
  const long long nf = XF ? (long long)P.ny * (P.nx + 1) : (long long)(P.ny + 1) * P.nx;
  const long long fi = (long long)blockIdx.x * TPB + threadIdx.x;
  if (fi >= nf) return;
  const long long n = P.n;
  const double dt = dts[step];
  const double t = stage == 1 ? tt[step] : tt[step] + dt;
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
  Lim lo, hi;
  if (hasLo) lo = cell_lim(Wfx, Zfx, n, kLo, fLo);
  if (hasHi) hi = cell_lim(Wfx, Zfx, n, kHi, fHi);
  if (!hasLo) lo = ghost(P, eLo, along, hi, t);
  if (!hasHi) hi = ghost(P, eHi, along, lo, t);
  const double zf = fmax(lo.z, hi.z);
  const Side<double> sLo = revise_h(lo.h, lo.qx, lo.qy, lo.z, zf, P.hd);
  const Side<double> sHi = revise_h(hi.h, hi.qx, hi.qy, hi.z, zf, P.hd);
  double lF[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int v = 0; v < 3; v++) {
    if (hasLo) lF[v] += cF[(fLo * 3 + v) * n + kLo];
    if (hasHi) lF[v] += cF[(fHi * 3 + v) * n + kHi];
  }
  double l6[6];
  if (XF) {
    hll_rev(sLo.hs, sLo.u, sLo.v, sHi.hs, sHi.u, sHi.v, P.g, P.hd, lF, l6);
  } else {
    const double lH[3] = {lF[0], lF[2], lF[1]};
    hll_rev(sLo.hs, sLo.v, sLo.u, sHi.hs, sHi.v, sHi.u, P.g, P.hd, lH, l6);
  }
  // cotangents of (hs, u, v, zr) of each side
  double rLo[4], rHi[4];
  rLo[0] = l6[0];
  rHi[0] = l6[3];
  if (XF) { rLo[1] = l6[1]; rLo[2] = l6[2]; rHi[1] = l6[4]; rHi[2] = l6[5]; }
  else { rLo[2] = l6[1]; rLo[1] = l6[2]; rHi[2] = l6[4]; rHi[1] = l6[5]; }
  rLo[3] = 0.0;
  rHi[3] = 0.0;
  if (hasLo)
    for (int q = 0; q < 4; q++) rLo[q] += cR[(fLo * 4 + q) * n + kLo];
  if (hasHi)
    for (int q = 0; q < 4; q++) rHi[q] += cR[(fHi * 4 + q) * n + kHi];
  double gLo[4], gHi[4], lzf = 0.0;
  revise_rev(lo, zf, P.hd, rLo[0], rLo[1], rLo[2], rLo[3], gLo, lzf);
  revise_rev(hi, zf, P.hd, rHi[0], rHi[1], rHi[2], rHi[3], gHi, lzf);
  tiemax_rev(lo.z, hi.z, lzf, gLo[3], gHi[3]);
  double lQ = 0.0;
  if (!hasLo) {
    double f4[4] = {0.0, 0.0, 0.0, 0.0};
    lQ = ghost_rev(P, eLo, along, hi, t, gLo, f4);
    for (int q = 0; q < 4; q++) { gHi[q] += f4[q]; gLo[q] = 0.0; }
    if (P.inflow_edge == eLo) lq[along] = lQ;
  }
  if (!hasHi) {
    double f4[4] = {0.0, 0.0, 0.0, 0.0};
    lQ = ghost_rev(P, eHi, along, lo, t, gHi, f4);
    for (int q = 0; q < 4; q++) { gLo[q] += f4[q]; gHi[q] = 0.0; }
    if (P.inflow_edge == eHi) lq[along] = lQ;
  }
#pragma unroll
  for (int q = 0; q < 4; q++) {
    lim[q * nf + fi] = gLo[q];
    lim[(4 + q) * nf + fi] = gHi[q];
  }
}

// hydrograph knots: the cotangent of Q(t) summed over the inflow edge in a
// fixed order, spread over the two knots around t
__global__ void k_rev_knots(Par P, int stage, const double *dts, const double *tt, int step, const double *lq,
                            double *gQ) {
  __shared__ double sh[TPB];
  const int nedge = (P.inflow_edge < 2) ? P.ny : P.nx;
  double acc = 0.0;
  for (int a = threadIdx.x; a < nedge; a += TPB)
    if (a >= P.c0 && a <= P.c1) acc += lq[a];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double dt = dts[step];
    const double t = stage == 1 ? tt[step] : tt[step] + dt;
    int k0, k1;
    double r;
    hydro(P, t, k0, k1, r);
    const double l = sh[0];
    if (k0 == k1) {
      gQ[k0] += l;
    } else {
      gQ[k0] += l - l * r;
      gQ[k1] += l * r;
    }
  }
}

// Face-limit transpose and the limiter in reverse for one cell: the
// cotangent of the stage input X of this cell (lXo) and the shares of its
// neighbours' averages (lnb: direction, side A/B, variable), the bed's own
// cotangents added to gz.
__global__ void __launch_bounds__(TPB) k_rev_limit(Par P, const double *X, const double *Z, const double *lWs,
                                                   const double *limx, const double *limy, const double *cD,
                                                   double *lXo, double *lnb, double *gz) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long n = P.n;
  const long long nfx = (long long)P.ny * (P.nx + 1), nfy = (long long)(P.ny + 1) * P.nx;
  const double s3 = S3();
  double ws[9], wf[9], ze[3];
  LimRec r;
  limit_cell(P, X, Z, i, j, ws, wf, ze, r);
  // cotangents of the face limits: E = low side of x face (j, i + 1), W =
  // high side of x face (j, i), N = low side of y face (j + 1, i), S = high
  // side of y face (j, i)
  double lf[4][4];
  const long long fE = (long long)j * (P.nx + 1) + i + 1, fW = (long long)j * (P.nx + 1) + i;
  const long long fN = (long long)(j + 1) * P.nx + i, fS = (long long)j * P.nx + i;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    lf[0][q] = limx[q * nfx + fE];
    lf[1][q] = limx[(4 + q) * nfx + fW];
    lf[2][q] = limy[q * nfy + fN];
    lf[3][q] = limy[(4 + q) * nfy + fS];
  }
  double lw[9], lz[3];
#pragma unroll
  for (int v = 0; v < 4; v++) {
    const double a = lf[0][v] + lf[1][v] + lf[2][v] + lf[3][v];
    const double bx = s3 * (lf[0][v] - lf[1][v]);
    const double by = s3 * (lf[2][v] - lf[3][v]);
    if (v < 3) { lw[3 * v] = a; lw[3 * v + 1] = bx; lw[3 * v + 2] = by; }
    else { lz[0] = a; lz[1] = bx; lz[2] = by; }
  }
  lw[1] += cD[k];
  lw[2] += cD[n + k];
  lz[1] += cD[2 * n + k];
  lz[2] += cD[3 * n + k];
  double lX[9], gzz[3] = {0.0, 0.0, 0.0}, nb[2][2][3] = {};
  double lsw[9];
#pragma unroll
  for (int m = 0; m < 9; m++) lsw[m] = lWs[m * n + k];
  if (r.red) {
#pragma unroll
    for (int m = 0; m < 9; m++) lX[m] = 0.0;
    lX[0] = lsw[0] + lw[0];
    lX[3] = lsw[3] + lw[3];
    lX[6] = lsw[6] + lw[6];
    gzz[1] -= lsw[1];
    gzz[2] -= lsw[2];
    gzz[0] += lz[0];
  } else {
    double lt[9];
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
        const double l = lt[coef];
        lX[coef] = 0.0;
        if (v == 0) gzz[cs] -= l;
        const double lmm = l / s3;
        double laC = 0.0;
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
__global__ void __launch_bounds__(TPB) k_rev_gather(Par P, const double *lXo, const double *lnb, double *lX,
                                                    double *gz) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long n = P.n;
  double in[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int v = 0; v < 3; v++) {
    if (i > 0) in[v] += lnb[((0 * 2 + 0) * 3 + v) * n + k - 1];
    if (i < P.nx - 1) in[v] += lnb[((0 * 2 + 1) * 3 + v) * n + k + 1];
    if (j > 0) in[v] += lnb[((1 * 2 + 0) * 3 + v) * n + k - P.nx];
    if (j < P.ny - 1) in[v] += lnb[((1 * 2 + 1) * 3 + v) * n + k + P.nx];
  }
#pragma unroll
  for (int m = 0; m < 9; m++) {
    double l = lXo[m * n + k];
    if (m % 3 == 0) l += in[m / 3];
    lX[m * n + k] = l;
  }
  gz[k] += in[0];
}

// friction (and rain) in reverse: lU = cotangent of the step's input state,
// Manning n's share added to gn
__global__ void __launch_bounds__(TPB) k_rev_friction(Par P, const double *U, const double *nman,
                                                      const double *dts, const double *tt, int step,
                                                      const double *lUn, double *lU, double *gn) {
  long long k;
  int i, j;
  if (!cell_of(P, k, i, j)) return;
  const long long n = P.n;
  const double dt = dts[step], t = tt[step], g = P.g;
  const double rain = (t < P.rain_t_end) ? P.rain_rate : 0.0;
  double w[9], l[9], lo[9];
#pragma unroll
  for (int m = 0; m < 9; m++) {
    w[m] = U[m * n + k];
    l[m] = lUn[m * n + k];
  }
  if (rain > 0.0) w[0] = w[0] + rain * dt;
  const double h0 = w[0];
  lo[0] = l[0];
  lo[1] = l[1];
  lo[2] = l[2];
  double lnm = 0.0;
  if (h0 > P.hd) {
    const double u = w[3] / h0, v = w[6] / h0;
    const double sp = sqrt(u * u + v * v);
    const double nm = nman[k];
    const double cr = newton_cbrt(h0);
    const double B = h0 * cr;
    const double A = dt * g * nm * nm;
    const double den = 1.0 + dt * g * nm * nm * sp / B;
    const double f = 1.0 / den;
    double lf = 0.0;
#pragma unroll
    for (int m = 3; m < 9; m++) {
      lo[m] = l[m] * f;
      lf += l[m] * w[m];
    }
    const double lden = -lf / (den * den);
    const double lsp = lden * A / B;
    const double lB = -lden * A * sp / (B * B);
    lnm = lden * sp / B * (dt * g * 2.0 * nm);
    double lh = lB * (cr + h0 / (3.0 * cr * cr));
    if (sp > 0.0) {
      const double lu = lsp * u / sp, lv = lsp * v / sp;
      lo[3] += lu / h0;
      lo[6] += lv / h0;
      lh -= (lu * u + lv * v) / h0;
    }
    lo[0] += lh;
  } else {
#pragma unroll
    for (int m = 3; m < 9; m++) lo[m] = 0.0;
  }
#pragma unroll
  for (int m = 0; m < 9; m++) lU[m * n + k] = lo[m];
  gn[k] += lnm;
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
  long long n = 0;
  int dev = 0;
  double *tape = nullptr;      // (max_steps + 1) x 9n: the state at the start of each step
  uint8_t *clip = nullptr;     // max_steps x n: bit s-1 set when stage s clipped
  double *tt = nullptr;        // max_steps + 1 step start times
  double *dtbuf = nullptr;     // max_steps time steps (fixed runs copy theirs here)
  unsigned long long *best = nullptr;
  double *Un = nullptr, *Ui = nullptr, *W1 = nullptr, *F1 = nullptr, *Z1 = nullptr;
  double *W2 = nullptr, *F2 = nullptr, *Z2 = nullptr;
  double *lU = nullptr, *lX = nullptr, *lWs = nullptr, *lW1 = nullptr, *cF = nullptr, *cR = nullptr,
         *cD = nullptr, *limx = nullptr, *limy = nullptr, *lXo = nullptr, *lnb = nullptr, *lq = nullptr;
  std::string err;
};

namespace {

void free_all(mwdg_adj *a) {
  void *ptrs[] = {a->tape, a->clip, a->tt, a->dtbuf, a->best, a->Un, a->Ui, a->W1, a->F1, a->Z1, a->W2,
                  a->F2, a->Z2, a->lU, a->lX, a->lWs, a->lW1, a->cF, a->cR, a->cD, a->limx, a->limy,
                  a->lXo, a->lnb, a->lq};
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

Par make_par(const mwdg_adj *a, int nknots, const double *kt, const double *kQ) {
  Par P;
  const mwdg_adj_params &p = a->p;
  P.nx = p.nx;
  P.ny = p.ny;
  P.n = a->n;
  P.dx = p.dx;
  P.g = p.g;
  P.hd = p.h_dry;
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

// the forward sweep of one step s from tape slot s into slot s + 1
void launch_step(const mwdg_adj *a, const Par &P, const double *z, const double *nman, int s, bool cfl,
                 double *dts, cudaStream_t st) {
  const long long n = a->n;
  const double *U = a->tape + (long long)s * 9 * n;
  double *Unext = a->tape + (long long)(s + 1) * 9 * n;
  uint8_t *clip = a->clip + (long long)s * n;
  const unsigned nb = blocks(n);
  if (cfl) {
    k_cfl<<<nb, TPB, 0, st>>>(P, U, a->tt, s, a->best);
    k_dt<<<1, 1, 0, st>>>(P, a->best, dts, a->tt, s);
  }
  k_friction<<<nb, TPB, 0, st>>>(P, U, nman, dts, a->tt, s, a->Un);
  k_limit<<<nb, TPB, 0, st>>>(P, a->Un, z, a->W1, a->F1, a->Z1);
  k_update<<<nb, TPB, 0, st>>>(P, 1, a->F1, a->Z1, a->W1, nullptr, dts, a->tt, s, a->Ui, clip);
  k_limit<<<nb, TPB, 0, st>>>(P, a->Ui, z, a->W2, a->F2, a->Z2);
  k_update<<<nb, TPB, 0, st>>>(P, 2, a->F2, a->Z2, a->W2, a->W1, dts, a->tt, s, Unext, clip);
}

mwdg_status check_run(mwdg_adj *a, const double *U0, const double *z, const double *n, int32_t nknots,
                      const double *kt, const double *kQ, int32_t steps, const double *dts) {
  if (!a) return MWDG_ERR_ARG;
  if (!U0 || !z || !n || !dts || steps < 0) return fail(a, MWDG_ERR_ARG, "NULL pointer or steps < 0");
  if (steps > a->p.max_steps) return fail(a, MWDG_ERR_CAPACITY, "steps > max_steps");
  if (a->p.inflow_edge >= 0 && (nknots < 1 || !kt || !kQ))
    return fail(a, MWDG_ERR_ARG, "an inflow edge needs nknots >= 1 knots");
  return MWDG_OK;
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
  return MWDG_OK;
}

mwdg_status mwdg_adj_create(const mwdg_adj_params *p, mwdg_adj **out) {
  if (!p || !out) return MWDG_ERR_ARG;
  *out = nullptr;
  if (p->nx < 1 || p->ny < 1 || (long long)p->nx * p->ny > (1LL << 28) || !(p->dx > 0.0) || p->max_steps < 1)
    return MWDG_ERR_DIMS;
  if (!(p->g > 0.0) || !(p->h_dry >= 0.0) || !(p->cfl > 0.0) || !(p->dt_max > 0.0) || p->rain_rate < 0.0)
    return MWDG_ERR_ARG;
  for (int e = 0; e < 4; e++)
    if (p->bc[e] != MWDG_WALL && p->bc[e] != MWDG_OPEN) return MWDG_ERR_ARG;
  if (p->inflow_edge >= 4 || p->inflow_edge < -1) return MWDG_ERR_ARG;
  if (p->inflow_edge >= 0) {
    const int len = p->inflow_edge < 2 ? p->ny : p->nx;
    if (p->inflow_c0 < 0 || p->inflow_c1 < p->inflow_c0 || p->inflow_c1 >= len) return MWDG_ERR_ARG;
  }
  mwdg_adj *a = new (std::nothrow) mwdg_adj;
  if (!a) return MWDG_ERR_CUDA;
  a->p = *p;
  a->n = (long long)p->nx * p->ny;
  cudaGetDevice(&a->dev);
  const long long n = a->n, S = p->max_steps;
  const long long nfx = (long long)p->ny * (p->nx + 1), nfy = (long long)(p->ny + 1) * p->nx;
  const long long nedge = p->nx > p->ny ? p->nx : p->ny;
  bool ok = true;
  auto alloc = [&](auto **ptr, long long count, size_t elem) {
    if (ok && cudaMalloc((void **)ptr, (size_t)count * elem) != cudaSuccess) ok = false;
  };
  alloc(&a->tape, (S + 1) * 9 * n, sizeof(double));
  alloc(&a->clip, S * n, 1);
  alloc(&a->tt, S + 1, sizeof(double));
  alloc(&a->dtbuf, S, sizeof(double));
  alloc(&a->best, 1, sizeof(unsigned long long));
  for (double **w : {&a->Un, &a->Ui, &a->W1, &a->F1, &a->W2, &a->F2, &a->lU, &a->lX, &a->lWs, &a->lW1,
                     &a->lXo})
    alloc(w, 9 * n, sizeof(double));
  alloc(&a->Z1, 3 * n, sizeof(double));
  alloc(&a->Z2, 3 * n, sizeof(double));
  alloc(&a->cF, 12 * n, sizeof(double));
  alloc(&a->cR, 16 * n, sizeof(double));
  alloc(&a->cD, 4 * n, sizeof(double));
  alloc(&a->lnb, 12 * n, sizeof(double));
  alloc(&a->limx, 8 * nfx, sizeof(double));
  alloc(&a->limy, 8 * nfy, sizeof(double));
  alloc(&a->lq, nedge, sizeof(double));
  if (ok) {
    const unsigned long long inf = 0x7ff0000000000000ull;
    ok = cudaMemcpy(a->best, &inf, sizeof inf, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(a->lq, 0, (size_t)nedge * sizeof(double)) == cudaSuccess;
  }
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

mwdg_status mwdg_adj_project(mwdg_adj *a, const double *vert, double *out, void *stream) {
  if (!a) return MWDG_ERR_ARG;
  if (!vert || !out) return fail(a, MWDG_ERR_ARG, "NULL pointer");
  const Par P = make_par(a, 0, nullptr, nullptr);
  k_project<<<blocks(a->n), TPB, 0, (cudaStream_t)stream>>>(P, vert, out);
  return cuda_check(a, "mwdg_adj_project");
}

mwdg_status mwdg_adj_project_transpose(mwdg_adj *a, const double *gp, double *gv, void *stream) {
  if (!a) return MWDG_ERR_ARG;
  if (!gp || !gv) return fail(a, MWDG_ERR_ARG, "NULL pointer");
  const Par P = make_par(a, 0, nullptr, nullptr);
  k_project_t<<<blocks((long long)(a->p.nx + 1) * (a->p.ny + 1)), TPB, 0, (cudaStream_t)stream>>>(P, gp, gv);
  return cuda_check(a, "mwdg_adj_project_transpose");
}

mwdg_status mwdg_adj_forward(mwdg_adj *a, const double *U0, const double *z, const double *nman, int32_t nknots,
                             const double *kt, const double *kQ, double t0, int32_t steps, int32_t fixed_dt,
                             double *dts, double *U_out, void *stream) {
  mwdg_status s = check_run(a, U0, z, nman, nknots, kt, kQ, steps, dts);
  if (s != MWDG_OK) return s;
  if (!U_out) return fail(a, MWDG_ERR_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const Par P = make_par(a, nknots, kt, kQ);
  const size_t bytes = (size_t)9 * a->n * sizeof(double);
  if (cudaMemcpyAsync(a->tape, U0, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return cuda_check(a, "mwdg_adj_forward copy-in");
  k_set_t0<<<1, 1, 0, st>>>(a->tt, t0);
  if (fixed_dt) k_times<<<1, 1, 0, st>>>(dts, steps, a->tt);
  for (int k = 0; k < steps; k++) launch_step(a, P, z, nman, k, !fixed_dt, dts, st);
  if (cudaMemcpyAsync(U_out, a->tape + (long long)steps * 9 * a->n, bytes, cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return cuda_check(a, "mwdg_adj_forward copy-out");
  return cuda_check(a, "mwdg_adj_forward");
}

mwdg_status mwdg_adj_backward(mwdg_adj *a, const double *U0, const double *z, const double *nman,
                              int32_t nknots, const double *kt, const double *kQ, double t0, int32_t steps,
                              const double *dts_in, const double *gUK, double *gU0, double *gz, double *gn,
                              double *gQ, void *stream) {
  mwdg_status s = check_run(a, U0, z, nman, nknots, kt, kQ, steps, dts_in);
  if (s != MWDG_OK) return s;
  if (!gUK || !gU0 || !gz || !gn || (a->p.inflow_edge >= 0 && !gQ)) return fail(a, MWDG_ERR_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const Par P = make_par(a, nknots, kt, kQ);
  const long long n = a->n;
  const size_t bytes = (size_t)9 * n * sizeof(double);
  const unsigned nb = blocks(n);
  const long long nfx = (long long)a->p.ny * (a->p.nx + 1), nfy = (long long)(a->p.ny + 1) * a->p.nx;
  // the tape: the run recomputed from its checkpoint U0 over the given steps
  if (steps > 0 && cudaMemcpyAsync(a->dtbuf, dts_in, (size_t)steps * sizeof(double), cudaMemcpyDeviceToDevice,
                                   st) != cudaSuccess)
    return cuda_check(a, "mwdg_adj_backward dts");
  if (cudaMemcpyAsync(a->tape, U0, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return cuda_check(a, "mwdg_adj_backward copy-in");
  k_set_t0<<<1, 1, 0, st>>>(a->tt, t0);
  k_times<<<1, 1, 0, st>>>(a->dtbuf, steps, a->tt);
  for (int k = 0; k < steps; k++) launch_step(a, P, z, nman, k, false, a->dtbuf, st);
  if (cudaMemcpyAsync(a->lU, gUK, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return cuda_check(a, "mwdg_adj_backward seed");
  const double *dts = a->dtbuf;
  for (int k = steps - 1; k >= 0; k--) {
    const double *U = a->tape + (long long)k * 9 * n;
    const double *Y2 = a->tape + (long long)(k + 1) * 9 * n;
    uint8_t *clip = a->clip + (long long)k * n;
    // recompute the stage inputs of step k (stage 1 rewrites its clip bit
    // with the same value and keeps stage 2's from the tape run)
    k_friction<<<nb, TPB, 0, st>>>(P, U, nman, dts, a->tt, k, a->Un);
    k_limit<<<nb, TPB, 0, st>>>(P, a->Un, z, a->W1, a->F1, a->Z1);
    k_update<<<nb, TPB, 0, st>>>(P, 1, a->F1, a->Z1, a->W1, nullptr, dts, a->tt, k, a->Ui, clip);
    k_limit<<<nb, TPB, 0, st>>>(P, a->Ui, z, a->W2, a->F2, a->Z2);
    for (int stage = 2; stage >= 1; stage--) {
      const double *X = stage == 2 ? a->Ui : a->Un;
      const double *Y = stage == 2 ? Y2 : a->Ui;
      const double *Wf = stage == 2 ? a->F2 : a->F1;
      const double *Zf = stage == 2 ? a->Z2 : a->Z1;
      const double *lY = stage == 2 ? a->lU : a->lX;
      k_rev_cell<<<nb, TPB, 0, st>>>(P, stage, lY, Y, clip, dts, a->tt, k, Wf, Zf, a->lWs, a->lW1, a->cF, a->cR,
                                     a->cD);
      k_rev_face<true><<<blocks(nfx), TPB, 0, st>>>(P, stage, dts, a->tt, k, Wf, Zf, a->cF, a->cR, a->limx, a->lq);
      k_rev_face<false><<<blocks(nfy), TPB, 0, st>>>(P, stage, dts, a->tt, k, Wf, Zf, a->cF, a->cR, a->limy,
                                                     a->lq);
      if (P.nknots > 0) k_rev_knots<<<1, TPB, 0, st>>>(P, stage, dts, a->tt, k, a->lq, gQ);
      k_rev_limit<<<nb, TPB, 0, st>>>(P, X, z, a->lWs, a->limx, a->limy, a->cD, a->lXo, a->lnb, gz);
      k_rev_gather<<<nb, TPB, 0, st>>>(P, a->lXo, a->lnb, a->lX, gz);
    }
    k_rev_friction<<<nb, TPB, 0, st>>>(P, U, nman, dts, a->tt, k, a->lX, a->lU, gn);
  }
  if (cudaMemcpyAsync(gU0, a->lU, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return cuda_check(a, "mwdg_adj_backward copy-out");
  return cuda_check(a, "mwdg_adj_backward");
}

}  // extern "C"
