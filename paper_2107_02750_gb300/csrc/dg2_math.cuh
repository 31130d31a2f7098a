// Device arithmetic of the DG2 shallow-water operator and the multiwavelet
// filters (Sharifian & Kesserwani, arXiv 2107.02750, Sect. 2.1.1-2.3).
//
// Template parameters: T is the coefficient type (double or float); ETA
// selects the storage form of the first variable: depth h (false) or free
// surface eta = h + z (true, used by the FP32 path so that a flat surface is
// stored exactly).  The FP64 build of this header is compiled without FMA
// contraction so that every expression rounds as written.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mwdg {

enum : uint8_t { K_BELOW = 0, K_LEAF = 1, K_SIG = 2 };

template <typename T> __device__ __forceinline__ T s3v();
template <> __device__ __forceinline__ double s3v<double>() { return 1.7320508075688772; }
template <> __device__ __forceinline__ float s3v<float>() { return 1.7320508f; }

template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return fmax(a, b); }
template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return fmin(a, b); }
template <typename T> __device__ __forceinline__ T tinf();
template <> __device__ __forceinline__ float tinf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double tinf<double>() { return __longlong_as_double(0x7ff0000000000000LL); }
template <typename T> __device__ __forceinline__ T tsqrt(T a) { return sqrt(a); }
// Cube root.  FP32: the library's.  FP64: Newton's method on y^3 = x seeded
// by dividing the exponent field by three (W. Kahan, "Computing a real cube
// root", 1991), six iterations of y <- y - (y^3 - x) / (3 y^2) with basic
// IEEE operations only, so the result is the same on any IEEE machine.
__device__ __forceinline__ double newton_cbrt(double x) {
  if (x == 0.0 || x != x) return x;
  double sgn = 1.0, scale = 1.0;
  if (x < 0.0) { x = -x; sgn = -1.0; }
  if (x < 1e-290) { x = x * 0x1p300; scale = 0x1p-100; }
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  b = b / 3ull + (682ull << 52);
  double y = __longlong_as_double((long long)b);
#pragma unroll
  for (int it = 0; it < 6; it++) y = y - (y * y * y - x) / (3.0 * y * y);
  return sgn * scale * y;
}
template <typename T> __device__ __forceinline__ T tcbrt(T a);
template <> __device__ __forceinline__ float tcbrt<float>(float a) { return cbrtf(a); }
template <> __device__ __forceinline__ double tcbrt<double>(double a) { return newton_cbrt(a); }
template <typename T> __device__ __forceinline__ T tabs(T a) { return fabs(a); }

// Limit of a plane (Eq. 2-3) at the interface centre of face f:
// 0 east (+x), 1 west, 2 north (+y), 3 south.
template <typename T>
__device__ __forceinline__ T face_value(T c0, T c1x, T c1y, int f) {
  const T s3 = s3v<T>();
  switch (f) {
    case 0: return c0 + s3 * c1x;
    case 1: return c0 - s3 * c1x;
    case 2: return c0 + s3 * c1y;
    default: return c0 - s3 * c1y;
  }
}

// One side of an interface after the wet/dry, well-balanced revision:
// interface bed zf = max of the two sides' beds, revised depth
// h* = eta - zf where that exceeds h_dry, else 0 (dry for flux and source
// alike), the bed the source term sees (zf on a wet face, eta on a dry one,
// so h* + z' = eta), and velocities from the unrevised limit (zero when it is
// not wetter than h_dry).
template <typename T>
struct Side {
  T hs, u, v, zr;
};

// depth-form limit (h, qx, qy, z)
template <typename T>
__device__ __forceinline__ Side<T> revise_h(T h, T qx, T qy, T z, T zf, T hd) {
  Side<T> s;
  T eta = h + z;
  T d = eta - zf;
  if (d > hd) {
    s.hs = d;
    s.zr = zf;
  } else {
    s.hs = T(0);
    s.zr = eta;
  }
  if (h > hd) {
    s.u = qx / h;
    s.v = qy / h;
  } else {
    s.u = T(0);
    s.v = T(0);
  }
  return s;
}

// free-surface-form limit (eta, qx, qy, z)
template <typename T>
__device__ __forceinline__ Side<T> revise_eta(T eta, T qx, T qy, T z, T zf, T hd) {
  Side<T> s;
  T h = eta - z;
  T d = eta - zf;
  if (d > hd) {
    s.hs = d;
    s.zr = zf;
  } else {
    s.hs = T(0);
    s.zr = eta;
  }
  if (h > hd) {
    s.u = qx / h;
    s.v = qy / h;
  } else {
    s.u = T(0);
    s.v = T(0);
  }
  return s;
}

// HLL flux in the interface-normal frame (normal velocity un, tangential ut);
// F = (mass, normal momentum, tangential momentum).  Wave speeds are the
// two-rarefaction estimates with the dry-bed forms on a dry side.
template <typename T>
__device__ __forceinline__ void hll(T hL, T unL, T utL, T hR, T unR, T utR, T g, T hd, T F[3]) {
  const bool dryL = !(hL > hd), dryR = !(hR > hd);
  if (dryL && dryR) {
    F[0] = F[1] = F[2] = T(0);
    return;
  }
  const T cL = tsqrt(g * hL), cR = tsqrt(g * hR);
  T sL, sR;
  if (dryL) {
    sL = unR - T(2) * cR;
    sR = unR + cR;
  } else if (dryR) {
    sL = unL - cL;
    sR = unL + T(2) * cL;
  } else {
    const T us = T(0.5) * (unL + unR) + cL - cR;
    const T cs = T(0.5) * (cL + cR) + T(0.25) * (unL - unR);
    sL = tmin(unL - cL, us - cs);
    sR = tmax(unR + cR, us + cs);
  }
  const T qL = hL * unL, qR = hR * unR;
  const T FL0 = qL, FL1 = qL * unL + T(0.5) * g * hL * hL, FL2 = qL * utL;
  const T FR0 = qR, FR1 = qR * unR + T(0.5) * g * hR * hR, FR2 = qR * utR;
  if (sL >= T(0)) {
    F[0] = FL0; F[1] = FL1; F[2] = FL2;
  } else if (sR <= T(0)) {
    F[0] = FR0; F[1] = FR1; F[2] = FR2;
  } else {
    const T UL1 = qL, UL2 = hL * utL, UR1 = qR, UR2 = hR * utR;
    const T den = sR - sL;
    F[0] = (sR * FL0 - sL * FR0 + sL * sR * (hR - hL)) / den;
    F[1] = (sR * FL1 - sL * FR1 + sL * sR * (UR1 - UL1)) / den;
    F[2] = (sR * FL2 - sL * FR2 + sL * sR * (UR2 - UL2)) / den;
  }
}

// Outflow limited by content (Sect. 2.1.1: the wet/dry treatment keeps
// depths non-negative).  The donor leaf's content h0 dx^2 is split among its
// four interfaces in proportion to e_f = max(0, outward average velocity
// through f) + sqrt(g h0), and the volume that leaves through one interface
// during a forward-Euler stage of length dt is limited to its share: the
// draining time step of Bollermann, Chen, Kurganov & Noelle (2013), applied
// per interface so that both sides of an interface evaluate the same limit.
// F (per unit length, along +x or +y; F0 > 0 means the donor is the west or
// south side) is scaled as a whole so that |F0| dt <= share * h0 dx.  The
// donor is given by its flux-view averages: depth h0, discharge qn normal to
// the interface (along +x or +y) and qt along it.  A donor without content
// passes nothing.
template <typename T>
__device__ __forceinline__ void drain_limit(T &F0, T &F1, T &F2, T h0, T qn, T qt, T g, T hd, T dx, T dt) {
  if (!(h0 > T(0))) {
    F0 = F1 = F2 = T(0);
    return;
  }
  T un = T(0), ut = T(0);
  if (h0 > hd) {
    un = qn / h0;
    ut = qt / h0;
  }
  const T c = tsqrt(g * h0);
  const T out = F0 > T(0) ? un : -un;
  const T e = tmax(out, T(0)) + c;
  const T S = (tabs(un) + tabs(ut)) + T(4) * c;
  const T cap = (h0 * dx / dt) * (e / S);
  const T a = tabs(F0);
  if (a > cap) {
    const T th = cap / a;
    F0 = F0 > T(0) ? cap : -cap;
    F1 = F1 * th;
    F2 = F2 * th;
  }
}

template <typename T>
__device__ __forceinline__ T minmod2(T a, T b) {
  if (a > T(0) && b > T(0)) return tmin(a, b);
  if (a < T(0) && b < T(0)) return tmax(a, b);
  return T(0);
}

template <typename T>
__device__ __forceinline__ T minmod3(T a, T b, T c) {
  if (a > T(0) && b > T(0) && c > T(0)) return tmin(a, tmin(b, c));
  if (a < T(0) && b < T(0) && c < T(0)) return tmax(a, tmax(b, c));
  return T(0);
}

// ---------------------------------------------------------------------------
// Multiwavelet filters (Eq. 9-10) for one variable's three coefficients.
// Children c = ix + 2 iy; sigma_x = +-1 is the sign of the child centre's x
// offset.  Low pass: parent = 1/4 sum_c A_c child_c with
//   A_c = [[1,0,0],[sqrt3/2 sx, 1/2, 0],[sqrt3/2 sy, 0, 1/2]].
// High pass (orthonormal completion of the parent rows, Haar patterns H =
// sign(y), V = sign(x), D = product on each child basis function):
//   d_H = sum_c (sy/4 s0 - sqrt3/4 s1y, sy/2 s1x, sy/2 s1y)
//   d_V = sum_c (sx/4 s0 - sqrt3/4 s1x, sx/2 s1x, sx/2 s1y)
//   d_D = sum_c (sx sy/2 s0, sx sy/2 s1x, sx sy/2 s1y)
// ---------------------------------------------------------------------------
// Haar wavelets (HWFV1): the parent average and the largest of the three
// orthonormal Haar details (west-east, south-north, diagonal) of four child
// averages (child c = ix + 2 iy)
template <typename T>
__device__ __forceinline__ T haar_avg(T s0, T s1, T s2, T s3) {
  return T(0.25) * (((s0 + s1) + s2) + s3);
}
template <typename T>
__device__ __forceinline__ T haar_detail_max(T s0, T s1, T s2, T s3) {
  const T dx = T(0.5) * (((-s0 + s1) - s2) + s3);
  const T dy = T(0.5) * (((-s0 - s1) + s2) + s3);
  const T dd = T(0.5) * (((s0 - s1) - s2) + s3);
  return tmax(tabs(dx), tmax(tabs(dy), tabs(dd)));
}

template <typename T>
__device__ __forceinline__ void encode3(const T (&ch)[4][3], T sp[3]) {
  const T hs3 = T(0.5) * s3v<T>();
  T a0 = ch[0][0];
  a0 = a0 + ch[1][0];
  a0 = a0 + ch[2][0];
  a0 = a0 + ch[3][0];
  T a1 = T(0), a2 = T(0);
#pragma unroll
  for (int c = 0; c < 4; c++) {
    const T sx = (c & 1) ? hs3 : -hs3, sy = (c & 2) ? hs3 : -hs3;
    a1 = a1 + sx * ch[c][0];
    a1 = a1 + T(0.5) * ch[c][1];
    a2 = a2 + sy * ch[c][0];
    a2 = a2 + T(0.5) * ch[c][2];
  }
  sp[0] = T(0.25) * a0;
  sp[1] = T(0.25) * a1;
  sp[2] = T(0.25) * a2;
}

// largest |detail| of one variable over the nine details
template <typename T>
__device__ __forceinline__ T detail_max3(const T (&ch)[4][3]) {
  const T q3 = T(0.25) * s3v<T>();
  T dH0 = 0, dH1 = 0, dH2 = 0, dV0 = 0, dV1 = 0, dV2 = 0, dD0 = 0, dD1 = 0, dD2 = 0;
#pragma unroll
  for (int c = 0; c < 4; c++) {
    const T sx = (c & 1) ? T(1) : T(-1), sy = (c & 2) ? T(1) : T(-1);
    dH0 += T(0.25) * sy * ch[c][0] - q3 * ch[c][2];
    dH1 += T(0.5) * sy * ch[c][1];
    dH2 += T(0.5) * sy * ch[c][2];
    dV0 += T(0.25) * sx * ch[c][0] - q3 * ch[c][1];
    dV1 += T(0.5) * sx * ch[c][1];
    dV2 += T(0.5) * sx * ch[c][2];
    dD0 += T(0.5) * sx * sy * ch[c][0];
    dD1 += T(0.5) * sx * sy * ch[c][1];
    dD2 += T(0.5) * sx * sy * ch[c][2];
  }
  T m = tabs(dH0);
  m = tmax(m, tabs(dH1));
  m = tmax(m, tabs(dH2));
  m = tmax(m, tabs(dV0));
  m = tmax(m, tabs(dV1));
  m = tmax(m, tabs(dV2));
  m = tmax(m, tabs(dD0));
  m = tmax(m, tabs(dD1));
  m = tmax(m, tabs(dD2));
  return m;
}

// prolongation of a plane to child c (Eq. 10 with zero details)
template <typename T>
__device__ __forceinline__ void prolong3(T s0, T s1x, T s1y, int c, T out[3]) {
  const T hs3 = T(0.5) * s3v<T>();
  const T ax = (c & 1) ? hs3 : -hs3, ay = (c & 2) ? hs3 : -hs3;
  out[0] = (s0 + ax * s1x) + ay * s1y;
  out[1] = T(0.5) * s1x;
  out[2] = T(0.5) * s1y;
}

}  // namespace mwdg
