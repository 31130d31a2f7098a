/*
 * FP64 CPU oracle for the DG2 / multiwavelet-MRA flood solvers of
 * Sharifian & Kesserwani, "Benchmarking (multi)wavelet-based dynamic and
 * static non-uniform grid solvers for flood inundation modelling"
 * (arXiv 2107.02750).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product library
 * never links, calls or falls back to it, and it shares no code, header or
 * table with the CUDA sources.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC (no FMA
 * contraction, so every expression rounds exactly as written).
 *
 * Everything is written per element, in the order of the paper:
 *   Sect. 2.1.1 / Eq. 1-4   DG2 shallow-water operator and RK2 step
 *   Sect. 2.1.4 / Eq. 8     projection of vertex rasters on the planar basis
 *   Sect. 2.2   / Eq. 9-10  multiwavelet encode / decode, normalised details,
 *                           threshold, parent closure
 *   Sect. 2.2.1             non-homogeneous interfaces, grading (Fig. 2b)
 *   Sect. 2.3               adaptive MWDG2 (MRA each step, local encoding of
 *                           finer elements at non-homogeneous interfaces)
 * The paper delegates the DG2 operator details (HLL, wet/dry revisions,
 * friction, limiter, filter entries) to cited works; the readings used here
 * are listed beside each function.  The wet/dry treatment keeps depths
 * non-negative, as Sect. 2.1.1 states it does, by limiting each interface's
 * outflow to the donor leaf's share of its content (drain_limit); pinned by
 * non-negative depths and a closed mass budget on the rapid-flow valley and
 * a dam break over a steep dry slope, and by a mound drained in one stage.  Friction is pinned by the exact decay
 * of a uniform flow and the limiter by hand-evaluated minmod cases.  The
 * non-homogeneous interface rule is pinned on planar data, where each
 * leaf's stage equals the uniform grid's of the leaf's level (views of a
 * plane are exact); with a plane's details zero, that fixes which views and
 * faces the rule uses but not its arithmetic on non-planar data beyond the
 * invariants (lake at rest, mass budget).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LMAX 14

enum { ORC_UNIFORM = 0, ORC_STATIC = 1, ORC_ADAPTIVE = 2 };
enum { ORC_WALL = 0, ORC_OPEN = 1 };
enum { K_BELOW = 0, K_LEAF = 1, K_SIG = 2 };

/* Parameters (SI units).  Edges: 0 west, 1 east, 2 south, 3 north. */
typedef struct {
  int32_t M, N, L;        /* coarsest grid M x N, maximum level L (Sect. 2.2) */
  int32_t mode;           /* uniform / static non-uniform / adaptive MWDG2   */
  double R;               /* finest resolution (cell size) in metres         */
  double eps;             /* MRA threshold epsilon (Sect. 2.2)               */
  double cfl;             /* Courant number, 0.33 for DG2 (Sect. 2.1.1)      */
  double g;               /* gravity                                         */
  double h_dry;           /* dry-depth tolerance                             */
  double dt_max;          /* upper bound on dt                               */
  int32_t limiter;        /* 0 off, 1 minmod                                 */
  int32_t bc[4];          /* wall / open per edge                            */
  int32_t inflow_edge;    /* -1: none                                        */
  int32_t inflow_c0, inflow_c1; /* finest cell range along the edge, incl.   */
  double rain_rate;       /* m/s                                             */
  double rain_t_end;      /* s                                               */
  int32_t iface_rule;     /* static grids: 0 each side from its own view,    */
                          /* 1 coarse side takes the mean fine flux (reflux) */
  int32_t scheme;         /* 0 DG2 (Sect. 2.1.1), 1 FV1 (Sect. 2.1.2; with   */
                          /* the adaptive mode HWFV1, Sect. 2.3), 2 ACC      */
                          /* (Sect. 2.1.3; uniform and static grids)         */
} orc_params;

typedef struct {
  orc_params p;
  int L;                   /* number of levels - 1 actually stored           */
  int M, N;                /* coarsest grid actually stored                  */
  int nx[ORC_LMAX + 1], ny[ORC_LMAX + 1];
  double dx[ORC_LMAX + 1];
  double *U[ORC_LMAX + 1];   /* 9 coefficients per node (h, qx, qy) x (0,1x,1y) */
  double *z[ORC_LMAX + 1];   /* 3 coefficients per node, full static pyramid */
  double *nm[ORC_LMAX + 1];  /* Manning n per node (averages)                */
  double *dz[ORC_LMAX + 1];  /* normalised topography detail per node        */
  uint8_t *kind[ORC_LMAX + 1];
  /* work arrays */
  double *Wn[ORC_LMAX + 1], *Wi[ORC_LMAX + 1], *Ui[ORC_LMAX + 1];
  double *V[ORC_LMAX + 1], *Vz[ORC_LMAX + 1], *Ze[ORC_LMAX + 1], *F[ORC_LMAX + 1];
  double *D[ORC_LMAX + 1];   /* 27 flow details per node (adaptive)          */
  double *eta_init;          /* finest free-surface coefficients, or NULL    */
  uint8_t *flag[ORC_LMAX + 1];
  int n_knots;
  double *knot_t, *knot_Q;
  double t;
  int64_t steps;
  int64_t n_clip;
  double v_clip, v_in, v_out, v_rain;
  double last_dt;
} orc_sim;

/* Cube root by Newton's method on y^3 = x, seeded by dividing the exponent
 * field of x by three (W. Kahan, "Computing a real cube root", 1991): the
 * seed is within a few per cent, six iterations of
 * y <- y - (y^3 - x) / (3 y^2) reach the rounding level.  Used for the
 * friction depth power h^(4/3) and the critical depth; written out with
 * basic operations only, so the result does not depend on a math library. */
static double cube_root(double x) {
  if (x == 0.0 || x != x) return x;
  double sgn = 1.0, scale = 1.0;
  if (x < 0.0) { x = -x; sgn = -1.0; }
  if (x < 1e-290) { x = x * 0x1p300; scale = 0x1p-100; }
  uint64_t b;
  memcpy(&b, &x, sizeof b);
  b = b / 3u + ((uint64_t)682 << 52);
  double y;
  memcpy(&y, &b, sizeof y);
  for (int it = 0; it < 6; it++) y = y - (y * y * y - x) / (3.0 * y * y);
  return sgn * scale * y;
}

/* ------------------------------------------------------------------------ */
/* Basis and filters                                                         */
/* ------------------------------------------------------------------------ */

/* sqrt(3): the scaled Legendre basis is [1, 2 sqrt3 (x-xc)/R, 2 sqrt3 (y-yc)/R]
 * (Eq. 2-3), so the limit of a plane at an interface centre is
 * v0 +- sqrt3 v1.                                                          */
static double S3(void) { return sqrt(3.0); }

/* Child numbering c = ix + 2 iy (0 SW, 1 SE, 2 NW, 3 NE); sigma = +-1 is the
 * sign of the child centre offset from the parent centre.  The paper's
 * numbering (Eq. 9) pairs child [1] with HH^2 and child [2] with HH^1; that
 * is a relabelling of the same four children. */
static int sgx(int c) { return (c & 1) ? 1 : -1; }
static int sgy(int c) { return (c & 2) ? 1 : -1; }

/* Low-pass filter A_c (3x3): the parent coefficients of a field that is
 * planar on child c, with average-normalised coefficients:
 *   parent = 1/4 sum_c A_c child_c                                (Eq. 9a)
 * Derived from projecting the child plane on the parent basis: on child c
 * the parent slope function 2 sqrt3 x equals 1/2 (child slope function)
 * + sqrt3/2 sigma_x. */
void orc_lowpass(int c, double A[3][3]) {
  double s3 = S3();
  A[0][0] = 1.0; A[0][1] = 0.0; A[0][2] = 0.0;
  A[1][0] = 0.5 * s3 * sgx(c); A[1][1] = 0.5; A[1][2] = 0.0;
  A[2][0] = 0.5 * s3 * sgy(c); A[2][1] = 0.0; A[2][2] = 0.5;
}

/* Symmetric Jacobi eigen-decomposition of a small matrix (n <= 12). */
static void jacobi_eig(int n, double *a /* n*n, destroyed */, double *vec, double *val) {
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) vec[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0.0;
    for (int i = 0; i < n; i++)
      for (int j = i + 1; j < n; j++) off += a[i * n + j] * a[i * n + j];
    if (off < 1e-30) break;
    for (int p = 0; p < n; p++)
      for (int q = p + 1; q < n; q++) {
        double apq = a[p * n + q];
        if (fabs(apq) < 1e-300) continue;
        double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; k++) {
          double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = cs * akp - sn * akq;
          a[k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; k++) {
          double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = cs * apk - sn * aqk;
          a[q * n + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; k++) {
          double vkp = vec[k * n + p], vkq = vec[k * n + q];
          vec[k * n + p] = cs * vkp - sn * vkq;
          vec[k * n + q] = sn * vkp + cs * vkq;
        }
      }
  }
  for (int i = 0; i < n; i++) val[i] = a[i * n + i];
}

/* High-pass filters G_c (9x3 per child): the entries are not printed in the
 * paper (Sect. 2.2, "generated from the MWs decomposition of the basis").
 * Reading: in the 12-dimensional space of piecewise-planar functions on the
 * four children, with coordinates a_c = s_c / 2 (orthonormal for the
 * parent-averaged inner product), the parent rows are 1/2 A_c.  For each
 * Haar pattern P in (H: sign(y), V: sign(x), D: sign(x)sign(y)) and each
 * child basis function b in (1, slope x, slope y) take P*b, remove its
 * projection on the parent rows, then orthonormalise the nine vectors
 * symmetrically (Loewdin, (R R^T)^(-1/2) R).  Details are then scaled to the
 * average-normalised convention d = sum_c G_c s_c, so that decoding is
 * s_c = A_c^T parent + G_c^T d (Eq. 10).
 * Detail row order: 3*p + m with p = H,V,D and m = (1, x, y).             */
void orc_highpass(double G[4][9][3]) {
  double par[3][12], r[9][12];
  for (int c = 0; c < 4; c++) {
    double A[3][3];
    orc_lowpass(c, A);
    for (int k = 0; k < 3; k++)
      for (int m = 0; m < 3; m++) par[k][3 * c + m] = 0.5 * A[k][m];
  }
  for (int p = 0; p < 3; p++)
    for (int m = 0; m < 3; m++)
      for (int c = 0; c < 4; c++)
        for (int mm = 0; mm < 3; mm++) {
          double pat = (p == 0) ? sgy(c) : (p == 1) ? sgx(c) : sgx(c) * sgy(c);
          r[3 * p + m][3 * c + mm] = (mm == m) ? pat : 0.0;
        }
  /* remove the parent component */
  for (int i = 0; i < 9; i++)
    for (int k = 0; k < 3; k++) {
      double dot = 0.0;
      for (int e = 0; e < 12; e++) dot += r[i][e] * par[k][e];
      for (int e = 0; e < 12; e++) r[i][e] -= dot * par[k][e];
    }
  /* Loewdin: G = (R R^T)^{-1/2} R */
  double S[81], vec[81], val[9], Sm[81];
  for (int i = 0; i < 9; i++)
    for (int j = 0; j < 9; j++) {
      double dot = 0.0;
      for (int e = 0; e < 12; e++) dot += r[i][e] * r[j][e];
      S[i * 9 + j] = dot;
    }
  jacobi_eig(9, S, vec, val);
  for (int i = 0; i < 9; i++)
    for (int j = 0; j < 9; j++) {
      double acc = 0.0;
      for (int k = 0; k < 9; k++) acc += vec[i * 9 + k] * vec[j * 9 + k] / sqrt(val[k]);
      Sm[i * 9 + j] = acc;
    }
  for (int i = 0; i < 9; i++)
    for (int c = 0; c < 4; c++)
      for (int m = 0; m < 3; m++) {
        double acc = 0.0;
        for (int k = 0; k < 9; k++) acc += Sm[i * 9 + k] * r[k][3 * c + m];
        /* orthonormal coordinates use a_c = s_c/2, so d = sum_c (2 g_c) (s_c/2) */
        G[c][i][m] = acc;
      }
}

/* Filters are derived once and cached. */
static double gA[4][3][3], gG[4][9][3];
static int g_filters_ready = 0;
static void ensure_filters(void) {
  if (g_filters_ready) return;
  for (int c = 0; c < 4; c++) orc_lowpass(c, gA[c]);
  orc_highpass(gG);
  g_filters_ready = 1;
}

/* Export of the filters (HH_c = A_c/4 is what multiplies the child in
 * Eq. 9a; the tests inspect A_c and G_c). */
void orc_filters(double *A /*4*3*3*/, double *G /*4*9*3*/) {
  ensure_filters();
  memcpy(A, gA, sizeof gA);
  memcpy(G, gG, sizeof gG);
}

/* Eq. 9: parent scale coefficients and details of one variable from the
 * four children's coefficients s[c][0..2]. */
void orc_encode_node(const double *s /*4x3*/, double *sp /*3*/, double *d /*9*/) {
  ensure_filters();
  for (int k = 0; k < 3; k++) {
    double acc = 0.0;
    for (int c = 0; c < 4; c++)
      for (int m = 0; m < 3; m++) acc += gA[c][k][m] * s[3 * c + m];
    sp[k] = 0.25 * acc;
  }
  for (int i = 0; i < 9; i++) {
    double acc = 0.0;
    for (int c = 0; c < 4; c++)
      for (int m = 0; m < 3; m++) acc += gG[c][i][m] * s[3 * c + m];
    d[i] = acc;
  }
}

/* Eq. 10: the four children from the parent and its (kept) details. */
void orc_decode_node(const double *sp /*3*/, const double *d /*9 or NULL*/, double *s /*4x3*/) {
  ensure_filters();
  for (int c = 0; c < 4; c++)
    for (int m = 0; m < 3; m++) {
      double acc = 0.0;
      for (int k = 0; k < 3; k++) acc += gA[c][k][m] * sp[k];
      if (d)
        for (int i = 0; i < 9; i++) acc += gG[c][i][m] * d[i];
      s[3 * c + m] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 8: planar coefficients from the four vertex values of each cell.     */
/* vert is (ny+1) x (nx+1), row j = south to north, column i = west to east. */
/* The printed four-vertex form of Eq. 8a has a factor 1/2; the E/W and N/S  */
/* forms on the same line require 1/4, which is used.                        */
/* ------------------------------------------------------------------------ */
/* Haar wavelets (HWFV1, Sect. 2.3): piecewise-constant children s_c (c =
 * ix + 2 iy) -> parent average p = 1/4 sum s_c and three details from the
 * orthonormal Haar transform (rows 1/2 (+-1, ...)): d_x (west-east),
 * d_y (south-north), d_xy; decode s_c = p + 1/2 (sx d_x + sy d_y + sx sy d_xy)
 * with sx, sy = -1 / +1 on the west / east and south / north children. */
void orc_haar_encode(const double *sc /*4*/, double *p, double *d /*3*/) {
  *p = 0.25 * (sc[0] + sc[1] + sc[2] + sc[3]);
  d[0] = 0.5 * (-sc[0] + sc[1] - sc[2] + sc[3]);
  d[1] = 0.5 * (-sc[0] - sc[1] + sc[2] + sc[3]);
  d[2] = 0.5 * (sc[0] - sc[1] - sc[2] + sc[3]);
}

void orc_haar_decode(double p, const double *d /*3*/, double *sc /*4*/) {
  for (int c = 0; c < 4; c++) {
    double sx = (c & 1) ? 1.0 : -1.0, sy = (c & 2) ? 1.0 : -1.0;
    sc[c] = p + 0.5 * (sx * d[0] + sy * d[1] + sx * sy * d[2]);
  }
}

void orc_project(const double *vert, int nx, int ny, double *c0, double *c1x, double *c1y) {
  double s3 = S3();
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      double sw = vert[(size_t)j * (nx + 1) + i], se = vert[(size_t)j * (nx + 1) + i + 1];
      double nw = vert[(size_t)(j + 1) * (nx + 1) + i], ne = vert[(size_t)(j + 1) * (nx + 1) + i + 1];
      double zn = 0.5 * (nw + ne), zs = 0.5 * (sw + se);
      double ze = 0.5 * (ne + se), zw = 0.5 * (nw + sw);
      size_t k = (size_t)j * nx + i;
      c0[k] = 0.5 * (ze + zw);
      c1x[k] = (ze - zw) / (2.0 * s3);
      c1y[k] = (zn - zs) / (2.0 * s3);
    }
}

/* ------------------------------------------------------------------------ */
/* Simulation object                                                         */
/* ------------------------------------------------------------------------ */
static size_t nn(const orc_sim *s, int l) { return (size_t)s->nx[l] * s->ny[l]; }
static size_t id(const orc_sim *s, int l, int i, int j) { return (size_t)j * s->nx[l] + i; }

orc_sim *orc_create(const orc_params *p) {
  orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
  s->p = *p;
  if (p->mode == ORC_UNIFORM) {
    /* a uniform grid is the single level of an L = 0 hierarchy */
    s->L = 0;
    s->M = p->M << p->L;
    s->N = p->N << p->L;
  } else {
    s->L = p->L;
    s->M = p->M;
    s->N = p->N;
  }
  for (int l = 0; l <= s->L; l++) {
    s->nx[l] = s->M << l;
    s->ny[l] = s->N << l;
    s->dx[l] = p->R * (double)(1 << (s->L - l));
    size_t n = nn(s, l);
    s->U[l] = calloc(9 * n, sizeof(double));
    s->z[l] = calloc(3 * n, sizeof(double));
    s->nm[l] = calloc(n, sizeof(double));
    s->dz[l] = calloc(n, sizeof(double));
    s->kind[l] = calloc(n, 1);
    s->Wn[l] = calloc(9 * n, sizeof(double));
    s->Wi[l] = calloc(9 * n, sizeof(double));
    s->Ui[l] = calloc(9 * n, sizeof(double));
    s->V[l] = calloc(9 * n, sizeof(double));
    s->Vz[l] = calloc(3 * n, sizeof(double));
    s->Ze[l] = calloc(3 * n, sizeof(double));
    s->F[l] = calloc(9 * n, sizeof(double));
    s->D[l] = calloc(27 * n, sizeof(double));
    s->flag[l] = calloc(n, 1);
  }
  ensure_filters();
  return s;
}

void orc_destroy(orc_sim *s) {
  if (!s) return;
  for (int l = 0; l <= s->L; l++) {
    free(s->U[l]); free(s->z[l]); free(s->nm[l]); free(s->dz[l]); free(s->kind[l]);
    free(s->Wn[l]); free(s->Wi[l]); free(s->Ui[l]); free(s->V[l]); free(s->Vz[l]); free(s->Ze[l]); free(s->F[l]);
    free(s->D[l]); free(s->flag[l]);
  }
  free(s->knot_t); free(s->knot_Q); free(s->eta_init);
  free(s);
}

int orc_levels(const orc_sim *s) { return s->L; }

/* Topography: Eq. 8 on the finest level, then the full static pyramid by
 * Eq. 9 and the normalised topography detail of every node (Sect. 2.2):
 * max |d| over the nine details, divided by max(1, max |z0| at level L). */
void orc_load_dem(orc_sim *s, const double *vert) {
  int L = s->L;
  size_t n = nn(s, L);
  orc_project(vert, s->nx[L], s->ny[L], s->z[L], s->z[L] + n, s->z[L] + 2 * n);
  double zmax = 0.0;
  for (size_t k = 0; k < n; k++) zmax = fmax(zmax, fabs(s->z[L][k]));
  double norm = fmax(1.0, zmax);
  for (int l = L - 1; l >= 0; l--) {
    size_t nl = nn(s, l), nf = nn(s, l + 1);
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        double ch[12], sp[3], d[9];
        for (int c = 0; c < 4; c++) {
          size_t kc = id(s, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
          for (int m = 0; m < 3; m++) ch[3 * c + m] = s->z[l + 1][m * nf + kc];
        }
        orc_encode_node(ch, sp, d);
        size_t k = id(s, l, i, j);
        for (int m = 0; m < 3; m++) s->z[l][m * nl + k] = sp[m];
        double dm = 0.0;
        for (int q = 0; q < 9; q++) dm = fmax(dm, fabs(d[q]));
        s->dz[l][k] = dm / norm;
      }
  }
  if (s->p.scheme == 1 || s->p.scheme == 2) {
    /* FV1 and ACC see the bed as one level per element (Eq. 6): the pyramid keeps
     * the averages (the multiwavelet average is the children's mean) and
     * drops the slopes.  The static grid keeps the multiwavelet details of
     * the planar topography (Sect. 2.2); HWFV1 thresholds Haar details of
     * the piecewise-constant bed (Sect. 2.3). */
    if (s->p.mode == ORC_ADAPTIVE && s->p.scheme == 1)
      for (int l = L - 1; l >= 0; l--)
        for (int j = 0; j < s->ny[l]; j++)
          for (int i = 0; i < s->nx[l]; i++) {
            double a[4], pa, d[3];
            for (int c = 0; c < 4; c++) a[c] = s->z[l + 1][id(s, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1))];
            orc_haar_encode(a, &pa, d);
            s->dz[l][id(s, l, i, j)] = fmax(fabs(d[0]), fmax(fabs(d[1]), fabs(d[2]))) / norm;
          }
    for (int l = 0; l <= L; l++) {
      size_t nl = nn(s, l);
      for (size_t k = 0; k < nl; k++) s->z[l][nl + k] = s->z[l][2 * nl + k] = 0.0;
    }
  }
}

/* Manning n on the finest cells; coarser nodes hold the mean of their
 * children. */
void orc_load_roughness(orc_sim *s, const double *n_cell) {
  int L = s->L;
  memcpy(s->nm[L], n_cell, nn(s, L) * sizeof(double));
  for (int l = L - 1; l >= 0; l--)
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        double acc = 0.0;
        for (int c = 0; c < 4; c++) acc += s->nm[l + 1][id(s, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1))];
        s->nm[l][id(s, l, i, j)] = 0.25 * acc;
      }
}

void orc_set_inflow(orc_sim *s, int n, const double *t, const double *Q) {
  free(s->knot_t); free(s->knot_Q);
  s->n_knots = n;
  s->knot_t = malloc(n * sizeof(double));
  s->knot_Q = malloc(n * sizeof(double));
  memcpy(s->knot_t, t, n * sizeof(double));
  memcpy(s->knot_Q, Q, n * sizeof(double));
}

/* piecewise-linear hydrograph, held constant outside the knots */
static double inflow_Q(const orc_sim *s, double t) {
  int n = s->n_knots;
  if (n <= 0) return 0.0;
  if (t <= s->knot_t[0]) return s->knot_Q[0];
  if (t >= s->knot_t[n - 1]) return s->knot_Q[n - 1];
  int k = 0;
  while (k + 1 < n && !(t < s->knot_t[k + 1])) k++;
  double tk = s->knot_t[k], tk1 = s->knot_t[k + 1], Qk = s->knot_Q[k], Qk1 = s->knot_Q[k + 1];
  return Qk + (Qk1 - Qk) * (t - tk) / (tk1 - tk);
}

/* encode/decode of one variable's node from its children (4 x 3 coefficients):
 * DG2 multiwavelets (Eq. 9, 10), or for FV1 Haar wavelets on the averages
 * (slopes stay zero; the details beyond the three Haar ones are zero) */
static void encode_node_scheme(const orc_sim *s, const double *ch /*4x3*/, double *sp /*3*/, double *d /*9*/) {
  if (s->p.scheme != 1) {
    orc_encode_node(ch, sp, d);
    return;
  }
  double a[4] = {ch[0], ch[3], ch[6], ch[9]};
  for (int q = 0; q < 9; q++) d[q] = 0.0;
  orc_haar_encode(a, &sp[0], d);
  sp[1] = sp[2] = 0.0;
}

static void decode_node_scheme(const orc_sim *s, const double *sp, const double *d, double *ch /*4x3*/) {
  if (s->p.scheme != 1) {
    orc_decode_node(sp, d, ch);
    return;
  }
  double a[4];
  orc_haar_decode(sp[0], d, a);
  for (int c = 0; c < 4; c++) {
    ch[3 * c] = a[c];
    ch[3 * c + 1] = ch[3 * c + 2] = 0.0;
  }
}

/* full encode of the 9 flow coefficients from level `from` down to 0, all
 * nodes; details of every node are stored when D != NULL */
static void encode_flow_all(orc_sim *s, double **X, int from, int store_details) {
  for (int l = from - 1; l >= 0; l--) {
    size_t nl = nn(s, l), nf = nn(s, l + 1);
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        for (int v = 0; v < 3; v++) {
          double ch[12], sp[3], d[9];
          for (int c = 0; c < 4; c++) {
            size_t kc = id(s, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
            for (int m = 0; m < 3; m++) ch[3 * c + m] = X[l + 1][(3 * v + m) * nf + kc];
          }
          encode_node_scheme(s, ch, sp, d);
          for (int m = 0; m < 3; m++) X[l][(3 * v + m) * nl + k] = sp[m];
          if (store_details)
            for (int q = 0; q < 9; q++) s->D[l][(9 * v + q) * nl + k] = d[q];
        }
      }
  }
}

/* Initial condition: vertex rasters of h (or eta = h + z), qx, qy at the
 * finest level, projected by Eq. 8 (Sect. 2.1.4).  With is_eta, cells whose
 * average eta does not exceed z0 start dry (h = q = 0); elsewhere
 * h = eta - z coefficient-wise. */
void orc_load_initial(orc_sim *s, const double *hv, const double *qxv, const double *qyv, int is_eta) {
  int L = s->L;
  size_t n = nn(s, L);
  double *U = s->U[L];
  orc_project(hv, s->nx[L], s->ny[L], U, U + n, U + 2 * n);
  orc_project(qxv, s->nx[L], s->ny[L], U + 3 * n, U + 4 * n, U + 5 * n);
  orc_project(qyv, s->nx[L], s->ny[L], U + 6 * n, U + 7 * n, U + 8 * n);
  free(s->eta_init);
  s->eta_init = NULL;
  if (is_eta) {
    s->eta_init = malloc(3 * n * sizeof(double));
    memcpy(s->eta_init, U, 3 * n * sizeof(double));
    for (size_t k = 0; k < n; k++) {
      double eta0 = U[k], eta1x = U[n + k], eta1y = U[2 * n + k];
      if (eta0 > s->z[L][k]) {
        U[k] = eta0 - s->z[L][k];
        U[n + k] = eta1x - s->z[L][n + k];
        U[2 * n + k] = eta1y - s->z[L][2 * n + k];
      } else {
        for (int m = 0; m < 9; m++) U[m * n + k] = 0.0;
      }
    }
  }
  if (s->p.scheme == 1 || s->p.scheme == 2)  /* FV1, ACC: averages only (Eq. 5) */
    for (size_t k = 0; k < n; k++)
      for (int v = 0; v < 3; v++) U[(3 * v + 1) * n + k] = U[(3 * v + 2) * n + k] = 0.0;
  if (s->p.scheme == 2)  /* ACC: face discharges start at zero */
    for (int l = 0; l <= L; l++) memset(s->Wi[l], 0, 4 * nn(s, l) * sizeof(double));
  s->t = 0.0;
  s->steps = 0;
  s->n_clip = 0;
  s->v_clip = s->v_in = s->v_out = s->v_rain = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Grid generation (Sect. 2.2 and 2.2.1)                                     */
/* ------------------------------------------------------------------------ */
static int in_dom(const orc_sim *s, int l, int i, int j) {
  return i >= 0 && j >= 0 && i < s->nx[l] && j < s->ny[l];
}

/* parent closure: a flagged child flags all its ancestors (Sect. 2.2) */
static void closure(orc_sim *s) {
  for (int l = s->L - 1; l >= 1; l--)
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++)
        if (s->flag[l][id(s, l, i, j)]) s->flag[l - 1][id(s, l - 1, i / 2, j / 2)] = 1;
}

/* 2:1 grading (Sect. 2.2.1, Fig. 2b): every face neighbour of a flagged
 * node must itself exist, i.e. have a flagged parent; repeated with closure
 * until nothing changes. */
static void grading(orc_sim *s) {
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int l = s->L - 1; l >= 1; l--)
      for (int j = 0; j < s->ny[l]; j++)
        for (int i = 0; i < s->nx[l]; i++) {
          if (!s->flag[l][id(s, l, i, j)]) continue;
          static const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
          for (int f = 0; f < 4; f++) {
            int a = i + di[f], b = j + dj[f];
            if (!in_dom(s, l, a, b)) continue;
            size_t kp = id(s, l - 1, a / 2, b / 2);
            if (!s->flag[l - 1][kp]) {
              s->flag[l - 1][kp] = 1;
              changed = 1;
            }
          }
        }
    closure(s);
  }
}

/* kinds from flags: a flagged node is refined (SIG); a node whose parent is
 * refined (or that is a root) and that is not refined is an active leaf. */
static void kinds_from_flags(orc_sim *s) {
  for (int l = 0; l <= s->L; l++)
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        int f = (l < s->L) ? s->flag[l][k] : 0;
        int parent_sig = (l == 0) ? 1 : (s->kind[l - 1][id(s, l - 1, i / 2, j / 2)] == K_SIG);
        s->kind[l][k] = f ? K_SIG : (parent_sig ? K_LEAF : K_BELOW);
      }
}

/* Builds the starting grid: uniform (one level), static (MRA once on the
 * topography, closure, grading) or adaptive (all finest elements active;
 * the first step adapts).  Flow coefficients of every node are the encoded
 * finest coefficients. */
void orc_init_grid(orc_sim *s) {
  int L = s->L;
  if (s->p.mode == ORC_UNIFORM || L == 0) {
    for (size_t k = 0; k < nn(s, 0); k++) s->kind[0][k] = K_LEAF;
    return;
  }
  encode_flow_all(s, s->U, L, 0);
  for (int l = 0; l <= L; l++) memset(s->flag[l], 0, nn(s, l));
  if (s->p.mode == ORC_STATIC) {
    for (int l = 0; l < L; l++)
      for (size_t k = 0; k < nn(s, l); k++) s->flag[l][k] = (s->dz[l][k] >= s->p.eps);
    closure(s);
    grading(s);
  } else {
    for (int l = 0; l < L; l++) memset(s->flag[l], 1, nn(s, l));
  }
  kinds_from_flags(s);
  if (s->eta_init) {
    /* a free-surface initial state is encoded as eta and split into depth
     * per leaf with the same wet/dry rule as on the finest level, so that a
     * state at rest is at rest on the generated grid too */
    size_t nL = nn(s, L);
    for (int m = 0; m < 3; m++) memcpy(s->V[L] + m * nL, s->eta_init + m * nL, nL * sizeof(double));
    for (int l = L - 1; l >= 0; l--) {
      size_t nl = nn(s, l), nf = nn(s, l + 1);
      for (int j = 0; j < s->ny[l]; j++)
        for (int i = 0; i < s->nx[l]; i++) {
          double ch[12], sp[3], d[9];
          for (int c = 0; c < 4; c++) {
            size_t kc = id(s, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
            for (int m = 0; m < 3; m++) ch[3 * c + m] = s->V[l + 1][m * nf + kc];
          }
          encode_node_scheme(s, ch, sp, d);
          for (int m = 0; m < 3; m++) s->V[l][m * nl + id(s, l, i, j)] = sp[m];
        }
    }
    for (int l = 0; l <= L; l++) {
      size_t n = nn(s, l);
      for (size_t k = 0; k < n; k++) {
        if (s->kind[l][k] != K_LEAF) continue;
        double *U = s->U[l];
        if (s->V[l][k] > s->z[l][k]) {
          for (int m = 0; m < 3; m++) U[m * n + k] = s->V[l][m * n + k] - s->z[l][m * n + k];
          if (s->p.scheme != 0) U[n + k] = U[2 * n + k] = 0.0;
        } else {
          for (int m = 0; m < 9; m++) U[m * n + k] = 0.0;
        }
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* MWDG2 adaptation (Sect. 2.3): encode flow from the uniform level-L view,  */
/* normalise, threshold, predict, close, decode.                             */
/* ------------------------------------------------------------------------ */

/* prolongation of a plane to child c: the decode of Eq. 10 with zero details */
static void prolong_child(const double *sp /*3*/, int c, double *sc /*3*/) {
  for (int m = 0; m < 3; m++) {
    double acc = 0.0;
    for (int k = 0; k < 3; k++) acc += gA[c][k][m] * sp[k];
    sc[m] = acc;
  }
}

/* Positivity of a refined leaf's depth (Sect. 2.1.1 and 2.3: the wet/dry
 * treatment keeps depths non-negative; a leaf stored as a flat free surface
 * over a steep bed, or one with a steep depth plane, would otherwise give
 * children of negative average depth).  Before a depth plane sp is prolonged
 * to its children, its slopes are scaled about its average so that none of
 * the four children's averages is negative: the scaling limiter of Zhang &
 * Shu (2010) applied at the children's centres.  A plane whose children are
 * all non-negative is prolonged as it is; one without content loses its
 * slopes. */
static void depth_plane_for_children(double sp[3]) {
  double m = INFINITY;
  for (int c = 0; c < 4; c++) {
    double sc[3];
    prolong_child(sp, c, sc);
    m = fmin(m, sc[0]);
  }
  if (!(m < 0.0)) return;
  if (sp[0] > 0.0) {
    double th = sp[0] / (sp[0] - m);
    sp[1] = sp[1] * th;
    sp[2] = sp[2] * th;
  } else {
    sp[1] = 0.0;
    sp[2] = 0.0;
  }
}

void orc_adapt(orc_sim *s) {
  int L = s->L;
  if (s->p.mode != ORC_ADAPTIVE || L == 0) return;
  /* normalisation maxima over the current active leaves */
  double mx[3] = {0, 0, 0};
  for (int l = 0; l <= L; l++) {
    size_t n = nn(s, l);
    for (size_t k = 0; k < n; k++)
      if (s->kind[l][k] == K_LEAF)
        for (int v = 0; v < 3; v++) mx[v] = fmax(mx[v], fabs(s->U[l][3 * v * n + k]));
  }
  /* the current solution on the uniform grid at level L: leaves are
   * prolonged down to the finest level */
  for (int l = 1; l <= L; l++) {
    size_t n = nn(s, l), np = nn(s, l - 1);
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        if (s->kind[l][k] != K_BELOW) continue;
        size_t kp = id(s, l - 1, i / 2, j / 2);
        int c = (i & 1) + 2 * (j & 1);
        for (int v = 0; v < 3; v++) {
          double sp[3], sc[3];
          for (int m = 0; m < 3; m++) sp[m] = s->U[l - 1][(3 * v + m) * np + kp];
          if (v == 0) depth_plane_for_children(sp);
          prolong_child(sp, c, sc);
          /* rounding residue of a child brought to zero depth */
          if (v == 0) sc[0] = fmax(sc[0], 0.0);
          for (int m = 0; m < 3; m++) s->U[l][(3 * v + m) * n + k] = sc[m];
        }
      }
  }
  /* Eq. 9 from the leaves upwards, keeping the details: a refined node's
   * scale coefficients and details come from its children's coefficients;
   * a leaf keeps its own, and a node at or below a leaf carries no flow
   * detail (its data are the prolongation of the leaf's plane, whose
   * details vanish) */
  for (int l = L - 1; l >= 0; l--) {
    size_t nl = nn(s, l), nf = nn(s, l + 1);
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        if (s->kind[l][k] != K_SIG) {
          for (int q = 0; q < 27; q++) s->D[l][q * nl + k] = 0.0;
          continue;
        }
        for (int v = 0; v < 3; v++) {
          double ch[12], sp[3], d[9];
          for (int c = 0; c < 4; c++) {
            size_t kc = id(s, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
            for (int m = 0; m < 3; m++) ch[3 * c + m] = s->U[l + 1][(3 * v + m) * nf + kc];
          }
          encode_node_scheme(s, ch, sp, d);
          for (int m = 0; m < 3; m++) s->U[l][(3 * v + m) * nl + k] = sp[m];
          for (int q = 0; q < 9; q++) s->D[l][(9 * v + q) * nl + k] = d[q];
        }
      }
  }
  /* normalised details against epsilon; topography details are static */
  for (int l = 0; l < L; l++) {
    size_t n = nn(s, l);
    for (size_t k = 0; k < n; k++) {
      double dmax = s->dz[l][k];
      for (int v = 0; v < 3; v++) {
        double dm = 0.0;
        for (int q = 0; q < 9; q++) dm = fmax(dm, fabs(s->D[l][(9 * v + q) * n + k]));
        dmax = fmax(dmax, dm / fmax(1.0, mx[v]));
      }
      s->flag[l][k] = (dmax >= s->p.eps);
    }
  }
  /* prediction: a significant node also flags its eight same-level
   * neighbours, so that the tree can follow the flow */
  for (int l = 0; l < L; l++) {
    size_t n = nn(s, l);
    uint8_t *f0 = malloc(n);
    memcpy(f0, s->flag[l], n);
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        if (!f0[id(s, l, i, j)]) continue;
        for (int b = j - 1; b <= j + 1; b++)
          for (int a = i - 1; a <= i + 1; a++)
            if (in_dom(s, l, a, b)) s->flag[l][id(s, l, a, b)] = 1;
      }
    free(f0);
  }
  closure(s);
  kinds_from_flags(s);
  /* Eq. 10: the new leaves' coefficients.  Decoding from level 0 with the
   * kept details reproduces, at every node, the coefficients the encode
   * gave it (Eq. 9 and Eq. 10 are inverse); those are already in place: a
   * leaf that stays keeps its coefficients, a coarsened leaf has its
   * encoded scale coefficients, and a refined leaf the prolongation of its
   * old leaf's plane.  So the decode is taken as that identity, exactly,
   * rather than recomputed with rounding (orc_decode_node states it and the
   * tests pin the round trip). */
}

/* ------------------------------------------------------------------------ */
/* DG2 operator pieces (Sect. 2.1.1)                                         */
/* ------------------------------------------------------------------------ */
static double minmod2(double a, double b) {
  if (a > 0.0 && b > 0.0) return fmin(a, b);
  if (a < 0.0 && b < 0.0) return fmax(a, b);
  return 0.0;
}

static double minmod3(double a, double b, double c) {
  if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
  if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
  return 0.0;
}

/* Revision of one side's limit at an interface (wet/dry, well-balanced):
 * hydrostatic reconstruction with the interface bed z_f = max(z_L, z_R):
 * h* = eta - z_f where that exceeds h_dry, else 0 (a face not wetter than
 * h_dry is dry for the flux and the source alike); the bed seen by the
 * source term is z' = z_f on a wet face and eta on a dry one, so that
 * h* + z' = eta and the pressure and bed-slope terms cancel at rest;
 * velocities come from the unrevised limit (zero when it is not wetter
 * than h_dry). */
static void revise(double h, double qx, double qy, double z, double zf, double hd,
                   double *hs, double *u, double *v, double *zr) {
  double eta = h + z;
  double d = eta - zf;
  if (d > hd) {
    *hs = d;
    *zr = zf;
  } else {
    *hs = 0.0;
    *zr = eta;
  }
  if (h > hd) {
    *u = qx / h;
    *v = qy / h;
  } else {
    *u = 0.0;
    *v = 0.0;
  }
}

/* HLL flux in the interface-normal frame (un normal, ut tangential);
 * F = (mass, normal momentum, tangential momentum).  Wave speeds: two-rarefaction
 * estimate with the dry-bed forms. */
static void hll(double hL, double unL, double utL, double hR, double unR, double utR,
                double g, double hd, double F[3]) {
  int dryL = !(hL > hd), dryR = !(hR > hd);
  if (dryL && dryR) {
    F[0] = F[1] = F[2] = 0.0;
    return;
  }
  double cL = sqrt(g * hL), cR = sqrt(g * hR);
  double sL, sR;
  if (dryL) {
    sL = unR - 2.0 * cR;
    sR = unR + cR;
  } else if (dryR) {
    sL = unL - cL;
    sR = unL + 2.0 * cL;
  } else {
    double us = 0.5 * (unL + unR) + cL - cR;
    double cs = 0.5 * (cL + cR) + 0.25 * (unL - unR);
    sL = fmin(unL - cL, us - cs);
    sR = fmax(unR + cR, us + cs);
  }
  double qL = hL * unL, qR = hR * unR;
  double FL[3] = {qL, qL * unL + 0.5 * g * hL * hL, qL * utL};
  double FR[3] = {qR, qR * unR + 0.5 * g * hR * hR, qR * utR};
  if (sL >= 0.0) {
    F[0] = FL[0]; F[1] = FL[1]; F[2] = FL[2];
  } else if (sR <= 0.0) {
    F[0] = FR[0]; F[1] = FR[1]; F[2] = FR[2];
  } else {
    double UL[3] = {hL, qL, hL * utL}, UR[3] = {hR, qR, hR * utR};
    double den = sR - sL;
    for (int k = 0; k < 3; k++) F[k] = (sR * FL[k] - sL * FR[k] + sL * sR * (UR[k] - UL[k])) / den;
  }
}

/* critical depth of a unit discharge q */
static double crit_depth(double q, double g) { return cube_root(q * q / g); }

/* inflow unit discharge through the boundary face of a leaf (level l, index
 * k along the edge): the hydrograph Q(t) spread over the inflow cells, times
 * the overlap of the face with them */
static double inflow_q(const orc_sim *s, int edge, int l, int k, double t) {
  if (s->p.inflow_edge != edge) return 0.0;
  int sh = s->L - l;
  long a = (long)k << sh, b = (long)(k + 1) << sh;
  long lo = a > s->p.inflow_c0 ? a : s->p.inflow_c0;
  long hi = b < (long)s->p.inflow_c1 + 1 ? b : (long)s->p.inflow_c1 + 1;
  long ov = hi - lo;
  if (ov <= 0) return 0.0;
  long nin = (long)s->p.inflow_c1 - s->p.inflow_c0 + 1;
  return inflow_Q(s, t) * (double)ov / ((double)nin * s->dx[l]);
}

/* ------------------------------------------------------------------------ */
/* Step helpers                                                              */
/* ------------------------------------------------------------------------ */

/* plane limits: face 0 E, 1 W, 2 N, 3 S */
static double face_lim(const double *c /*3 coeffs*/, int f) {
  double s3 = S3();
  switch (f) {
    case 0: return c[0] + s3 * c[1];
    case 1: return c[0] - s3 * c[1];
    case 2: return c[0] + s3 * c[2];
    default: return c[0] - s3 * c[2];
  }
}

static void get9(double *const *X, const orc_sim *s, int l, size_t k, double *w) {
  size_t n = nn(s, l);
  for (int m = 0; m < 9; m++) w[m] = X[l][m * n + k];
}
static void put9(double **X, const orc_sim *s, int l, size_t k, const double *w) {
  size_t n = nn(s, l);
  for (int m = 0; m < 9; m++) X[l][m * n + k] = w[m];
}

/* CFL time step over the active leaves (Courant number p.cfl, Sect. 2.1.1),
 * including the inflow ghost states; bounded by dt_max and t_end - t. */
static double compute_dt(orc_sim *s, double t_end) {
  double g = s->p.g, hd = s->p.h_dry;
  double best = INFINITY;
  for (int l = 0; l <= s->L; l++) {
    size_t n = nn(s, l);
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        if (s->kind[l][k] != K_LEAF) continue;
        double h0 = s->U[l][k];
        double dxl = s->dx[l];
        if (s->p.scheme == 2) {  /* ACC: gravity-wave celerity only (Bates et al. 2010) */
          if (h0 > hd) best = fmin(best, dxl / sqrt(g * h0));
          continue;
        }
        if (h0 > hd) {
          double u = s->U[l][3 * n + k] / h0, v = s->U[l][6 * n + k] / h0;
          double c = sqrt(g * h0);
          best = fmin(best, fmin(dxl / (fabs(u) + c), dxl / (fabs(v) + c)));
        }
        /* inflow ghost at the critical depth */
        for (int e = 0; e < 4; e++) {
          int onedge = (e == 0 && i == 0) || (e == 1 && i == s->nx[l] - 1) || (e == 2 && j == 0) ||
                       (e == 3 && j == s->ny[l] - 1);
          if (!onedge) continue;
          double q = inflow_q(s, e, l, (e < 2) ? j : i, s->t);
          if (q > 0.0) {
            double hc = crit_depth(q, g);
            if (hc > hd) best = fmin(best, dxl / (q / hc + sqrt(g * hc)));
          }
        }
      }
  }
  double dt = s->p.dt_max;
  if (best < INFINITY) dt = fmin(dt, s->p.cfl * best);
  return fmin(dt, t_end - s->t);
}

/* Split implicit friction at the start of a step (Sect. 2.1.1): linearised
 * backward Euler of dq/dt = -g n^2 |u| q / h^(4/3), the same factor on the
 * average and slope coefficients; dry leaves lose their discharge. */
static void friction(double *w, double nman, double dt, double g, double hd) {
  double h0 = w[0];
  if (h0 > hd) {
    double u = w[3] / h0, v = w[6] / h0;
    double sp = sqrt(u * u + v * v);
    double den = 1.0 + dt * g * nman * nman * sp / (h0 * cube_root(h0));
    double f = 1.0 / den;
    for (int m = 3; m < 9; m++) w[m] = w[m] * f;
  } else {
    for (int m = 3; m < 9; m++) w[m] = 0.0;
  }
}

/* positivity clip and dry-leaf reset after each stage */
static void post_stage(orc_sim *s, double *w, double area) {
  if (w[0] < 0.0) {
    s->n_clip++;
    s->v_clip += -w[0] * area;
    w[0] = 0.0;
  }
  if (!(w[0] > s->p.h_dry)) {
    w[1] = 0.0;
    w[2] = 0.0;
    for (int m = 3; m < 9; m++) w[m] = 0.0;
  }
}

/* Stage-input limiting of one leaf.  Outputs the limited coefficients in
 * two views: w_st, which the RK2 combination (Eq. 4) and the stored state
 * use, and w_fx with its bed planes ze, which the interface fluxes and the
 * operator use.
 * (1) Partially wet leaves drop to first order.  A leaf is partially wet
 *     when its average is not wetter than h_dry, when the depth limit of
 *     its plane at any interface centre is not wetter than h_dry, or when a
 *     flat free surface h0 + z0 would leave any interface centre of its
 *     planar bed not wetter than h_dry (water shallower than the leaf's own
 *     bed relief, e.g. a rain film on a slope).  Such a leaf stores a flat
 *     free surface over its planar bed (h1 = -z1, discharge slopes zero)
 *     and is seen by the fluxes as flat depth over a flat bed (z0, 0, 0), so
 *     its interface depths are its average and a shoreline leaf at rest
 *     stays at rest.  The paper delegates its wet/dry treatment to cited works;
 *     this is the reading used here.
 * (2) Otherwise, the slope limiter (the paper names none; the DG2 step it
 *     cites limits its slopes): minmod on the face-limit offsets sqrt3*v1 of eta, qx and qy
 *     against the differences of the averages of the same-level leaf
 *     neighbours, per direction (two-argument minmod against the one
 *     difference where only one such neighbour exists: domain edges and
 *     level transitions); eta only where the leaf and its neighbours are
 *     wet, the discharges also next to dry neighbours (whose discharge is
 *     zero), so that slopes at wet/dry fronts and edges stay bounded. */
static void limit_leaf(const orc_sim *s, double *const *X, int l, int i, int j, const double *w_in,
                       double *w_st, double *w_fx, double *ze) {
  double s3 = S3();
  size_t n = nn(s, l);
  size_t kc = id(s, l, i, j);
  double hd = s->p.h_dry;
  for (int m = 0; m < 9; m++) w_st[m] = w_in[m];
  for (int m = 0; m < 3; m++) ze[m] = s->z[l][m * n + kc];
  if (s->p.scheme == 1) {  /* FV1: first order, nothing to limit */
    for (int m = 0; m < 9; m++) w_fx[m] = w_in[m];
    return;
  }
  double h0 = w_in[0];
  double eta0 = h0 + ze[0];
  int reduced = !(h0 > hd);
  for (int f = 0; f < 4; f++) {
    if (!(face_lim(w_in, f) > hd)) reduced = 1;
    if (!(eta0 - face_lim(ze, f) > hd)) reduced = 1;
  }
  if (reduced) {
    w_st[1] = -ze[1]; w_st[2] = -ze[2];
    w_st[4] = 0.0; w_st[5] = 0.0;
    w_st[7] = 0.0; w_st[8] = 0.0;
    for (int m = 0; m < 9; m++) w_fx[m] = w_st[m];
    w_fx[1] = 0.0; w_fx[2] = 0.0;
    ze[1] = 0.0; ze[2] = 0.0;
    return;
  }
  for (int m = 0; m < 9; m++) w_fx[m] = w_in[m];
  if (!s->p.limiter) return;
  for (int dir = 0; dir < 2; dir++) {
    int ia = i + (dir == 0), ja = j + (dir == 1), ib = i - (dir == 0), jb = j - (dir == 1);
    int hasA = in_dom(s, l, ia, ja) && s->kind[l][id(s, l, ia, ja)] == K_LEAF;
    int hasB = in_dom(s, l, ib, jb) && s->kind[l][id(s, l, ib, jb)] == K_LEAF;
    if (!hasA && !hasB) continue;
    size_t ka = hasA ? id(s, l, ia, ja) : kc, kb = hasB ? id(s, l, ib, jb) : kc;
    double hC = X[l][kc], hA = X[l][ka], hB = X[l][kb];
    int wet = (hC > hd) && (!hasA || hA > hd) && (!hasB || hB > hd);
    int cs = 1 + dir; /* slope coefficient index */
    for (int v = 0; v < 3; v++) {
      if (v == 0 && !wet) continue;
      double a0, aC, aB, slope, zs = s->z[l][cs * n + kc];
      if (v == 0) {
        aC = hC + s->z[l][kc];
        a0 = hA + s->z[l][ka];
        aB = hB + s->z[l][kb];
        slope = w_in[cs] + zs;
      } else {
        aC = X[l][3 * v * n + kc];
        a0 = X[l][3 * v * n + ka];
        aB = X[l][3 * v * n + kb];
        slope = w_in[3 * v + cs];
      }
      double a = s3 * slope, mm;
      if (hasA && hasB) mm = minmod3(a, a0 - aC, aC - aB);
      else if (hasA) mm = minmod2(a, a0 - aC);
      else mm = minmod2(a, aC - aB);
      if (mm != a) {
        double ns = mm / s3;
        if (v == 0) w_st[cs] = ns - zs;
        else w_st[3 * v + cs] = ns;
      }
    }
  }
  for (int m = 0; m < 9; m++) w_fx[m] = w_st[m];
}

/* Same-level view of every node for the limited stage state X and its bed
 * planes Z: leaves keep their coefficients, refined nodes hold the local
 * encoding of their finer leaves (Eq. 9, Sect. 2.3), nodes under a coarser
 * leaf hold the prolongation of that leaf's plane (Eq. 10 with zero
 * details).  Beds are viewed the same way. */
static void build_view(orc_sim *s, double **X, double **Z) {
  int L = s->L;
  for (int l = 0; l <= L; l++) {
    size_t n = nn(s, l);
    for (size_t k = 0; k < n; k++)
      if (s->kind[l][k] == K_LEAF) {
        for (int m = 0; m < 9; m++) s->V[l][m * n + k] = X[l][m * n + k];
        for (int m = 0; m < 3; m++) s->Vz[l][m * n + k] = Z[l][m * n + k];
      }
  }
  for (int l = L - 1; l >= 0; l--) {
    size_t n = nn(s, l), nf = nn(s, l + 1);
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        if (s->kind[l][k] != K_SIG) continue;
        for (int v = 0; v < 3; v++) {
          double ch[12], sp[3], d[9];
          for (int c = 0; c < 4; c++) {
            size_t kc = id(s, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
            for (int m = 0; m < 3; m++) ch[3 * c + m] = s->V[l + 1][(3 * v + m) * nf + kc];
          }
          encode_node_scheme(s, ch, sp, d);
          for (int m = 0; m < 3; m++) s->V[l][(3 * v + m) * n + k] = sp[m];
        }
        double ch[12], sp[3], d[9];
        for (int c = 0; c < 4; c++) {
          size_t kc = id(s, l + 1, 2 * i + (c & 1), 2 * j + (c >> 1));
          for (int m = 0; m < 3; m++) ch[3 * c + m] = s->Vz[l + 1][m * nf + kc];
        }
        encode_node_scheme(s, ch, sp, d);
        for (int m = 0; m < 3; m++) s->Vz[l][m * n + k] = sp[m];
      }
  }
  for (int l = 1; l <= L; l++) {
    size_t n = nn(s, l), np = nn(s, l - 1);
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        if (s->kind[l][k] != K_BELOW) continue;
        size_t kp = id(s, l - 1, i / 2, j / 2);
        int c = (i & 1) + 2 * (j & 1);
        double sp[3], sc[3];
        for (int v = 0; v < 3; v++) {
          for (int m = 0; m < 3; m++) sp[m] = s->V[l - 1][(3 * v + m) * np + kp];
          prolong_child(sp, c, sc);
          for (int m = 0; m < 3; m++) s->V[l][(3 * v + m) * n + k] = sc[m];
        }
        for (int m = 0; m < 3; m++) sp[m] = s->Vz[l - 1][m * np + kp];
        prolong_child(sp, c, sc);
        for (int m = 0; m < 3; m++) s->Vz[l][m * n + k] = sc[m];
      }
  }
}

/* neighbour limit (h, qx, qy, z) across face f of leaf (l,i,j) and the
 * averages (h0, qx0, qy0) of the view it comes from (the mean of the two
 * finer leaves' averages on the coarse side of a static grid's face);
 * returns 0 when the face is on the domain boundary */
static int nbr_limit(const orc_sim *s, int l, int i, int j, int f, double out[4], double avg[3]) {
  static const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
  int a = i + di[f], b = j + dj[f];
  if (!in_dom(s, l, a, b)) return 0;
  int fo = f ^ 1; /* the neighbour's face that touches ours */
  size_t n = nn(s, l);
  size_t k = id(s, l, a, b);
  if (s->p.mode == ORC_STATIC && s->kind[l][k] == K_SIG) {
    /* Sect. 2.2.1: the coarse side interpolates the limit from the two finer
     * interface centres (graded grid, so those are level l+1 leaves) */
    size_t nf = nn(s, l + 1);
    int c1, c2;
    if (f == 0) { c1 = 0; c2 = 2; }      /* neighbour's west children */
    else if (f == 1) { c1 = 1; c2 = 3; } /* east children */
    else if (f == 2) { c1 = 0; c2 = 1; } /* south children */
    else { c1 = 2; c2 = 3; }             /* north children */
    size_t k1 = id(s, l + 1, 2 * a + (c1 & 1), 2 * b + (c1 >> 1));
    size_t k2 = id(s, l + 1, 2 * a + (c2 & 1), 2 * b + (c2 >> 1));
    for (int v = 0; v < 3; v++) {
      double p1[3], p2[3];
      for (int m = 0; m < 3; m++) {
        p1[m] = s->V[l + 1][(3 * v + m) * nf + k1];
        p2[m] = s->V[l + 1][(3 * v + m) * nf + k2];
      }
      out[v] = 0.5 * (face_lim(p1, fo) + face_lim(p2, fo));
      avg[v] = 0.5 * (p1[0] + p2[0]);
    }
    double z1[3], z2[3];
    for (int m = 0; m < 3; m++) {
      z1[m] = s->Vz[l + 1][m * nf + k1];
      z2[m] = s->Vz[l + 1][m * nf + k2];
    }
    out[3] = 0.5 * (face_lim(z1, fo) + face_lim(z2, fo));
    return 1;
  }
  for (int v = 0; v < 3; v++) {
    double p[3];
    for (int m = 0; m < 3; m++) p[m] = s->V[l][(3 * v + m) * n + k];
    out[v] = face_lim(p, f ^ 1);
    avg[v] = p[0];
  }
  double zp[3];
  for (int m = 0; m < 3; m++) zp[m] = s->Vz[l][m * n + k];
  out[3] = face_lim(zp, f ^ 1);
  return 1;
}

/* ghost limit at a boundary face: wall (mirror, normal discharge negated),
 * open (copy) or inflow (critical-depth ghost carrying the hydrograph) */
static void ghost_limit(const orc_sim *s, int l, int i, int j, int f, const double own[4], double t,
                        double out[4]) {
  /* faces E, W, N, S lie on the east, west, north, south edges */
  int e = (f == 0) ? 1 : (f == 1) ? 0 : (f == 2) ? 3 : 2;
  double q = inflow_q(s, e, l, (e < 2) ? j : i, t);
  out[3] = own[3];
  if (q > 0.0) {
    double hc = crit_depth(q, s->p.g);
    out[0] = fmax(own[0], hc);
    double qn = (e == 0 || e == 2) ? q : -q;
    if (e < 2) { out[1] = qn; out[2] = 0.0; }
    else { out[1] = 0.0; out[2] = qn; }
    return;
  }
  if (s->p.bc[e] == ORC_OPEN) {
    out[0] = own[0]; out[1] = own[1]; out[2] = own[2];
    return;
  }
  out[0] = own[0];
  if (e < 2) { out[1] = -own[1]; out[2] = own[2]; }
  else { out[1] = own[1]; out[2] = -own[2]; }
}

/* Outflow limited by content (Sect. 2.1.1 states that the wet/dry treatment
 * keeps depths non-negative; the revisions alone do not where a thin leaf's
 * interface limits carry large velocities).  Reading: a leaf's content
 * h0 dx^2 is split among its four interfaces, and the volume that leaves
 * through interface f during a forward-Euler stage is limited to its share
 * s_f h0 dx^2, so that the average stays non-negative whatever the other
 * interfaces do (the draining time step of Bollermann, Chen, Kurganov &
 * Noelle 2013, with the donor's content divided among its interfaces so
 * that each interface is limited on its own).  The shares follow the
 * donor's average flow: s_f = e_f / (e_E + e_W + e_N + e_S) with
 * e_f = max(0, outward average velocity through f) + sqrt(g h0), so a
 * leaf's content goes mostly to the interfaces it flows towards and a leaf
 * at rest splits it evenly.  The mass flux F[0] (per unit length, along +x
 * or +y) is limited to |F[0]| dt <= s_f h0 dx, and the momentum components
 * are scaled by the same factor.  don = the donor's (the side the mass
 * leaves) flux-view averages (h0, q_n0 normal to the interface along +x or
 * +y, q_t0); F[0] > 0 means the donor is the west or south side.  Both sides
 * of an interface between two leaves of one level evaluate it from the same
 * operands, so the flux stays conservative there. */
static void drain_limit(double F[3], const double don[3], double g, double hd, double dx, double dt) {
  double h0 = don[0];
  if (!(h0 > 0.0)) {
    F[0] = F[1] = F[2] = 0.0;
    return;
  }
  double un = 0.0, ut = 0.0;
  if (h0 > hd) {
    un = don[1] / h0;
    ut = don[2] / h0;
  }
  double c = sqrt(g * h0);
  double out = F[0] > 0.0 ? un : -un;
  double e = fmax(out, 0.0) + c;
  double S = (fabs(un) + fabs(ut)) + 4.0 * c;
  double cap = (h0 * dx / dt) * (e / S);
  double a = fabs(F[0]);
  if (a > cap) {
    double th = cap / a;
    F[0] = F[0] > 0.0 ? cap : -cap;
    F[1] = F[1] * th;
    F[2] = F[2] * th;
  }
}

/* Numerical flux through face f of leaf (l, i, j) with flux-view
 * coefficients w and beds zc: own interface limit and the neighbour's (same-
 * level view or boundary ghost), both revised, HLL in (h, qx, qy) order,
 * oriented along +x (E, W) or +y (N, S), then (DG2, stage step dt > 0) the
 * outflow limit of the donor side; a boundary ghost is never a donor that is
 * limited.  The own revised limit goes to hs, us, vs, zr; returns 1 inside
 * the domain, 0 on the boundary. */
static int face_flux(const orc_sim *s, int l, int i, int j, const double *w, const double *zc, int f,
                     double t, double dt, double F[3], double *hs, double *us, double *vs, double *zr) {
  double g = s->p.g, hd = s->p.h_dry;
  double own[4];
  own[0] = face_lim(w + 0, f);
  own[1] = face_lim(w + 3, f);
  own[2] = face_lim(w + 6, f);
  own[3] = face_lim(zc, f);
  double nb[4], nbavg[3];
  int inside = nbr_limit(s, l, i, j, f, nb, nbavg);
  if (!inside) ghost_limit(s, l, i, j, f, own, t, nb);
  double zf = fmax(own[3], nb[3]);
  double hn, un, vn, zn;
  revise(own[0], own[1], own[2], own[3], zf, hd, hs, us, vs, zr);
  revise(nb[0], nb[1], nb[2], nb[3], zf, hd, &hn, &un, &vn, &zn);
  double H[3];
  if (f == 0) { /* east: own on the left */
    hll(*hs, *us, *vs, hn, un, vn, g, hd, H);
    F[0] = H[0]; F[1] = H[1]; F[2] = H[2];
  } else if (f == 1) {
    hll(hn, un, vn, *hs, *us, *vs, g, hd, H);
    F[0] = H[0]; F[1] = H[1]; F[2] = H[2];
  } else if (f == 2) { /* north: own below */
    hll(*hs, *vs, *us, hn, vn, un, g, hd, H);
    F[0] = H[0]; F[1] = H[2]; F[2] = H[1];
  } else {
    hll(hn, vn, un, *hs, *vs, *us, g, hd, H);
    F[0] = H[0]; F[1] = H[2]; F[2] = H[1];
  }
  if (dt > 0.0 && F[0] != 0.0) {
    /* the donor: own side when the mass leaves it (own is the west side of
     * an E face and the south side of an N face); a boundary ghost is never
     * limited */
    int own_first = (f == 0 || f == 2);
    int from_own = own_first ? (F[0] > 0.0) : (F[0] < 0.0);
    int xf = f < 2;
    double don[3];
    if (from_own) {
      don[0] = w[0]; don[1] = xf ? w[3] : w[6]; don[2] = xf ? w[6] : w[3];
      drain_limit(F, don, g, hd, s->dx[l], dt);
    } else if (inside) {
      don[0] = nbavg[0]; don[1] = xf ? nbavg[1] : nbavg[2]; don[2] = xf ? nbavg[2] : nbavg[1];
      drain_limit(F, don, g, hd, s->dx[l], dt);
    }
  }
  return inside;
}

/* Reflux rule on static grids (the coarse side of a face whose neighbour
 * is refined): the flux is the mean of the two fine leaves' own fluxes
 * through their halves of the face, computed as they compute them, so the
 * mass leaving one side enters the other. */
static int reflux_face(const orc_sim *s, int l, int i, int j, int f, double t, double dt, double F[3]) {
  static const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
  if (s->p.mode != ORC_STATIC || s->p.iface_rule != 1) return 0;
  int a = i + di[f], b = j + dj[f];
  if (!in_dom(s, l, a, b) || s->kind[l][id(s, l, a, b)] != K_SIG) return 0;
  int c1, c2;
  if (f == 0) { c1 = 0; c2 = 2; }
  else if (f == 1) { c1 = 1; c2 = 3; }
  else if (f == 2) { c1 = 0; c2 = 1; }
  else { c1 = 2; c2 = 3; }
  int cs[2] = {c1, c2};
  double Fc[2][3];
  size_t nf = nn(s, l + 1);
  for (int q = 0; q < 2; q++) {
    int ic = 2 * a + (cs[q] & 1), jc = 2 * b + (cs[q] >> 1);
    size_t kc = id(s, l + 1, ic, jc);
    double wc[9], zcc[3], hs, us, vs, zr;
    get9(s->F, s, l + 1, kc, wc);
    for (int m = 0; m < 3; m++) zcc[m] = s->Ze[l + 1][m * nf + kc];
    face_flux(s, l + 1, ic, jc, wc, zcc, f ^ 1, t, dt, Fc[q], &hs, &us, &vs, &zr);
  }
  for (int v = 0; v < 3; v++) F[v] = 0.5 * (Fc[0][v] + Fc[1][v]);
  return 1;
}

/* DG2 spatial operator L = [L0, L1x, L1y] of one leaf (Eq. 4, Sect. 2.1.1),
 * evaluated on limited coefficients w and the same-level neighbour view.
 * Average: flux difference over the four faces plus the bed source with the
 * revised face beds.  Slopes: two-point (interface-centre) rule for the
 * volume flux integral, midpoint rule on the faces, and the bed source
 * written so that it cancels the hydrostatic quadrature error at rest:
 * S1 = -(2 sqrt3 g / dx) h1 (h1 + z1).  Returns the outward boundary mass
 * flux (m^3/s) in *bnd_out. */
static void leaf_operator(const orc_sim *s, int l, int i, int j, const double *w, const double *zc,
                          double t, double dt, double *Lo, double *bnd_out) {
  double g = s->p.g, s3 = S3();
  double dxl = s->dx[l];
  double Fh[4][3];                 /* numerical flux per face in (h,qx,qy) */
  double hs[4], us[4], vs[4], zr[4]; /* own revised limits */
  double bout = 0.0;
  for (int f = 0; f < 4; f++) {
    int inside = face_flux(s, l, i, j, w, zc, f, t, dt, Fh[f], &hs[f], &us[f], &vs[f], &zr[f]);
    double Fr[3];
    if (inside && reflux_face(s, l, i, j, f, t, dt, Fr))
      for (int v = 0; v < 3; v++) Fh[f][v] = Fr[v];
    if (!inside) {
      double outward = (f == 0 || f == 2) ? Fh[f][0] : -Fh[f][0];
      bout += outward * dxl;
    }
  }
  /* physical fluxes of the own revised limits */
  double Fx[2][3], Gy[2][3];
  for (int a = 0; a < 2; a++) {
    int f = a; /* E, W */
    double q = hs[f] * us[f];
    Fx[a][0] = q;
    Fx[a][1] = q * us[f] + 0.5 * g * hs[f] * hs[f];
    Fx[a][2] = q * vs[f];
    f = 2 + a; /* N, S */
    double r = hs[f] * vs[f];
    Gy[a][0] = r;
    Gy[a][1] = r * us[f];
    Gy[a][2] = r * vs[f] + 0.5 * g * hs[f] * hs[f];
  }
  for (int v = 0; v < 3; v++) {
    double L0 = -(Fh[0][v] - Fh[1][v]) / dxl - (Fh[2][v] - Fh[3][v]) / dxl;
    if (v == 1) L0 = L0 + -g * 0.5 * (hs[0] + hs[1]) * (zr[0] - zr[1]) / dxl;
    if (v == 2) L0 = L0 + -g * 0.5 * (hs[2] + hs[3]) * (zr[2] - zr[3]) / dxl;
    double L1x = -(s3 / dxl) * (Fh[0][v] + Fh[1][v] - Fx[0][v] - Fx[1][v]);
    double L1y = -(s3 / dxl) * (Fh[2][v] + Fh[3][v] - Gy[0][v] - Gy[1][v]);
    if (v == 1) L1x = L1x + -(2.0 * s3 * g / dxl) * w[1] * (w[1] + zc[1]);
    if (v == 2) L1y = L1y + -(2.0 * s3 * g / dxl) * w[2] * (w[2] + zc[2]);
    if (s->p.scheme == 1) L1x = L1y = 0.0;  /* FV1: L0 only (Sect. 2.1.2) */
    Lo[3 * v + 0] = L0;
    Lo[3 * v + 1] = L1x;
    Lo[3 * v + 2] = L1y;
  }
  *bnd_out = bout;
}

/* One RK2 stage (Eq. 4a when Wcomb == NULL, Eq. 4b otherwise): limit the
 * stage input Xin on every leaf (stored view into Wout, flux view into
 * s->F with beds s->Ze), then update every leaf into Out. */
static double rk_stage(orc_sim *s, double **Xin, double **Wout, double **Wcomb, double **Out,
                       double dt, double t_force) {
  int L = s->L;
  for (int l = 0; l <= L; l++)
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        if (s->kind[l][k] != K_LEAF) continue;
        double w_in[9], w[9], wf[9], ze[3];
        get9(Xin, s, l, k, w_in);
        limit_leaf(s, Xin, l, i, j, w_in, w, wf, ze);
        put9(Wout, s, l, k, w);
        put9(s->F, s, l, k, wf);
        for (int m = 0; m < 3; m++) s->Ze[l][m * nn(s, l) + k] = ze[m];
      }
  build_view(s, s->F, s->Ze);
  double bnd = 0.0;
  for (int l = 0; l <= L; l++)
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        if (s->kind[l][k] != K_LEAF) continue;
        double w[9], wf[9], zc[3], Lo[9], o[9], b;
        get9(Wout, s, l, k, w);
        get9(s->F, s, l, k, wf);
        for (int m = 0; m < 3; m++) zc[m] = s->Ze[l][m * nn(s, l) + k];
        leaf_operator(s, l, i, j, wf, zc, t_force, dt, Lo, &b);
        bnd += b;
        if (!Wcomb) {
          for (int m = 0; m < 9; m++) o[m] = w[m] + dt * Lo[m];
        } else {
          double wn[9];
          get9(Wcomb, s, l, k, wn);
          for (int m = 0; m < 9; m++) o[m] = 0.5 * (wn[m] + w[m] + dt * Lo[m]);
        }
        post_stage(s, o, s->dx[l] * s->dx[l]);
        put9(Out, s, l, k, o);
      }
  return bnd;
}

/* ------------------------------------------------------------------------ */
/* ACC: the local inertial solver (Sect. 2.1.3)                              */
/* ------------------------------------------------------------------------ */
/* The paper describes ACC by reference (Bates et al. 2010, De Almeida et al.
 * 2012): piecewise-constant depth and bed, a discharge per interface from
 * the momentum equation without convective acceleration coupled to the
 * Manning resistance, continuity from the four interface discharges,
 * Courant number 0.7.  Reading used here: the explicit scheme of Bates et
 * al. with the resistance taken semi-implicitly in the discharge,
 *   q^{n+1} = (q^n - g h_f dt (eta_b - eta_a) / d)
 *             / (1 + g dt n_f^2 |q^n| / h_f^{7/3}),
 * h_f = max(eta_a, eta_b) - max(z_a, z_b) (no flow where h_f <= h_dry),
 * n_f the mean of the two cells' Manning n, d the distance between the cell
 * centres; rain enters continuity.  On graded static grids each finer
 * element computes the discharge of its half of a face with the coarser
 * element, and the coarser element sums them (Sect. 2.2.1, "aggregated").
 * Face discharges (m^2/s, positive towards +x / +y) are held per leaf and
 * face (E, W, N, S) in s->Wi; a face between two leaves of one level is
 * computed by both with the same operands, so both hold the same value.
 * Discharges start at zero.  Boundaries: walls carry none, inflow faces the
 * hydrograph's unit discharge, and an open face carries the discharge of
 * the element's opposite face (zero gradient of the discharge; a zero
 * surface gradient would let friction stop the outflow). */
static double acc_face_q(double q0, double ha, double za, double hb, double zb, double d, double nf,
                         double dt, double g, double hd) {
  double ea = ha + za, eb = hb + zb;
  double hf = fmax(ea, eb) - fmax(za, zb);
  if (!(hf > hd)) return 0.0;
  double num = q0 - g * hf * dt * (eb - ea) / d;
  double den = 1.0 + g * dt * nf * nf * fabs(q0) / (hf * hf * cube_root(hf));
  return num / den;
}

/* the leaf covering node (l, a, b) at that level or above: its level */
static int acc_cover(const orc_sim *s, int l, int a, int b, int *la, int *ia, int *ja) {
  while (l > 0 && s->kind[l][id(s, l, a, b)] == K_BELOW) {
    a /= 2;
    b /= 2;
    l--;
  }
  *la = l; *ia = a; *ja = b;
  return s->kind[l][id(s, l, a, b)];
}

/* one ACC step of length dt; returns the outward boundary mass flux */
static double acc_step(orc_sim *s, double dt) {
  static const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
  const double g = s->p.g, hd = s->p.h_dry;
  const int L = s->L;
  /* discharges of every leaf's faces, from the old state, into s->Ui */
  for (int l = 0; l <= L; l++) {
    size_t n = nn(s, l);
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        if (s->kind[l][k] != K_LEAF) continue;
        double h = s->U[l][k], z = s->z[l][k], nm = s->nm[l][k];
        for (int f = 0; f < 4; f++) {
          double q0 = s->Wi[l][f * n + k], qn = 0.0;
          int a = i + di[f], b = j + dj[f];
          if (!in_dom(s, l, a, b)) {
            int e = (f == 0) ? 1 : (f == 1) ? 0 : (f == 2) ? 3 : 2;
            double qin = inflow_q(s, e, l, (e < 2) ? j : i, s->t);
            if (qin > 0.0) qn = (e == 0 || e == 2) ? qin : -qin;
            else if (s->p.bc[e] == ORC_OPEN) qn = s->Wi[l][(f ^ 1) * n + k];  /* discharge carried through */
          } else {
            int la, ia, ja;
            int kd = acc_cover(s, l, a, b, &la, &ia, &ja);
            if (kd == K_SIG) {
              qn = 0.0; /* finer neighbour: its elements hold the half-face discharges */
            } else {
              size_t kb = id(s, la, ia, ja);
              double hb = s->U[la][kb], zb = s->z[la][kb], nb = s->nm[la][kb];
              double d = 0.5 * (s->dx[l] + s->dx[la]), nf = 0.5 * (nm + nb);
              if (f == 0 || f == 2) qn = acc_face_q(q0, h, z, hb, zb, d, nf, dt, g, hd);
              else qn = acc_face_q(q0, hb, zb, h, z, d, 0.5 * (nb + nm), dt, g, hd);
            }
          }
          s->Ui[l][f * n + k] = qn;
        }
      }
  }
  for (int l = 0; l <= L; l++) memcpy(s->Wi[l], s->Ui[l], 4 * nn(s, l) * sizeof(double));
  /* continuity */
  double bnd = 0.0;
  double rain = (s->t < s->p.rain_t_end) ? s->p.rain_rate : 0.0;
  for (int l = 0; l <= L; l++) {
    size_t n = nn(s, l);
    double dxl = s->dx[l];
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        if (s->kind[l][k] != K_LEAF) continue;
        double F[4];
        for (int f = 0; f < 4; f++) {
          int a = i + di[f], b = j + dj[f];
          F[f] = s->Wi[l][f * n + k] * dxl;
          if (in_dom(s, l, a, b) && s->kind[l][id(s, l, a, b)] == K_SIG) {
            int c1, c2;
            if (f == 0) { c1 = 0; c2 = 2; }
            else if (f == 1) { c1 = 1; c2 = 3; }
            else if (f == 2) { c1 = 0; c2 = 1; }
            else { c1 = 2; c2 = 3; }
            size_t nf = nn(s, l + 1);
            size_t k1 = id(s, l + 1, 2 * a + (c1 & 1), 2 * b + (c1 >> 1));
            size_t k2 = id(s, l + 1, 2 * a + (c2 & 1), 2 * b + (c2 >> 1));
            double q1 = s->Wi[l + 1][(f ^ 1) * nf + k1], q2 = s->Wi[l + 1][(f ^ 1) * nf + k2];
            F[f] = q1 * s->dx[l + 1] + q2 * s->dx[l + 1];
            s->Wi[l][f * n + k] = 0.5 * (q1 + q2);  /* the face's mean, for the read-out */
          }
          if (!in_dom(s, l, a, b)) bnd += (f == 0 || f == 2) ? F[f] : -F[f];
        }
        double h = s->U[l][k] + rain * dt;
        if (rain > 0.0) s->v_rain += rain * dt * dxl * dxl;
        h = h + dt * ((F[1] - F[0]) + (F[3] - F[2])) / (dxl * dxl);
        if (h < 0.0) {
          s->n_clip++;
          s->v_clip += -h * dxl * dxl;
          h = 0.0;
        }
        s->U[l][k] = h;
        s->U[l][3 * n + k] = 0.5 * (s->Wi[l][0 * n + k] + s->Wi[l][1 * n + k]);
        s->U[l][6 * n + k] = 0.5 * (s->Wi[l][2 * n + k] + s->Wi[l][3 * n + k]);
      }
  }
  return bnd;
}

/* One time step (Sect. 2.1.1 and 2.3): adapt (MWDG2), dt, rain, friction,
 * stage 1 (Eq. 4a), stage 2 (Eq. 4b).  Returns dt. */
/* One step with a time step given by the caller (dt_given > 0) or chosen by
 * the CFL condition (dt_given <= 0).  A given dt serves the discrete adjoint:
 * the step map differentiated there is the one with the recorded dt held
 * fixed, and its central differences must be taken on that same map. */
static double step_with(orc_sim *s, double t_end, double dt_given, int adapt) {
  if (adapt) orc_adapt(s);
  double dt = dt_given > 0.0 ? dt_given : compute_dt(s, t_end);
  if (!(dt > 0.0)) return 0.0;
  if (s->p.scheme == 2) {
    double net_out = dt * acc_step(s, dt);
    if (net_out >= 0.0) s->v_out += net_out;
    else s->v_in += -net_out;
    s->t = s->t + dt;
    s->steps++;
    s->last_dt = dt;
    return dt;
  }
  int L = s->L;
  double rain = (s->t < s->p.rain_t_end) ? s->p.rain_rate : 0.0;
  for (int l = 0; l <= L; l++) {
    size_t n = nn(s, l);
    for (size_t k = 0; k < n; k++) {
      if (s->kind[l][k] != K_LEAF) continue;
      double w[9];
      get9(s->U, s, l, k, w);
      if (rain > 0.0) {
        w[0] = w[0] + rain * dt;
        s->v_rain += rain * dt * s->dx[l] * s->dx[l];
      }
      friction(w, s->nm[l][k], dt, s->p.g, s->p.h_dry);
      put9(s->U, s, l, k, w);
    }
  }
  double net_out;
  if (s->p.scheme == 1) {
    /* FV1: forward Euler, Eq. 7 */
    double b1 = rk_stage(s, s->U, s->Wn, NULL, s->U, dt, s->t);
    net_out = dt * b1;
  } else {
    double b1 = rk_stage(s, s->U, s->Wn, NULL, s->Ui, dt, s->t);
    double b2 = rk_stage(s, s->Ui, s->Wi, s->Wn, s->U, dt, s->t + dt);
    net_out = 0.5 * dt * (b1 + b2);
  }
  if (net_out >= 0.0) s->v_out += net_out;
  else s->v_in += -net_out;
  s->t = s->t + dt;
  s->steps++;
  s->last_dt = dt;
  return dt;
}

double orc_step(orc_sim *s, double t_end) { return step_with(s, t_end, 0.0, 1); }

/* One forward-Euler stage of Eq. 4a on the current active leaves, with no
 * adaptation, rain or friction and the clock left where it is: the stage
 * operator of Sect. 2.1.1 applied once, so that tests can compare it
 * between grids (the interface rule of Sect. 2.3). */
void orc_stage(orc_sim *s, double dt) { (void)rk_stage(s, s->U, s->Wn, NULL, s->U, dt, s->t); }

double orc_step_dt(orc_sim *s, double dt) { return step_with(s, INFINITY, dt, 1); }

/* A step of the given dt on the current active set, without the MWDG2
 * regridding at its start: the map that an adjoint differentiates when it
 * freezes the adaptive grid over a checkpoint segment (test entry point; on
 * uniform and static grids it equals orc_step_dt). */
double orc_step_frozen(orc_sim *s, double dt) { return step_with(s, INFINITY, dt, 0); }

int64_t orc_run_to(orc_sim *s, double t_end, int64_t max_steps) {
  int64_t k = 0;
  while (s->t < t_end && k < max_steps) {
    double dt = orc_step(s, t_end);
    if (!(dt > 0.0)) break;
    k++;
  }
  return k;
}

/* ------------------------------------------------------------------------ */
/* Read-back                                                                 */
/* ------------------------------------------------------------------------ */
double orc_time(const orc_sim *s) { return s->t; }
int64_t orc_steps(const orc_sim *s) { return s->steps; }
double orc_last_dt(const orc_sim *s) { return s->last_dt; }

void orc_diag(const orc_sim *s, double *out /*6*/) {
  double vol = 0.0;
  for (int l = 0; l <= s->L; l++)
    for (size_t k = 0; k < nn(s, l); k++)
      if (s->kind[l][k] == K_LEAF) vol += s->U[l][k] * s->dx[l] * s->dx[l];
  out[0] = vol;
  out[1] = s->v_in;
  out[2] = s->v_out;
  out[3] = s->v_rain;
  out[4] = s->v_clip;
  out[5] = (double)s->n_clip;
}

int64_t orc_n_leaves(const orc_sim *s) {
  int64_t c = 0;
  for (int l = 0; l <= s->L; l++)
    for (size_t k = 0; k < nn(s, l); k++) c += (s->kind[l][k] == K_LEAF);
  return c;
}

/* leaves ordered by level, then row-major (j, then i); coefficients in the
 * order h0 h1x h1y qx0 qx1x qx1y qy0 qy1x qy1y.  For a uniform run the
 * single stored level is reported as level L of the parameters. */
void orc_get_leaves(const orc_sim *s, int32_t *lev, int32_t *ii, int32_t *jj, double *coef) {
  int64_t c = 0;
  int loff = (s->p.mode == ORC_UNIFORM) ? s->p.L : 0;
  for (int l = 0; l <= s->L; l++) {
    size_t n = nn(s, l);
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        if (s->kind[l][k] != K_LEAF) continue;
        if (lev) lev[c] = l + loff;
        if (ii) ii[c] = i;
        if (jj) jj[c] = j;
        if (coef)
          for (int m = 0; m < 9; m++) coef[9 * c + m] = s->U[l][m * n + k];
        c++;
      }
  }
}

/* finest-resolution cell averages of h, u, v (each leaf's plane evaluated
 * at the centre of every finest cell it covers) */
void orc_read_fields(const orc_sim *s, double *h, double *u, double *v) {
  int L = s->L;
  int nxL = s->nx[L];
  double s3 = S3();
  for (int l = 0; l <= L; l++) {
    size_t n = nn(s, l);
    int sh = L - l, w = 1 << sh;
    for (int j = 0; j < s->ny[l]; j++)
      for (int i = 0; i < s->nx[l]; i++) {
        size_t k = id(s, l, i, j);
        if (s->kind[l][k] != K_LEAF) continue;
        for (int b = 0; b < w; b++)
          for (int a = 0; a < w; a++) {
            double xi = ((double)a + 0.5) / (double)w - 0.5, et = ((double)b + 0.5) / (double)w - 0.5;
            double val[3];
            for (int q = 0; q < 3; q++) {
              const double *X = s->U[l];
              val[q] = X[3 * q * n + k] + 2.0 * s3 * xi * X[(3 * q + 1) * n + k] +
                       2.0 * s3 * et * X[(3 * q + 2) * n + k];
            }
            size_t kf = (size_t)(j * w + b) * nxL + (size_t)(i * w + a);
            h[kf] = val[0];
            if (val[0] > s->p.h_dry) {
              u[kf] = val[1] / val[0];
              v[kf] = val[2] / val[0];
            } else {
              u[kf] = 0.0;
              v[kf] = 0.0;
            }
          }
      }
  }
}

/* access to the static topography pyramid and normalised details (tests) */
void orc_get_z(const orc_sim *s, int l, double *out /*3*n*/, double *dz /*n*/) {
  size_t n = nn(s, l);
  if (out) memcpy(out, s->z[l], 3 * n * sizeof(double));
  if (dz) memcpy(dz, s->dz[l], n * sizeof(double));
}
