/*
 * oracle.c - plain serial FP64 reference of the free-stream-preserving (FP) upwind
 * conservative finite-difference residual (Su, Cai, Pan & Hu, arXiv 2101.05886).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline of the benchmark.  It shares no code with the CUDA library.
 *
 * Every function follows the paper's equations in the paper's order, with plain
 * loops and no blocking, fusion or reordering.  Where the paper is silent or
 * garbled, the reading taken is stated at the point of use.  Compile with
 * -O2 -ffp-contract=off.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Sec. 3, Eq. (metric_discret): central midpoint interpolation at order M.  */
/* x_{i+1/2} = sum_m w_m x_{i-M/2+1+m} / den; derivative x_i = x_{i+1/2}-x_{i-1/2}. */
/* ------------------------------------------------------------------------ */
static const double W2[2] = {1, 1};
static const double W4[4] = {-1, 7, 7, -1};
static const double W6[6] = {1, -8, 37, 37, -8, 1};
static const double W8[8] = {-3, 29, -139, 533, 533, -139, 29, -3};

static const double *interp_w(int M, double *den) {
  switch (M) {
    case 2: *den = 2.0; return W2;
    case 4: *den = 12.0; return W4;
    case 6: *den = 60.0; return W6;
    case 8: *den = 840.0; return W8;
    default: *den = 0.0; return NULL;
  }
}

int or_ghost(int M) { return M / 2 > 3 ? M / 2 : 3; }
int or_node_ghost(int M) { return or_ghost(M) + 3 * (M / 2); }
/* the 7th-order stencil reaches four points past a face */
int or_ghost_s(int M, int scheme) {
  int r = scheme == 2 ? 4 : 3;
  return M / 2 > r ? M / 2 : r;
}
int or_node_ghost_s(int M, int scheme) { return or_ghost_s(M, scheme) + 3 * (M / 2); }

void or_interp_coef(int M, double c[8]) {
  double den;
  const double *w = interp_w(M, &den);
  for (int m = 0; m < 8; ++m) c[m] = (w && m < M) ? w[m] / den : 0.0;
}

/* interpolation of f (given at the M points i-M/2+1 .. i+M/2, f[0] first) to i+1/2 */
static double interp_face(int M, const double *f) {
  double den;
  const double *w = interp_w(M, &den);
  double s = 0.0;
  for (int m = 0; m < M; ++m) s += w[m] * f[m];
  return s / den;
}

/* ------------------------------------------------------------------------ */
/* Arrays over an index box (lo inclusive, hi exclusive), i fastest.          */
/* ------------------------------------------------------------------------ */
typedef struct { int lo[3], hi[3]; double *a; } arr3;

static size_t box_size(const int lo[3], const int hi[3]) {
  return (size_t)(hi[0] - lo[0]) * (size_t)(hi[1] - lo[1]) * (size_t)(hi[2] - lo[2]);
}
static arr3 arr_new(const int lo[3], const int hi[3]) {
  arr3 r;
  memcpy(r.lo, lo, sizeof r.lo);
  memcpy(r.hi, hi, sizeof r.hi);
  r.a = (double *)calloc(box_size(lo, hi), sizeof(double));
  return r;
}
static size_t at3(const arr3 *A, int i, int j, int k) {
  return ((size_t)(k - A->lo[2]) * (size_t)(A->hi[1] - A->lo[1]) + (size_t)(j - A->lo[1])) *
             (size_t)(A->hi[0] - A->lo[0]) + (size_t)(i - A->lo[0]);
}
static double get3(const arr3 *A, const int p[3]) { return A->a[at3(A, p[0], p[1], p[2])]; }

/* derivative along direction e at point p: I_M(f)_{p+1/2} - I_M(f)_{p-1/2} (Eq. metric_discret).
   The value at p is subtracted from the stencil first (the weights sum to one, so the
   derivative is unchanged) to keep the sums at the size of the differences. */
static double deriv(const arr3 *F, int M, int e, const int p[3]) {
  double fp[8], fm[8];
  int q[3];
  const double f0 = get3(F, p);
  for (int m = 0; m < M; ++m) {
    q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
    q[e] = p[e] - M / 2 + 1 + m;
    fp[m] = get3(F, q) - f0;
    q[e] = p[e] - M / 2 + m;
    fm[m] = get3(F, q) - f0;
  }
  return interp_face(M, fp) - interp_face(M, fm);
}

/* derivative from the M+1 values f(p + t e), t = -M/2 .. M/2 (vals[t + M/2]) */
static double deriv_vals(int M, const double *vals) {
  return interp_face(M, vals + 1) - interp_face(M, vals);
}

/* ------------------------------------------------------------------------ */
/* Metrics: symmetric conservative metrics (Eq. JBabc) and Jacobian (Eq. JB). */
/* The discrete SCMM does not change when the coordinates are translated (the */
/* central derivative operators commute, the coordinate invariance the SCMM is */
/* built to keep), so every metric and Jacobian value at a point p is formed  */
/* from coordinates measured from the node at p.  This keeps the products in  */
/* Eqs. JBabc and JB of the size of the metric itself and the discrete SCL    */
/* residual at the round-off of the metrics rather than of the coordinates.  */
/* Each metric is (1/2) * sum of four signed terms (A B)_outer, where A and B  */
/* are a coordinate or one of its first derivatives.  Table transcribed from   */
/* Eq. JBabc: {sign, outer, coordA, derivA, coordB, derivB}, -1 = no derivative. */
/* coordinates x=0,y=1,z=2; directions xi=0, eta=1, zeta=2.                   */
/* ------------------------------------------------------------------------ */
#define X 0
#define Y 1
#define Z 2
#define XI 0
#define ET 1
#define ZE 2
#define NO (-1)
static const int SCMM[9][4][6] = {
  /* xi_x/J  = 1/2[(y_eta z)_zeta - (y_zeta z)_eta + (y z_zeta)_eta - (y z_eta)_zeta] */
  {{+1, ZE, Y, ET, Z, NO}, {-1, ET, Y, ZE, Z, NO}, {+1, ET, Y, NO, Z, ZE}, {-1, ZE, Y, NO, Z, ET}},
  /* xi_y/J  = 1/2[(x z_eta)_zeta - (x z_zeta)_eta + (x_zeta z)_eta - (x_eta z)_zeta] */
  {{+1, ZE, X, NO, Z, ET}, {-1, ET, X, NO, Z, ZE}, {+1, ET, X, ZE, Z, NO}, {-1, ZE, X, ET, Z, NO}},
  /* xi_z/J  = 1/2[(x_eta y)_zeta - (x_zeta y)_eta + (x y_zeta)_eta - (x y_eta)_zeta] */
  {{+1, ZE, X, ET, Y, NO}, {-1, ET, X, ZE, Y, NO}, {+1, ET, X, NO, Y, ZE}, {-1, ZE, X, NO, Y, ET}},
  /* eta_x/J = 1/2[(y_zeta z)_xi - (y_xi z)_zeta + (y z_xi)_zeta - (y z_zeta)_xi] */
  {{+1, XI, Y, ZE, Z, NO}, {-1, ZE, Y, XI, Z, NO}, {+1, ZE, Y, NO, Z, XI}, {-1, XI, Y, NO, Z, ZE}},
  /* eta_y/J = 1/2[(x z_zeta)_xi - (x z_xi)_zeta + (x_xi z)_zeta - (x_zeta z)_xi] */
  {{+1, XI, X, NO, Z, ZE}, {-1, ZE, X, NO, Z, XI}, {+1, ZE, X, XI, Z, NO}, {-1, XI, X, ZE, Z, NO}},
  /* eta_z/J = 1/2[(x_zeta y)_xi - (x_xi y)_zeta + (x y_xi)_zeta - (x y_zeta)_xi] */
  {{+1, XI, X, ZE, Y, NO}, {-1, ZE, X, XI, Y, NO}, {+1, ZE, X, NO, Y, XI}, {-1, XI, X, NO, Y, ZE}},
  /* zeta_x/J = 1/2[(y_xi z)_eta - (y_eta z)_xi + (y z_eta)_xi - (y z_xi)_eta] */
  {{+1, ET, Y, XI, Z, NO}, {-1, XI, Y, ET, Z, NO}, {+1, XI, Y, NO, Z, ET}, {-1, ET, Y, NO, Z, XI}},
  /* zeta_y/J = 1/2[(x z_xi)_eta - (x z_eta)_xi + (x_eta z)_xi - (x_xi z)_eta] */
  {{+1, ET, X, NO, Z, XI}, {-1, XI, X, NO, Z, ET}, {+1, XI, X, ET, Z, NO}, {-1, ET, X, XI, Z, NO}},
  /* zeta_z/J = 1/2[(x_xi y)_eta - (x_eta y)_xi + (x y_eta)_xi - (x y_xi)_eta] */
  {{+1, ET, X, XI, Y, NO}, {-1, XI, X, ET, Y, NO}, {+1, XI, X, NO, Y, ET}, {-1, ET, X, NO, Y, XI}},
};

static int valid_cfg(const or_cfg *c) {
  if (!c) return 0;
  if (c->dims != 2 && c->dims != 3) return 0;
  if (c->M != 2 && c->M != 4 && c->M != 6 && c->M != 8) return 0;
  if (c->scheme < 0 || c->scheme > 3) return 0;
  for (int d = 0; d < 3; ++d) if (c->n[d] < 1) return 0;
  if (c->dims == 2 && c->n[2] != 1) return 0;
  for (int d = 0; d < c->dims; ++d)
    for (int s = 0; s < 2; ++s) if (c->bc[d][s] < 0 || c->bc[d][s] > 4) return 0;
  if (c->cut < 0) return 0;
  return 1;
}

int or_metrics(const or_cfg *c, const double *nodes, int Gn, double *met) {
  if (!valid_cfg(c) || !nodes || !met) return 1;
  const int M = c->M, h = M / 2, G = or_ghost_s(M, c->scheme), D = c->dims;
  if (Gn < G + 3 * h) return 1;
  int nlo[3], nhi[3], b1lo[3], b1hi[3], b2lo[3], b2hi[3], b3lo[3], b3hi[3];
  for (int d = 0; d < 3; ++d) {
    int on = d < D;
    nlo[d] = on ? -Gn : 0;            nhi[d] = on ? c->n[d] + Gn : 1;
    b1lo[d] = on ? -(G + M) : 0;      b1hi[d] = on ? c->n[d] + G + M : 1;      /* products */
    b2lo[d] = on ? -(G + h) : 0;      b2hi[d] = on ? c->n[d] + G + h : 1;      /* metrics  */
    b3lo[d] = on ? -G : 0;            b3hi[d] = on ? c->n[d] + G : 1;          /* output   */
  }
  arr3 xyz[3];
  size_t nn = box_size(nlo, nhi);
  for (int a = 0; a < 3; ++a) {
    xyz[a] = arr_new(nlo, nhi);
    if (a < D) memcpy(xyz[a].a, nodes + (size_t)a * nn, nn * sizeof(double));
  }
  /* first derivatives of the node coordinates over the product box */
  arr3 d1[3][3];
  for (int a = 0; a < 3; ++a)
    for (int e = 0; e < 3; ++e) {
      d1[a][e] = arr_new(b1lo, b1hi);
      if (a >= D || e >= D) continue;
      for (int k = b1lo[2]; k < b1hi[2]; ++k)
        for (int j = b1lo[1]; j < b1hi[1]; ++j)
          for (int i = b1lo[0]; i < b1hi[0]; ++i) {
            int p[3] = {i, j, k};
            d1[a][e].a[at3(&d1[a][e], i, j, k)] = deriv(&xyz[a], M, e, p);
          }
    }
  arr3 m9[9];
  for (int t = 0; t < 9; ++t) m9[t] = arr_new(b2lo, b2hi);
  if (D == 3) {
    for (int t = 0; t < 9; ++t)
      for (int k = b2lo[2]; k < b2hi[2]; ++k)
        for (int j = b2lo[1]; j < b2hi[1]; ++j)
          for (int i = b2lo[0]; i < b2hi[0]; ++i) {
            int p[3] = {i, j, k};
            double x0[3];
            for (int a = 0; a < 3; ++a) x0[a] = get3(&xyz[a], p);
            double acc = 0.0;
            for (int term = 0; term < 4; ++term) {
              const int *T = SCMM[t][term];
              double vals[9];
              for (int tt = -M / 2; tt <= M / 2; ++tt) {
                int r[3] = {i, j, k};
                r[T[1]] += tt;
                double A = T[3] == NO ? get3(&xyz[T[2]], r) - x0[T[2]] : get3(&d1[T[2]][T[3]], r);
                double B = T[5] == NO ? get3(&xyz[T[4]], r) - x0[T[4]] : get3(&d1[T[4]][T[5]], r);
                vals[tt + M / 2] = A * B;
              }
              acc += (double)T[0] * deriv_vals(M, vals);
            }
            m9[t].a[at3(&m9[t], i, j, k)] = 0.5 * acc;
          }
  } else {
    /* 2-D reading of Eq. JBabc with z = zeta and z_zeta = 1:
       xi_x/J = y_eta, xi_y/J = -x_eta, eta_x/J = -y_xi, eta_y/J = x_xi. */
    for (int j = b2lo[1]; j < b2hi[1]; ++j)
      for (int i = b2lo[0]; i < b2hi[0]; ++i) {
        size_t s = at3(&m9[0], i, j, 0);
        m9[0].a[s] = get3(&d1[Y][ET], (int[3]){i, j, 0});
        m9[1].a[s] = -get3(&d1[X][ET], (int[3]){i, j, 0});
        m9[3].a[s] = -get3(&d1[Y][XI], (int[3]){i, j, 0});
        m9[4].a[s] = get3(&d1[X][XI], (int[3]){i, j, 0});
      }
  }
  /* Jacobian, Eq. JB: 1/J = (1/D) sum_d ( sum_a x_a (d_{x_a}/J) )_d  (factor 1/2 in 2-D),
     with x measured from the node at the point */
  arr3 invJ = arr_new(b3lo, b3hi);
  for (int k = b3lo[2]; k < b3hi[2]; ++k)
    for (int j = b3lo[1]; j < b3hi[1]; ++j)
      for (int i = b3lo[0]; i < b3hi[0]; ++i) {
        int p[3] = {i, j, k};
        double x0[3];
        for (int a = 0; a < 3; ++a) x0[a] = get3(&xyz[a], p);
        double s = 0.0;
        for (int d = 0; d < D; ++d) {
          double vals[9];
          for (int tt = -M / 2; tt <= M / 2; ++tt) {
            int r[3] = {i, j, k};
            r[d] += tt;
            double v = 0.0;
            for (int a = 0; a < D; ++a) v += (get3(&xyz[a], r) - x0[a]) * get3(&m9[3 * d + a], r);
            vals[tt + M / 2] = v;
          }
          s += deriv_vals(M, vals);
        }
        invJ.a[at3(&invJ, i, j, k)] = s;
      }
  size_t n3 = box_size(b3lo, b3hi);
  for (size_t s = 0; s < n3; ++s) invJ.a[s] = invJ.a[s] / (double)D;
  /* output: 9 metrics cropped to the ghosted cell box, then 1/J */
  arr3 out = {{b3lo[0], b3lo[1], b3lo[2]}, {b3hi[0], b3hi[1], b3hi[2]}, NULL};
  for (int t = 0; t < 9; ++t)
    for (int k = b3lo[2]; k < b3hi[2]; ++k)
      for (int j = b3lo[1]; j < b3hi[1]; ++j)
        for (int i = b3lo[0]; i < b3hi[0]; ++i)
          met[(size_t)t * n3 + at3(&out, i, j, k)] = m9[t].a[at3(&m9[t], i, j, k)];
  memcpy(met + 9 * n3, invJ.a, n3 * sizeof(double));
  for (int a = 0; a < 3; ++a) free(xyz[a].a);
  for (int a = 0; a < 3; ++a) for (int e = 0; e < 3; ++e) free(d1[a][e].a);
  for (int t = 0; t < 9; ++t) free(m9[t].a);
  free(invJ.a);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.2, Eq. (weno) and (weno_wights): WENO5-JS at i+1/2 from          */
/* v = f_{i-2}, ..., f_{i+2}.  Reading: the first coefficient set is         */
/* (1/3, -7/6, 11/6) (the printed 7/6 for f_i cannot sum to one), and the     */
/* weight denominator sums C_r/(beta_r + eps)^2 over r.                       */
/* ------------------------------------------------------------------------ */
static void weno5_parts(const double v[5], double q[3], double beta[3]) {
  q[0] = (1.0 / 3.0) * v[0] - (7.0 / 6.0) * v[1] + (11.0 / 6.0) * v[2];
  q[1] = -(1.0 / 6.0) * v[1] + (5.0 / 6.0) * v[2] + (1.0 / 3.0) * v[3];
  q[2] = (1.0 / 3.0) * v[2] + (5.0 / 6.0) * v[3] - (1.0 / 6.0) * v[4];
  double a, b;
  a = v[0] - 4.0 * v[1] + 3.0 * v[2];  b = v[0] - 2.0 * v[1] + v[2];
  beta[0] = 0.25 * a * a + (13.0 / 12.0) * b * b;
  a = -v[1] + v[3];                    b = v[1] - 2.0 * v[2] + v[3];
  beta[1] = 0.25 * a * a + (13.0 / 12.0) * b * b;
  a = -3.0 * v[2] + 4.0 * v[3] - v[4]; b = v[2] - 2.0 * v[3] + v[4];
  beta[2] = 0.25 * a * a + (13.0 / 12.0) * b * b;
}

static const double C_OPT[3] = {0.1, 0.6, 0.3};

/* the sub-stencil face values and smoothness indicators, exposed for the pins */
void or_weno5_parts(const double v[5], double q[3], double beta[3]) { weno5_parts(v, q, beta); }

double or_weno5(const double v[5]) {
  const double eps = 1.0e-6;
  double q[3], beta[3], alpha[3], s = 0.0;
  weno5_parts(v, q, beta);
  for (int k = 0; k < 3; ++k) {
    double t = beta[k] + eps;
    alpha[k] = C_OPT[k] / (t * t);
    s += alpha[k];
  }
  double r = 0.0;
  for (int k = 0; k < 3; ++k) r += (alpha[k] / s) * q[k];
  return r;
}

/* Standard 7th-order WENO (cited in Sec. 4; Remark 2 extends the FP form to it), from
   the general WENO construction: four 4-point sub-stencils, face values q_k of the
   cubic reconstructions, smoothness indicators from the integral definition
   beta_k = sum_{l=1..3} int_{cell} h^(2l-1) (p_k^(l))^2 (the quadratic forms below are
   240 beta_k), optimal weights (1, 12, 18, 4)/35, eps = 1e-6, power 2. */
void or_weno7_parts(const double v[7], double q[4], double beta[4]) {
  q[0] = (-3.0 * v[0] + 13.0 * v[1] - 23.0 * v[2] + 25.0 * v[3]) / 12.0;
  q[1] = (v[1] - 5.0 * v[2] + 13.0 * v[3] + 3.0 * v[4]) / 12.0;
  q[2] = (-v[2] + 7.0 * v[3] + 7.0 * v[4] - v[5]) / 12.0;
  q[3] = (3.0 * v[3] + 13.0 * v[4] - 5.0 * v[5] + v[6]) / 12.0;
  const double *a = v;
  beta[0] = (a[0] * (547.0 * a[0] - 3882.0 * a[1] + 4642.0 * a[2] - 1854.0 * a[3]) +
             a[1] * (7043.0 * a[1] - 17246.0 * a[2] + 7042.0 * a[3]) +
             a[2] * (11003.0 * a[2] - 9402.0 * a[3]) + 2107.0 * a[3] * a[3]) / 240.0;
  beta[1] = (a[1] * (267.0 * a[1] - 1642.0 * a[2] + 1602.0 * a[3] - 494.0 * a[4]) +
             a[2] * (2843.0 * a[2] - 5966.0 * a[3] + 1922.0 * a[4]) +
             a[3] * (3443.0 * a[3] - 2522.0 * a[4]) + 547.0 * a[4] * a[4]) / 240.0;
  beta[2] = (a[2] * (547.0 * a[2] - 2522.0 * a[3] + 1922.0 * a[4] - 494.0 * a[5]) +
             a[3] * (3443.0 * a[3] - 5966.0 * a[4] + 1602.0 * a[5]) +
             a[4] * (2843.0 * a[4] - 1642.0 * a[5]) + 267.0 * a[5] * a[5]) / 240.0;
  beta[3] = (a[3] * (2107.0 * a[3] - 9402.0 * a[4] + 7042.0 * a[5] - 1854.0 * a[6]) +
             a[4] * (11003.0 * a[4] - 17246.0 * a[5] + 4642.0 * a[6]) +
             a[5] * (7043.0 * a[5] - 3882.0 * a[6]) + 547.0 * a[6] * a[6]) / 240.0;
}

double or_weno7(const double v[7]) {
  static const double C7[4] = {1.0 / 35.0, 12.0 / 35.0, 18.0 / 35.0, 4.0 / 35.0};
  const double eps = 1.0e-6;
  double q[4], beta[4], alpha[4], s = 0.0;
  or_weno7_parts(v, q, beta);
  for (int k = 0; k < 4; ++k) {
    double t = beta[k] + eps;
    alpha[k] = C7[k] / (t * t);
    s += alpha[k];
  }
  double r = 0.0;
  for (int k = 0; k < 4; ++k) r += (alpha[k] / s) * q[k];
  return r;
}

/* WENOCU6, the sixth-order adaptive central-upwind WENO scheme that Remark 2 names (its
   formulas are in the cited scheme paper, not here).  Four 3-point sub-stencils over the
   cells i-2..i+3: the three upwind ones of WENO5 and the downwind {i+1, i+2, i+3}; their
   parabolic face values q_k; linear weights d = (1, 9, 9, 1)/20, which make the combination
   the 6-point central face value (1, -8, 37, 37, -8, 1)/60 (the M6 weights of Sec. 3).  The
   downwind stencil's smoothness indicator is that of the whole 6-point stencil, beta6, the
   integral definition sum_{l=1..5} int_{cell} h^(2l-1) (p^(l))^2 of its quintic (the quadratic
   form below is 120960 beta6).  The reference indicator is tau6 = |beta6 - (beta0 + 4 beta1 +
   beta2)/6| and the weights alpha_k = d_k (C + tau6/(beta_k + eps))^q with C = 20, q = 2,
   eps = 1e-40.  Parity unpinned for C, q and eps (taken from the cited scheme paper, which is
   not at hand): the pins cover the sub-stencils, the linear weights, beta6 and the scheme's
   order, and hold for any C, q and eps. */
void or_wenocu6_parts(const double v[6], double q[4], double beta[4], double *tau) {
  double q3[3], b3[3];
  weno5_parts(v, q3, b3);
  for (int k = 0; k < 3; ++k) { q[k] = q3[k]; beta[k] = b3[k]; }
  q[3] = (11.0 * v[3] - 7.0 * v[4] + 2.0 * v[5]) / 6.0;
  const double *a = v;
  beta[3] = (a[0] * (271779.0 * a[0] - 2380800.0 * a[1] + 4086352.0 * a[2] - 3462252.0 * a[3] +
                     1458762.0 * a[4] - 245620.0 * a[5]) +
             a[1] * (5653317.0 * a[1] - 20427884.0 * a[2] + 17905032.0 * a[3] - 7727988.0 * a[4] +
                     1325006.0 * a[5]) +
             a[2] * (19510972.0 * a[2] - 35817664.0 * a[3] + 15929912.0 * a[4] - 2792660.0 * a[5]) +
             a[3] * (17195652.0 * a[3] - 15880404.0 * a[4] + 2863984.0 * a[5]) +
             a[4] * (3824847.0 * a[4] - 1429976.0 * a[5]) + 139633.0 * a[5] * a[5]) / 120960.0;
  *tau = fabs(beta[3] - (beta[0] + 4.0 * beta[1] + beta[2]) / 6.0);
}

double or_wenocu6(const double v[6]) {
  static const double D6[4] = {0.05, 0.45, 0.45, 0.05};
  const double C = 20.0, eps = 1.0e-40;
  double q[4], beta[4], tau, alpha[4], s = 0.0;
  or_wenocu6_parts(v, q, beta, &tau);
  for (int k = 0; k < 4; ++k) {
    const double t = C + tau / (beta[k] + eps);
    alpha[k] = D6[k] * t * t;
    s += alpha[k];
  }
  double r = 0.0;
  for (int k = 0; k < 4; ++k) r += (alpha[k] / s) * q[k];
  return r;
}

/* Appendix, Eq. (new_form_linear_upwind): the linear upwind scheme is WENO with
   the optimal weights C_k, which reproduces Eq. (linear_upwind). */
double or_lu5(const double v[5]) {
  double q[3], beta[3];
  weno5_parts(v, q, beta);
  return C_OPT[0] * q[0] + C_OPT[1] * q[1] + C_OPT[2] * q[2];
}

/* ------------------------------------------------------------------------ */
/* Euler fluxes (Eqs. F, G, H, EOS) contracted with a metric vector k:        */
/* (k_x F + k_y G + k_z H)(Q), Eq. (FGH).                                     */
/* ------------------------------------------------------------------------ */
static void flux_k(const double Q[5], const double k[3], double gamma, double out[5]) {
  double rho = Q[0], u = Q[1] / rho, v = Q[2] / rho, w = Q[3] / rho;
  double p = (gamma - 1.0) * (Q[4] - 0.5 * rho * (u * u + v * v + w * w));
  double Fx[5] = {rho * u, rho * u * u + p, rho * v * u, rho * w * u, (Q[4] + p) * u};
  double Fy[5] = {rho * v, rho * u * v, rho * v * v + p, rho * w * v, (Q[4] + p) * v};
  double Fz[5] = {rho * w, rho * u * w, rho * v * w, rho * w * w + p, (Q[4] + p) * w};
  for (int c = 0; c < 5; ++c) out[c] = k[0] * Fx[c] + k[1] * Fy[c] + k[2] * Fz[c];
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.2: Roe-averaged eigensystem of A = dF~/dQ~ at i+1/2 in the face   */
/* normal n = k/|k|.  The paper does not print the eigenvectors; the basis   */
/* taken is: acoustic (U -+ c), entropy, and two shear waves along unit       */
/* tangents t1, t2 with t1 = normalise(e_z x n) when n_z^2 <= 1/2, else        */
/* normalise(n x e_x), and t2 = n x t1.  R columns, L rows (L = R^-1).         */
/* ------------------------------------------------------------------------ */
void or_eigensystem(const double qL[5], const double qR[5], const double k[3], double gamma,
                    double L[25], double R[25]) {
  double rl = sqrt(qL[0]), rr = sqrt(qR[0]);
  double uL[3] = {qL[1] / qL[0], qL[2] / qL[0], qL[3] / qL[0]};
  double uR[3] = {qR[1] / qR[0], qR[2] / qR[0], qR[3] / qR[0]};
  double pL = (gamma - 1.0) * (qL[4] - 0.5 * qL[0] * (uL[0] * uL[0] + uL[1] * uL[1] + uL[2] * uL[2]));
  double pR = (gamma - 1.0) * (qR[4] - 0.5 * qR[0] * (uR[0] * uR[0] + uR[1] * uR[1] + uR[2] * uR[2]));
  double HL = (qL[4] + pL) / qL[0], HR = (qR[4] + pR) / qR[0];
  double u[3];
  for (int a = 0; a < 3; ++a) u[a] = (rl * uL[a] + rr * uR[a]) / (rl + rr);
  double H = (rl * HL + rr * HR) / (rl + rr);
  double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double c = sqrt((gamma - 1.0) * (H - 0.5 * q2));
  double kn = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
  double n[3] = {k[0] / kn, k[1] / kn, k[2] / kn};
  double t1[3], t2[3];
  if (n[2] * n[2] <= 0.5) {
    double s = sqrt(n[0] * n[0] + n[1] * n[1]);
    t1[0] = -n[1] / s; t1[1] = n[0] / s; t1[2] = 0.0;
  } else {
    double s = sqrt(n[1] * n[1] + n[2] * n[2]);
    t1[0] = 0.0; t1[1] = n[2] / s; t1[2] = -n[1] / s;
  }
  t2[0] = n[1] * t1[2] - n[2] * t1[1];
  t2[1] = n[2] * t1[0] - n[0] * t1[2];
  t2[2] = n[0] * t1[1] - n[1] * t1[0];
  double U = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  double ut1 = u[0] * t1[0] + u[1] * t1[1] + u[2] * t1[2];
  double ut2 = u[0] * t2[0] + u[1] * t2[1] + u[2] * t2[2];
  double b = (gamma - 1.0) / (c * c);
  /* right eigenvectors (columns s = 0..4) */
  double Rc[5][5] = {
    {1.0, u[0] - c * n[0], u[1] - c * n[1], u[2] - c * n[2], H - c * U},
    {1.0, u[0], u[1], u[2], 0.5 * q2},
    {0.0, t1[0], t1[1], t1[2], ut1},
    {0.0, t2[0], t2[1], t2[2], ut2},
    {1.0, u[0] + c * n[0], u[1] + c * n[1], u[2] + c * n[2], H + c * U},
  };
  for (int s = 0; s < 5; ++s)
    for (int r = 0; r < 5; ++r) R[r * 5 + s] = Rc[s][r];
  /* left eigenvectors (rows) */
  double Lr[5][5] = {
    {0.5 * (0.5 * b * q2 + U / c), 0.5 * (-b * u[0] - n[0] / c), 0.5 * (-b * u[1] - n[1] / c),
     0.5 * (-b * u[2] - n[2] / c), 0.5 * b},
    {1.0 - 0.5 * b * q2, b * u[0], b * u[1], b * u[2], -b},
    {-ut1, t1[0], t1[1], t1[2], 0.0},
    {-ut2, t2[0], t2[1], t2[2], 0.0},
    {0.5 * (0.5 * b * q2 - U / c), 0.5 * (-b * u[0] + n[0] / c), 0.5 * (-b * u[1] + n[1] / c),
     0.5 * (-b * u[2] + n[2] / c), 0.5 * b},
  };
  for (int s = 0; s < 5; ++s)
    for (int r = 0; r < 5; ++r) L[s * 5 + r] = Lr[s][r];
}

/* eigenvalues of dF~/dQ~ at one point: U -+ c|grad xi| and U, grad xi = J k */
static void point_eigs(const double Q[5], const double km[3], double invJ, double gamma, double lam[5]) {
  double rho = Q[0], u = Q[1] / rho, v = Q[2] / rho, w = Q[3] / rho;
  double p = (gamma - 1.0) * (Q[4] - 0.5 * rho * (u * u + v * v + w * w));
  double c = sqrt(gamma * p / rho);
  double g[3] = {km[0] / invJ, km[1] / invJ, km[2] / invJ};
  double U = u * g[0] + v * g[1] + w * g[2];
  double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  lam[0] = U - c * gn; lam[1] = U; lam[2] = U; lam[3] = U; lam[4] = U + c * gn;
}

/* ------------------------------------------------------------------------ */
/* The face flux F'_{i+1/2} (Sec. 3.2) from the 8 cells i-3..i+4.            */
/* ------------------------------------------------------------------------ */
static void face_flux_impl(const or_cfg *c, const double q8[40], const double met8[32],
                           const double *lam_given, double out[5]);

void or_face_flux(const or_cfg *c, const double q8[40], const double met8[32], double out[5]) {
  face_flux_impl(c, q8, met8, NULL, out);
}

void or_face_flux_lam(const or_cfg *c, const double q8[40], const double met8[32], const double lam[5],
                      double out[5]) {
  face_flux_impl(c, q8, met8, lam, out);
}

static void face_flux_impl(const or_cfg *c, const double q8[40], const double met8[32],
                           const double *lam_given, double out[5]) {
  const int M = c->M;
  const double gamma = c->gamma;
  const int i0 = 3;                     /* position of cell i in the 8-cell window */
  /* Eqs. (QdJ_star), (1dJ), (xidJ) at order M (Remark 3): Q~_{i+1/2}, (1/J)_{i+1/2}, k_{i+1/2} */
  double qt[8][5], invJ[8], fw[8];
  for (int m = 0; m < 8; ++m) {
    invJ[m] = met8[m * 4 + 3];
    for (int v = 0; v < 5; ++v) qt[m][v] = q8[m * 5 + v] * invJ[m];
  }
  int first = i0 - M / 2 + 1;           /* first cell of the interpolation stencil */
  double kf[3], invJf, Qtf[5], Qs[5];
  for (int a = 0; a < 3; ++a) {
    for (int m = 0; m < M; ++m) fw[m] = met8[(first + m) * 4 + a];
    kf[a] = interp_face(M, fw);
  }
  for (int m = 0; m < M; ++m) fw[m] = invJ[first + m];
  invJf = interp_face(M, fw);
  for (int v = 0; v < 5; ++v) {
    for (int m = 0; m < M; ++m) fw[m] = qt[first + m][v];
    Qtf[v] = interp_face(M, fw);
    Qs[v] = Qtf[v] / invJf;             /* Eq. (Q_star) */
  }
  /* stencil values m = i-2..i+3 (window positions 1..6), i-3..i+4 for WENO7 (0..7) */
  const int ns = c->scheme == 2 ? 8 : 6, m0 = c->scheme == 2 ? 0 : 1;
  double gF[8][5], gQ[8][5];
  for (int s = 0; s < ns; ++s) {
    int m = s + m0;
    const double *Qm = q8 + m * 5;
    double km[3] = {met8[m * 4 + 0], met8[m * 4 + 1], met8[m * 4 + 2]};
    double Ft[5];
    flux_k(Qm, km, gamma, Ft);                          /* F~_m, Eq. (FGH) */
    if (!c->fp) {
      for (int v = 0; v < 5; ++v) { gF[s][v] = Ft[v]; gQ[s][v] = qt[m][v]; }
    } else if (c->form == 1) {
      /* Eq. (my_point1): WENO acts on F~_m - F~*_m and on (Q_m - Q*)/J_m */
      double Fs[5];
      flux_k(Qs, km, gamma, Fs);                        /* F~*_m = F(Q*) . k_m, Eq. (flux_split_detail) */
      for (int v = 0; v < 5; ++v) {
        gF[s][v] = Ft[v] - Fs[v];
        gQ[s][v] = (Qm[v] - Qs[v]) * invJ[m];
      }
    } else {
      /* Eq. (my_point2)/(my_point3): F~_m - F~*_m + F~*_{i+1/2} = F~_m - F(Q*).(k_m - k_face), and
         Eq. (Linear_upwind_LFspliting): (Q-Q*)/J_m + Q*(1/J)_face = Q~_m - Q*((1/J)_m - (1/J)_face) */
      double dk[3] = {km[0] - kf[0], km[1] - kf[1], km[2] - kf[2]};
      double Fd[5];
      flux_k(Qs, dk, gamma, Fd);
      for (int v = 0; v < 5; ++v) {
        gF[s][v] = Ft[v] - Fd[v];
        gQ[s][v] = qt[m][v] - Qs[v] * (invJ[m] - invJf);
      }
    }
  }
  /* eigensystem at i+1/2 (Roe average of cells i, i+1; normal from the face metric) */
  double Lm[25], Rm[25];
  if (c->charwise) {
    or_eigensystem(q8 + i0 * 5, q8 + (i0 + 1) * 5, kf, gamma, Lm, Rm);
  } else {
    for (int r = 0; r < 25; ++r) { Lm[r] = (r % 6 == 0) ? 1.0 : 0.0; Rm[r] = Lm[r]; }
  }
  /* local Lax-Friedrichs speeds: max over the stencil cells of |eigenvalue| (Sec. 4: local LF),
     or the global speeds passed in */
  double lam[5] = {0, 0, 0, 0, 0};
  if (lam_given)
    for (int v = 0; v < 5; ++v) lam[v] = lam_given[v];
  for (int s = 0; s < ns && !lam_given; ++s) {
    int m = s + m0;
    double km[3] = {met8[m * 4 + 0], met8[m * 4 + 1], met8[m * 4 + 2]};
    double e[5];
    point_eigs(q8 + m * 5, km, invJ[m], gamma, e);
    if (c->charwise) {
      for (int v = 0; v < 5; ++v) if (fabs(e[v]) > lam[v]) lam[v] = fabs(e[v]);
    } else {
      double mx = fabs(e[0]) > fabs(e[4]) ? fabs(e[0]) : fabs(e[4]);
      for (int v = 0; v < 5; ++v) if (mx > lam[v]) lam[v] = mx;
    }
  }
  /* characteristic Lax-Friedrichs splitting and reconstruction per field */
  double h[5];
  for (int sf = 0; sf < 5; ++sf) {
    double fpl[8], fmi[8];
    for (int s = 0; s < ns; ++s) {
      double a = 0.0, b = 0.0;
      for (int v = 0; v < 5; ++v) { a += Lm[sf * 5 + v] * gF[s][v]; b += Lm[sf * 5 + v] * gQ[s][v]; }
      fpl[s] = 0.5 * (a + lam[sf] * b);
      fmi[s] = 0.5 * (a - lam[sf] * b);
    }
    double rp, rm;
    if (c->scheme == 2) {
      double vp[7], vm[7];
      for (int t = 0; t < 7; ++t) { vp[t] = fpl[t]; vm[t] = fmi[7 - t]; }   /* i-3..i+3 and i+4..i-2 */
      rp = or_weno7(vp);
      rm = or_weno7(vm);
    } else if (c->scheme == 3) {
      double vp[6], vm[6];
      for (int t = 0; t < 6; ++t) { vp[t] = fpl[t]; vm[t] = fmi[5 - t]; }   /* i-2..i+3 and i+3..i-2 */
      rp = or_wenocu6(vp);
      rm = or_wenocu6(vm);
    } else {
      double vp[5] = {fpl[0], fpl[1], fpl[2], fpl[3], fpl[4]};        /* i-2 .. i+2 */
      double vm[5] = {fmi[5], fmi[4], fmi[3], fmi[2], fmi[1]};        /* i+3 .. i-1 */
      rp = c->scheme == 1 ? or_lu5(vp) : or_weno5(vp);
      rm = c->scheme == 1 ? or_lu5(vm) : or_weno5(vm);
    }
    h[sf] = rp + rm;
  }
  for (int v = 0; v < 5; ++v) {
    double s = 0.0;
    for (int sf = 0; sf < 5; ++sf) s += Rm[v * 5 + sf] * h[sf];
    out[v] = s;
  }
  if (c->fp && c->form == 1) {
    double Fsf[5];
    flux_k(Qs, kf, gamma, Fsf);                         /* + F~*_{i+1/2} */
    for (int v = 0; v < 5; ++v) out[v] += Fsf[v];
  }
}

/* ------------------------------------------------------------------------ */
/* Ghosted state: interior copy plus boundary layers (periodic image,          */
/* far-field state, or zero-gradient copy of the nearest interior point).      */
/* ------------------------------------------------------------------------ */
static int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

/* unit normal n = k/|k| of the boundary face of direction d on side s of the grid line
   through p, with k the order-M face metric (Sec. 3, Eq. xidJ) */
static void boundary_normal(const or_cfg *c, const double *met, const arr3 *A, size_t nb, int d, int s,
                            const int p[3], double nrm[3]) {
  double w[8], k[3] = {0.0, 0.0, 0.0};
  or_interp_coef(c->M, w);
  const int f = s ? c->n[d] - 1 : -1;          /* face f+1/2 */
  for (int m = 0; m < c->M; ++m) {
    int r[3] = {p[0], p[1], p[2]};
    r[d] = f - c->M / 2 + 1 + m;
    const size_t o = at3(A, r[0], r[1], r[2]);
    for (int a = 0; a < 3; ++a) k[a] += w[m] * met[(size_t)(3 * d + a) * nb + o];
  }
  const double len = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
  for (int a = 0; a < 3; ++a) nrm[a] = k[a] / len;
}

static double *ghost_state(const or_cfg *c, const double *met, const double *q, int G, int lo[3], int hi[3]) {
  for (int d = 0; d < 3; ++d) {
    int on = d < c->dims;
    lo[d] = on ? -G : 0;
    hi[d] = on ? c->n[d] + G : 1;
  }
  size_t nb = box_size(lo, hi);
  double *g = (double *)malloc(5 * nb * sizeof(double));
  const int ni = c->n[0], nj = c->n[1], nk = c->n[2];
  arr3 A = {{lo[0], lo[1], lo[2]}, {hi[0], hi[1], hi[2]}, NULL};
  for (int k = lo[2]; k < hi[2]; ++k)
    for (int j = lo[1]; j < hi[1]; ++j)
      for (int i = lo[0]; i < hi[0]; ++i) {
        int p[3] = {i, j, k}, src[3];
        int far = 0, nwall = 0, wd[3], ws[3];
        for (int d = 0; d < 3; ++d) src[d] = p[d];
        for (int d = 0; d < 3; ++d) {
          if (p[d] < 0 || p[d] >= c->n[d]) {
            int side = p[d] < 0 ? 0 : 1;
            int b = c->bc[d][side];
            const int mirror = side ? 2 * c->n[d] - 1 - p[d] : -1 - p[d];
            if (b == 0) src[d] = wrap(p[d], c->n[d]);
            else if (b == 1) far = 1;
            else if (b == 2) src[d] = p[d] < 0 ? 0 : c->n[d] - 1;
            else {
              const int t = d == 0 ? 1 : 0;           /* direction reversed through a cut */
              const int tt = p[t] < 0 ? 0 : (p[t] >= c->n[t] ? c->n[t] - 1 : p[t]);
              src[d] = mirror;
              if (b == 4 && (tt < c->cut || tt >= c->n[t] - c->cut)) {
                src[t] = c->n[t] - 1 - p[t];
              } else {
                wd[nwall] = d; ws[nwall] = side; ++nwall;
              }
            }
          }
        }
        for (int d = 0; d < 3; ++d)                   /* corner points: clamp what is left */
          if (src[d] < 0 || src[d] >= c->n[d]) src[d] = src[d] < 0 ? 0 : c->n[d] - 1;
        size_t o = at3(&A, i, j, k);
        double Q[5];
        for (int v = 0; v < 5; ++v)
          Q[v] = far ? c->qinf[v]
                     : q[(size_t)v * ni * nj * nk + ((size_t)src[2] * nj + src[1]) * ni + src[0]];
        for (int w = 0; w < nwall && !far; ++w) {
          double nrm[3];
          boundary_normal(c, met, &A, nb, wd[w], ws[w], p, nrm);
          const double mn = Q[1] * nrm[0] + Q[2] * nrm[1] + Q[3] * nrm[2];
          for (int a = 0; a < 3; ++a) Q[1 + a] -= 2.0 * mn * nrm[a];
        }
        for (int v = 0; v < 5; ++v) g[(size_t)v * nb + o] = Q[v];
      }
  return g;
}

int or_rhs(const or_cfg *c, const double *met, const double *q, double *R, double *dqdt) {
  if (!valid_cfg(c) || !met || !q) return 1;
  const int G = or_ghost_s(c->M, c->scheme);
  for (int d = 0; d < c->dims; ++d) if (c->n[d] < G) return 1;
  int lo[3], hi[3];
  double *g = ghost_state(c, met, q, G, lo, hi);
  arr3 A = {{lo[0], lo[1], lo[2]}, {hi[0], hi[1], hi[2]}, NULL};
  size_t nb = box_size(lo, hi);
  const int ni = c->n[0], nj = c->n[1], nk = c->n[2];
  size_t nc = (size_t)ni * nj * nk;
  double *Rl = (double *)calloc(5 * nc, sizeof(double));
  for (int d = 0; d < c->dims; ++d) {
    int nd = c->n[d];
    /* global Lax-Friedrichs (Sec. 4: used for the shock cases): the max of |eigenvalue|
       over every interior point of the block, per characteristic field */
    double glam[5] = {0, 0, 0, 0, 0};
    if (c->global_lf) {
      for (int k = 0; k < nk; ++k)
        for (int j = 0; j < nj; ++j)
          for (int i = 0; i < ni; ++i) {
            size_t o = at3(&A, i, j, k);
            double Q[5], km[3], e[5];
            for (int v = 0; v < 5; ++v) Q[v] = g[(size_t)v * nb + o];
            for (int a2 = 0; a2 < 3; ++a2) km[a2] = met[(size_t)(3 * d + a2) * nb + o];
            point_eigs(Q, km, met[(size_t)9 * nb + o], c->gamma, e);
            if (c->charwise) {
              for (int v = 0; v < 5; ++v) if (fabs(e[v]) > glam[v]) glam[v] = fabs(e[v]);
            } else {
              double mx = fabs(e[0]) > fabs(e[4]) ? fabs(e[0]) : fabs(e[4]);
              for (int v = 0; v < 5; ++v) if (mx > glam[v]) glam[v] = mx;
            }
          }
    }
    double *Fline = (double *)malloc((size_t)(nd + 1) * 5 * sizeof(double));
    int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;   /* transverse directions */
    for (int b = 0; b < c->n[t2]; ++b)
      for (int a = 0; a < c->n[t1]; ++a) {
        for (int f = -1; f < nd; ++f) {                 /* face f+1/2 between cells f, f+1 */
          double q8[40], met8[32];
          for (int m = 0; m < 8; ++m) {
            int p[3];
            p[d] = f - 3 + m; p[t1] = a; p[t2] = b;
            if (p[d] < -G || p[d] >= nd + G) {          /* outside every stencil when M < 8 */
              for (int v = 0; v < 5; ++v) q8[m * 5 + v] = NAN;
              for (int a2 = 0; a2 < 4; ++a2) met8[m * 4 + a2] = NAN;
              continue;
            }
            size_t o = at3(&A, p[0], p[1], p[2]);
            for (int v = 0; v < 5; ++v) q8[m * 5 + v] = g[(size_t)v * nb + o];
            for (int a2 = 0; a2 < 3; ++a2) met8[m * 4 + a2] = met[(size_t)(3 * d + a2) * nb + o];
            met8[m * 4 + 3] = met[(size_t)9 * nb + o];
          }
          if (c->global_lf) or_face_flux_lam(c, q8, met8, glam, Fline + (size_t)(f + 1) * 5);
          else or_face_flux(c, q8, met8, Fline + (size_t)(f + 1) * 5);
        }
        for (int i = 0; i < nd; ++i) {                  /* Eq. (aderivative) with Delta xi = 1 */
          int p[3];
          p[d] = i; p[t1] = a; p[t2] = b;
          size_t o = ((size_t)p[2] * nj + p[1]) * ni + p[0];
          for (int v = 0; v < 5; ++v)
            Rl[(size_t)v * nc + o] += Fline[(size_t)(i + 1) * 5 + v] - Fline[(size_t)i * 5 + v];
        }
      }
    free(Fline);
  }
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        size_t o = ((size_t)k * nj + j) * ni + i;
        double Jc = 1.0 / met[(size_t)9 * nb + at3(&A, i, j, k)];
        for (int v = 0; v < 5; ++v) {
          if (R) R[(size_t)v * nc + o] = Rl[(size_t)v * nc + o];
          if (dqdt) dqdt[(size_t)v * nc + o] = -Jc * Rl[(size_t)v * nc + o];   /* dQ/dt = -J R */
        }
      }
  free(Rl);
  free(g);
  return 0;
}

/* 3rd-order TVD Runge-Kutta of Gottlieb & Shu (Sec. 2.2), one step in place. */
int or_rk3_step(const or_cfg *c, const double *met, double *q, double dt) {
  if (!valid_cfg(c)) return 1;
  size_t nc = (size_t)c->n[0] * c->n[1] * c->n[2] * 5;
  double *L = (double *)malloc(nc * sizeof(double));
  double *q1 = (double *)malloc(nc * sizeof(double));
  double *q2 = (double *)malloc(nc * sizeof(double));
  int rc = or_rhs(c, met, q, NULL, L);
  for (size_t s = 0; s < nc; ++s) q1[s] = q[s] + dt * L[s];
  rc |= or_rhs(c, met, q1, NULL, L);
  for (size_t s = 0; s < nc; ++s) q2[s] = 0.75 * q[s] + 0.25 * (q1[s] + dt * L[s]);
  rc |= or_rhs(c, met, q2, NULL, L);
  for (size_t s = 0; s < nc; ++s) q[s] = (1.0 / 3.0) * q[s] + (2.0 / 3.0) * (q2[s] + dt * L[s]);
  free(L); free(q1); free(q2);
  return rc;
}

/* dt = CFL / max over points of sum_d (|U_d| + c |grad d|), grad d = J k_d. */
double or_cfl_dt(const or_cfg *c, const double *met, const double *q, double cfl) {
  const int G = or_ghost_s(c->M, c->scheme), ni = c->n[0], nj = c->n[1], nk = c->n[2];
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    int on = d < c->dims;
    lo[d] = on ? -G : 0;
    hi[d] = on ? c->n[d] + G : 1;
  }
  arr3 A = {{lo[0], lo[1], lo[2]}, {hi[0], hi[1], hi[2]}, NULL};
  size_t nb = box_size(lo, hi), nc = (size_t)ni * nj * nk;
  double smax = 0.0;
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        size_t o = ((size_t)k * nj + j) * ni + i, om = at3(&A, i, j, k);
        double Q[5];
        for (int v = 0; v < 5; ++v) Q[v] = q[(size_t)v * nc + o];
        double s = 0.0;
        for (int d = 0; d < c->dims; ++d) {
          double km[3] = {met[(size_t)(3 * d) * nb + om], met[(size_t)(3 * d + 1) * nb + om],
                          met[(size_t)(3 * d + 2) * nb + om]};
          double e[5];
          point_eigs(Q, km, met[(size_t)9 * nb + om], c->gamma, e);
          s += fabs(e[0]) > fabs(e[4]) ? fabs(e[0]) : fabs(e[4]);
        }
        if (s > smax) smax = s;
      }
  return cfl / smax;
}
