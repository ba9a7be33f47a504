/*
 * oracle.h - plain, serial, FP64 CPU reference of the free-stream-preserving (FP)
 * upwind conservative finite-difference residual of Su, Cai, Pan & Hu,
 * "Reformulated dissipation for the free-stream preserving of the conservative
 * finite difference schemes on curvilinear grids" (arXiv 2101.05886).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or helper with the CUDA library; the two are compared on the same seeded
 * inputs.
 *
 * Pins: every function is checked against values the paper prints, closed forms,
 * invariants or brute force (tests/test_oracle_pins.py), with one exception: parity
 * unpinned for the constants C = 20, q = 2, eps = 1e-40 of or_wenocu6, which come from
 * the cited WENOCU6 paper (not at hand); its other parts are pinned.
 *
 * Layouts (all C order, i fastest, float64):
 *   nodes : [dims][nk+2Gn][nj+2Gn][ni+2Gn]   (2-D: [2][nj+2Gn][ni+2Gn])
 *   met   : [10][nk+2G][nj+2G][ni+2G]         (2-D: [10][1][nj+2G][ni+2G])
 *           entry 3*d+a = (d-th curvilinear coordinate)_(x_a) / J, entry 9 = 1/J
 *   q, R  : [5][nk][nj][ni]  conserved variables (rho, rho u, rho v, rho w, rho E)
 * with G = max(3, M/2) and Gn >= G + 3M/2.
 */
#ifndef FP_ORACLE_H
#define FP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dims;        /* 2 or 3 */
  int n[3];        /* ni, nj, nk (nk = 1 in 2-D) */
  int M;           /* metric and face-interpolation order: 2, 4, 6 or 8 */
  int scheme;      /* 0 = WENO5-JS, 1 = 5th-order linear upwind, 2 = WENO7-JS, 3 = WENOCU6 */
  int fp;          /* 1 = free-stream-preserving form, 0 = plain scheme */
  int charwise;    /* 1 = characteristic-wise (Roe eigenvectors), 0 = component-wise */
  int form;        /* 2 = WENO(F_m - F*_m + F*_face) (Eq. my_point2), 1 = WENO(F_m - F*_m) + F*_face (Eq. my_point1) */
  int global_lf;   /* 0 = local Lax-Friedrichs speeds (stencil max), 1 = global (max over the block) */
  int bc[3][2];    /* 0 periodic, 1 far field (q_inf), 2 zero gradient, 3 slip wall,
                      4 C-grid cut (see below) */
  double gamma;
  double qinf[5];
  int cut;         /* code 4 only: cells t < cut and t >= n_t - cut of the reversed direction t
                      connect across the cut; the cells in between are slip wall */
} or_cfg;

/* Boundary rules for a ghost point at index x of direction d (x < 0 on side 0, x >= n_d on
   side 1), with the mirror index x' = -1 - x (side 0) or 2 n_d - 1 - x (side 1):
   - 3 slip wall: the wall is the boundary face; the ghost state is the state at x' with its
     momentum reflected about that face's unit normal n = k/|k| (k = the order-M face metric
     of direction d at the boundary face of the same grid line): m - 2 (m.n) n.
   - 4 C-grid cut: the boundary face of direction d is a cut through which the block meets
     itself with the transverse index t reversed (t = j for d = 0, t = i for d = 1, 2): the
     ghost state is the state at (x', t' = n_t - 1 - t) as it is.  Points with
     cut <= t < n_t - cut use the slip-wall rule instead (the body of a C-grid). */

int or_ghost(int M);                 /* G = max(3, M/2) for the 5th-order schemes */
int or_node_ghost(int M);            /* G + 3M/2 */
int or_ghost_s(int M, int scheme);   /* G = max(3 or 4 (WENO7), M/2) */
int or_node_ghost_s(int M, int scheme);
void or_interp_coef(int M, double c[8]);      /* face interpolation weights (Sec. 3) */
double or_weno5(const double v[5]);           /* WENO5-JS of v[0..4] = f_{i-2..i+2} at i+1/2 */
void or_weno5_parts(const double v[5], double q[3], double beta[3]);  /* its q_k and beta_k */
double or_lu5(const double v[5]);             /* linear upwind 5 = WENO with optimal weights */
double or_weno7(const double v[7]);           /* WENO7-JS of v[0..6] = f_{i-3..i+3} at i+1/2 */
void or_weno7_parts(const double v[7], double q[4], double beta[4]);
double or_wenocu6(const double v[6]);         /* WENOCU6 of v[0..5] = f_{i-2..i+3} at i+1/2 */
void or_wenocu6_parts(const double v[6], double q[4], double beta[4], double *tau);
void or_eigensystem(const double qL[5], const double qR[5], const double k[3], double gamma,
                    double L[25], double R[25]);
int or_metrics(const or_cfg *c, const double *nodes, int Gn, double *met);
/* face flux at i+1/2 from 8 consecutive cells i-3..i+4 along one direction d:
   q8 [8][5], met8 [8][4] = (k_x, k_y, k_z, 1/J) of that direction */
void or_face_flux(const or_cfg *c, const double q8[40], const double met8[32], double out[5]);
/* as or_face_flux with the Lax-Friedrichs speeds lam[5] given (global splitting) */
void or_face_flux_lam(const or_cfg *c, const double q8[40], const double met8[32], const double lam[5],
                      double out[5]);
int or_rhs(const or_cfg *c, const double *met, const double *q, double *R, double *dqdt);
int or_rk3_step(const or_cfg *c, const double *met, double *q, double dt);
double or_cfl_dt(const or_cfg *c, const double *met, const double *q, double cfl);

#ifdef __cplusplus
}
#endif
#endif
