/*
 * hope_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU reference ("oracle") of the HOPE cubed-sphere
 * shallow-water spatial operator and its Runge-Kutta stepping
 * (Zhou, "HOPE: an automatically differentiable high-order non-oscillatory
 * finite-volume shallow-water dynamic core", arXiv 2411.19185).
 *
 * Only the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code, header, table or
 * constant generator with the CUDA library; neither includes the other.
 *
 * Conventions (identical in meaning to the CUDA library, written separately):
 *   state q[v][p][j][i]   v = 0..2  (sqrtG*phi, sqrtG*phi*u, sqrtG*phi*v),
 *                         p = 0..5  (the paper's panels 1..6), j, i = 0..N-1,
 *                         i (x direction) fastest.
 *   sqrtG is the unit-sphere metric Jacobian (eq. 2.8 divided by r^2);
 *   phi in m^2/s^2, (u, v) contravariant in rad/s.
 *   extended arrays e[v][p][jj][ii], jj, ii = 0..N+2H-1, interior at offset H.
 *   per-cell reconstruction points (n_poc = 4*me + me*me), in this order:
 *     [0, me)        west edge   (xi = -1/2, eta = g_r)
 *     [me, 2me)      east edge   (xi = +1/2, eta = g_r)
 *     [2me, 3me)     south edge  (xi = g_r,  eta = -1/2)
 *     [3me, 4me)     north edge  (xi = g_r,  eta = +1/2)
 *     [4me + h*me + g]  cell point (xi = g_g, eta = g_h)
 *   with g_r the Gauss-Legendre nodes on [-1/2, 1/2].
 */
#ifndef HOPE_ORACLE_H
#define HOPE_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_TPP 0
#define ORC_WENO 1
#define ORC_WENO1D 2   /* dimension-by-dimension WENO-Z (fifth order only), section 5.5 */
#define ORC_SSPRK3 0
#define ORC_WSRK3 1

/* initial-condition cases for orc_ic */
#define ORC_IC_GEOSTROPHIC 2   /* params: alpha, u0, phi0                         */
#define ORC_IC_ROSSBY 6        /* params: omega_rh, K, R, h0                      */
#define ORC_IC_DAMBREAK 7      /* params: lon_c, lat_c, radius_rad, h_in, h_out   */
#define ORC_IC_BUMPS 8         /* geostrophic + n Gaussian bumps; params: alpha,u0,phi0,amp_m,
                                  radius_rad; extra = n pairs (lon, lat)          */
#define ORC_IC_GALEWSKY 11     /* perturbed jet, eqs. 5.16-5.18; params: umax, theta0, theta1,
                                  theta2, alpha, beta, hhat_m, phi0 (0: mean depth 10 km) */

/* analytic bottom surfaces for orc_set_topography_case; params (4 doubles):
   MOUNTAIN  hs0_m, R_rad, lon_c, lat_c   isolated cone of eq. 5.8
   ZONAL     hs0_m, alpha                  hs0 cos^2 of the latitude about the tilted axis
   HILL      hs0_m, R_rad, lon_c, lat_c   Gaussian hs0 exp(-(d/R)^2), d great-circle */
#define ORC_TOPO_MOUNTAIN 1
#define ORC_TOPO_ZONAL 2
#define ORC_TOPO_HILL 3

typedef struct orc orc;

orc *orc_new(int N, int k, int scheme, double radius, double gravity, double omega,
             double weno_eps, int ghost_iters);
void orc_free(orc *o);
/* Tilt the rotation axis by alpha_c (Williamson case-2 Coriolis parameter); 0 = eq. 2.5. */
void orc_set_coriolis_tilt(orc *o, double alpha_c);
int orc_npoc(const orc *o);
int orc_halo(const orc *o);

/* One evaluation of the spatial operator L(q) = dq/dt (eq. 3.1). */
void orc_tendency(orc *o, const double *q, double *dqdt);
/* L(q) at n selected cells (cells[c] = p*N*N + j*N + i): the same computation as
   orc_tendency with the reconstruction restricted to the cells the selected cells'
   edge fluxes and sources need; out[3][n]. */
void orc_tendency_cells(orc *o, const double *q, int n, const int *cells, double *out);
/* nsteps Runge-Kutta steps in place (rk = ORC_SSPRK3 or ORC_WSRK3). */
void orc_step(orc *o, double *q, double dt, int nsteps, int rk);
/* Total mass dx*dy*sum(q0) (the I() weighted sum of eq. 5.7), long-double accumulation. */
double orc_mass(const orc *o, const double *q);
/* Ghost fill by the iteration of section 3.3.1; ext receives the extended array.
   resid (may be NULL) receives the 2-norm of the last sweep's increment per variable. */
void orc_fill_ghosts(orc *o, const double *q, double *ext, double *resid);
/* Reconstruction at every point of every interior cell from an extended array:
   pts[v][p][j][i][n_poc]. */
void orc_reconstruct_all(orc *o, const double *ext, double *pts);
/* Cell averages of an analytic initial condition by me x me Gauss quadrature. */
void orc_ic(const orc *o, int ic_case, const double *params, int n_extra, const double *extra,
            double *q);
/* Bottom topography (eqs. 2.13-2.14): cell averages of sqrtG phi_s [p][j][i] (copied;
   NULL removes it), or an analytic surface averaged by the me x me Gauss rule.  With an
   analytic surface set, orc_ic reads its phi as phi_t and stores the depth phi_t - phi_s. */
void orc_set_topography(orc *o, const double *sbar);
void orc_set_topography_case(orc *o, int tcase, const double *params4);
void orc_get_topography(const orc *o, double *sbar);
double orc_topography_point(const orc *o, int panel, double X, double Y);
/* 0 (default): the total-geopotential form of eqs. 2.13-2.14; 1: the depth form of eqs.
   2.1 and 2.4 (for comparisons only). */
void orc_set_topography_form(orc *o, int form);
/* The cell average of psi_B (eq. 2.14) alone for state q: out[2][6][N][N]. */
void orc_topo_psib(orc *o, const double *q, double *out);
/* phi, u_s, v_s of an initial condition at one (lambda, theta) (params as orc_ic,
   8 doubles; no topography, no extra). */
void orc_ic_point(const orc *o, int ic_case, const double *params8, double lam, double th, double *out3);
/* Cell-averaged sqrtG (unit sphere) per cell, [p][j][i]. */
void orc_cell_sqrtg(const orc *o, double *out);
/* L1, L2, Linf error norms of phi (eqs. 5.4-5.7). */
void orc_norms(const orc *o, const double *q, const double *qref, double *out3);

/* ---- building blocks exposed for the pin tests ---- */
void orc_gauss(int m, double *x, double *w);
void orc_weights_1d(int n, int o0, double xi, double *out);
void orc_tpp_weights_2d(int k, double xi, double eta, double *out);
void orc_tpp_weights_2d_literal(int k, double xi, double eta, double *out);
void orc_tpp_dweights_2d(int k, double xi, double eta, int dir, double *out);
void orc_sqrtg_grad(double X, double Y, double *out2);
int orc_weno_gamma(int k, double xi, double eta, double *gam, double *resid);
double orc_weno_beta(int l, int o0x, int o0y, const double *Qsub);
double orc_weno_point(const orc *o, const double *stencil, int pt);
/* 1-D WENO-Z (dimension-by-dimension comparator): linear weights at xi and the value at
   xi from k cell averages v (offsets -H..H) with the given epsilon. */
int orc_weno1d_gamma(int k, double xi, double *gam, double *resid);
double orc_weno1d_point(int k, const double *v, double xi, double eps);
void orc_metric(double X, double Y, double *out7);
void orc_jacobian(int panel, double X, double Y, double *J4);
void orc_xyz(int panel, double X, double Y, double *xyz);
int orc_locate(const double *xyz, double *XY);
void orc_lmars(const orc *o, int dir, double X, double Y, const double *qL, const double *qR,
               double *F);
void orc_sources(const orc *o, int panel, double X, double Y, const double *qv, double *S);
/* LMARS with topography: sL, sR = sqrtG phi_s at the point on each side. */
void orc_lmars_topo(const orc *o, int dir, double X, double Y, const double *qL, const double *qR,
                    double sL, double sR, double *F);

/* ---- table exports for the PyTorch reference composition ---- */
int orc_ghost_count(const orc *o);
/* per ghost Gauss point two owner slots (w = 1 and 0, or 1/2 and 1/2 on a cube edge) */
void orc_ghost_tables(const orc *o, int *ring, int *B, int *ic, int *jc, double *wx, double *wy,
                      double *ratio, double *C, double *w);
void orc_edge_tables(const orc *o, int *B, int *sideB, int *tB, int *gB, double *ratio, double *C);
double orc_coriolis(const orc *o, int panel, double X, double Y);

#ifdef __cplusplus
}
#endif
#endif
