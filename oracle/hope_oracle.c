/*
 * hope_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct FP64 CPU reference ("oracle") of the HOPE
 * cubed-sphere shallow-water core (arXiv 2411.19185): geometry (section 2),
 * TPP reconstruction (section 3.1), genuine-2D WENO-Z (section 3.2), ghost-cell
 * interpolation (section 3.3.1 and the appendix), panel conversion (section
 * 3.3.2), the LMARS flux (section 3.4), Gauss quadrature (eqs. 3.5-3.6), the
 * finite-volume tendency (eq. 3.1) and Runge-Kutta stepping (section 3.5).
 *
 * Only the tests, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it.  No code is shared with the CUDA library.
 *
 * Small setup solves (1-D cell-average systems, the WENO least-squares normal
 * equations) run in long double; everything on the data path is double.
 * Loops over cells carry OpenMP pragmas; every iteration writes only its own
 * outputs, so results do not depend on the thread count.
 *
 * Readings of passages that are garbled or silent in the paper are marked
 * "reading:" at the point of use.
 */
#include "hope_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI_L 3.141592653589793238462643383279502884L
#define QPI (M_PI / 4.0)
#define MAXK 15

/* ------------------------------------------------------------------------- */
/* small dense long-double solve with partial pivoting: A (n x n, row major)  */
/* is overwritten, b receives the solution.                                   */
/* ------------------------------------------------------------------------- */
static void solve_ld(int n, long double *A, long double *b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r * n + c]) > fabsl(A[piv * n + c])) piv = r;
    if (piv != c) {
      for (int j = 0; j < n; ++j) {
        long double t = A[c * n + j];
        A[c * n + j] = A[piv * n + j];
        A[piv * n + j] = t;
      }
      long double t = b[c];
      b[c] = b[piv];
      b[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      long double f = A[r * n + c] / A[c * n + c];
      if (f == 0.0L) continue;
      for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    long double s = b[r];
    for (int j = r + 1; j < n; ++j) s -= A[r * n + j] * b[j];
    b[r] = s / A[r * n + r];
  }
}

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre rule on [-1/2, 1/2] (weights sum to 1), used for the edge   */
/* averages (eq. 3.5) and the cell averages (eq. 3.6).  Newton iteration on   */
/* the Legendre polynomial P_m from the standard cosine initial guess.        */
/* ------------------------------------------------------------------------- */
void orc_gauss(int m, double *x, double *w) {
  for (int i = 0; i < m; ++i) {
    long double z = cosl(PI_L * (i + 0.75L) / (m + 0.5L));
    long double dp = 0.0L;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1.0L, p1 = z;
      for (int n = 2; n <= m; ++n) {
        long double p2 = ((2 * n - 1) * z * p1 - (n - 1) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      if (m == 1) { p1 = z; p0 = 1.0L; }
      /* P_m = p1, P_{m-1} = p0 */
      dp = m * (z * p1 - p0) / (z * z - 1.0L);
      long double dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-30L) break;
    }
    {
      long double p0 = 1.0L, p1 = z;
      for (int n = 2; n <= m; ++n) {
        long double p2 = ((2 * n - 1) * z * p1 - (n - 1) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      if (m == 1) { p1 = z; p0 = 1.0L; }
      dp = m * (z * p1 - p0) / (z * z - 1.0L);
    }
    /* ascending order on [-1/2, 1/2] */
    x[m - 1 - i] = (double)(0.5L * z);
    w[m - 1 - i] = (double)(1.0L / ((1.0L - z * z) * dp * dp));
  }
}

/* ------------------------------------------------------------------------- */
/* 1-D cell-average reconstruction weights (1-D slice of eqs. 3.7-3.15):      */
/* the stencil is n unit cells centred at offsets o0, o0+1, ..., o0+n-1 from  */
/* the target cell; the polynomial has monomials xi^a, a = 0..n-1 (reading    */
/* of eq. 3.7: exponents start at 0, origin at the target-cell centre);       */
/* out[j] is the weight of cell j in the value at xi:  r = A^{-T} c(xi).      */
/* Monomials are scaled by s = max|offset|+1/2 for conditioning only.         */
/* ------------------------------------------------------------------------- */
static void weights_1d_any(int n, int o0, long double xi, int deriv, long double *out) {
  long double A[MAXK * MAXK], b[MAXK];
  long double s = 0.5L;
  for (int j = 0; j < n; ++j) {
    long double a = fabsl((long double)(o0 + j)) + 0.5L;
    if (a > s) s = a;
  }
  /* M[a][j] = integral over cell j of (x/s)^a dx  (transpose of eq. 3.11's A) */
  for (int j = 0; j < n; ++j) {
    long double lo = ((long double)(o0 + j) - 0.5L) / s;
    long double hi = ((long double)(o0 + j) + 0.5L) / s;
    long double plo = lo, phi = hi;
    for (int a = 0; a < n; ++a) {
      A[a * n + j] = s * (phi - plo) / (long double)(a + 1);
      plo *= lo;
      phi *= hi;
    }
  }
  long double c = 1.0L;
  if (!deriv) {
    for (int a = 0; a < n; ++a) {
      b[a] = c;
      c *= xi / s;
    }
  } else { /* d/dxi (xi/s)^a = a (xi/s)^(a-1) / s */
    b[0] = 0.0L;
    for (int a = 1; a < n; ++a) {
      b[a] = (long double)a * c / s;
      c *= xi / s;
    }
  }
  solve_ld(n, A, b);
  for (int j = 0; j < n; ++j) out[j] = b[j];
}

static void weights_1d_ld(int n, int o0, long double xi, long double *out) {
  weights_1d_any(n, o0, xi, 0, out);
}

void orc_weights_1d(int n, int o0, double xi, double *out) {
  long double t[MAXK];
  weights_1d_ld(n, o0, (long double)xi, t);
  for (int j = 0; j < n; ++j) out[j] = (double)t[j];
}

/* TPP weights of a central k x k stencil at (xi, eta): R = r_x (x) r_y, the   */
/* tensor-product form of R = C A^{-1} (eq. 3.15) for the tensor-product      */
/* basis of eq. 3.7.  Layout out[b*k + a]: a = x offset + H, b = y offset + H. */
void orc_tpp_weights_2d(int k, double xi, double eta, double *out) {
  int H = (k - 1) / 2;
  long double rx[MAXK], ry[MAXK];
  weights_1d_ld(k, -H, xi, rx);
  weights_1d_ld(k, -H, eta, ry);
  for (int b = 0; b < k; ++b)
    for (int a = 0; a < k; ++a) out[b * k + a] = (double)(rx[a] * ry[b]);
}

/* Weights of the x- (dir 0) or y-derivative (dir 1), with respect to the      */
/* cell-unit coordinate, of the same tensor-product polynomial at (xi, eta):    */
/* r_x' (x) r_y or r_x (x) r_y'.  Used for the gradient of phi_t in eq. 2.14.   */
void orc_tpp_dweights_2d(int k, double xi, double eta, int dir, double *out) {
  int H = (k - 1) / 2;
  long double rx[MAXK], ry[MAXK];
  weights_1d_any(k, -H, xi, dir == 0, rx);
  weights_1d_any(k, -H, eta, dir == 1, ry);
  for (int b = 0; b < k; ++b)
    for (int a = 0; a < k; ++a) out[b * k + a] = (double)(rx[a] * ry[b]);
}

/* The same weights by the literal 2-D route of eqs. 3.7-3.15: assemble the    */
/* k^2 x k^2 cell-average matrix A of the monomials x^a y^b and solve          */
/* A^T r = c(xi, eta).  Only for small k (used to pin the tensor form).       */
void orc_tpp_weights_2d_literal(int k, double xi, double eta, double *out) {
  int H = (k - 1) / 2, n = k * k;
  long double *A = (long double *)malloc(sizeof(long double) * n * n);
  long double *b = (long double *)malloc(sizeof(long double) * n);
  long double s = H + 0.5L;
  for (int cb = 0; cb < k; ++cb)
    for (int ca = 0; ca < k; ++ca) {
      int cell = cb * k + ca; /* cell offsets (ca-H, cb-H) */
      for (int eb = 0; eb < k; ++eb)
        for (int ea = 0; ea < k; ++ea) {
          int term = eb * k + ea; /* monomial (x/s)^ea (y/s)^eb */
          long double xl = (ca - H - 0.5L) / s, xh = (ca - H + 0.5L) / s;
          long double yl = (cb - H - 0.5L) / s, yh = (cb - H + 0.5L) / s;
          long double ix = s * (powl(xh, ea + 1) - powl(xl, ea + 1)) / (ea + 1);
          long double iy = s * (powl(yh, eb + 1) - powl(yl, eb + 1)) / (eb + 1);
          A[term * n + cell] = ix * iy;
        }
    }
  for (int eb = 0; eb < k; ++eb)
    for (int ea = 0; ea < k; ++ea)
      b[eb * k + ea] = powl((long double)xi / s, ea) * powl((long double)eta / s, eb);
  solve_ld(n, A, b);
  for (int i = 0; i < n; ++i) out[i] = (double)b[i];
  free(A);
  free(b);
}

/* ------------------------------------------------------------------------- */
/* Genuine-2D WENO building blocks (section 3.2).                              */
/* Sub-stencil (sx, sy), sx, sy = 0..l-1, covers the l x l cells with offsets  */
/* [sx-H, sx-H+l-1] x [sy-H, sy-H+l-1]; it is sub-stencil number sy*l + sx.    */
/* ------------------------------------------------------------------------- */
static void sub_weights_2d(int k, int sx, int sy, long double xi, long double eta, long double *out) {
  int H = (k - 1) / 2, l = (k + 1) / 2;
  long double rx[MAXK], ry[MAXK];
  weights_1d_ld(l, sx - H, xi, rx);
  weights_1d_ld(l, sy - H, eta, ry);
  for (int b = 0; b < l; ++b)
    for (int a = 0; a < l; ++a) out[b * l + a] = rx[a] * ry[b];
}

/* Optimal linear weights gamma at (xi, eta) by the least-squares procedure of */
/* eqs. 3.16-3.19: R_L gamma = R_H with R_L's columns the sub-stencil weights  */
/* extended into the k x k stencil (matrix E), solved through the normal       */
/* equations in long double.  Returns s; resid = max |R_L gamma - R_H|.        */
int orc_weno_gamma(int k, double xi, double eta, double *gam, double *resid) {
  int H = (k - 1) / 2, l = (k + 1) / 2, s = l * l, m = k * k;
  long double *RL = (long double *)calloc((size_t)m * s, sizeof(long double));
  long double RH[MAXK * MAXK], sub[MAXK * MAXK];
  long double rx[MAXK], ry[MAXK];
  weights_1d_ld(k, -H, xi, rx);
  weights_1d_ld(k, -H, eta, ry);
  for (int b = 0; b < k; ++b)
    for (int a = 0; a < k; ++a) RH[b * k + a] = rx[a] * ry[b];
  for (int sy = 0; sy < l; ++sy)
    for (int sx = 0; sx < l; ++sx) {
      int i = sy * l + sx;
      sub_weights_2d(k, sx, sy, xi, eta, sub);
      for (int b = 0; b < l; ++b)
        for (int a = 0; a < l; ++a) /* extension: sub-stencil cell -> big-stencil cell */
          RL[(size_t)((sy + b) * k + (sx + a)) * s + i] = sub[b * l + a];
    }
  long double *NE = (long double *)calloc((size_t)s * s, sizeof(long double));
  long double rhs[MAXK * MAXK];
  for (int i = 0; i < s; ++i) {
    long double t = 0.0L;
    for (int r = 0; r < m; ++r) t += RL[(size_t)r * s + i] * RH[r];
    rhs[i] = t;
    for (int j = 0; j < s; ++j) {
      long double u = 0.0L;
      for (int r = 0; r < m; ++r) u += RL[(size_t)r * s + i] * RL[(size_t)r * s + j];
      NE[i * s + j] = u;
    }
  }
  solve_ld(s, NE, rhs);
  long double mx = 0.0L;
  for (int r = 0; r < m; ++r) {
    long double t = -RH[r];
    for (int i = 0; i < s; ++i) t += RL[(size_t)r * s + i] * rhs[i];
    if (fabsl(t) > mx) mx = fabsl(t);
  }
  for (int i = 0; i < s; ++i) gam[i] = (double)rhs[i];
  if (resid) *resid = (double)mx;
  free(RL);
  free(NE);
  return s;
}

/* Monomial coefficients of a sub-stencil's 1-D polynomial: C[a][j] such that  */
/* p(xi) = sum_a (sum_j C[a][j] qbar_j) xi^a (no scaling).                     */
static void coeffs_1d(int l, int o0, long double *C) {
  long double A[MAXK * MAXK], e[MAXK];
  for (int j = 0; j < l; ++j) {
    for (int r = 0; r < l; ++r) {
      long double lo = (long double)(o0 + r) - 0.5L, hi = (long double)(o0 + r) + 0.5L;
      for (int a = 0; a < l; ++a) A[r * l + a] = (powl(hi, a + 1) - powl(lo, a + 1)) / (a + 1);
    }
    for (int r = 0; r < l; ++r) e[r] = (r == j) ? 1.0L : 0.0L;
    solve_ld(l, A, e); /* column j of A^{-1} */
    for (int a = 0; a < l; ++a) C[a * l + j] = e[a];
  }
}

/* d^al/dx^al of x^a at x */
static long double dmono(int a, int al, long double x) {
  if (al > a) return 0.0L;
  long double c = 1.0L;
  for (int t = 0; t < al; ++t) c *= (long double)(a - t);
  return c * powl(x, a - al);
}

/* Smoothness indicator of one sub-stencil on the target cell [-1/2,1/2]^2.    */
/* reading (eq. 3.25 is garbled): beta = sum over (al1, al2) != (0,0),         */
/* al1, al2 <= l-1, of the integral of the SQUARED mixed derivative            */
/* d^(al1+al2) p / dx^al1 dy^al2 over the unit target cell (no length weights, */
/* the cell is a unit square).  The integral is taken with an l x l            */
/* Gauss-Legendre rule, exact for these degree-2(l-1) integrands.              */
/* Qsub[b*l + a] holds the sub-stencil cell averages, first cell at offset     */
/* (o0x, o0y).                                                                 */
double orc_weno_beta(int l, int o0x, int o0y, const double *Qsub) {
  long double Cx[MAXK * MAXK], Cy[MAXK * MAXK], c2[MAXK * MAXK];
  coeffs_1d(l, o0x, Cx);
  coeffs_1d(l, o0y, Cy);
  for (int eb = 0; eb < l; ++eb)
    for (int ea = 0; ea < l; ++ea) {
      long double t = 0.0L;
      for (int b = 0; b < l; ++b)
        for (int a = 0; a < l; ++a) t += Cx[ea * l + a] * Cy[eb * l + b] * Qsub[b * l + a];
      c2[eb * l + ea] = t;
    }
  double gx[MAXK], gw[MAXK];
  orc_gauss(l, gx, gw);
  long double beta = 0.0L;
  for (int a2 = 0; a2 < l; ++a2)
    for (int a1 = 0; a1 < l; ++a1) {
      if (a1 == 0 && a2 == 0) continue;
      for (int qy = 0; qy < l; ++qy)
        for (int qx = 0; qx < l; ++qx) {
          long double v = 0.0L;
          for (int eb = 0; eb < l; ++eb)
            for (int ea = 0; ea < l; ++ea)
              v += c2[eb * l + ea] * dmono(ea, a1, gx[qx]) * dmono(eb, a2, gx[qy]);
          beta += (long double)gw[qx] * gw[qy] * v * v;
        }
    }
  return (double)beta;
}


/* ------------------------------------------------------------------------- */
/* Dimension-by-dimension WENO-Z, the 1-D comparator of section 5.5 (fifth     */
/* order): the 1-D WENO-Z of Borges et al. (2008) on the k cell averages of a  */
/* line, at xi.  Sub-stencil s (s = 0..l-1) covers offsets [s-H, s-H+l-1];     */
/* the linear weights solve sum_s gamma_s r_s = r_k (the 1-D form of eqs.      */
/* 3.16-3.19, least squares in long double), split with theta = 3 as in eq.    */
/* 3.20 (reading c2); beta_s is the Jiang-Shu indicator sum_{m=1}^{l-1} of the  */
/* integral of (p_s^(m))^2 over the unit target cell; tau = |beta_0 -          */
/* beta_{l-1}|; alpha = gamma (1 + tau / (beta + eps)) (reading c31).          */
/* ------------------------------------------------------------------------- */
int orc_weno1d_gamma(int k, double xi, double *gam, double *resid) {
  int H = (k - 1) / 2, l = (k + 1) / 2;
  long double RH[MAXK], RL[MAXK * MAXK], sub[MAXK], NE[MAXK * MAXK], rhs[MAXK];
  weights_1d_ld(k, -H, xi, RH);
  for (int r = 0; r < k * l; ++r) RL[r] = 0.0L;
  for (int sb = 0; sb < l; ++sb) {
    weights_1d_ld(l, sb - H, xi, sub);
    for (int a = 0; a < l; ++a) RL[(sb + a) * l + sb] = sub[a];
  }
  for (int i = 0; i < l; ++i) {
    long double t = 0.0L;
    for (int r = 0; r < k; ++r) t += RL[r * l + i] * RH[r];
    rhs[i] = t;
    for (int j = 0; j < l; ++j) {
      long double u = 0.0L;
      for (int r = 0; r < k; ++r) u += RL[r * l + i] * RL[r * l + j];
      NE[i * l + j] = u;
    }
  }
  solve_ld(l, NE, rhs);
  long double mx = 0.0L;
  for (int r = 0; r < k; ++r) {
    long double t = -RH[r];
    for (int i = 0; i < l; ++i) t += RL[r * l + i] * rhs[i];
    if (fabsl(t) > mx) mx = fabsl(t);
  }
  for (int i = 0; i < l; ++i) gam[i] = (double)rhs[i];
  if (resid) *resid = (double)mx;
  return l;
}

static double beta_1d(int l, int o0, const double *v) {
  long double C[MAXK * MAXK], c[MAXK];
  coeffs_1d(l, o0, C);
  for (int a = 0; a < l; ++a) {
    long double t = 0.0L;
    for (int j = 0; j < l; ++j) t += C[a * l + j] * v[j];
    c[a] = t;
  }
  double gx[MAXK], gw[MAXK];
  orc_gauss(l, gx, gw);
  long double b = 0.0L;
  for (int m = 1; m < l; ++m)
    for (int q = 0; q < l; ++q) {
      long double d = 0.0L;
      for (int a = 0; a < l; ++a) d += c[a] * dmono(a, m, gx[q]);
      b += (long double)gw[q] * d * d;
    }
  return (double)b;
}

/* 1-D tables at one position: sub-stencil weights r[l][l] and the split weights */
typedef struct {
  double r[MAXK * MAXK], gp[MAXK], gm[MAXK], sp, sm;
} w1d_t;

static void w1d_tables(int k, double xi, w1d_t *t) {
  int H = (k - 1) / 2, l = (k + 1) / 2;
  long double sub[MAXK];
  for (int sb = 0; sb < l; ++sb) {
    weights_1d_ld(l, sb - H, xi, sub);
    for (int a = 0; a < l; ++a) t->r[sb * l + a] = (double)sub[a];
  }
  double gam[MAXK];
  orc_weno1d_gamma(k, xi, gam, NULL);
  t->sp = t->sm = 0.0;
  for (int i = 0; i < l; ++i) {
    t->gp[i] = 0.5 * (3.0 * fabs(gam[i]) + gam[i]);
    t->gm[i] = 0.5 * (3.0 * fabs(gam[i]) - gam[i]);
    t->sp += t->gp[i];
    t->sm += t->gm[i];
  }
}

static double w1d_value(int k, const w1d_t *t, const double *v, double eps) {
  int H = (k - 1) / 2, l = (k + 1) / 2;
  double beta[MAXK], p[MAXK], ap[MAXK], am[MAXK], sap = 0.0, sam = 0.0;
  for (int sb = 0; sb < l; ++sb) {
    double u = 0.0;
    for (int a = 0; a < l; ++a) u += t->r[sb * l + a] * v[sb + a];
    p[sb] = u;
    beta[sb] = beta_1d(l, sb - H, v + sb);
  }
  double tau = fabs(beta[0] - beta[l - 1]);
  for (int sb = 0; sb < l; ++sb) {
    double f = 1.0 + tau / (beta[sb] + eps);
    ap[sb] = t->gp[sb] / t->sp * f;
    am[sb] = t->gm[sb] / t->sm * f;
    sap += ap[sb];
    sam += am[sb];
  }
  double qp = 0.0, qm = 0.0;
  for (int sb = 0; sb < l; ++sb) {
    qp += ap[sb] / sap * p[sb];
    qm += am[sb] / sam * p[sb];
  }
  return t->sp * qp - t->sm * qm;
}

double orc_weno1d_point(int k, const double *v, double xi, double eps) {
  w1d_t t;
  w1d_tables(k, xi, &t);
  return w1d_value(k, &t, v, eps);
}
/* ------------------------------------------------------------------------- */
/* Geometry (section 2): gnomonic equiangular cube, unit sphere.               */
/* Panel p (0-based, paper's panel p+1) maps (X, Y) = (tan x, tan y) to        */
/* (n_p + X e1_p + Y e2_p)/delta.  Panels 1-4 are centred on the equator at    */
/* longitude (p-1)*pi/2 with X = tan(lambda - lambda_c) and                    */
/* Y = tan(theta)/cos(lambda - lambda_c); panel 5 (north) has                  */
/* X = sin(lambda)/tan(theta), Y = -cos(lambda)/tan(theta); panel 6 (south)    */
/* X = -sin(lambda)/tan(theta), Y = -cos(lambda)/tan(theta): the forms for     */
/* which the paper's J (eqs. 2.10-2.11) and sin(theta) (eq. 2.5) hold.         */
/* ------------------------------------------------------------------------- */
static const double FR_N[6][3] = {{1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const double FR_E1[6][3] = {{0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {1, 0, 0}, {0, 1, 0}, {0, 1, 0}};
static const double FR_E2[6][3] = {{0, 0, 1}, {0, 0, 1}, {0, 0, 1}, {0, 0, 1}, {-1, 0, 0}, {1, 0, 0}};

void orc_xyz(int p, double X, double Y, double *xyz) {
  double d = sqrt(1.0 + X * X + Y * Y);
  for (int c = 0; c < 3; ++c) xyz[c] = (FR_N[p][c] + X * FR_E1[p][c] + Y * FR_E2[p][c]) / d;
}

/* Panels owning a point: largest projection on the panel normal.  Returns the */
/* number of owners, 1, or 2 for a point on a cube edge (projections within    */
/* 1e-12), and the owners in B[0], B[1] (lower panel first).                   */
static int owner_panels(const double *xyz, int exclude, int *B) {
  double d[6], bv = -2.0;
  for (int p = 0; p < 6; ++p) {
    d[p] = xyz[0] * FR_N[p][0] + xyz[1] * FR_N[p][1] + xyz[2] * FR_N[p][2];
    if (p != exclude && d[p] > bv) bv = d[p];
  }
  int n = 0;
  for (int p = 0; p < 6 && n < 2; ++p)
    if (p != exclude && d[p] > bv - 1e-12) B[n++] = p;
  return n;
}

/* Panel owning a point: largest projection on the panel normal; a tie (point */
/* on a cube edge, up to 1e-12) goes to the lower panel number.                 */
static int owner_panel(const double *xyz, int exclude) {
  int best = -1;
  double bv = -2.0;
  for (int p = 0; p < 6; ++p) {
    if (p == exclude) continue;
    double d = xyz[0] * FR_N[p][0] + xyz[1] * FR_N[p][1] + xyz[2] * FR_N[p][2];
    if (d > bv + 1e-12) { bv = d; best = p; }
  }
  return best;
}

static void to_panel(int p, const double *xyz, double *XY) {
  double t = xyz[0] * FR_N[p][0] + xyz[1] * FR_N[p][1] + xyz[2] * FR_N[p][2];
  XY[0] = (xyz[0] * FR_E1[p][0] + xyz[1] * FR_E1[p][1] + xyz[2] * FR_E1[p][2]) / t;
  XY[1] = (xyz[0] * FR_E2[p][0] + xyz[1] * FR_E2[p][1] + xyz[2] * FR_E2[p][2]) / t;
}

int orc_locate(const double *xyz, double *XY) {
  int p = owner_panel(xyz, -1);
  to_panel(p, xyz, XY);
  return p;
}

/* Metric terms (unit sphere), eqs. 2.6-2.8; reading c5: the denominator of    */
/* eq. 2.6 is (1+X^2)(1+Y^2).  out7 = sqrtG, G^11, G^12, G^22, G_11, G_12, G_22. */
void orc_metric(double X, double Y, double *o) {
  double d2 = 1.0 + X * X + Y * Y, d = sqrt(d2);
  double ax = 1.0 + X * X, ay = 1.0 + Y * Y;
  o[0] = ax * ay / (d2 * d);
  double c = d2 / (ax * ay);
  o[1] = c * ay;
  o[2] = c * X * Y;
  o[3] = c * ax;
  double cl = ax * ay / (d2 * d2);
  o[4] = cl * ax;
  o[5] = -cl * X * Y;
  o[6] = cl * ay;
}

/* Gradient of the unit-sphere sqrtG of eq. 2.8 with respect to (x, y):        */
/* with A = (1+X^2)(1+Y^2) and delta^2 = 1+X^2+Y^2, d(A delta^-3)/dX =          */
/* X (1+Y^2)(2Y^2 - X^2 - 1) / delta^5, and dX/dx = 1 + X^2 (symmetric in y).   */
void orc_sqrtg_grad(double X, double Y, double *out2) {
  double d2 = 1.0 + X * X + Y * Y, d5 = d2 * d2 * sqrt(d2);
  double ax = 1.0 + X * X, ay = 1.0 + Y * Y;
  out2[0] = X * ay * (2.0 * Y * Y - X * X - 1.0) / d5 * ax;
  out2[1] = Y * ax * (2.0 * X * X - Y * Y - 1.0) / d5 * ay;
}

static void lonlat(const double *xyz, double *lam, double *th) {
  *lam = atan2(xyz[1], xyz[0]);
  *th = atan2(xyz[2], sqrt(xyz[0] * xyz[0] + xyz[1] * xyz[1]));
}

/* J of eq. 2.10 (r = 1), row major: (u_s, v_s) = r J (u, v). */
void orc_jacobian(int p, double X, double Y, double *J) {
  double xyz[3], lam, th;
  orc_xyz(p, X, Y, xyz);
  lonlat(xyz, &lam, &th);
  double ct = cos(th), st = sin(th);
  if (p < 4) {
    double lp = lam - 0.5 * M_PI * p; /* eq. 2.11 */
    J[0] = ct;
    J[1] = 0.0;
    J[2] = -st * ct * tan(lp);
    J[3] = cos(lp) * ct * ct + st * st / cos(lp);
  } else {
    double tt = tan(th);
    double g1 = 1.0 + sin(lam) * sin(lam) / (tt * tt);
    double g2 = 1.0 + cos(lam) * cos(lam) / (tt * tt);
    double sgn = (p == 4) ? 1.0 : -1.0;
    J[0] = sgn * cos(lam) * st * g1;
    J[1] = sin(lam) * st * g2;
    J[2] = -sgn * sin(lam) * st * st * g1;
    J[3] = cos(lam) * st * st * g2;
  }
}

/* sin(latitude) by eq. 2.5 */
static double sin_lat(int p, double X, double Y) {
  double d = sqrt(1.0 + X * X + Y * Y);
  if (p < 4) return Y / d;
  return (p == 4) ? 1.0 / d : -1.0 / d;
}

static void inv2(const double *A, double *B) {
  double det = A[0] * A[3] - A[1] * A[2];
  B[0] = A[3] / det;
  B[1] = -A[1] / det;
  B[2] = -A[2] / det;
  B[3] = A[0] / det;
}
static void mul2(const double *A, const double *B, double *C) {
  C[0] = A[0] * B[0] + A[1] * B[2];
  C[1] = A[0] * B[1] + A[1] * B[3];
  C[2] = A[2] * B[0] + A[3] * B[2];
  C[3] = A[2] * B[1] + A[3] * B[3];
}

/* Conversion of a field value from panel B at (XB, YB) to panel A at         */
/* (XA, YA), the same point of the sphere: mass ratio sqrtG_A/sqrtG_B          */
/* (eq. 3.26) and momentum matrix C = (sqrtG_A/sqrtG_B) J_A^{-1} J_B           */
/* (eqs. 3.27-3.29).                                                            */
static void conversion(int A, double XA, double YA, int B, double XB, double YB, double *ratio,
                       double *C) {
  double mA[7], mB[7], JA[4], JB[4], JAi[4];
  orc_metric(XA, YA, mA);
  orc_metric(XB, YB, mB);
  *ratio = mA[0] / mB[0];
  orc_jacobian(A, XA, YA, JA);
  orc_jacobian(B, XB, YB, JB);
  inv2(JA, JAi);
  mul2(JAi, JB, C);
  for (int i = 0; i < 4; ++i) C[i] *= *ratio;
}

/* ------------------------------------------------------------------------- */
/* The oracle object                                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
  int B, ic, jc;  /* source panel and containing cell */
  double wx[MAXK], wy[MAXK];
  double ratio, C[4];
  double w;       /* share of the point's value: 1, or 1/2 for each panel of a tie */
} gqp_t;

typedef struct {
  int B, sideB, tB, gB;
  double ratio, C[4]; /* conversion B -> A at the point */
} nbr_t;

struct orc {
  int N, k, H, me, npoc, scheme, l, s, ghost_iters, ne;
  double r, g, omega, eps, dx;
  double alpha_c; /* tilt of the rotation axis (0: f = 2 Omega sin(theta), eq. 2.5) */
  double gx[MAXK], gw[MAXK];
  double *px, *py; /* [npoc] */
  double *R;       /* [npoc][k*k] */
  double *Rsub;    /* [npoc][s][l*l] */
  double *gp, *gm; /* [npoc][s] */
  double *sigp, *sigm;
  int nring;       /* ghost cells per panel */
  int *ring;       /* [nring] jj*ne + ii */
  gqp_t *gq;       /* [6][nring][me*me][2]: two owner slots per ghost Gauss point */
  nbr_t *nb;       /* [6][4][N][me] */
  /* bottom topography (eqs. 2.13-2.14); sbar == NULL: none */
  double *sbar;    /* [6][N][N] cell averages of sqrtG phi_s */
  int tcase;       /* analytic surface behind sbar (ORC_TOPO_*), 0 if set from averages */
  double tpar[4];
  double *Rd;      /* [me*me][2][k*k] x- and y-derivative weights at the cell points */
  void *w1d;       /* [me+2] 1-D WENO-Z tables at xi = -1/2, +1/2, g_0.. (ORC_WENO1D) */
  int tform;       /* 0: total-geopotential form (eqs. 2.13-2.14); 1: depth form (2.1, 2.4) */
  const unsigned char *rmask; /* [6][N][N]: cells to reconstruct (NULL: all), orc_tendency_cells */
};

int orc_npoc(const orc *o) { return o->npoc; }
int orc_halo(const orc *o) { return o->H; }

static double cell_centre(const orc *o, int i) { return -QPI + (i + 0.5) * o->dx; }

/* side s: 0 west (x=-pi/4), 1 east, 2 south (y=-pi/4), 3 north */
static void edge_point(const orc *o, int side, int t, int gidx, double *x, double *y) {
  double along = cell_centre(o, t) + o->gx[gidx] * o->dx;
  switch (side) {
    case 0: *x = -QPI; *y = along; break;
    case 1: *x = QPI; *y = along; break;
    case 2: *x = along; *y = -QPI; break;
    default: *x = along; *y = QPI; break;
  }
}

orc *orc_new(int N, int k, int scheme, double radius, double gravity, double omega, double weno_eps,
             int ghost_iters) {
  if (N < 2 || k < 1 || k > MAXK || (k % 2) == 0) return NULL;
  orc *o = (orc *)calloc(1, sizeof(orc));
  o->N = N;
  o->k = k;
  o->H = (k - 1) / 2;
  o->me = (k + 1) / 2;
  o->npoc = 4 * o->me + o->me * o->me;
  o->scheme = scheme;
  o->l = (k + 1) / 2;
  o->s = o->l * o->l;
  o->ghost_iters = ghost_iters;
  o->ne = N + 2 * o->H;
  o->r = radius;
  o->g = gravity;
  o->omega = omega;
  o->eps = weno_eps;
  o->dx = M_PI / (2.0 * N);
  if (2 * o->H >= N) { free(o); return NULL; }
  orc_gauss(o->me, o->gx, o->gw);
  int me = o->me, np = o->npoc, kk = k * k;
  o->px = (double *)malloc(sizeof(double) * np);
  o->py = (double *)malloc(sizeof(double) * np);
  for (int r = 0; r < me; ++r) {
    o->px[r] = -0.5; o->py[r] = o->gx[r];
    o->px[me + r] = 0.5; o->py[me + r] = o->gx[r];
    o->px[2 * me + r] = o->gx[r]; o->py[2 * me + r] = -0.5;
    o->px[3 * me + r] = o->gx[r]; o->py[3 * me + r] = 0.5;
  }
  for (int h = 0; h < me; ++h)
    for (int g = 0; g < me; ++g) {
      o->px[4 * me + h * me + g] = o->gx[g];
      o->py[4 * me + h * me + g] = o->gx[h];
    }
  o->R = (double *)malloc(sizeof(double) * np * kk);
  for (int pt = 0; pt < np; ++pt) orc_tpp_weights_2d(k, o->px[pt], o->py[pt], o->R + (size_t)pt * kk);

  if (scheme == ORC_WENO1D) {
    if (k != 5) { orc_free(o); return NULL; } /* the comparator of section 5.5 is fifth order */
    w1d_t *t = (w1d_t *)malloc(sizeof(w1d_t) * (me + 2));
    w1d_tables(k, -0.5, &t[0]);
    w1d_tables(k, 0.5, &t[1]);
    for (int g = 0; g < me; ++g) w1d_tables(k, o->gx[g], &t[2 + g]);
    o->w1d = t;
  }
  if (scheme == ORC_WENO) {
    int l = o->l, s = o->s;
    o->Rsub = (double *)malloc(sizeof(double) * np * s * l * l);
    o->gp = (double *)malloc(sizeof(double) * np * s);
    o->gm = (double *)malloc(sizeof(double) * np * s);
    o->sigp = (double *)malloc(sizeof(double) * np);
    o->sigm = (double *)malloc(sizeof(double) * np);
    long double sub[MAXK * MAXK];
    for (int pt = 0; pt < np; ++pt) {
      for (int sy = 0; sy < l; ++sy)
        for (int sx = 0; sx < l; ++sx) {
          sub_weights_2d(k, sx, sy, o->px[pt], o->py[pt], sub);
          for (int c = 0; c < l * l; ++c)
            o->Rsub[((size_t)pt * s + sy * l + sx) * l * l + c] = (double)sub[c];
        }
      double gam[MAXK * MAXK], res;
      orc_weno_gamma(k, o->px[pt], o->py[pt], gam, &res);
      /* eq. 3.20 with theta = 3; reading c2: sigma+- = sum gamma+- */
      double sp = 0.0, sm = 0.0;
      for (int i = 0; i < s; ++i) {
        double gpl = 0.5 * (3.0 * fabs(gam[i]) + gam[i]);
        double gmi = 0.5 * (3.0 * fabs(gam[i]) - gam[i]);
        o->gp[(size_t)pt * s + i] = gpl;
        o->gm[(size_t)pt * s + i] = gmi;
        sp += gpl;
        sm += gmi;
      }
      o->sigp[pt] = sp;
      o->sigm[pt] = sm;
    }
  }

  /* ghost ring cells */
  int ne = o->ne, H = o->H;
  o->nring = ne * ne - N * N;
  o->ring = (int *)malloc(sizeof(int) * o->nring);
  {
    int c = 0;
    for (int jj = 0; jj < ne; ++jj)
      for (int ii = 0; ii < ne; ++ii) {
        int i = ii - H, j = jj - H;
        if (i >= 0 && i < N && j >= 0 && j < N) continue;
        o->ring[c++] = jj * ne + ii;
      }
  }
  /* ghost quadrature-point tables (section 3.3.1): each ghost cell's me x me  */
  /* Gauss points, located on the sphere, assigned to the owning panel, and    */
  /* given that panel's central k x k TPP stencil around the containing cell.  */
  o->gq = (gqp_t *)malloc(sizeof(gqp_t) * 6 * o->nring * me * me * 2);
  for (int p = 0; p < 6; ++p)
    for (int c = 0; c < o->nring; ++c) {
      int ii = o->ring[c] % ne, jj = o->ring[c] / ne;
      int i = ii - H, j = jj - H;
      for (int h = 0; h < me; ++h)
        for (int g = 0; g < me; ++g) {
          gqp_t *q2 = &o->gq[(((size_t)p * o->nring + c) * me * me + h * me + g) * 2];
          double x = cell_centre(o, i) + o->gx[g] * o->dx;
          double y = cell_centre(o, j) + o->gx[h] * o->dx;
          double X = tan(x), Y = tan(y), xyz[3], XB[2];
          int own[2];
          orc_xyz(p, X, Y, xyz);
          /* reading c11: a point on a cube edge takes the mean of both panels' values */
          int nown = owner_panels(xyz, -1, own);
          for (int sl = 0; sl < 2; ++sl) {
            gqp_t *q = &q2[sl];
            int B = own[sl < nown ? sl : 0];
            to_panel(B, xyz, XB);
            double xb = atan(XB[0]), yb = atan(XB[1]);
            int ic = (int)floor((xb + QPI) / o->dx), jc = (int)floor((yb + QPI) / o->dx);
            if (ic < 0) ic = 0;
            if (ic > N - 1) ic = N - 1;
            if (jc < 0) jc = 0;
            if (jc > N - 1) jc = N - 1;
            double xi = (xb - cell_centre(o, ic)) / o->dx, eta = (yb - cell_centre(o, jc)) / o->dx;
            q->B = B;
            q->ic = ic;
            q->jc = jc;
            q->w = nown == 2 ? 0.5 : (sl == 0 ? 1.0 : 0.0);
            orc_weights_1d(k, -H, xi, q->wx);
            orc_weights_1d(k, -H, eta, q->wy);
            conversion(p, X, Y, B, XB[0], XB[1], &q->ratio, q->C);
          }
        }
    }
  /* panel-edge neighbours of every edge Gauss point (for reading c10) */
  o->nb = (nbr_t *)malloc(sizeof(nbr_t) * 6 * 4 * N * me);
  for (int p = 0; p < 6; ++p)
    for (int side = 0; side < 4; ++side)
      for (int t = 0; t < N; ++t)
        for (int g = 0; g < me; ++g) {
          nbr_t *nb = &o->nb[((p * 4 + side) * N + t) * me + g];
          double x, y, xyz[3], XB[2];
          edge_point(o, side, t, g, &x, &y);
          double X = tan(x), Y = tan(y);
          orc_xyz(p, X, Y, xyz);
          int B = owner_panel(xyz, p);
          to_panel(B, xyz, XB);
          double xb = atan(XB[0]), yb = atan(XB[1]);
          int sB;
          double along;
          if (fabs(xb) > fabs(yb)) { sB = xb < 0 ? 0 : 1; along = yb; }
          else { sB = yb < 0 ? 2 : 3; along = xb; }
          int tB = (int)floor((along + QPI) / o->dx);
          if (tB < 0) tB = 0;
          if (tB > N - 1) tB = N - 1;
          double eta = (along - cell_centre(o, tB)) / o->dx;
          int gB = 0;
          for (int q = 1; q < me; ++q)
            if (fabs(o->gx[q] - eta) < fabs(o->gx[gB] - eta)) gB = q;
          nb->B = B;
          nb->sideB = sB;
          nb->tB = tB;
          nb->gB = gB;
          conversion(p, X, Y, B, XB[0], XB[1], &nb->ratio, nb->C);
        }
  return o;
}

void orc_free(orc *o) {
  if (!o) return;
  free(o->px); free(o->py); free(o->R); free(o->Rsub); free(o->gp); free(o->gm);
  free(o->sigp); free(o->sigm); free(o->ring); free(o->gq); free(o->nb);
  free(o->sbar); free(o->Rd); free(o->w1d);
  free(o);
}

/* ------------------------------------------------------------------------- */
/* Ghost fill (section 3.3.1, appendix eqs. 7.1-7.12): g^(0) = 0, then         */
/* ghost_iters Jacobi sweeps; each sweep interpolates every ghost Gauss point  */
/* with the owning panel's TPP stencil (which reads that panel's current       */
/* ghosts), converts it to the ghost's panel (eqs. 3.26-3.29, per Gauss point) */
/* and averages with the 2-D Gauss rule (eq. 3.6).                             */
/* reading c11: a fixed count of sweeps (the paper sets it to 10).             */
/* ------------------------------------------------------------------------- */
void orc_fill_ghosts(orc *o, const double *q, double *ext, double *resid) {
  int N = o->N, H = o->H, ne = o->ne, me = o->me, k = o->k;
  size_t pe = (size_t)ne * ne, pi = (size_t)N * N;
  memset(ext, 0, sizeof(double) * 3 * 6 * pe);
  for (int v = 0; v < 3; ++v)
    for (int p = 0; p < 6; ++p)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i)
          ext[(v * 6 + p) * pe + (size_t)(j + H) * ne + (i + H)] = q[(v * 6 + p) * pi + (size_t)j * N + i];
  double *newg = (double *)malloc(sizeof(double) * 3 * 6 * o->nring);
  double res[3] = {0, 0, 0};
  for (int it = 0; it < o->ghost_iters; ++it) {
#pragma omp parallel for schedule(static)
    for (int pc = 0; pc < 6 * o->nring; ++pc) {
      int p = pc / o->nring, c = pc % o->nring;
      double acc[3] = {0, 0, 0};
      for (int r2 = 0; r2 < me * me * 2; ++r2) {
        const int r = r2 / 2;
        const gqp_t *g = &o->gq[(size_t)pc * me * me * 2 + r2];
        if (g->w == 0.0) continue;
        double wq = o->gw[r % me] * o->gw[r / me] * g->w;
        double val[3];
        for (int v = 0; v < 3; ++v) {
          const double *src = ext + (v * 6 + g->B) * pe;
          double s = 0.0;
          for (int b = 0; b < k; ++b)
            for (int a = 0; a < k; ++a)
              s += g->wx[a] * g->wy[b] * src[(size_t)(g->jc + b) * ne + (g->ic + a)];
          val[v] = s;
        }
        acc[0] += wq * g->ratio * val[0];
        acc[1] += wq * (g->C[0] * val[1] + g->C[1] * val[2]);
        acc[2] += wq * (g->C[2] * val[1] + g->C[3] * val[2]);
      }
      for (int v = 0; v < 3; ++v) newg[(v * 6 + p) * o->nring + c] = acc[v];
    }
    for (int v = 0; v < 3; ++v) {
      double s = 0.0;
      for (int p = 0; p < 6; ++p)
        for (int c = 0; c < o->nring; ++c) {
          double *dst = ext + (v * 6 + p) * pe + o->ring[c];
          double d = newg[(v * 6 + p) * o->nring + c] - *dst;
          s += d * d;
          *dst = newg[(v * 6 + p) * o->nring + c];
        }
      res[v] = sqrt(s);
    }
  }
  if (resid)
    for (int v = 0; v < 3; ++v) resid[v] = res[v];
  free(newg);
}

/* ------------------------------------------------------------------------- */
/* Reconstruction at one point of one cell from its k x k stencil.             */
/* ------------------------------------------------------------------------- */
static double tpp_point(const orc *o, const double *st, int pt) {
  const double *w = o->R + (size_t)pt * o->k * o->k;
  double s = 0.0;
  for (int c = 0; c < o->k * o->k; ++c) s += w[c] * st[c];
  return s;
}

/* tau of eq. 3.24 (reading c4: the double sum as printed, exponent 1) */
static double weno_tau(int s, const double *beta) {
  double t = 0.0;
  for (int e = 0; e < s - 1; ++e)
    for (int ps = e; ps < s; ++ps) t += fabs(beta[ps] - beta[e]);
  return 2.0 / ((s + 1.0) * s) * t;
}

static void weno_betas(const orc *o, const double *st, double *beta) {
  int k = o->k, l = o->l, H = o->H;
  double Qs[MAXK * MAXK];
  for (int sy = 0; sy < l; ++sy)
    for (int sx = 0; sx < l; ++sx) {
      for (int b = 0; b < l; ++b)
        for (int a = 0; a < l; ++a) Qs[b * l + a] = st[(sy + b) * k + (sx + a)];
      beta[sy * l + sx] = orc_weno_beta(l, sx - H, sy - H, Qs);
    }
}

/* WENO-Z value at one point (eqs. 3.21-3.23) given the cell's betas and tau.  */
/* reading c2: q = sigma+ sum(w+ p) - sigma- sum(w- p), sigma+- = sum gamma+-. */
static double weno_value(const orc *o, const double *st, int pt, const double *beta, double tau) {
  int k = o->k, l = o->l, s = o->s;
  double ap[MAXK * MAXK], am[MAXK * MAXK], pv[MAXK * MAXK], sap = 0.0, sam = 0.0;
  for (int sy = 0; sy < l; ++sy)
    for (int sx = 0; sx < l; ++sx) {
      int i = sy * l + sx;
      const double *w = o->Rsub + ((size_t)pt * s + i) * l * l;
      double v = 0.0;
      for (int b = 0; b < l; ++b)
        for (int a = 0; a < l; ++a) v += w[b * l + a] * st[(sy + b) * k + (sx + a)];
      pv[i] = v;
      double f = 1.0 + tau / (beta[i] + o->eps);
      ap[i] = o->gp[(size_t)pt * s + i] / o->sigp[pt] * f;
      am[i] = o->gm[(size_t)pt * s + i] / o->sigm[pt] * f;
      sap += ap[i];
      sam += am[i];
    }
  double qp = 0.0, qm = 0.0;
  for (int i = 0; i < s; ++i) {
    qp += ap[i] / sap * pv[i];
    qm += am[i] / sam * pv[i];
  }
  return o->sigp[pt] * qp - o->sigm[pt] * qm;
}

double orc_weno_point(const orc *o, const double *st, int pt) {
  double beta[MAXK * MAXK];
  weno_betas(o, st, beta);
  return weno_value(o, st, pt, beta, weno_tau(o->s, beta));
}

void orc_reconstruct_all(orc *o, const double *ext, double *pts) {
  int N = o->N, k = o->k, ne = o->ne, np = o->npoc;
  size_t pe = (size_t)ne * ne;
#pragma omp parallel for schedule(static)
  for (int row = 0; row < 3 * 6 * N; ++row) {
    int v = row / (6 * N), p = (row / N) % 6, j = row % N;
    double st[MAXK * MAXK], beta[MAXK * MAXK];
    const double *src = ext + (v * 6 + p) * pe;
    for (int i = 0; i < N; ++i) {
      for (int b = 0; b < k; ++b)
        for (int a = 0; a < k; ++a) st[b * k + a] = src[(size_t)(j + b) * ne + (i + a)];
      double *out = pts + ((((size_t)v * 6 + p) * N + j) * N + i) * np;
      if (o->rmask && !o->rmask[((size_t)p * N + j) * N + i]) { /* not needed by the sample */
        for (int pt = 0; pt < np; ++pt) out[pt] = NAN;
        continue;
      }
      if (o->scheme == ORC_WENO) {
        weno_betas(o, st, beta);
        double tau = weno_tau(o->s, beta);
        for (int pt = 0; pt < np; ++pt) out[pt] = weno_value(o, st, pt, beta, tau);
      } else if (o->scheme == ORC_WENO1D) {
        /* x on every stencil row at the point's xi, then y on the row values; the     */
        /* x pass depends only on (row, xi position), so it is evaluated once for each */
        const w1d_t *t = (const w1d_t *)o->w1d;
        int me = o->me;
        double Lx[MAXK + 2][MAXK];
        for (int ix = 0; ix < me + 2; ++ix)
          for (int b = 0; b < k; ++b) Lx[ix][b] = w1d_value(k, &t[ix], st + b * k, o->eps);
        for (int pt = 0; pt < np; ++pt) {
          int ix, iy;
          if (pt < 4 * me) {
            int side = pt / me, r = pt % me;
            ix = side == 0 ? 0 : (side == 1 ? 1 : 2 + r);
            iy = side == 2 ? 0 : (side == 3 ? 1 : 2 + r);
          } else {
            ix = 2 + (pt - 4 * me) % me;
            iy = 2 + (pt - 4 * me) / me;
          }
          out[pt] = w1d_value(k, &t[iy], Lx[ix], o->eps);
        }
      } else {
        for (int pt = 0; pt < np; ++pt) out[pt] = tpp_point(o, st, pt);
      }
    }
  }
}

/* ------------------------------------------------------------------------- */
/* LMARS flux (section 3.4, eqs. 3.30-3.38) at an edge point (X, Y) of one     */
/* panel; dir 0: x-edge (i = 1), 1: y-edge (i = 2).  q in the unit-sphere      */
/* scaling: q = sqrtG_u (phi, phi u, phi v), true metric G^ij = G_u^ij / r^2.   */
/* reading c1: |m| (q_R - q_L), i.e. m*sign(m); reading c9: P uses the         */
/* interface value phi of eq. 3.33.                                            */
/* With topography (eqs. 2.13, 3.38) sL, sR are sqrtG phi_s at the point on    */
/* each side; reading c26: the depth phi = q0/sqrtG gives the wave speed c     */
/* (eq. 3.35) and the upwinded q, the total phi_t = phi + phi_s enters the      */
/* pressure jump of eq. 3.32 and the interface value of eq. 3.33 that P uses.  */
/* Without topography sL = sR = 0 and phi_t = phi exactly.                      */
/* ------------------------------------------------------------------------- */
static void lmars_core(const orc *o, int dir, double X, double Y, const double *qL, const double *qR,
                       double sL, double sR, double *F) {
  double m7[7];
  orc_metric(X, Y, m7);
  double sG = m7[0], r2 = o->r * o->r;
  double Gii = (dir == 0 ? m7[1] : m7[3]) / r2; /* true G^ii */
  double G1i = (dir == 0 ? m7[1] : m7[2]) / r2, G2i = (dir == 0 ? m7[2] : m7[3]) / r2;
  double phL = qL[0] / sG, phR = qR[0] / sG;
  double ptL = phL + sL / sG, ptR = phR + sR / sG;              /* phi_t */
  double uL = qL[1 + dir] / qL[0], uR = qR[1 + dir] / qR[0];
  double upL = uL / sqrt(Gii), upR = uR / sqrt(Gii);          /* eq. 3.31 */
  double c = 0.5 * (sqrt(phL) + sqrt(phR));                     /* eqs. 3.34-3.35 */
  double ms = 0.5 * (upL + upR - (ptR - ptL) / c);              /* eq. 3.32 */
  double ph = 0.5 * (ptL + ptR - c * (upR - upL));              /* eq. 3.33 */
  double m = ms * sqrt(Gii);                                    /* eq. 3.36 */
  double am = fabs(m);
  for (int v = 0; v < 3; ++v) F[v] = 0.5 * (m * (qL[v] + qR[v]) - am * (qR[v] - qL[v])); /* eq. 3.37 */
  F[1] += 0.5 * sG * G1i * ph * ph;                             /* eq. 3.38 */
  F[2] += 0.5 * sG * G2i * ph * ph;
}

void orc_lmars(const orc *o, int dir, double X, double Y, const double *qL, const double *qR,
               double *F) {
  lmars_core(o, dir, X, Y, qL, qR, 0.0, 0.0, F);
}

void orc_lmars_topo(const orc *o, int dir, double X, double Y, const double *qL, const double *qR,
                    double sL, double sR, double *F) {
  lmars_core(o, dir, X, Y, qL, qR, sL, sR, F);
}

/* Coriolis parameter.  With alpha_c = 0 it is 2 Omega sin(theta) with sin(theta)   */
/* of eq. 2.5.  reading c21: for the geostrophic case rotated by alpha (eqs.        */
/* 5.1-5.3 with alpha != 0) to stay steady, the rotation axis is tilted with it, as */
/* in Williamson et al. (1992) case 2: f = 2 Omega (-cos(lambda) cos(theta)         */
/* sin(alpha_c) + sin(theta) cos(alpha_c)).                                         */
static double coriolis(const orc *o, int p, double X, double Y) {
  if (o->alpha_c == 0.0) return 2.0 * o->omega * sin_lat(p, X, Y);
  double xyz[3], lam, th;
  orc_xyz(p, X, Y, xyz);
  lonlat(xyz, &lam, &th);
  return 2.0 * o->omega * (-cos(lam) * cos(th) * sin(o->alpha_c) + sin(th) * cos(o->alpha_c));
}

void orc_set_coriolis_tilt(orc *o, double alpha_c) { o->alpha_c = alpha_c; }

/* Source terms (eqs. 2.2, 2.3; psi_B = 0 without topography) at one point of */
/* panel p, unit-sphere scaling (both sides of eq. 2.1 divided by r^2).        */
void orc_sources(const orc *o, int p, double X, double Y, const double *q, double *S) {
  double m7[7];
  orc_metric(X, Y, m7);
  double sG = m7[0], d2 = 1.0 + X * X + Y * Y;
  double phi = q[0] / sG, u = q[1] / q[0], v = q[2] / q[0];
  double f = coriolis(o, p, X, Y);
  double pm1 = 2.0 * sG / d2 * (-X * Y * Y * phi * u * u + Y * (1.0 + Y * Y) * phi * u * v);
  double pm2 = 2.0 * sG / d2 * (X * (1.0 + X * X) * phi * u * v - X * X * Y * phi * v * v);
  double pc1 = sG * f * (-m7[2] * q[1] + m7[1] * q[2]);
  double pc2 = sG * f * (-m7[3] * q[1] + m7[2] * q[2]);
  S[0] = 0.0;
  S[1] = pm1 + pc1;
  S[2] = pm2 + pc2;
}

/* ------------------------------------------------------------------------- */
/* Bottom topography (section 2, eqs. 2.13-2.14; section 5.2, eq. 5.8).        */
/* The state keeps the depth, q0 = sqrtG phi; the mass variable is             */
/* reconstructed as sqrtG phi_t = q0 + sqrtG phi_s (the cell averages of        */
/* sqrtG phi_s are added before the ghost fill), and phi_s at the points is     */
/* the linear reconstruction of its own cell averages (reading c26).            */
/* ------------------------------------------------------------------------- */
static double gc_dist(double l1, double t1, double l2, double t2);

static double topo_lonlat(const orc *o, double lam, double th) {
  const double *P = o->tpar;
  if (o->tcase == ORC_TOPO_MOUNTAIN) {
    /* eq. 5.8: hs = hs0 (1 - r/R), r = sqrt(min(R^2, dlam^2 + dtheta^2));     */
    /* reading c27: the longitude difference is taken modulo 2 pi.             */
    double dl = remainder(lam - P[2], 2.0 * M_PI), dt = th - P[3];
    double r = sqrt(fmin(P[1] * P[1], dl * dl + dt * dt));
    return o->g * P[0] * (1.0 - r / P[1]);
  }
  if (o->tcase == ORC_TOPO_ZONAL) {
    /* hs = hs0 cos^2(theta'), theta' the latitude about the axis tilted by    */
    /* alpha (the same rotated latitude as eq. 5.1)                             */
    double t = -cos(lam) * cos(th) * sin(P[1]) + sin(th) * cos(P[1]);
    return o->g * P[0] * (1.0 - t * t);
  }
  if (o->tcase == ORC_TOPO_HILL) {
    double d = gc_dist(lam, th, P[2], P[3]) / P[1];
    return o->g * P[0] * exp(-d * d);
  }
  return 0.0;
}

double orc_topography_point(const orc *o, int p, double X, double Y) {
  double xyz[3], lam, th;
  orc_xyz(p, X, Y, xyz);
  lonlat(xyz, &lam, &th);
  return topo_lonlat(o, lam, th);
}

static void topo_prepare(orc *o) {
  int k = o->k, me = o->me, kk = k * k;
  if (!o->Rd) o->Rd = (double *)malloc(sizeof(double) * me * me * 2 * kk);
  for (int h = 0; h < me; ++h)
    for (int g = 0; g < me; ++g)
      for (int d = 0; d < 2; ++d)
        orc_tpp_dweights_2d(k, o->gx[g], o->gx[h], d, o->Rd + ((size_t)(h * me + g) * 2 + d) * kk);
}

void orc_set_topography(orc *o, const double *sbar) {
  size_t n = (size_t)6 * o->N * o->N;
  free(o->sbar);
  o->sbar = NULL;
  o->tcase = 0;
  if (!sbar) return;
  o->sbar = (double *)malloc(sizeof(double) * n);
  memcpy(o->sbar, sbar, sizeof(double) * n);
  topo_prepare(o);
}

/* Analytic surface: cell averages of sqrtG phi_s by the me x me Gauss rule    */
/* (reading c15); initial conditions then read their phi as phi_t (c28).       */
void orc_set_topography_case(orc *o, int tcase, const double *P) {
  int N = o->N, me = o->me;
  double *sb = (double *)malloc(sizeof(double) * 6 * N * N);
  o->tcase = tcase;
  for (int i = 0; i < 4; ++i) o->tpar[i] = P[i];
  for (int p = 0; p < 6; ++p)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int h = 0; h < me; ++h)
          for (int g = 0; g < me; ++g) {
            double X = tan(cell_centre(o, i) + o->gx[g] * o->dx);
            double Y = tan(cell_centre(o, j) + o->gx[h] * o->dx);
            double m7[7];
            orc_metric(X, Y, m7);
            acc += o->gw[g] * o->gw[h] * m7[0] * orc_topography_point(o, p, X, Y);
          }
        sb[((size_t)p * N + j) * N + i] = acc;
      }
  orc_set_topography(o, sb);
  o->tcase = tcase;
  free(sb);
}

/* Which form of the topography terms the tendency uses: 0 (default) the paper's        */
/* total-geopotential form, eqs. 2.13-2.14 (reconstruct sqrtG phi_t, pressure with     */
/* phi_t, psi_B = sqrtG phi_s G^ij d_j phi_t); 1 the depth form of eqs. 2.1 and 2.4     */
/* that section 2 replaces (reconstruct sqrtG phi, pressure with phi, psi_B =           */
/* -sqrtG phi G^ij d_j phi_s, the gradient of the surface's own TPP polynomial).        */
void orc_set_topography_form(orc *o, int form) { o->tform = form ? 1 : 0; }

void orc_get_topography(const orc *o, double *out) {
  size_t n = (size_t)6 * o->N * o->N;
  for (size_t c = 0; c < n; ++c) out[c] = o->sbar ? o->sbar[c] : 0.0;
}

/* Point values for the topography terms of one tendency evaluation.          */
/* ext holds the extended sqrtG phi_t (and momentum); pts its reconstruction.  */
/* On return spt[p][j][i][pt] = sqrtG phi_s (TPP of its averages), pts' mass    */
/* variable is the depth sqrtG phi_t - sqrtG phi_s, and dpt[p][j][i][c][2] is    */
/* the gradient of phi_t at cell point c, reading c29: phi_t = P / sqrtG with P  */
/* the TPP polynomial of sqrtG phi_t, so d phi_t = (dP - phi_t d sqrtG) / sqrtG. */
static void topo_points(orc *o, const double *ext, double *pts, double *spt, double *dpt, int depth_form) {
  int N = o->N, k = o->k, ne = o->ne, np = o->npoc, me = o->me, kk = k * k;
  size_t pe = (size_t)ne * ne, pi = (size_t)N * N;
  double *s3 = (double *)calloc(3 * 6 * pi, sizeof(double));
  double *exs = (double *)malloc(sizeof(double) * 3 * 6 * pe);
  memcpy(s3, o->sbar, sizeof(double) * 6 * pi);
  orc_fill_ghosts(o, s3, exs, NULL);
#pragma omp parallel for schedule(static)
  for (int pj = 0; pj < 6 * N; ++pj) {
    int p = pj / N, j = pj % N;
    double st[MAXK * MAXK], tt[MAXK * MAXK];
    for (int i = 0; i < N; ++i) {
      for (int b = 0; b < k; ++b)
        for (int a = 0; a < k; ++a) {
          st[b * k + a] = exs[p * pe + (size_t)(j + b) * ne + (i + a)];
          tt[b * k + a] = ext[p * pe + (size_t)(j + b) * ne + (i + a)];
        }
      size_t cell = ((size_t)p * N + j) * N + i;
      for (int pt = 0; pt < np; ++pt) {
        double sv = tpp_point(o, st, pt);
        spt[cell * np + pt] = sv;
        if (!depth_form) pts[cell * np + pt] -= sv; /* the v = 0 block of pts */
      }
      const double *G = depth_form ? st : tt; /* the field whose gradient the source takes */
      for (int h = 0; h < me; ++h)
        for (int g = 0; g < me; ++g) {
          int c = h * me + g;
          double X = tan(cell_centre(o, i) + o->gx[g] * o->dx);
          double Y = tan(cell_centre(o, j) + o->gx[h] * o->dx);
          double m7[7], gs[2];
          orc_metric(X, Y, m7);
          orc_sqrtg_grad(X, Y, gs);
          double P = tpp_point(o, G, 4 * me + c);
          double dP[2] = {0.0, 0.0};
          for (int d = 0; d < 2; ++d) {
            const double *w = o->Rd + ((size_t)c * 2 + d) * kk;
            for (int q = 0; q < kk; ++q) dP[d] += w[q] * G[q];
            dP[d] /= o->dx;
          }
          double pt_t = P / m7[0];
          for (int d = 0; d < 2; ++d) dpt[(cell * me * me + c) * 2 + d] = (dP[d] - pt_t * gs[d]) / m7[0];
        }
    }
  }
  free(s3);
  free(exs);
}

/* psi_B of eq. 2.14 at a cell point, unit-sphere scaling like the pressure    */
/* term: sqrtG phi_s G^ij d phi_t / dx^j with the true G^ij = G_unit^ij / r^2.  */
static void topo_source(const orc *o, double X, double Y, double s, const double *dphit, double *S) {
  double m7[7];
  orc_metric(X, Y, m7);
  double sG = m7[0], r2 = o->r * o->r, fs = s / sG;
  S[1] += sG * fs * (m7[1] * dphit[0] + m7[2] * dphit[1]) / r2;
  S[2] += sG * fs * (m7[2] * dphit[0] + m7[3] * dphit[1]) / r2;
}

/* The cell average of psi_B (eq. 2.14) alone, out[2][6][N][N] (momentum x, y), */
/* by the same steps as the tendency's sources: zero without a surface.        */
void orc_topo_psib(orc *o, const double *q, double *out) {
  int N = o->N, ne = o->ne, np = o->npoc, me = o->me;
  size_t pn = (size_t)6 * N * N, nq = 3 * pn;
  memset(out, 0, sizeof(double) * 2 * pn);
  if (!o->sbar) return;
  double *qt = (double *)malloc(sizeof(double) * nq);
  double *ext = (double *)malloc(sizeof(double) * 3 * 6 * ne * ne);
  double *pts = (double *)malloc(sizeof(double) * nq * np);
  double *spt = (double *)malloc(sizeof(double) * pn * np);
  double *dpt = (double *)malloc(sizeof(double) * pn * me * me * 2);
  memcpy(qt, q, sizeof(double) * nq);
  for (size_t c = 0; c < pn; ++c) qt[c] += o->sbar[c];
  orc_fill_ghosts(o, qt, ext, NULL);
  orc_reconstruct_all(o, ext, pts);
  topo_points(o, ext, pts, spt, dpt, 0);
  for (int p = 0; p < 6; ++p)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        size_t cell = ((size_t)p * N + j) * N + i;
        for (int h = 0; h < me; ++h)
          for (int g = 0; g < me; ++g) {
            double x = cell_centre(o, i) + o->gx[g] * o->dx, y = cell_centre(o, j) + o->gx[h] * o->dx;
            double S[3] = {0.0, 0.0, 0.0};
            topo_source(o, tan(x), tan(y), spt[cell * np + 4 * me + h * me + g],
                        dpt + (cell * me * me + h * me + g) * 2, S);
            out[cell] += o->gw[g] * o->gw[h] * S[1];
            out[pn + cell] += o->gw[g] * o->gw[h] * S[2];
          }
      }
  free(qt);
  free(ext);
  free(pts);
  free(spt);
  free(dpt);
}

/* ------------------------------------------------------------------------- */
/* Tendency (eq. 3.1, reading c6: F_{i+1/2} - F_{i-1/2} over dx = pi/(2N)).    */
/* ------------------------------------------------------------------------- */
#define PTS(v, p, j, i, pt) pts[((((size_t)(v) * 6 + (p)) * N + (j)) * N + (i)) * np + (pt)]

static int side_point(int me, int side, int g) { return side * me + g; }

void orc_tendency(orc *o, const double *q, double *dqdt) {
  int N = o->N, ne = o->ne, np = o->npoc, me = o->me;
  double dx = o->dx;
  double *ext = (double *)malloc(sizeof(double) * 3 * 6 * ne * ne);
  double *pts = (double *)malloc(sizeof(double) * 3 * 6 * (size_t)N * N * np);
  double *qt = NULL, *spt = NULL, *dpt = NULL;
  if (o->sbar && !o->tform) { /* eq. 2.13: reconstruct sqrtG phi_t = q0 + sqrtG phi_s */
    size_t nq = (size_t)3 * 6 * N * N;
    qt = (double *)malloc(sizeof(double) * nq);
    memcpy(qt, q, sizeof(double) * nq);
    for (size_t c = 0; c < (size_t)6 * N * N; ++c) qt[c] += o->sbar[c];
  }
  if (o->sbar) {
    spt = (double *)malloc(sizeof(double) * 6 * (size_t)N * N * np);
    dpt = (double *)malloc(sizeof(double) * 6 * (size_t)N * N * me * me * 2);
  }
  orc_fill_ghosts(o, qt ? qt : q, ext, NULL);
  orc_reconstruct_all(o, ext, pts);
  if (o->sbar) topo_points(o, ext, pts, spt, dpt, o->tform);
  /* the depth form of eqs. 2.1 and 2.4 keeps phi in LMARS: no surface there */
#define SPT(p, j, i, pt) (spt && !o->tform ? spt[((((size_t)(p)) * N + (j)) * N + (i)) * np + (pt)] : 0.0)
  /* edge-averaged fluxes: Fx[v][p][j][i'] i' = 0..N, Fy[v][p][j'][i] j' = 0..N */
  size_t fe = (size_t)N * (N + 1);
  double *Fx = (double *)calloc(3 * 6 * fe, sizeof(double));
  double *Fy = (double *)calloc(3 * 6 * fe, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int pj = 0; pj < 6 * N; ++pj) {
    int p = pj / N, j = pj % N;
    for (int e = 1; e < N; ++e) { /* interior x-edges of row j, between cells e-1 and e */
      double acc[3] = {0, 0, 0};
      for (int g = 0; g < me; ++g) {
        double qL[3], qR[3], F[3];
        for (int v = 0; v < 3; ++v) {
          qL[v] = PTS(v, p, j, e - 1, side_point(me, 1, g));
          qR[v] = PTS(v, p, j, e, side_point(me, 0, g));
        }
        double x = -QPI + e * dx, y = cell_centre(o, j) + o->gx[g] * dx;
        lmars_core(o, 0, tan(x), tan(y), qL, qR, SPT(p, j, e - 1, side_point(me, 1, g)),
                   SPT(p, j, e, side_point(me, 0, g)), F);
        for (int v = 0; v < 3; ++v) acc[v] += o->gw[g] * F[v];
      }
      for (int v = 0; v < 3; ++v) Fx[(v * 6 + p) * fe + (size_t)j * (N + 1) + e] = acc[v];
    }
    for (int e = 1; e < N; ++e) { /* interior y-edges of column j (cells (j, e-1) | (j, e)) */
      int i = j;
      double acc[3] = {0, 0, 0};
      for (int g = 0; g < me; ++g) {
        double qL[3], qR[3], F[3];
        for (int v = 0; v < 3; ++v) {
          qL[v] = PTS(v, p, e - 1, i, side_point(me, 3, g));
          qR[v] = PTS(v, p, e, i, side_point(me, 2, g));
        }
        double x = cell_centre(o, i) + o->gx[g] * dx, y = -QPI + e * dx;
        lmars_core(o, 1, tan(x), tan(y), qL, qR, SPT(p, e - 1, i, side_point(me, 3, g)),
                   SPT(p, e, i, side_point(me, 2, g)), F);
        for (int v = 0; v < 3; ++v) acc[v] += o->gw[g] * F[v];
      }
      for (int v = 0; v < 3; ++v) Fy[(v * 6 + p) * fe + (size_t)e * N + i] = acc[v];
    }
  }
  /* panel-boundary edges, reading c10: the flux is computed once, in the      */
  /* lower-numbered panel's frame, from that panel's boundary-cell             */
  /* reconstruction and the neighbour panel's own boundary-cell reconstruction */
  /* converted by eqs. 3.26-3.29; the other panel receives the mass flux with  */
  /* its orientation sign and the momentum flux converted back by C.           */
  for (int A = 0; A < 6; ++A)
    for (int side = 0; side < 4; ++side) {
      const nbr_t *nb0 = &o->nb[((A * 4 + side) * N + 0) * me];
      int B = nb0->B;
      if (B < A) continue;
      int sideB = nb0->sideB;
      double sA = (side == 1 || side == 3) ? 1.0 : -1.0;
      double sB = (sideB == 1 || sideB == 3) ? 1.0 : -1.0;
      int dirA = side / 2, dirB = sideB / 2;
      for (int t = 0; t < N; ++t) {
        double accA[3] = {0, 0, 0};
        double FB[MAXK][3];
        int tB = -1;
        for (int g = 0; g < me; ++g) {
          const nbr_t *nb = &o->nb[((A * 4 + side) * N + t) * me + g];
          tB = nb->tB;
          int ci = side == 0 ? 0 : (side == 1 ? N - 1 : t);
          int cj = side == 2 ? 0 : (side == 3 ? N - 1 : t);
          int bi = nb->sideB == 0 ? 0 : (nb->sideB == 1 ? N - 1 : nb->tB);
          int bj = nb->sideB == 2 ? 0 : (nb->sideB == 3 ? N - 1 : nb->tB);
          double qin[3], qb[3], qo[3];
          for (int v = 0; v < 3; ++v) {
            qin[v] = PTS(v, A, cj, ci, side_point(me, side, g));
            qb[v] = PTS(v, B, bj, bi, side_point(me, nb->sideB, nb->gB));
          }
          qo[0] = nb->ratio * qb[0];
          qo[1] = nb->C[0] * qb[1] + nb->C[1] * qb[2];
          qo[2] = nb->C[2] * qb[1] + nb->C[3] * qb[2];
          double sin_ = SPT(A, cj, ci, side_point(me, side, g));
          double so = nb->ratio * SPT(B, bj, bi, side_point(me, nb->sideB, nb->gB));
          double x, y, F[3];
          edge_point(o, side, t, g, &x, &y);
          if (sA > 0) lmars_core(o, dirA, tan(x), tan(y), qin, qo, sin_, so, F);
          else lmars_core(o, dirA, tan(x), tan(y), qo, qin, so, sin_, F);
          for (int v = 0; v < 3; ++v) accA[v] += o->gw[g] * F[v];
          /* back to B: C_{A->B} is the inverse of C_{B->A} at the same point */
          double Ci[4];
          inv2(nb->C, Ci);
          double sg = -sA * sB;
          FB[nb->gB][0] = sg * F[0];
          FB[nb->gB][1] = sg * (Ci[0] * F[1] + Ci[1] * F[2]);
          FB[nb->gB][2] = sg * (Ci[2] * F[1] + Ci[3] * F[2]);
        }
        double accB[3] = {0, 0, 0};
        for (int g = 0; g < me; ++g)
          for (int v = 0; v < 3; ++v) accB[v] += o->gw[g] * FB[g][v];
        accB[0] = -sA * sB * accA[0]; /* the single mass flux, exactly */
        double *FA = dirA == 0 ? Fx : Fy;
        double *FBp = dirB == 0 ? Fx : Fy;
        size_t ia = dirA == 0 ? (size_t)t * (N + 1) + (side == 1 ? N : 0)
                              : (size_t)(side == 3 ? N : 0) * N + t;
        size_t ib = dirB == 0 ? (size_t)tB * (N + 1) + (sideB == 1 ? N : 0)
                              : (size_t)(sideB == 3 ? N : 0) * N + tB;
        for (int v = 0; v < 3; ++v) {
          FA[(v * 6 + A) * fe + ia] = accA[v];
          FBp[(v * 6 + B) * fe + ib] = accB[v];
        }
      }
    }
  /* sources at the cell points (eq. 3.6) and the tendency */
#pragma omp parallel for schedule(static)
  for (int pj = 0; pj < 6 * N; ++pj) {
    int p = pj / N, j = pj % N;
    for (int i = 0; i < N; ++i) {
      double sb[3] = {0, 0, 0};
      for (int h = 0; h < me; ++h)
        for (int g = 0; g < me; ++g) {
          int pt = 4 * me + h * me + g;
          double qv[3], S[3];
          for (int v = 0; v < 3; ++v) qv[v] = PTS(v, p, j, i, pt);
          double x = cell_centre(o, i) + o->gx[g] * dx, y = cell_centre(o, j) + o->gx[h] * dx;
          orc_sources(o, p, tan(x), tan(y), qv, S);
          if (spt && !o->tform) /* eq. 2.14: sqrtG phi_s G^ij d_j phi_t */
            topo_source(o, tan(x), tan(y), SPT(p, j, i, pt),
                        dpt + ((((size_t)p * N + j) * N + i) * me * me + h * me + g) * 2, S);
          else if (spt) /* eq. 2.4: -sqrtG phi G^ij d_j phi_s */
            topo_source(o, tan(x), tan(y), -PTS(0, p, j, i, pt),
                        dpt + ((((size_t)p * N + j) * N + i) * me * me + h * me + g) * 2, S);
          for (int v = 0; v < 3; ++v) sb[v] += o->gw[g] * o->gw[h] * S[v];
        }
      for (int v = 0; v < 3; ++v) {
        const double *fx = Fx + (v * 6 + p) * fe + (size_t)j * (N + 1);
        const double *fy = Fy + (v * 6 + p) * fe;
        double d = -(fx[i + 1] - fx[i]) / dx - (fy[(size_t)(j + 1) * N + i] - fy[(size_t)j * N + i]) / dx + sb[v];
        dqdt[((size_t)(v * 6 + p) * N + j) * N + i] = d;
      }
    }
  }
#undef SPT
  free(ext);
  free(pts);
  free(Fx);
  free(Fy);
  free(qt);
  free(spt);
  free(dpt);
}

/* L(q) at selected cells only: the cells' own reconstructions and those of   */
/* their four edge neighbours (across panel edges, the neighbour panel's       */
/* boundary cell) are computed, every other cell's reconstruction is skipped;  */
/* then orc_tendency runs unchanged.  The ghost fill stays global.  out[3][n]. */
void orc_tendency_cells(orc *o, const double *q, int n, const int *cells, double *out) {
  int N = o->N, me = o->me;
  size_t pn = (size_t)6 * N * N;
  unsigned char *mask = (unsigned char *)calloc(pn, 1);
  double *full = (double *)malloc(sizeof(double) * 3 * pn);
  for (int c = 0; c < n; ++c) {
    int p = cells[c] / (N * N), j = (cells[c] / N) % N, i = cells[c] % N;
    mask[cells[c]] = 1;
    int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
    for (int side = 0; side < 4; ++side) {
      int ii = i + di[side], jj = j + dj[side];
      if (ii >= 0 && ii < N && jj >= 0 && jj < N) {
        mask[((size_t)p * N + jj) * N + ii] = 1;
      } else { /* the cell across the cube edge */
        int t = side < 2 ? j : i;
        const nbr_t *nb = &o->nb[((p * 4 + side) * N + t) * me];
        int bi = nb->sideB == 0 ? 0 : (nb->sideB == 1 ? N - 1 : nb->tB);
        int bj = nb->sideB == 2 ? 0 : (nb->sideB == 3 ? N - 1 : nb->tB);
        mask[((size_t)nb->B * N + bj) * N + bi] = 1;
      }
    }
  }
  o->rmask = mask;
  orc_tendency(o, q, full);
  o->rmask = NULL;
  for (int v = 0; v < 3; ++v)
    for (int c = 0; c < n; ++c) out[(size_t)v * n + c] = full[v * pn + cells[c]];
  free(full);
  free(mask);
}

/* ------------------------------------------------------------------------- */
/* Time stepping: SSP-RK3 (Shu-Osher form) and the Wicker-Skamarock RK3 of    */
/* eqs. 3.39-3.41 (reading c8: the second stage starts from q^n).             */
/* ------------------------------------------------------------------------- */
void orc_step(orc *o, double *q, double dt, int nsteps, int rk) {
  size_t n = (size_t)3 * 6 * o->N * o->N;
  double *L = (double *)malloc(sizeof(double) * n);
  double *q1 = (double *)malloc(sizeof(double) * n);
  double *q2 = (double *)malloc(sizeof(double) * n);
  for (int s = 0; s < nsteps; ++s) {
    if (rk == ORC_WSRK3) {
      orc_tendency(o, q, L);
      for (size_t i = 0; i < n; ++i) q1[i] = q[i] + dt / 3.0 * L[i];
      orc_tendency(o, q1, L);
      for (size_t i = 0; i < n; ++i) q2[i] = q[i] + dt / 2.0 * L[i];
      orc_tendency(o, q2, L);
      for (size_t i = 0; i < n; ++i) q[i] = q[i] + dt * L[i];
    } else {
      orc_tendency(o, q, L);
      for (size_t i = 0; i < n; ++i) q1[i] = q[i] + dt * L[i];
      orc_tendency(o, q1, L);
      for (size_t i = 0; i < n; ++i) q2[i] = 0.75 * q[i] + 0.25 * (q1[i] + dt * L[i]);
      orc_tendency(o, q2, L);
      for (size_t i = 0; i < n; ++i) q[i] = q[i] / 3.0 + 2.0 / 3.0 * (q2[i] + dt * L[i]);
    }
  }
  free(L);
  free(q1);
  free(q2);
}

double orc_mass(const orc *o, const double *q) {
  long double s = 0.0L;
  for (size_t i = 0; i < (size_t)6 * o->N * o->N; ++i) s += q[i];
  return (double)(s * o->dx * o->dx);
}

/* ------------------------------------------------------------------------- */
/* Initial conditions (section 5), cell averages by the me x me Gauss rule of  */
/* sqrtG times the analytic field (reading c15).                               */
/* ------------------------------------------------------------------------- */
static double gc_dist(double l1, double t1, double l2, double t2) {
  double c = sin(t1) * sin(t2) + cos(t1) * cos(t2) * cos(l1 - l2);
  if (c > 1.0) c = 1.0;
  if (c < -1.0) c = -1.0;
  return acos(c);
}

/* Perturbed jet of section 5.4 (Galewsky et al. 2004), P = (umax, theta0, theta1,     */
/* theta2, alpha, beta, hhat, phi0).  u(theta) of eq. 5.16, zero outside (theta0,       */
/* theta1).                                                                            */
static double jet_u(const double *P, double th) {
  if (th <= P[1] || th >= P[2]) return 0.0;
  double en = exp(-4.0 / ((P[2] - P[1]) * (P[2] - P[1])));
  return P[0] / en * exp(1.0 / ((th - P[1]) * (th - P[2])));
}

/* The balance integral of eq. 5.17, int_{-pi/2}^{theta} a u (f + tan(t) u / a) dt,     */
/* f = 2 Omega sin(t), by composite Gauss-Legendre (16 panels of 8 nodes) over          */
/* (theta0, min(theta, theta1)); u vanishes elsewhere.                                  */
static double jet_integral(const orc *o, const double *P, double th) {
  double hi = th < P[2] ? th : P[2];
  if (hi <= P[1]) return 0.0;
  double x[8], w[8], s = 0.0, h = (hi - P[1]) / 16.0;
  orc_gauss(8, x, w);
  for (int pnl = 0; pnl < 16; ++pnl)
    for (int q = 0; q < 8; ++q) {
      double t = P[1] + (pnl + 0.5 + x[q]) * h, u = jet_u(P, t);
      s += w[q] * h * o->r * u * (2.0 * o->omega * sin(t) + tan(t) * u / o->r);
    }
  return s;
}

/* reading c30: phi0 = 0 in the parameters means Galewsky's choice, the constant that   */
/* makes the area mean of the balanced phi (without phi') equal g * 10 km:              */
/* phi0 = g 1e4 + (1/2) int_{-pi/2}^{pi/2} I(theta) cos(theta) d theta.                 */
static double jet_phi0(const orc *o, const double *P) {
  double x[8], w[8], s = 0.0, h = (P[2] - P[1]) / 16.0;
  orc_gauss(8, x, w);
  for (int pnl = 0; pnl < 16; ++pnl)
    for (int q = 0; q < 8; ++q) {
      double t = P[1] + (pnl + 0.5 + x[q]) * h;
      s += w[q] * h * jet_integral(o, P, t) * cos(t);
    }
  s += jet_integral(o, P, P[2]) * (1.0 - sin(P[2]));
  return o->g * 1.0e4 + 0.5 * s;
}

static void ic_point(const orc *o, int cs, const double *P, int n_extra, const double *ex, double lam,
                     double th, double *phi, double *us, double *vs) {
  double a = o->r, Om = o->omega, g = o->g;
  if (cs == ORC_IC_GALEWSKY) {
    /* eqs. 5.16-5.18, lambda in (-pi, pi] */
    double d2 = (lam / P[4]) * (lam / P[4]) + ((P[3] - th) / P[5]) * ((P[3] - th) / P[5]);
    *phi = P[7] + g * P[6] * cos(th) * exp(-d2) - jet_integral(o, P, th);
    *us = jet_u(P, th);
    *vs = 0.0;
    return;
  }
  if (cs == ORC_IC_GEOSTROPHIC || cs == ORC_IC_BUMPS) {
    double al = P[0], u0 = P[1], phi0 = P[2];
    double t = -cos(lam) * cos(th) * sin(al) + sin(th) * cos(al);
    *phi = phi0 - (a * Om * u0 + 0.5 * u0 * u0) * t * t;            /* eq. 5.1 */
    *us = u0 * (cos(th) * cos(al) + cos(lam) * sin(th) * sin(al));  /* eq. 5.2 */
    *vs = -u0 * sin(lam) * sin(al);                                 /* eq. 5.3 */
    if (cs == ORC_IC_BUMPS) {
      double amp = P[3], rad = P[4];
      for (int b = 0; b < n_extra / 2; ++b) {
        double d = gc_dist(lam, th, ex[2 * b], ex[2 * b + 1]);
        *phi += g * amp * exp(-(d / rad) * (d / rad));
      }
    }
  } else if (cs == ORC_IC_ROSSBY) {
    double w = P[0], K = P[1], R = P[2], h0 = P[3];
    double ct = cos(th), st = sin(th);
    double A = 0.5 * w * (2.0 * Om + w) * ct * ct +
               0.25 * K * K * pow(ct, 2 * R) * ((R + 1) * ct * ct + 2 * R * R - R - 2 - 2 * R * R / (ct * ct));
    double B = 2.0 * (Om + w) * K / ((R + 1) * (R + 2)) * pow(ct, R) * (R * R + 2 * R + 2 - (R + 1) * (R + 1) * ct * ct);
    double C = 0.25 * K * K * pow(ct, 2 * R) * ((R + 1) * ct * ct - R - 2);
    *phi = g * h0 + a * a * (A + B * cos(R * lam) + C * cos(2 * R * lam));   /* eqs. 5.10, 5.13-5.15 */
    *us = a * w * ct + a * K * pow(ct, R - 1) * (R * st * st - ct * ct) * cos(R * lam); /* eq. 5.11 */
    *vs = -a * K * R * pow(ct, R - 1) * st * sin(R * lam);                    /* eq. 5.12 */
  } else { /* dam break, reading c18: great-circle distance, fluid at rest */
    double d = gc_dist(lam, th, P[0], P[1]);
    *phi = g * (d < P[2] ? P[3] : P[4]);
    *us = 0.0;
    *vs = 0.0;
  }
}

void orc_ic(const orc *o, int cs, const double *P_in, int n_extra, const double *ex, double *q) {
  int N = o->N, me = o->me;
  size_t pi = (size_t)N * N;
  double P[8];
  for (int t = 0; t < 8; ++t) P[t] = P_in[t];
  if (cs == ORC_IC_GALEWSKY && P[7] == 0.0) P[7] = jet_phi0(o, P);
#pragma omp parallel for schedule(static)
  for (int pj = 0; pj < 6 * N; ++pj) {
    int p = pj / N, j = pj % N;
    for (int i = 0; i < N; ++i) {
      double acc[3] = {0, 0, 0};
      for (int h = 0; h < me; ++h)
        for (int g = 0; g < me; ++g) {
          double X = tan(cell_centre(o, i) + o->gx[g] * o->dx);
          double Y = tan(cell_centre(o, j) + o->gx[h] * o->dx);
          double xyz[3], lam, th, phi, us, vs, m7[7], J[4], Ji[4];
          orc_xyz(p, X, Y, xyz);
          lonlat(xyz, &lam, &th);
          ic_point(o, cs, P, n_extra, ex, lam, th, &phi, &us, &vs);
          if (o->tcase) phi -= topo_lonlat(o, lam, th); /* reading c28: depth = phi_t - phi_s */
          orc_metric(X, Y, m7);
          orc_jacobian(p, X, Y, J);
          inv2(J, Ji);
          double u = (Ji[0] * us + Ji[1] * vs) / o->r, v = (Ji[2] * us + Ji[3] * vs) / o->r;
          double w = o->gw[g] * o->gw[h];
          acc[0] += w * m7[0] * phi;
          acc[1] += w * m7[0] * phi * u;
          acc[2] += w * m7[0] * phi * v;
        }
      for (int v = 0; v < 3; ++v) q[(size_t)(v * 6 + p) * pi + (size_t)j * N + i] = acc[v];
    }
  }
}

void orc_ic_point(const orc *o, int cs, const double *P_in, double lam, double th, double *out3) {
  double P[8];
  for (int t = 0; t < 8; ++t) P[t] = P_in[t];
  if (cs == ORC_IC_GALEWSKY && P[7] == 0.0) P[7] = jet_phi0(o, P);
  ic_point(o, cs, P, 0, NULL, lam, th, out3, out3 + 1, out3 + 2);
}

void orc_cell_sqrtg(const orc *o, double *out) {
  int N = o->N, me = o->me;
  for (int p = 0; p < 6; ++p)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int h = 0; h < me; ++h)
          for (int g = 0; g < me; ++g) {
            double m7[7];
            orc_metric(tan(cell_centre(o, i) + o->gx[g] * o->dx), tan(cell_centre(o, j) + o->gx[h] * o->dx), m7);
            acc += o->gw[g] * o->gw[h] * m7[0];
          }
        out[((size_t)p * N + j) * N + i] = acc;
      }
}

/* Error norms of phi (eqs. 5.4-5.7), reading c16: phi = q0 / <sqrtG>, the     */
/* I() weights are <sqrtG>, the L1 numerator takes absolute values.            */
void orc_norms(const orc *o, const double *q, const double *qr, double *out) {
  size_t n = (size_t)6 * o->N * o->N;
  double *sg = (double *)malloc(sizeof(double) * n);
  orc_cell_sqrtg(o, sg);
  long double n1 = 0, d1 = 0, n2 = 0, d2 = 0;
  double mx = 0, mr = 0;
  for (size_t c = 0; c < n; ++c) {
    double ph = q[c] / sg[c], pr = qr[c] / sg[c], d = ph - pr;
    n1 += sg[c] * fabs(d);
    d1 += sg[c] * fabs(pr);
    n2 += sg[c] * d * d;
    d2 += sg[c] * pr * pr;
    if (fabs(d) > mx) mx = fabs(d);
    if (fabs(pr) > mr) mr = fabs(pr);
  }
  out[0] = (double)(n1 / d1);
  out[1] = (double)sqrtl(n2 / d2);
  out[2] = mx / mr;
  free(sg);
}

/* ------------------------------------------------------------------------- */
/* Table exports for the PyTorch reference composition (test infrastructure). */
/* ------------------------------------------------------------------------- */
int orc_ghost_count(const orc *o) { return o->nring; }

void orc_ghost_tables(const orc *o, int *ring, int *B, int *ic, int *jc, double *wx, double *wy,
                      double *ratio, double *C, double *w) {
  int me = o->me, k = o->k;
  for (int c = 0; c < o->nring; ++c) ring[c] = o->ring[c];
  for (size_t r = 0; r < (size_t)6 * o->nring * me * me * 2; ++r) {
    const gqp_t *g = &o->gq[r];
    w[r] = g->w;
    B[r] = g->B;
    ic[r] = g->ic;
    jc[r] = g->jc;
    for (int a = 0; a < k; ++a) {
      wx[r * k + a] = g->wx[a];
      wy[r * k + a] = g->wy[a];
    }
    ratio[r] = g->ratio;
    for (int t = 0; t < 4; ++t) C[r * 4 + t] = g->C[t];
  }
}

void orc_edge_tables(const orc *o, int *B, int *sideB, int *tB, int *gB, double *ratio, double *C) {
  for (size_t r = 0; r < (size_t)6 * 4 * o->N * o->me; ++r) {
    const nbr_t *n = &o->nb[r];
    B[r] = n->B;
    sideB[r] = n->sideB;
    tB[r] = n->tB;
    gB[r] = n->gB;
    ratio[r] = n->ratio;
    for (int t = 0; t < 4; ++t) C[r * 4 + t] = n->C[t];
  }
}

double orc_coriolis(const orc *o, int p, double X, double Y) { return coriolis(o, p, X, Y); }
