// hope_setup_math.cuh -- FP64 setup mathematics shared by the host-side table
// assembly and the device-side setup kernels of the HOPE GB300 library.
//
// Everything here is evaluated once per grid at set-up; nothing runs per stage.
// Routes are chosen for conditioning in FP64:
//   * cell-average reconstruction weights through the derivative of the Lagrange
//     interpolant of the primitive function at the cell interfaces (the unique
//     polynomial of degree n-1 with the given cell averages, section 3.1);
//   * panel conversions through the tangent and dual bases of the two panels' maps
//     (the same matrices as eqs. 3.26-3.29, obtained without latitude/longitude);
//   * WENO linear weights as tensor products of 1-D least-squares weights
//     (eq. 3.19 factorises for the tensor-product basis).
#pragma once
#include <math.h>

#ifndef HOPE_HD
#define HOPE_HD __host__ __device__ inline
#endif

#define HOPE_MAXK 11
#define HOPE_MAXME 6
#define HOPE_PI 3.14159265358979323846
#define HOPE_QPI (HOPE_PI / 4.0)

namespace hope {

// Panel frames: panel p maps (X, Y) to (n + X e1 + Y e2)/delta (see include/hope.h).
HOPE_HD void panel_frame(int p, double n[3], double e1[3], double e2[3]) {
  for (int c = 0; c < 3; ++c) n[c] = e1[c] = e2[c] = 0.0;
  switch (p) {
    case 0: n[0] = 1; e1[1] = 1; e2[2] = 1; break;
    case 1: n[1] = 1; e1[0] = -1; e2[2] = 1; break;
    case 2: n[0] = -1; e1[1] = -1; e2[2] = 1; break;
    case 3: n[1] = -1; e1[0] = 1; e2[2] = 1; break;
    case 4: n[2] = 1; e1[1] = 1; e2[0] = -1; break;
    default: n[2] = -1; e1[1] = 1; e2[0] = 1; break;
  }
}

HOPE_HD double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

HOPE_HD void panel_point(int p, double X, double Y, double P[3]) {
  double n[3], e1[3], e2[3];
  panel_frame(p, n, e1, e2);
  double d = sqrt(1.0 + X * X + Y * Y);
  for (int c = 0; c < 3; ++c) P[c] = (n[c] + X * e1[c] + Y * e2[c]) / d;
}

// Panel whose face contains P: largest projection on the face normal.  Projections
// within 1e-12 of each other (a point on a cube edge) resolve to the lower panel index.
HOPE_HD int face_of(const double P[3], int exclude) {
  int best = -1;
  double bv = -2.0;
  for (int p = 0; p < 6; ++p) {
    if (p == exclude) continue;
    double n[3], e1[3], e2[3];
    panel_frame(p, n, e1, e2);
    double d = dot3(P, n);
    if (d > bv + 1e-12) {
      bv = d;
      best = p;
    }
  }
  return best;
}

HOPE_HD void panel_coords(int p, const double P[3], double *X, double *Y) {
  double n[3], e1[3], e2[3];
  panel_frame(p, n, e1, e2);
  double t = dot3(P, n);
  *X = dot3(P, e1) / t;
  *Y = dot3(P, e2) / t;
}

HOPE_HD double sqrtg_unit(double X, double Y) {
  double d2 = 1.0 + X * X + Y * Y;
  return (1.0 + X * X) * (1.0 + Y * Y) / (d2 * sqrt(d2));
}

// Unit-sphere tangent vectors a_x = dP/dx, a_y = dP/dy of panel p at (X, Y).
HOPE_HD void tangent_basis(int p, double X, double Y, double ax[3], double ay[3]) {
  double n[3], e1[3], e2[3], P[3];
  panel_frame(p, n, e1, e2);
  double d = sqrt(1.0 + X * X + Y * Y);
  for (int c = 0; c < 3; ++c) P[c] = (n[c] + X * e1[c] + Y * e2[c]) / d;
  double pe1 = dot3(P, e1), pe2 = dot3(P, e2);
  for (int c = 0; c < 3; ++c) {
    ax[c] = (1.0 + X * X) * (e1[c] - P[c] * pe1) / d;
    ay[c] = (1.0 + Y * Y) * (e2[c] - P[c] * pe2) / d;
  }
}

// Conversion of a state at one point of the sphere from panel B (at XB, YB) to panel A
// (at XA, YA): mass factor sqrtG_A/sqrtG_B and momentum matrix
// C = (sqrtG_A/sqrtG_B) [dual basis of A]^T [tangent basis of B]  (= eq. 3.29's C).
HOPE_HD void panel_conversion(int A, double XA, double YA, int B, double XB, double YB,
                              double *ratio, double C[4]) {
  double ax[3], ay[3], bx[3], by[3];
  tangent_basis(A, XA, YA, ax, ay);
  tangent_basis(B, XB, YB, bx, by);
  double g11 = dot3(ax, ax), g12 = dot3(ax, ay), g22 = dot3(ay, ay);
  double det = g11 * g22 - g12 * g12;
  double i11 = g22 / det, i12 = -g12 / det, i22 = g11 / det;
  double dx[3], dy[3];
  for (int c = 0; c < 3; ++c) {
    dx[c] = i11 * ax[c] + i12 * ay[c];
    dy[c] = i12 * ax[c] + i22 * ay[c];
  }
  double r = sqrtg_unit(XA, YA) / sqrtg_unit(XB, YB);
  *ratio = r;
  C[0] = r * dot3(dx, bx);
  C[1] = r * dot3(dx, by);
  C[2] = r * dot3(dy, bx);
  C[3] = r * dot3(dy, by);
}

// Gauss-Legendre nodes (ascending) and weights (summing to 1) on [-1/2, 1/2].
HOPE_HD void gauss_legendre(int m, double *x, double *w) {
  for (int i = 0; i < m; ++i) {
    double z = cos(HOPE_PI * (i + 0.75) / (m + 0.5));
    double pm = 0.0, pm1 = 0.0;
    for (int it = 0; it < 60; ++it) {
      double a = 1.0, b = z;  // P_0, P_1
      for (int n = 2; n <= m; ++n) {
        double c = ((2.0 * n - 1.0) * z * b - (n - 1.0) * a) / n;
        a = b;
        b = c;
      }
      pm = (m == 1) ? z : b;
      pm1 = (m == 1) ? 1.0 : a;
      double dp = m * (z * pm - pm1) / (z * z - 1.0);
      double dz = pm / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    double a = 1.0, b = z;
    for (int n = 2; n <= m; ++n) {
      double c = ((2.0 * n - 1.0) * z * b - (n - 1.0) * a) / n;
      a = b;
      b = c;
    }
    pm = (m == 1) ? z : b;
    pm1 = (m == 1) ? 1.0 : a;
    double dp = m * (z * pm - pm1) / (z * z - 1.0);
    x[m - 1 - i] = 0.5 * z;
    w[m - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Cell-average reconstruction weights of an n-cell stencil of unit cells whose first
// cell is centred at offset o0 from the target cell, evaluated at xi (target-cell
// coordinates): with interfaces z_m = o0 - 1/2 + m (m = 0..n) and L_m the Lagrange basis
// on them, p(xi) = sum_m P(z_m) L_m'(xi) with P the primitive, so w_j = sum_{m>j} L_m'(xi).
HOPE_HD void cell_avg_weights(int n, int o0, double xi, double *w) {
  double z[HOPE_MAXK + 2];
  for (int m = 0; m <= n; ++m) z[m] = o0 - 0.5 + m;
  double dl[HOPE_MAXK + 2];
  for (int m = 0; m <= n; ++m) {
    double s = 0.0;
    for (int a = 0; a <= n; ++a) {
      if (a == m) continue;
      double t = 1.0 / (z[m] - z[a]);
      for (int b = 0; b <= n; ++b) {
        if (b == m || b == a) continue;
        t *= (xi - z[b]) / (z[m] - z[b]);
      }
      s += t;
    }
    dl[m] = s;
  }
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int m = j + 1; m <= n; ++m) s += dl[m];
    w[j] = s;
  }
}

// Weights of the first derivative (in target-cell units) of the same polynomial at xi:
// p'(xi) = sum_m P(z_m) L_m''(xi), so w'_j = sum_{m>j} L_m''(xi), with
// L_m'' = sum over ordered pairs a != b (both != m) of prod_{c != m, a, b} (xi - z_c)
// over prod_{c != m} (z_m - z_c).
HOPE_HD void cell_avg_dweights(int n, int o0, double xi, double *w) {
  double z[HOPE_MAXK + 2];
  for (int m = 0; m <= n; ++m) z[m] = o0 - 0.5 + m;
  double d2[HOPE_MAXK + 2];
  for (int m = 0; m <= n; ++m) {
    double den = 1.0;
    for (int c = 0; c <= n; ++c)
      if (c != m) den *= z[m] - z[c];
    double s = 0.0;
    for (int a = 0; a <= n; ++a) {
      if (a == m) continue;
      for (int b = 0; b <= n; ++b) {
        if (b == m || b == a) continue;
        double t = 1.0;
        for (int c = 0; c <= n; ++c)
          if (c != m && c != a && c != b) t *= xi - z[c];
        s += t;
      }
    }
    d2[m] = s / den;
  }
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int m = j + 1; m <= n; ++m) s += d2[m];
    w[j] = s;
  }
}

// Gradient of the unit-sphere sqrtG = (1+X^2)(1+Y^2)/delta^3 with respect to the panel
// angles: d/dX = X (1+Y^2)(2Y^2 - X^2 - 1)/delta^5 and dX/dx = 1+X^2 (symmetric in y).
HOPE_HD void sqrtg_unit_grad(double X, double Y, double *gx, double *gy) {
  const double d2 = 1.0 + X * X + Y * Y, d5 = d2 * d2 * sqrt(d2);
  const double ax = 1.0 + X * X, ay = 1.0 + Y * Y;
  *gx = X * ay * (2.0 * Y * Y - X * X - 1.0) / d5 * ax;
  *gy = Y * ax * (2.0 * X * X - Y * Y - 1.0) / d5 * ay;
}

// 1-D WENO linear weights: the l sub-stencils of width l inside the central stencil of
// width k = 2l-1 (sub-stencil s covers offsets s-H .. s-H+l-1), gamma minimising
// |R_L gamma - R_H| (normal equations, partial pivoting).  Returns the max residual.
HOPE_HD double weno_linear_weights_1d(int k, double xi, double *gam) {
  int H = (k - 1) / 2, l = (k + 1) / 2;
  double RH[HOPE_MAXK], RL[HOPE_MAXK][HOPE_MAXME], sub[HOPE_MAXME];
  cell_avg_weights(k, -H, xi, RH);
  for (int c = 0; c < k; ++c)
    for (int s = 0; s < l; ++s) RL[c][s] = 0.0;
  for (int s = 0; s < l; ++s) {
    cell_avg_weights(l, s - H, xi, sub);
    for (int a = 0; a < l; ++a) RL[s + a][s] = sub[a];
  }
  double M[HOPE_MAXME][HOPE_MAXME + 1];
  for (int i = 0; i < l; ++i) {
    for (int j = 0; j < l; ++j) {
      double t = 0.0;
      for (int c = 0; c < k; ++c) t += RL[c][i] * RL[c][j];
      M[i][j] = t;
    }
    double t = 0.0;
    for (int c = 0; c < k; ++c) t += RL[c][i] * RH[c];
    M[i][l] = t;
  }
  for (int c = 0; c < l; ++c) {
    int piv = c;
    for (int r = c + 1; r < l; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    for (int j = 0; j <= l; ++j) {
      double t = M[c][j];
      M[c][j] = M[piv][j];
      M[piv][j] = t;
    }
    for (int r = 0; r < l; ++r) {
      if (r == c) continue;
      double f = M[r][c] / M[c][c];
      for (int j = c; j <= l; ++j) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = 0; i < l; ++i) gam[i] = M[i][l] / M[i][i];
  double res = 0.0;
  for (int c = 0; c < k; ++c) {
    double t = -RH[c];
    for (int s = 0; s < l; ++s) t += RL[c][s] * gam[s];
    if (fabs(t) > res) res = fabs(t);
  }
  return res;
}

// Smoothness-indicator 1-D forms of the l-cell sub-stencil starting at offset o0:
// B0[i][j] = integral over [-1/2,1/2] of phi_i phi_j and S[i][j] = sum_{a=0}^{l-1} of the
// same integral of the a-th derivatives, phi_i the cell-average basis polynomial of
// cell i.  With them beta = Q.(S_y Q S_x^T) - Q.(B0_y Q B0_x^T) (eq. 3.25 read as the sum
// of squared mixed derivatives of orders (a1, a2) != (0, 0), a1, a2 <= l-1).
HOPE_HD void weno_beta_forms_1d(int l, int o0, double *S, double *B0) {
  // monomial coefficients of phi_i: phi_i = sum_{m>i} L_m'
  double z[HOPE_MAXME + 2];
  for (int m = 0; m <= l; ++m) z[m] = o0 - 0.5 + m;
  double Lc[HOPE_MAXME + 2][HOPE_MAXME + 2];  // L_m monomial coefficients, degree l
  for (int m = 0; m <= l; ++m) {
    double c[HOPE_MAXME + 2];
    for (int t = 0; t <= l; ++t) c[t] = 0.0;
    c[0] = 1.0;
    int deg = 0;
    double den = 1.0;
    for (int b = 0; b <= l; ++b) {
      if (b == m) continue;
      // multiply by (xi - z_b)
      for (int t = deg + 1; t >= 1; --t) c[t] = c[t - 1] - z[b] * c[t];
      c[0] = -z[b] * c[0];
      ++deg;
      den *= (z[m] - z[b]);
    }
    for (int t = 0; t <= l; ++t) Lc[m][t] = c[t] / den;
  }
  double ph[HOPE_MAXME][HOPE_MAXME];  // phi_i coefficients, degree l-1
  for (int i = 0; i < l; ++i)
    for (int t = 0; t < l; ++t) {
      double s = 0.0;
      for (int m = i + 1; m <= l; ++m) s += (t + 1) * Lc[m][t + 1];
      ph[i][t] = s;
    }
  for (int i = 0; i < l; ++i)
    for (int j = 0; j < l; ++j) {
      S[i * l + j] = 0.0;
      B0[i * l + j] = 0.0;
    }
  for (int a = 0; a < l; ++a) {
    // a-th derivative coefficients
    double da[HOPE_MAXME][HOPE_MAXME];
    for (int i = 0; i < l; ++i)
      for (int t = 0; t < l; ++t) {
        if (t + a < l) {
          double f = 1.0;
          for (int u = 0; u < a; ++u) f *= (double)(t + a - u);
          da[i][t] = f * ph[i][t + a];
        } else {
          da[i][t] = 0.0;
        }
      }
    for (int i = 0; i < l; ++i)
      for (int j = 0; j < l; ++j) {
        double s = 0.0;
        for (int t = 0; t < l; ++t)
          for (int u = 0; u < l; ++u) {
            int e = t + u;
            if (e % 2) continue;
            s += da[i][t] * da[j][u] * 2.0 * pow(0.5, e + 1) / (e + 1);
          }
        S[i * l + j] += s;
        if (a == 0) B0[i * l + j] = s;
      }
  }
}

// Simultaneous diagonalisation of the smoothness forms of one sub-stencil: with
// B0 = L L^T (Cholesky) and L^{-1} S L^{-T} = U diag(lam) U^T (cyclic Jacobi), the matrix
// Winv = U^T L^T gives q^T B0 q = |Winv q|^2 and q^T S q = sum_k lam_k (Winv q)_k^2, so the
// 2-D indicator is beta = sum_{k,k'} (lam_y,k lam_x,k' - 1) Z_{k k'}^2, Z = Winv_y Q Winv_x^T.
// Returns 0 on success.
inline int weno_beta_diag(int l, const double *S, const double *B0, double *Winv, double *lam) {
  double L[HOPE_MAXME][HOPE_MAXME] = {}, Li[HOPE_MAXME][HOPE_MAXME] = {};
  for (int i = 0; i < l; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = B0[i * l + j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(s > 0)) return -1;
        L[i][i] = sqrt(s);
      } else {
        L[i][j] = s / L[j][j];
      }
    }
  for (int c = 0; c < l; ++c) {  // Li = L^{-1} by forward substitution
    for (int i = 0; i < l; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[i][k] * Li[k][c];
      Li[i][c] = s / L[i][i];
    }
  }
  double M[HOPE_MAXME][HOPE_MAXME], U[HOPE_MAXME][HOPE_MAXME];
  for (int i = 0; i < l; ++i)
    for (int j = 0; j < l; ++j) {
      double s = 0.0;
      for (int a = 0; a < l; ++a)
        for (int b = 0; b < l; ++b) s += Li[i][a] * S[a * l + b] * Li[j][b];
      M[i][j] = s;
      U[i][j] = (i == j) ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < l; ++p)
      for (int q = p + 1; q < l; ++q) off += M[p][q] * M[p][q];
    if (off < 1e-32) break;
    for (int p = 0; p < l; ++p)
      for (int q = p + 1; q < l; ++q) {
        if (fabs(M[p][q]) < 1e-300) continue;
        double th = (M[q][q] - M[p][p]) / (2.0 * M[p][q]);
        double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < l; ++k) {  // M <- J^T M J
          double mkp = M[k][p], mkq = M[k][q];
          M[k][p] = c * mkp - s * mkq;
          M[k][q] = s * mkp + c * mkq;
        }
        for (int k = 0; k < l; ++k) {
          double mpk = M[p][k], mqk = M[q][k];
          M[p][k] = c * mpk - s * mqk;
          M[q][k] = s * mpk + c * mqk;
        }
        for (int k = 0; k < l; ++k) {
          double ukp = U[k][p], ukq = U[k][q];
          U[k][p] = c * ukp - s * ukq;
          U[k][q] = s * ukp + c * ukq;
        }
      }
  }
  for (int k = 0; k < l; ++k) {
    lam[k] = M[k][k];
    for (int a = 0; a < l; ++a) {  // Winv = U^T L^T: row k = sum_i U[i][k] L[a][i]
      double s = 0.0;
      for (int i = 0; i < l; ++i) s += U[i][k] * L[a][i];
      Winv[k * l + a] = s;
    }
  }
  return 0;
}

}  // namespace hope
