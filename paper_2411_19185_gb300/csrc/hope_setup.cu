// hope_setup.cu -- per-grid table construction of the HOPE GB300 library (setup only,
// never on the per-stage path): device-side FP64 tables (1-D reconstruction weights,
// metric terms), host-side assembly of the ghost operator G (appendix eq. 7.12) and of
// the cube-edge topology.
#include <math.h>
#include <omp.h>

#include <algorithm>
#include <string>
#include <vector>

#include "hope_internal.h"
#include "hope_setup.h"
#include "hope_setup_math.cuh"

namespace hope {

// -------------------------------------------------------------------------------
// Device setup kernels (FP64), writing tables in the context precision T.
// -------------------------------------------------------------------------------
// w1 holds [me+2][K] point weights, then [npair][K] mirror-pair weights: a cell's weights
// at -xi are its weights at +xi in reverse tap order (the stencil is symmetric about the
// cell), so with the line folded into sums s_b = v_b + v_{K-1-b} and differences
// d_b = v_b - v_{K-1-b} (b < H), E = c v_H + sum e_b s_b and O = sum o_b d_b give
// p(+xi) = E + O and p(-xi) = E - O; e_b, o_b are the even and odd halves of the +xi
// weights (stored at taps b and K-1-b, the centre weight c at tap H).  Pairs: the edges
// -1/2, +1/2; the Gauss nodes g and me-1-g; for odd me the middle node alone (o = 0).
template <typename T>
__global__ void k_setup_order(int K, int me, T *w1, T *gw, double *nodes_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double x[HOPE_MAXME], w[HOPE_MAXME], r[HOPE_MAXK];
  gauss_legendre(me, x, w);
  const int H = (K - 1) / 2;
  for (int t = 0; t < me + 2; ++t) {
    double xi = t == 0 ? -0.5 : (t == 1 ? 0.5 : x[t - 2]);
    cell_avg_weights(K, -H, xi, r);
    for (int b = 0; b < K; ++b) w1[t * K + b] = (T)r[b];
  }
  const int npair = 1 + (me + 1) / 2;
  T *eo = w1 + (me + 2) * K;
  for (int pi = 0; pi < npair; ++pi) {
    const bool self = (me & 1) && pi == npair - 1;
    const double xi = pi == 0 ? 0.5 : x[me - pi];  // the +xi member of the pair
    cell_avg_weights(K, -H, xi, r);
    for (int b = 0; b < H; ++b) {
      eo[pi * K + b] = (T)(0.5 * (r[b] + r[K - 1 - b]));
      eo[pi * K + K - 1 - b] = self ? T(0) : (T)(0.5 * (r[b] - r[K - 1 - b]));
    }
    eo[pi * K + H] = (T)r[H];
  }
  for (int g = 0; g < me; ++g) {
    gw[g] = (T)w[g];
    nodes_out[g] = x[g];
    nodes_out[me + g] = w[g];
  }
}

template <typename T>
__global__ void k_setup_grid(int N, int me, double radius, const double *__restrict__ nw, T *Xg, T *t1w,
                             T *mx, T *src8) {
  const double dx = HOPE_PI / (2.0 * N);
  const double r2 = radius * radius;
  const long long nX = (long long)N * me, nT = (long long)N * N * me * me, nM = (long long)(N + 1) * N * me;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nX + nT + nM;
       idx += (long long)gridDim.x * blockDim.x) {
    if (idx < nX) {
      int i = (int)(idx / me), g = (int)(idx % me);
      Xg[idx] = (T)tan(-HOPE_QPI + (i + 0.5 + nw[g]) * dx);
    } else if (idx < nX + nT) {
      long long r = idx - nX;
      int g = (int)(r % me);
      long long t = r / me;
      int h = (int)(t % me);
      t /= me;
      int i = (int)(t % N), j = (int)(t / N);
      double X = tan(-HOPE_QPI + (i + 0.5 + nw[g]) * dx);
      double Y = tan(-HOPE_QPI + (j + 0.5 + nw[h]) * dx);
      const double tw = 2.0 / (1.0 + X * X + Y * Y) * nw[me + g] * nw[me + h];
      t1w[r] = (T)tw;
      // source polynomials with the weight folded in (eqs. 2.2, 2.3 times W_gh 2/delta^2):
      //   a1 = (c1 q1 + c2 q2) q1/q0 + os (e1 q1 + e2 q2)
      //   a2 = (c3 q1 + c4 q2) q2/q0 + os (e3 q1 + e4 q2),  os = Omega sin(lat) delta
      if (!src8) continue;
      T *o = src8 + r * 8;
      o[0] = (T)(-tw * X * Y * Y);
      o[1] = (T)(tw * Y * (1.0 + Y * Y));
      o[2] = (T)(tw * X * (1.0 + X * X));
      o[3] = (T)(-tw * X * X * Y);
      o[4] = (T)(-tw * X * Y);
      o[5] = (T)(tw * (1.0 + Y * Y));
      o[6] = (T)(-tw * (1.0 + X * X));
      o[7] = (T)(tw * X * Y);
    } else {
      long long r = idx - nX - nT;
      int g = (int)(r % me);
      long long t = r / me;
      int j = (int)(t % N), e = (int)(t / N);
      double X = tan(-HOPE_QPI + e * dx);
      double Y = tan(-HOPE_QPI + (j + 0.5 + nw[g]) * dx);
      double d2 = 1.0 + X * X + Y * Y, d = sqrt(d2);
      double sg = (1.0 + X * X) * (1.0 + Y * Y) / (d2 * d);
      double g11 = d2 / (1.0 + X * X);  // unit-sphere G^11 (eq. 2.6)
      double s11 = sqrt(g11) / radius;
      const T v[5] = {(T)(1.0 / sg), (T)s11, (T)(1.0 / s11),
                      (T)(0.5 * (1.0 + Y * Y) / (d * r2)),  // sqrtG G^11 / 2 (true metric)
                      (T)(0.5 * X * Y / (d * r2))};         // sqrtG G^12 / 2
      // five planes, stored with e fastest and again with the position j fastest
      const size_t plane = (size_t)me * N * (N + 1);
      const size_t ox = ((size_t)g * N + j) * (N + 1) + e, oy = 5 * plane + ((size_t)g * (N + 1) + e) * N + j;
      for (int c = 0; c < 5; ++c) {
        mx[c * plane + ox] = v[c];
        mx[c * plane + oy] = v[c];
      }
    }
  }
}

template __global__ void k_setup_order<double>(int, int, double *, double *, double *);
template __global__ void k_setup_order<float>(int, int, float *, float *, double *);
template __global__ void k_setup_grid<double>(int, int, double, const double *, double *, double *, double *,
                                              double *);
template __global__ void k_setup_grid<float>(int, int, double, const double *, float *, float *, float *, float *);

int setup_order_tables(hope_ctx *ctx, std::vector<double> &nodes, std::vector<double> &weights) {
  const int K = ctx->k, me = ctx->me;
  double *d_nw = nullptr;
  if (cudaMalloc(&d_nw, sizeof(double) * 2 * me) != cudaSuccess) return HOPE_ENOMEM;
  if (cudaMalloc(&ctx->w1, ctx->esize * (me + 2 + 1 + (me + 1) / 2) * K) != cudaSuccess) return HOPE_ENOMEM;
  if (cudaMalloc(&ctx->gw, ctx->esize * me) != cudaSuccess) return HOPE_ENOMEM;
  if (ctx->prec == HOPE_FP64)
    k_setup_order<double><<<1, 1>>>(K, me, (double *)ctx->w1, (double *)ctx->gw, d_nw);
  else
    k_setup_order<float><<<1, 1>>>(K, me, (float *)ctx->w1, (float *)ctx->gw, d_nw);
  std::vector<double> nw(2 * me);
  ctx->w1_host.resize((size_t)ctx->esize * (me + 2 + 1 + (me + 1) / 2) * K);
  if (cudaMemcpy(nw.data(), d_nw, sizeof(double) * 2 * me, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(ctx->w1_host.data(), ctx->w1, ctx->w1_host.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaFree(d_nw);
    return HOPE_ECUDA;
  }
  cudaFree(d_nw);
  nodes.assign(nw.begin(), nw.begin() + me);
  weights.assign(nw.begin() + me, nw.end());
  return HOPE_OK;
}

int setup_grid_tables(hope_ctx *ctx, Grid &gr, const std::vector<double> &nodes,
                      const std::vector<double> &weights) {
  const int N = gr.N, me = ctx->me;
  std::vector<double> nw(nodes);
  nw.insert(nw.end(), weights.begin(), weights.end());
  double *d_nw = nullptr;
  if (cudaMalloc(&d_nw, sizeof(double) * 2 * me) != cudaSuccess) return HOPE_ENOMEM;
  cudaMemcpy(d_nw, nw.data(), sizeof(double) * 2 * me, cudaMemcpyHostToDevice);
  size_t es = ctx->esize;
  if (cudaMalloc(&gr.Xg, es * N * me) != cudaSuccess) return HOPE_ENOMEM;
  if (cudaMalloc(&gr.t1w, es * (size_t)N * N * me * me) != cudaSuccess) return HOPE_ENOMEM;
  if (cudaMalloc(&gr.mx, es * (size_t)(N + 1) * N * me * 10) != cudaSuccess) return HOPE_ENOMEM;
  // the tabulated source polynomials serve only the FP64 TPP reconstruction
  if (ctx->prec == HOPE_FP64 && ctx->scheme == HOPE_TPP &&
      cudaMalloc(&gr.src8, es * (size_t)N * N * me * me * 8) != cudaSuccess)
    return HOPE_ENOMEM;
  if (ctx->prec == HOPE_FP64)
    k_setup_grid<double><<<256, 256>>>(N, me, ctx->radius, d_nw, (double *)gr.Xg, (double *)gr.t1w,
                                       (double *)gr.mx, (double *)gr.src8);
  else
    k_setup_grid<float><<<256, 256>>>(N, me, ctx->radius, d_nw, (float *)gr.Xg, (float *)gr.t1w,
                                      (float *)gr.mx, (float *)gr.src8);
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(d_nw);
  return e == cudaSuccess ? HOPE_OK : HOPE_ECUDA;
}

// -------------------------------------------------------------------------------
// Host assembly of the ghost operator: the map from interior cells to ghost cells
// obtained by `iters` Jacobi sweeps of the ghost interpolation from zero
// (section 3.3.1): each sweep interpolates every ghost Gauss point with the owning
// panel's central TPP stencil (reading that panel's ghosts of the previous sweep),
// converts it (eqs. 3.26-3.29) and averages (eq. 3.6).  Composed symbolically: a
// row of G holds, per source cell, a mass weight and a 2x2 momentum block.
// -------------------------------------------------------------------------------
namespace {
struct Ent {
  int col;
  double m, c[4];
};
struct LocalEnt {
  int idx;     // interior cell id, or ghost row id
  bool ghost;
  double m, c[4];
};
}  // namespace

// The 24 rotations of the cube and, per rotation t and panel p, the image panel and the
// induced map of panel coordinates X' = a X + c Y, Y' = b X + d Y (A = {a, b, c, d}).
struct CubeRotations {
  int img[24][6];
  int A[24][6][4];
  int identity = -1;
};

static void cube_rotations(CubeRotations &cr) {
  static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int t = 0;
  for (int pi = 0; pi < 6; ++pi)
    for (int sg = 0; sg < 8; ++sg) {
      int m[3][3] = {};
      for (int i = 0; i < 3; ++i) m[i][perm[pi][i]] = (sg >> i & 1) ? -1 : 1;
      const int det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                      m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                      m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
      if (det != 1) continue;
      if (pi == 0 && sg == 0) cr.identity = t;
      for (int p = 0; p < 6; ++p) {
        double n[3], e1[3], e2[3], Rn[3], R1[3], R2[3];
        panel_frame(p, n, e1, e2);
        for (int i = 0; i < 3; ++i) {
          Rn[i] = R1[i] = R2[i] = 0.0;
          for (int j = 0; j < 3; ++j) {
            Rn[i] += m[i][j] * n[j];
            R1[i] += m[i][j] * e1[j];
            R2[i] += m[i][j] * e2[j];
          }
        }
        int q = 0;
        for (int f = 0; f < 6; ++f) {
          double fn[3], f1[3], f2[3];
          panel_frame(f, fn, f1, f2);
          if (dot3(fn, Rn) > 0.5) q = f;
        }
        double fn[3], f1[3], f2[3];
        panel_frame(q, fn, f1, f2);
        cr.img[t][p] = q;
        cr.A[t][p][0] = (int)lround(dot3(R1, f1));
        cr.A[t][p][1] = (int)lround(dot3(R1, f2));
        cr.A[t][p][2] = (int)lround(dot3(R2, f1));
        cr.A[t][p][3] = (int)lround(dot3(R2, f2));
      }
      ++t;
    }
}

// index (i, j) of an n x n array centred on the panel centre, mapped by rotation t from panel p
static inline void rot_index(const CubeRotations &cr, int t, int p, int i, int j, int n, int *p2, int *i2,
                             int *j2) {
  const int *A = cr.A[t][p];
  const int u = 2 * i - (n - 1), v = 2 * j - (n - 1);
  *p2 = cr.img[t][p];
  *i2 = (A[0] * u + A[2] * v + (n - 1)) / 2;
  *j2 = (A[1] * u + A[3] * v + (n - 1)) / 2;
}

// transform code of a 2x2 signed permutation: bit 0 swap, bit 1 negate the first output,
// bit 2 negate the second.  in: v = M^T u (M = [[a, c], [b, d]]); out: g = M s.
static inline int code_in(const int *A) {
  return A[0] != 0 ? ((A[0] < 0) << 1) | ((A[3] < 0) << 2) : 1 | ((A[1] < 0) << 1) | ((A[2] < 0) << 2);
}
static inline int code_out(const int *A) {
  return A[0] != 0 ? ((A[0] < 0) << 1) | ((A[3] < 0) << 2) : 1 | ((A[2] < 0) << 1) | ((A[1] < 0) << 2);
}

int build_ghost_operator(const hope_ctx *ctx, int N, const std::vector<double> &nodes,
                         const std::vector<double> &weights, std::vector<int> &rowptr,
                         std::vector<int> &cols, std::vector<double> &vals, std::vector<int> &dst,
                         GhostSplit *split, GhostSym *sym) {
  const int K = ctx->k, H = ctx->H, me = ctx->me, ne = N + 2 * H;
  const double dx = HOPE_PI / (2.0 * N);
  // ring enumeration
  std::vector<int> rowid((size_t)6 * ne * ne, -1);
  dst.clear();
  for (int p = 0; p < 6; ++p)
    for (int jj = 0; jj < ne; ++jj)
      for (int ii = 0; ii < ne; ++ii) {
        int i = ii - H, j = jj - H;
        if (i >= 0 && i < N && j >= 0 && j < N) continue;
        rowid[((size_t)p * ne + jj) * ne + ii] = (int)dst.size();
        dst.push_back((p * ne + jj) * ne + ii);
      }
  const int rows = (int)dst.size();
  // local operators
  std::vector<std::vector<LocalEnt>> loc(rows);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
  for (int r = 0; r < rows; ++r) {
    int p = dst[r] / (ne * ne), rem = dst[r] % (ne * ne), jj = rem / ne, ii = rem % ne;
    int i = ii - H, j = jj - H;
    std::vector<LocalEnt> acc;
    acc.reserve((K + 2) * (K + 2));
    for (int h = 0; h < me; ++h)
      for (int g = 0; g < me; ++g) {
        double x = -HOPE_QPI + (i + 0.5 + nodes[g]) * dx;
        double y = -HOPE_QPI + (j + 0.5 + nodes[h]) * dx;
        double X = tan(x), Y = tan(y), P[3], XB, YB;
        panel_point(p, X, Y, P);
        // owners: the face(s) with the largest projection; a point on a cube edge (two
        // projections within 1e-12) takes the mean of both panels' interpolations
        int own[2], nown = 0;
        {
          double d[6], bv = -2.0;
          for (int f = 0; f < 6; ++f) {
            double n[3], e1[3], e2[3];
            panel_frame(f, n, e1, e2);
            d[f] = dot3(P, n);
            bv = fmax(bv, d[f]);
          }
          for (int f = 0; f < 6 && nown < 2; ++f)
            if (d[f] > bv - 1e-12) own[nown++] = f;
        }
        for (int o = 0; o < nown; ++o) {
        const int B = own[o];
        if (B == p) {
#pragma omp atomic
          ++bad;
          continue;
        }
        panel_coords(B, P, &XB, &YB);
        double xb = atan(XB), yb = atan(YB);
        int ic = (int)floor((xb + HOPE_QPI) / dx), jc = (int)floor((yb + HOPE_QPI) / dx);
        ic = ic < 0 ? 0 : (ic > N - 1 ? N - 1 : ic);
        jc = jc < 0 ? 0 : (jc > N - 1 ? N - 1 : jc);
        double xi = (xb - (-HOPE_QPI + (ic + 0.5) * dx)) / dx;
        double eta = (yb - (-HOPE_QPI + (jc + 0.5) * dx)) / dx;
        double wx[HOPE_MAXK], wy[HOPE_MAXK], ratio, C[4];
        cell_avg_weights(K, -H, xi, wx);
        cell_avg_weights(K, -H, eta, wy);
        panel_conversion(p, X, Y, B, XB, YB, &ratio, C);
        double W = weights[g] * weights[h] / nown;
        for (int b = 0; b < K; ++b)
          for (int a = 0; a < K; ++a) {
            int ci = ic + a - H, cj = jc + b - H;
            double wt = W * wx[a] * wy[b];
            LocalEnt le;
            if (ci >= 0 && ci < N && cj >= 0 && cj < N) {
              le.ghost = false;
              le.idx = (B * N + cj) * N + ci;
            } else {
              le.ghost = true;
              le.idx = rowid[((size_t)B * ne + (cj + H)) * ne + (ci + H)];
            }
            le.m = wt * ratio;
            for (int t = 0; t < 4; ++t) le.c[t] = wt * C[t];
            bool merged = false;
            for (auto &e : acc)
              if (e.ghost == le.ghost && e.idx == le.idx) {
                e.m += le.m;
                for (int t = 0; t < 4; ++t) e.c[t] += le.c[t];
                merged = true;
                break;
              }
            if (!merged) acc.push_back(le);
          }
        }
      }
    loc[r] = std::move(acc);
  }
  if (bad) {
    set_error("ghost operator: a ghost Gauss point maps back onto its own panel");
    return HOPE_EINVAL;
  }
  // sweeps
  const int ncell = 6 * N * N;
  std::vector<std::vector<Ent>> G(rows), Gn(rows);
  for (int it = 0; it < ctx->ghost_iters; ++it) {
#pragma omp parallel
    {
      std::vector<double> am(ncell, 0.0), ac((size_t)4 * ncell, 0.0);
      std::vector<int> mark(ncell, 0), touched;
      touched.reserve(4096);
#pragma omp for schedule(dynamic, 8)
      for (int r = 0; r < rows; ++r) {
        touched.clear();
        auto add = [&](int col, double m, const double *c) {
          if (!mark[col]) {
            mark[col] = 1;
            touched.push_back(col);
          }
          am[col] += m;
          for (int t = 0; t < 4; ++t) ac[(size_t)4 * col + t] += c[t];
        };
        for (const auto &e : loc[r]) {
          if (!e.ghost) {
            add(e.idx, e.m, e.c);
          } else {
            for (const auto &s : G[e.idx]) {
              double c[4] = {e.c[0] * s.c[0] + e.c[1] * s.c[2], e.c[0] * s.c[1] + e.c[1] * s.c[3],
                             e.c[2] * s.c[0] + e.c[3] * s.c[2], e.c[2] * s.c[1] + e.c[3] * s.c[3]};
              add(s.col, e.m * s.m, c);
            }
          }
        }
        std::sort(touched.begin(), touched.end());
        std::vector<Ent> out;
        out.reserve(touched.size());
        for (int col : touched) {
          Ent en;
          en.col = col;
          en.m = am[col];
          for (int t = 0; t < 4; ++t) en.c[t] = ac[(size_t)4 * col + t];
          bool nz = en.m != 0.0 || en.c[0] != 0.0 || en.c[1] != 0.0 || en.c[2] != 0.0 || en.c[3] != 0.0;
          if (nz) out.push_back(en);
          am[col] = 0.0;
          for (int t = 0; t < 4; ++t) ac[(size_t)4 * col + t] = 0.0;
          mark[col] = 0;
        }
        Gn[r] = std::move(out);
      }
    }
    std::swap(G, Gn);
  }
  // Cube symmetry: every row as the rotated copy of its panel-0 representative (rows on
  // panel 0 with ii < H, jj < ne - H; one per orbit of the 24 rotations), in the
  // representative's entry order, so equivalent rows share one set of weights.
  std::vector<int> rep(rows, -1), rot(rows, -1);
  bool symmetric = sym != nullptr;
  CubeRotations cr;
  if (symmetric) {
    cube_rotations(cr);
    std::vector<int> rowid((size_t)6 * ne * ne, -1);
    for (int r = 0; r < rows; ++r) rowid[dst[r]] = r;
    for (int jj = 0; jj < ne - H && symmetric; ++jj)
      for (int ii = 0; ii < H && symmetric; ++ii) {
        const int r0 = rowid[(size_t)jj * ne + ii];
        if (r0 < 0) { symmetric = false; break; }
        for (int t = 0; t < 24; ++t) {
          int p2, i2, j2;
          rot_index(cr, t, 0, ii, jj, ne, &p2, &i2, &j2);
          const int r = rowid[((size_t)p2 * ne + j2) * ne + i2];
          if (r < 0 || rep[r] >= 0) { symmetric = false; break; }
          rep[r] = r0;
          rot[r] = t;
        }
      }
    for (int r = 0; r < rows && symmetric; ++r)
      if (rep[r] < 0) symmetric = false;
  }
  if (symmetric) {
    std::vector<std::vector<Ent>> S(rows);
    double worst = 0.0;
#pragma omp parallel for schedule(dynamic, 8) reduction(max : worst)
    for (int r = 0; r < rows; ++r) {
      const int t = rot[r];
      const int *Ap = cr.A[t][0];
      const double Mp[4] = {(double)Ap[0], (double)Ap[2], (double)Ap[1], (double)Ap[3]};  // [[a, c], [b, d]]
      std::vector<Ent> &out = S[r];
      out.reserve(G[rep[r]].size());
      double mx = 0.0, dev = 0.0;
      for (const auto &e : G[r]) {
        mx = fmax(mx, fabs(e.m));
        for (int u = 0; u < 4; ++u) mx = fmax(mx, fabs(e.c[u]));
      }
      for (const auto &e : G[rep[r]]) {
        const int q = e.col / (N * N), rem = e.col % (N * N);
        int q2, i2, j2;
        rot_index(cr, t, q, rem % N, rem / N, N, &q2, &i2, &j2);
        const int *Aq = cr.A[t][q];
        const double Mq[4] = {(double)Aq[0], (double)Aq[2], (double)Aq[1], (double)Aq[3]};
        // C' = Mp C Mq^T (signed permutations: exact)
        const double T0 = e.c[0] * Mq[0] + e.c[1] * Mq[1], T1 = e.c[0] * Mq[2] + e.c[1] * Mq[3];
        const double T2 = e.c[2] * Mq[0] + e.c[3] * Mq[1], T3 = e.c[2] * Mq[2] + e.c[3] * Mq[3];
        Ent n;
        n.col = (q2 * N + j2) * N + i2;
        n.m = e.m;
        n.c[0] = Mp[0] * T0 + Mp[1] * T2;
        n.c[1] = Mp[0] * T1 + Mp[1] * T3;
        n.c[2] = Mp[2] * T0 + Mp[3] * T2;
        n.c[3] = Mp[2] * T1 + Mp[3] * T3;
        out.push_back(n);
      }
      // deviation from the directly composed row (entries matched by column)
      std::vector<Ent> a = G[r], b = out;
      auto bycol = [](const Ent &x, const Ent &y) { return x.col < y.col; };
      std::sort(a.begin(), a.end(), bycol);
      std::sort(b.begin(), b.end(), bycol);
      size_t ia = 0, ib = 0;
      while (ia < a.size() || ib < b.size()) {
        const Ent *x = ia < a.size() ? &a[ia] : nullptr, *y = ib < b.size() ? &b[ib] : nullptr;
        double d = 0.0;
        if (x && y && x->col == y->col) {
          d = fabs(x->m - y->m);
          for (int u = 0; u < 4; ++u) d = fmax(d, fabs(x->c[u] - y->c[u]));
          ++ia;
          ++ib;
        } else if (x && (!y || x->col < y->col)) {
          d = fmax(fabs(x->m), fmax(fmax(fabs(x->c[0]), fabs(x->c[1])), fmax(fabs(x->c[2]), fabs(x->c[3]))));
          ++ia;
        } else {
          d = fmax(fabs(y->m), fmax(fmax(fabs(y->c[0]), fabs(y->c[1])), fmax(fabs(y->c[2]), fabs(y->c[3]))));
          ++ib;
        }
        dev = fmax(dev, d);
      }
      worst = fmax(worst, mx > 0.0 ? dev / mx : dev);
    }
    sym->max_dev = worst;
    if (worst < 1e-12) G = std::move(S);
    else symmetric = false;
  }
  // Drop the negligible tail of every row: entries whose largest weight is below
  // drop_rel times the row's largest weight (contributions of deep sweeps, which decay
  // geometrically).  The dropped weights sum to well under the precision's rounding
  // unit relative to the row (FP64: 1e-17, FP32: 1e-9 relative cut-off).
  const double drop_rel = ctx->prec == HOPE_FP64 ? 1e-17 : 1e-9;
#pragma omp parallel for schedule(dynamic, 8)
  for (int r = 0; r < rows; ++r) {
    double mx = 0.0;
    auto emax = [](const Ent &e) {
      double m = fabs(e.m);
      for (int t = 0; t < 4; ++t) m = fmax(m, fabs(e.c[t]));
      return m;
    };
    for (const auto &e : G[r]) mx = fmax(mx, emax(e));
    std::vector<Ent> kept;
    kept.reserve(G[r].size());
    for (const auto &e : G[r])
      if (emax(e) >= drop_rel * mx) kept.push_back(e);
    G[r] = std::move(kept);
  }
  rowptr.assign(rows + 1, 0);
  for (int r = 0; r < rows; ++r) rowptr[r + 1] = rowptr[r] + (int)G[r].size();
  // input transform code of entry k of row r (0 without symmetry)
  auto ecode = [&](int r, int k) -> int {
    if (!symmetric) return 0;
    return code_in(cr.A[rot[r]][G[rep[r]][k].col / (N * N)]);
  };
  if (split) {
    // Head/tail split for FP64 contexts: entries whose largest weight is at least
    // split_rel of the row's largest stay in FP64; the rest (at most ~2e-8 of a row's
    // weight) are evaluated in FP32, whose rounding then contributes ~1e-15 relative.
    const double split_rel = 1e-9;
    split->head_ptr.assign(rows + 1, 0);
    split->tail_ptr.assign(rows + 1, 0);
    split->head_col.clear();
    split->tail_col.clear();
    split->head_val.clear();
    split->tail_val.clear();
    for (int r = 0; r < rows; ++r) {
      double mx = 0.0;
      for (const auto &e : G[r]) {
        double m = fabs(e.m);
        for (int t = 0; t < 4; ++t) m = fmax(m, fabs(e.c[t]));
        mx = fmax(mx, m);
      }
      for (size_t k = 0; k < G[r].size(); ++k) {
        const Ent &e = G[r][k];
        double m = fabs(e.m);
        for (int t = 0; t < 4; ++t) m = fmax(m, fabs(e.c[t]));
        if (m >= split_rel * mx) {
          split->head_col.push_back(e.col | (ecode(r, (int)k) << 28));
          split->head_val.push_back(e.m);
          for (int t = 0; t < 4; ++t) split->head_val.push_back(e.c[t]);
        } else {
          split->tail_col.push_back(e.col | (ecode(r, (int)k) << 28));
          split->tail_val.push_back((float)e.m);
          for (int t = 0; t < 4; ++t) split->tail_val.push_back((float)e.c[t]);
        }
      }
      split->head_ptr[r + 1] = (int)split->head_col.size();
      split->tail_ptr[r + 1] = (int)split->tail_col.size();
    }
  }
  if (sym) {
    sym->symmetric = symmetric;
    sym->finfo.assign(rows, 0);
    sym->ccode.assign(rowptr[rows], 0);
    for (int r = 0; r < rows; ++r) {
      if (!symmetric) {
        sym->finfo[r] = r;
        continue;
      }
      sym->finfo[r] = rep[r] | (code_out(cr.A[rot[r]][0]) << 28);
      for (int e = rowptr[r], k = 0; e < rowptr[r + 1]; ++e, ++k) sym->ccode[e] = ecode(r, k);
    }
  }
  cols.resize(rowptr[rows]);
  vals.resize((size_t)5 * rowptr[rows]);
  for (int r = 0; r < rows; ++r) {
    int o = rowptr[r];
    for (size_t t = 0; t < G[r].size(); ++t) {
      cols[o + t] = G[r][t].col;
      vals[(size_t)5 * (o + t)] = G[r][t].m;
      for (int u = 0; u < 4; ++u) vals[(size_t)5 * (o + t) + 1 + u] = G[r][t].c[u];
    }
  }
  return HOPE_OK;
}

// -------------------------------------------------------------------------------
// Cube-edge topology and per-point conversions for the panel-boundary fluxes.
// -------------------------------------------------------------------------------
static void edge_coords(int N, int side, int t, double node, double *x, double *y) {
  double dx = HOPE_PI / (2.0 * N);
  double along = -HOPE_QPI + (t + 0.5 + node) * dx;
  switch (side) {
    case 0: *x = -HOPE_QPI; *y = along; break;
    case 1: *x = HOPE_QPI; *y = along; break;
    case 2: *x = along; *y = -HOPE_QPI; break;
    default: *x = along; *y = HOPE_QPI; break;
  }
}

int build_cube_edges(const hope_ctx *ctx, int N, const std::vector<double> &nodes, CubeEdge edges[12],
                     std::vector<double> &conv) {
  const int me = ctx->me;
  const double dx = HOPE_PI / (2.0 * N);
  int ne = 0;
  conv.assign((size_t)12 * N * me * 9, 0.0);
  for (int A = 0; A < 6; ++A)
    for (int sA = 0; sA < 4; ++sA) {
      int B = -1, sB = -1, flip = -1;
      for (int t = 0; t < N; ++t)
        for (int g = 0; g < me; ++g) {
          double x, y, P[3], XB, YB;
          edge_coords(N, sA, t, nodes[g], &x, &y);
          double XA = tan(x), YA = tan(y);
          panel_point(A, XA, YA, P);
          int b = face_of(P, A);
          panel_coords(b, P, &XB, &YB);
          double xb = atan(XB), yb = atan(YB), along;
          int s;
          if (fabs(xb) > fabs(yb)) {
            s = xb < 0 ? 0 : 1;
            along = yb;
          } else {
            s = yb < 0 ? 2 : 3;
            along = xb;
          }
          int tb = (int)floor((along + HOPE_QPI) / dx);
          tb = tb < 0 ? 0 : (tb > N - 1 ? N - 1 : tb);
          double eta = (along - (-HOPE_QPI + (tb + 0.5) * dx)) / dx;
          int gb = 0;
          for (int u = 1; u < me; ++u)
            if (fabs(nodes[u] - eta) < fabs(nodes[gb] - eta)) gb = u;
          if (fabs(nodes[gb] - eta) > 1e-8) {
            set_error("cube edges: edge Gauss points do not coincide across panels");
            return HOPE_EINVAL;
          }
          if (t == 0 && g == 0) {
            B = b;
            sB = s;
            flip = (tb == 0 && gb == 0) ? 0 : ((tb == N - 1 && gb == me - 1) ? 1 : -1);
          }
          const int tb_exp = flip ? N - 1 - t : t, gb_exp = flip ? me - 1 - g : g;
          if (b != B || s != sB || flip < 0 || tb != tb_exp || gb != gb_exp) {
            set_error("cube edges: inconsistent neighbour along a panel side");
            return HOPE_EINVAL;
          }
          if (A < B) {
            double ratio, C[4], r2, Ci[4];
            panel_conversion(A, XA, YA, B, XB, YB, &ratio, C);
            panel_conversion(B, XB, YB, A, XA, YA, &r2, Ci);
            double *o = &conv[(((size_t)ne * N + t) * me + g) * 9];
            o[0] = ratio;
            for (int u = 0; u < 4; ++u) {
              o[1 + u] = C[u];
              o[5 + u] = Ci[u];
            }
          }
        }
      if (A < B) {
        if (ne >= 12) {
          set_error("cube edges: more than 12 edges");
          return HOPE_EINVAL;
        }
        edges[ne++] = CubeEdge{A, sA, B, sB, flip};
      }
    }
  if (ne != 12) {
    set_error("cube edges: expected 12 edges");
    return HOPE_EINVAL;
  }
  return HOPE_OK;
}

}  // namespace hope

namespace hope {
// WENO2D tables (section 3.2), FP64 on the host, stored in the context precision:
//   wsub [me+2][l][l]  1-D sub-stencil weights at xi = -1/2, +1/2, g_0..g_{me-1}
//   gpm  [npoc][2][s]  gamma+ and gamma- of eq. 3.20 (theta = 3) at every point, gamma the
//                      tensor product of the 1-D least-squares weights (eq. 3.19)
//   sig  [npoc][2]     sigma+- = sum of gamma+-
//   bform [l][l*l + l] per sub-stencil offset: Winv (l x l) of the simultaneous
//                      diagonalisation of the smoothness forms (eq. 3.25), its row sums
//   bcoef [l][l][l][l] mode weights lam_y lam_x - 1 of the indicator
// Static tables of a bottom surface (eqs. 2.13-2.14) from the cell averages of sqrtG phi_s,
// all in FP64: the surface's ghost ring by the composed ghost operator (eq. 7.12), its TPP
// values at the edge points, sep[4][me][6][N][N] (west, east at the y-nodes; south, north
// at the x-nodes), and psi_B's cell average (the me x me Gauss rule of eq. 2.14 at the
// cell points) as an affine map of the k x k depth stencil, weights tw[2][k*k][6][N][N]
// and constants tb[2][6][N][N].  The gradient of phi_t = (P_depth + P_s)/sqrtG uses the
// derivative weights of the TPP polynomials and the closed-form gradient of sqrtG.
int build_topography_tables(const hope_ctx *ctx, int N, const double *phis_avg_host, std::vector<double> &sep,
                            std::vector<double> &tw, std::vector<double> &tb, std::vector<double> *sext,
                            std::vector<double> *scp) {
  const int K = ctx->k, H = ctx->H, ME = ctx->me, KK = K * K, ne = N + 2 * H;
  const size_t pn = (size_t)6 * N * N;
  std::vector<double> nodes(ME), weights(ME);
  gauss_legendre(ME, nodes.data(), weights.data());
  std::vector<int> rowptr, cols, dst;
  std::vector<double> vals;
  int rc = build_ghost_operator(ctx, N, nodes, weights, rowptr, cols, vals, dst);
  if (rc) return rc;
  // extended array of sqrtG phi_s: interior cells and the ghost ring
  std::vector<double> ext((size_t)6 * ne * ne, 0.0);
  for (int p = 0; p < 6; ++p)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i)
        ext[((size_t)p * ne + j + H) * ne + i + H] = phis_avg_host[((size_t)p * N + j) * N + i];
  for (size_t r = 0; r + 1 < rowptr.size(); ++r) {
    double v = 0.0;
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) v += vals[(size_t)5 * e] * phis_avg_host[cols[e]];
    ext[dst[r]] = v;
  }
  // 1-D weights: values at xi = -1/2, +1/2 and the Gauss nodes; derivatives at the nodes
  std::vector<double> wv((size_t)(ME + 2) * K), wd((size_t)ME * K);
  cell_avg_weights(K, -H, -0.5, &wv[0]);
  cell_avg_weights(K, -H, 0.5, &wv[K]);
  for (int t = 0; t < ME; ++t) {
    cell_avg_weights(K, -H, nodes[t], &wv[(size_t)(2 + t) * K]);
    cell_avg_dweights(K, -H, nodes[t], &wd[(size_t)t * K]);
  }
  const double dx = HOPE_PI / (2.0 * N), r2 = ctx->radius * ctx->radius;
  sep.assign((size_t)4 * ME * pn, 0.0);
  tw.assign((size_t)2 * KK * pn, 0.0);
  tb.assign(2 * pn, 0.0);
  if (sext) *sext = ext;
  if (scp) scp->assign((size_t)ME * ME * pn, 0.0);
  // every cell writes only its own entries, so the panel rows run in parallel
#pragma omp parallel for schedule(dynamic, 4)
  for (int pj = 0; pj < 6 * N; ++pj) {
    const int p = pj / N, j = pj % N;
    std::vector<double> st(KK);
    for (int i = 0; i < N; ++i) {
        const size_t cell = ((size_t)p * N + j) * N + i;
        for (int b = 0; b < K; ++b)
          for (int a = 0; a < K; ++a) st[b * K + a] = ext[((size_t)p * ne + j + b) * ne + i + a];
        auto tpp = [&](const double *wx, const double *wy) {
          double v = 0.0;
          for (int b = 0; b < K; ++b) {
            double row = 0.0;
            for (int a = 0; a < K; ++a) row += wx[a] * st[b * K + a];
            v += wy[b] * row;
          }
          return v;
        };
        for (int r = 0; r < ME; ++r) {
          const double *wn = &wv[(size_t)(2 + r) * K];
          sep[((size_t)0 * ME + r) * pn + cell] = tpp(&wv[0], wn);  // west
          sep[((size_t)1 * ME + r) * pn + cell] = tpp(&wv[K], wn);  // east
          sep[((size_t)2 * ME + r) * pn + cell] = tpp(wn, &wv[0]);  // south
          sep[((size_t)3 * ME + r) * pn + cell] = tpp(wn, &wv[K]);  // north
        }
        for (int h = 0; h < ME; ++h)
          for (int gg = 0; gg < ME; ++gg) {
            const double X = tan(-HOPE_QPI + (i + 0.5 + nodes[gg]) * dx);
            const double Y = tan(-HOPE_QPI + (j + 0.5 + nodes[h]) * dx);
            const double sG = sqrtg_unit(X, Y), d2 = 1.0 + X * X + Y * Y;
            double gx, gy;
            sqrtg_unit_grad(X, Y, &gx, &gy);
            const double G11 = d2 / (1.0 + X * X), G22 = d2 / (1.0 + Y * Y);
            const double G12 = d2 * X * Y / ((1.0 + X * X) * (1.0 + Y * Y));
            const double *vx = &wv[(size_t)(2 + gg) * K], *vy = &wv[(size_t)(2 + h) * K];
            const double *dxw = &wd[(size_t)gg * K], *dyw = &wd[(size_t)h * K];
            const double Ps = tpp(vx, vy);
            if (scp) (*scp)[((size_t)h * ME + gg) * pn + cell] = Ps;
            const double fs = Ps / sG;  // phi_s at the point
            const double dsx = (tpp(dxw, vy) / dx - fs * gx) / sG, dsy = (tpp(vx, dyw) / dx - fs * gy) / sG;
            // quadrature weight times sqrtG phi_s G^ij (true metric) of eq. 2.14
            const double W = weights[gg] * weights[h] * Ps / r2;
            const double A11 = W * G11, A12 = W * G12, A22 = W * G22;
            tb[cell] += A11 * dsx + A12 * dsy;
            tb[pn + cell] += A12 * dsx + A22 * dsy;
            for (int b = 0; b < K; ++b)
              for (int a = 0; a < K; ++a) {
                const double R = vy[b] * vx[a], Rx = vy[b] * dxw[a] / dx, Ry = dyw[b] * vx[a] / dx;
                const double ex = (Rx - R * gx / sG) / sG, ey = (Ry - R * gy / sG) / sG;
                const size_t c = (size_t)b * K + a;
                tw[c * pn + cell] += A11 * ex + A12 * ey;
                tw[((size_t)KK + c) * pn + cell] += A12 * ex + A22 * ey;
              }
          }
      }
  }
  return HOPE_OK;
}

static int upload_t(hope_ctx *ctx, void **dst, const std::vector<double> &v) {
  size_t bytes = (size_t)ctx->esize * v.size();
  if (cudaMalloc(dst, bytes) != cudaSuccess) return HOPE_ENOMEM;
  cudaError_t e;
  if (ctx->esize == 8) {
    e = cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice);
  } else {
    std::vector<float> f(v.begin(), v.end());
    e = cudaMemcpy(*dst, f.data(), bytes, cudaMemcpyHostToDevice);
  }
  return e == cudaSuccess ? HOPE_OK : HOPE_ECUDA;
}

int setup_weno_tables(hope_ctx *ctx, const std::vector<double> &nodes) {
  const int K = ctx->k, H = ctx->H, me = ctx->me, l = (K + 1) / 2, S = l * l, np = ctx->npoc;
  std::vector<double> pos(me + 2);
  pos[0] = -0.5;
  pos[1] = 0.5;
  for (int g = 0; g < me; ++g) pos[2 + g] = nodes[g];
  std::vector<double> wsub((size_t)(me + 2) * l * l), g1((size_t)(me + 2) * l);
  for (int t = 0; t < me + 2; ++t) {
    for (int sb = 0; sb < l; ++sb) cell_avg_weights(l, sb - H, pos[t], &wsub[((size_t)t * l + sb) * l]);
    double res = weno_linear_weights_1d(K, pos[t], &g1[(size_t)t * l]);
    if (res > 1e-10) {
      set_error("WENO linear weights: least-squares residual too large");
      return HOPE_EINVAL;
    }
  }
  std::vector<double> gpm((size_t)np * 2 * S), sig((size_t)np * 2);
  auto ptpos = [me](int pt, int *tx, int *ty) {
    if (pt < me) { *tx = 0; *ty = 2 + pt; }
    else if (pt < 2 * me) { *tx = 1; *ty = 2 + pt - me; }
    else if (pt < 3 * me) { *tx = 2 + pt - 2 * me; *ty = 0; }
    else if (pt < 4 * me) { *tx = 2 + pt - 3 * me; *ty = 1; }
    else { int c = pt - 4 * me; *tx = 2 + c % me; *ty = 2 + c / me; }
  };
  for (int pt = 0; pt < np; ++pt) {
    int tx, ty;
    ptpos(pt, &tx, &ty);
    double sp = 0.0, sm = 0.0;
    for (int sy = 0; sy < l; ++sy)
      for (int sx = 0; sx < l; ++sx) {
        double gm = g1[(size_t)tx * l + sx] * g1[(size_t)ty * l + sy];
        double gpl = 0.5 * (3.0 * fabs(gm) + gm), gmi = 0.5 * (3.0 * fabs(gm) - gm);
        gpm[((size_t)pt * 2 + 0) * S + sy * l + sx] = gpl;
        gpm[((size_t)pt * 2 + 1) * S + sy * l + sx] = gmi;
        sp += gpl;
        sm += gmi;
      }
    sig[(size_t)pt * 2] = sp;
    sig[(size_t)pt * 2 + 1] = sm;
  }
  // bform per sub-stencil offset: Winv (l x l) and its row sums (l); the indicator uses
  // Q minus the cell's own value (beta is blind to constants), whose transform is
  // Winv Q - q_c * rowsum.  bcoef[sy][k][sx][k'] = lam_y,k lam_x,k' - 1, set to exactly 0
  // for the constant mode (|.| < 1e-12) and clamped at 0, so beta >= 0 in any precision.
  std::vector<double> bf((size_t)l * (l * l + l)), lam((size_t)l * l);
  for (int sb = 0; sb < l; ++sb) {
    double Sm[HOPE_MAXME * HOPE_MAXME], B0[HOPE_MAXME * HOPE_MAXME];
    weno_beta_forms_1d(l, sb - H, Sm, B0);
    double *W = &bf[(size_t)sb * (l * l + l)];
    if (weno_beta_diag(l, Sm, B0, W, &lam[(size_t)sb * l])) {
      set_error("WENO smoothness forms: Cholesky failed");
      return HOPE_EINVAL;
    }
    for (int k = 0; k < l; ++k) {
      double rs = 0.0;
      for (int a = 0; a < l; ++a) rs += W[k * l + a];
      W[l * l + k] = rs;
    }
  }
  std::vector<double> bcoef((size_t)l * l * l * l);
  for (int sy = 0; sy < l; ++sy)
    for (int k = 0; k < l; ++k)
      for (int sx = 0; sx < l; ++sx)
        for (int kp = 0; kp < l; ++kp) {
          double c = lam[(size_t)sy * l + k] * lam[(size_t)sx * l + kp] - 1.0;
          if (c < 1e-12) c = 0.0;
          bcoef[(((size_t)sy * l + k) * l + sx) * l + kp] = c;
        }
  int rc;
  if (ctx->scheme == HOPE_WENO1D) {
    // 1-D tables of the dimension-by-dimension comparator: split 1-D linear weights per
    // position, and per sub-stencil the Jiang-Shu indicator form S - B0 (derivative orders
    // 1..l-1) as eigenpairs, its constant mode's eigenvalue set to 0 and negatives clamped
    std::vector<double> w1gpm((size_t)(me + 2) * 2 * l), w1sig((size_t)(me + 2) * 2);
    for (int t = 0; t < me + 2; ++t) {
      double sp = 0.0, sm = 0.0;
      for (int sb = 0; sb < l; ++sb) {
        const double gm = g1[(size_t)t * l + sb];
        const double gpl = 0.5 * (3.0 * fabs(gm) + gm), gmi = 0.5 * (3.0 * fabs(gm) - gm);
        w1gpm[((size_t)t * 2 + 0) * l + sb] = gpl;
        w1gpm[((size_t)t * 2 + 1) * l + sb] = gmi;
        sp += gpl;
        sm += gmi;
      }
      w1sig[(size_t)t * 2] = sp;
      w1sig[(size_t)t * 2 + 1] = sm;
    }
    std::vector<double> w1bf((size_t)l * (l * l + l));
    for (int sb = 0; sb < l; ++sb) {
      double Sm[HOPE_MAXME * HOPE_MAXME], B0[HOPE_MAXME * HOPE_MAXME], I[HOPE_MAXME * HOPE_MAXME];
      weno_beta_forms_1d(l, sb - H, Sm, B0);
      double mx = 0.0;
      for (int a = 0; a < l * l; ++a) {
        Sm[a] -= B0[a];
        I[a] = (a % (l + 1)) == 0 ? 1.0 : 0.0;
        mx = std::max(mx, fabs(Sm[a]));
      }
      double *Wv = &w1bf[(size_t)sb * (l * l + l)];
      if (weno_beta_diag(l, Sm, I, Wv, Wv + l * l)) {
        set_error("1-D WENO smoothness forms: eigen-decomposition failed");
        return HOPE_EINVAL;
      }
      for (int k = 0; k < l; ++k)
        if (Wv[l * l + k] < 1e-12 * mx) Wv[l * l + k] = 0.0;
    }
    if ((rc = upload_t(ctx, &ctx->w1gpm, w1gpm))) return rc;
    if ((rc = upload_t(ctx, &ctx->w1sig, w1sig))) return rc;
    if ((rc = upload_t(ctx, &ctx->w1bf, w1bf))) return rc;
  }
  if ((rc = upload_t(ctx, &ctx->wsub, wsub))) return rc;
  if ((rc = upload_t(ctx, &ctx->gpm, gpm))) return rc;
  if ((rc = upload_t(ctx, &ctx->sig, sig))) return rc;
  if ((rc = upload_t(ctx, &ctx->bform, bf))) return rc;
  if ((rc = upload_t(ctx, &ctx->bcoef, bcoef))) return rc;
  return HOPE_OK;
}
}  // namespace hope
