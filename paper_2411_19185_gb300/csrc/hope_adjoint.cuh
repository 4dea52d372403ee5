// hope_adjoint.cuh -- hand-written vector-Jacobian products of one stage L(q)
// (eq. 3.1) for sm_103a.  Given lam (the adjoint of dq/dt) the kernels compute
// (dL/dq)^T lam, in reverse order of the forward stage:
//   k_flux_adj     edge quadrature (eq. 3.5) and LMARS (eqs. 3.31-3.38) adjoints, per
//                  edge, from lam of the two adjacent cells; panel-boundary edges with
//                  the transposed conversions (eqs. 3.26-3.29); writes lam at every
//                  edge point of every cell (each point has exactly one writer)
//   k_recon_*_adj  per cell: adjoint of the cell-point sources (eqs. 2.2, 2.3, 3.6),
//                  then of the reconstruction (TPP: transposed sum factorisation), giving
//                  the gradient with respect to the k x k stencil values; TPP tiles add
//                  them up on the tile's extended region in shared memory (fixed order)
//                  and write that region per tile
//   k_gather_*     per extended cell: sum of the contributions of every cell (WENO: the
//                  per-cell stencil gradients) or tile (TPP: the tiles' extended regions)
//                  whose stencils cover it (deterministic, no atomics)
//   k_ghost_adj    interior cells += G^T lam_ring (transposed ghost operator, eq. 7.12),
//                  fused with the Runge-Kutta combination of adjoint states
#pragma once
#include "hope_kernels.cuh"

namespace hope {

// LMARS flux and its vector-Jacobian product at one edge point (same arithmetic as lmars():
// interface velocity 1/2 (uL + uR) - (sR - sL), s = sqrt(phi)).
// TOPO: LMARS over bottom topography (lmars_topo), zL, zR = sqrtG phi_s at the point; the
// surface enters the interface velocity through -(phi_s,R - phi_s,L)/(2c), whose derivative
// with respect to c joins the adjoint of c, and the interface value through constants.
template <typename T, bool TOPO = false>
__device__ __forceinline__ void lmars_vjp(const T qL[3], const T qR[3], const T *m5, size_t mstr, int dir,
                                          const T lF[3], T lqL[3], T lqR[3], T zL = T(0), T zR = T(0)) {
  const T isg = m5[0], s11 = m5[mstr], is11 = m5[2 * mstr], pn = m5[3 * mstr], pc = m5[4 * mstr];
  const T qnL = dir ? qL[2] : qL[1], qnR = dir ? qR[2] : qR[1];
  const T phL = qL[0] * isg, phR = qR[0] * isg;
  const T rLR = rcp(qL[0] * qR[0]);
  const T rL = qR[0] * rLR, rR = qL[0] * rLR;
  const T uL = qnL * rL * is11, uR = qnR * rR * is11;
  const T sL = sqrt_pos(phL), sR = sqrt_pos(phR);
  const T c = T(0.5) * (sL + sR);
  T ms = T(0.5) * (uL + uR) - (sR - sL);
  T ph = T(0.5) * (phL + phR - c * (uR - uL));
  T dfs = T(0);  // phi_s,R - phi_s,L
  if constexpr (TOPO) {
    const T fsL = zL * isg, fsR = zR * isg;
    dfs = fsR - fsL;
    ms = T(0.5) * (uL + uR) - (sR - sL) - dfs * rcp(c + c);
    ph = T(0.5) * ((phL + fsL) + (phR + fsR) - c * (uR - uL));
  }
  const T m = ms * s11;
  const T am = fabs(m);
  const T sg = m > T(0) ? T(1) : (m < T(0) ? T(-1) : T(0));
  // F_v = 1/2 (m (qL + qR) - |m| (qR - qL)) + P_v,  P_1 = a1 ph^2, P_2 = a2 ph^2
  T lm = 0;
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    lqL[v] = T(0.5) * (m + am) * lF[v];
    lqR[v] = T(0.5) * (m - am) * lF[v];
    lm += T(0.5) * ((qL[v] + qR[v]) - sg * (qR[v] - qL[v])) * lF[v];
  }
  const T a1 = dir ? pc : pn, a2 = dir ? pn : pc;
  const T lph = T(2) * ph * (a1 * lF[1] + a2 * lF[2]);
  const T lms = lm * s11;
  T luL = T(0.5) * lms, luR = T(0.5) * lms;
  T lsL = lms, lsR = -lms;
  T lphL = T(0.5) * lph, lphR = T(0.5) * lph;
  T lc = -T(0.5) * (uR - uL) * lph;
  if constexpr (TOPO) lc += lms * dfs * rcp(T(2) * c * c);  // d/dc of -dfs / (2c)
  luR -= T(0.5) * c * lph;
  luL += T(0.5) * c * lph;
  lsL += T(0.5) * lc;
  lsR += T(0.5) * lc;
  lphL += lsL / (T(2) * sL);
  lphR += lsR / (T(2) * sR);
  const T dL = rL * is11 * luL, dR = rR * is11 * luR;
  lqL[1] += dir ? T(0) : dL;
  lqL[2] += dir ? dL : T(0);
  lqR[1] += dir ? T(0) : dR;
  lqR[2] += dir ? dR : T(0);
  lqL[0] += -rL * (qnL * rL * is11 * luL) + isg * lphL;
  lqR[0] += -rR * (qnR * rR * is11 * luR) + isg * lphR;
}

// ---------------------------------------------------------------------------------
// Flux adjoint.  lamL: adjoint of the tendency [3][6][N][N]; lep: [4][3][me][6][N][N].
// ---------------------------------------------------------------------------------
// One edge item (interior x-edges, interior y-edges, then the 12 cube edges x N cells).
// TOPO: over a surface, sep[4][me][6][N][N] = sqrtG phi_s at the edge points.
template <typename T, int ME, bool TOPO = false>
__device__ __forceinline__ void flux_adj_item(int idx, const T *__restrict__ ep, const T *__restrict__ mx,
                                              const T *__restrict__ gwg, const int *__restrict__ bedge,
                                              const T *__restrict__ bconv, const T *__restrict__ lamL,
                                              T *__restrict__ lep, int N, T inv_dx,
                                              const T *__restrict__ sep = nullptr) {
  // 32-bit item arithmetic: 12 N (N + 1) < 2^31 for N <= 8192
  const int nx = 6 * N * (N - 1), ny = nx;
  const size_t pn = (size_t)6 * N * N;
  const size_t mstr = metric_plane(N, ME);
  T gw[ME];
#pragma unroll
  for (int g = 0; g < ME; ++g) gw[g] = gwg[g];
  if (idx < nx + ny) {
    const int dir = idx < nx ? 0 : 1;
    const unsigned r = (unsigned)(dir ? idx - nx : idx);
    int p, a, e;
    if (dir == 0) {
      const unsigned t = r / (unsigned)(N - 1);
      e = 1 + (int)(r - t * (unsigned)(N - 1));
      p = (int)(t / (unsigned)N);
      a = (int)(t - (unsigned)p * N);
    } else {
      const unsigned t = r / (unsigned)N;
      a = (int)(r - t * (unsigned)N);
      p = (int)(t / (unsigned)(N - 1));
      e = 1 + (int)(t - (unsigned)p * (N - 1));
    }
    size_t cl, cr;
    if (dir == 0) {
      cl = ((size_t)p * N + a) * N + (e - 1);
      cr = cl + 1;
    } else {
      cl = ((size_t)p * N + (e - 1)) * N + a;
      cr = cl + N;
    }
    const int sl = dir ? 3 : 1, sr = dir ? 2 : 0;
    T lFbar[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) lFbar[v] = (lamL[v * pn + cr] - lamL[v * pn + cl]) * inv_dx;
#pragma unroll
    for (int g = 0; g < ME; ++g) {
      T qL[3], qR[3], lF[3], lqL[3], lqR[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        qL[v] = ep[((size_t)(sl * 3 + v) * ME + g) * pn + cl];
        qR[v] = ep[((size_t)(sr * 3 + v) * ME + g) * pn + cr];
        lF[v] = gw[g] * lFbar[v];
      }
      const T *m5 = mx + (dir ? metric_y(N, ME, e, a, g) : metric_x(N, e, a, g));
      if constexpr (TOPO)
        lmars_vjp<T, true>(qL, qR, m5, mstr, dir, lF, lqL, lqR, sep[((size_t)sl * ME + g) * pn + cl],
                           sep[((size_t)sr * ME + g) * pn + cr]);
      else
        lmars_vjp(qL, qR, m5, mstr, dir, lF, lqL, lqR);
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        lep[((size_t)(sl * 3 + v) * ME + g) * pn + cl] = lqL[v];
        lep[((size_t)(sr * 3 + v) * ME + g) * pn + cr] = lqR[v];
      }
    }
    return;
  }
  const int r = idx - nx - ny;
  const int ce = r / N, t = r - ce * N;
  const int A = bedge[ce * 5 + 0], sA = bedge[ce * 5 + 1], B = bedge[ce * 5 + 2], sB = bedge[ce * 5 + 3],
            flip = bedge[ce * 5 + 4];
  const int tB = flip ? N - 1 - t : t;
  auto side_cell = [N](int P, int side, int tt) -> size_t {
    int ci = side == 0 ? 0 : (side == 1 ? N - 1 : tt);
    int cj = side == 2 ? 0 : (side == 3 ? N - 1 : tt);
    return ((size_t)P * N + cj) * N + ci;
  };
  const size_t cA = side_cell(A, sA, t), cB = side_cell(B, sB, tB);
  const int dirA = sA >> 1;
  const T sgA = (sA & 1) ? T(1) : T(-1), sgB = (sB & 1) ? T(1) : T(-1);
  const T sg = -sgA * sgB;
  const int eA = (sA & 1) ? N : 0;
  // d L(cell) / d Fbar(edge) = -1/dx on the cell's east/north edge, +1/dx on west/south
  T lFA[3], lFB[3];
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    lFA[v] = -sgA * lamL[v * pn + cA] * inv_dx;
    lFB[v] = -sgB * lamL[v * pn + cB] * inv_dx;
  }
#pragma unroll
  for (int g = 0; g < ME; ++g) {
    const int gB = flip ? ME - 1 - g : g;
    const T *cv = bconv + (((size_t)ce * N + t) * ME + g) * 9;
    T qin[3], qb[3], qo[3], lF[3], l1[3], l2[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      qin[v] = ep[((size_t)(sA * 3 + v) * ME + g) * pn + cA];
      qb[v] = ep[((size_t)(sB * 3 + v) * ME + gB) * pn + cB];
    }
    qo[0] = cv[0] * qb[0];
    qo[1] = cv[1] * qb[1] + cv[2] * qb[2];
    qo[2] = cv[3] * qb[1] + cv[4] * qb[2];
    // Fbar_A = sum_g w_g F_g; Fbar_B,0 = sg Fbar_A,0; Fbar_B,mom = sum_g w_gB sg C_AB F_g,mom
    lF[0] = gw[g] * (lFA[0] + sg * lFB[0]);
    lF[1] = gw[g] * lFA[1] + gw[gB] * sg * (cv[5] * lFB[1] + cv[7] * lFB[2]);
    lF[2] = gw[g] * lFA[2] + gw[gB] * sg * (cv[6] * lFB[1] + cv[8] * lFB[2]);
    const T *m5 = mx + metric_y(N, ME, eA, t, g);
    T lin[3], lo[3];
    T zin = T(0), zo = T(0);
    if constexpr (TOPO) {
      zin = sep[((size_t)sA * ME + g) * pn + cA];
      zo = cv[0] * sep[((size_t)sB * ME + gB) * pn + cB];
    }
    if (sA & 1) {
      lmars_vjp<T, TOPO>(qin, qo, m5, mstr, dirA, lF, l1, l2, zin, zo);
#pragma unroll
      for (int v = 0; v < 3; ++v) { lin[v] = l1[v]; lo[v] = l2[v]; }
    } else {
      lmars_vjp<T, TOPO>(qo, qin, m5, mstr, dirA, lF, l1, l2, zo, zin);
#pragma unroll
      for (int v = 0; v < 3; ++v) { lo[v] = l1[v]; lin[v] = l2[v]; }
    }
    T lb[3];
    lb[0] = cv[0] * lo[0];
    lb[1] = cv[1] * lo[1] + cv[3] * lo[2];
    lb[2] = cv[2] * lo[1] + cv[4] * lo[2];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      lep[((size_t)(sA * 3 + v) * ME + g) * pn + cA] = lin[v];
      lep[((size_t)(sB * 3 + v) * ME + gB) * pn + cB] = lb[v];
    }
  }
}

template <typename T, int ME, bool TOPO = false>
__global__ void __launch_bounds__(256)
    k_flux_adj(const T *__restrict__ ep, const T *__restrict__ mx, const T *__restrict__ gwg,
               const int *__restrict__ bedge, const T *__restrict__ bconv, const T *__restrict__ lamL,
               T *__restrict__ lep, int N, T inv_dx, const T *__restrict__ sep = nullptr) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 12LL * N * (N - 1) + 12LL * N) return;
  flux_adj_item<T, ME, TOPO>((int)idx, ep, mx, gwg, bedge, bconv, lamL, lep, N, inv_dx, sep);
}

// ---------------------------------------------------------------------------------
// psi_B (eq. 2.14) adjoint: the forward adds sum_c w[v][c] * stencil_c (the mass
// variable's k x k stencil) to the momentum sources (k_topo_src), so the mass variable's
// stencil gradient gains w[0][c] lam_1 + w[1][c] lam_2 at every cell (after the
// reconstruction adjoint has written it).
// ---------------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(256)
    k_topo_src_adj(const T *__restrict__ lamL, const T *__restrict__ tw, T *__restrict__ grad, int N) {
  const long long n = 6LL * N * N;
  const long long cid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cid >= n) return;
  const T l1 = lamL[n + cid], l2 = lamL[2 * n + cid];
#pragma unroll 1
  for (int c = 0; c < K * K; ++c)
    grad[(size_t)c * n + cid] += tw[(size_t)c * n + cid] * l1 + tw[((size_t)K * K + c) * n + cid] * l2;
}

// Vector-Jacobian product of the cell-point source (same arithmetic as the forward).
template <typename T>
__device__ __forceinline__ void source_vjp(const T q[3], T X, T Y, T os, T tw, T l1, T l2, T lq[3]) {
  const T rq = rcp(q[0]);
  const T XY = X * Y, X2 = X * X, Y2 = Y * Y;
  const T A1 = -XY * Y * q[1] + Y * (T(1) + Y2) * q[2];
  const T A2 = X * (T(1) + X2) * q[1] - X2 * Y * q[2];
  const T la1 = tw * l1, la2 = tw * l2;
  // a1 = A1 q1 / q0 + os (-XY q1 + (1+Y2) q2); a2 = A2 q2 / q0 + os (-(1+X2) q1 + XY q2)
  lq[0] = -(la1 * A1 * q[1] + la2 * A2 * q[2]) * rq * rq;
  lq[1] = la1 * ((-XY * Y) * q[1] * rq + A1 * rq - os * XY) + la2 * (X * (T(1) + X2) * q[2] * rq - os * (T(1) + X2));
  lq[2] = la1 * (Y * (T(1) + Y2) * q[1] * rq + os * (T(1) + Y2)) + la2 * ((-X2 * Y) * q[2] * rq + A2 * rq + os * XY);
}

// ---------------------------------------------------------------------------------
// TPP reconstruction + sources adjoint: per cell, the gradient with respect to its
// K x K stencil, summed over the tile's cells onto the tile's extended region
// ((TY + K - 1) x (TX + K - 1) cells, the region its stencils cover), which is written to
// slot tile_id of the tile buffer tbuf ([tile][3][TY+K-1][TX+K-1], valid part only).
// One tile of at most TX x TY cells of panel p with its first cell at (i0, j0), called by
// all threads of a block of at least TX*TY threads (the valid cells of a tile cut by the
// panel's edge are packed onto the first threads); ends with a barrier so the shared
// memory can be reused.  Shared memory: the forward tile's (raw tile, x-pass, weights)
// plus the adjoint at the cell points [3][me^2][NT], one stencil row's gradient per cell
// [3][K][NT] and the extended region [3][TY+K-1][TX+K-1] (NT = blockDim.x).
// ---------------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void recon_tpp_adj_tile(unsigned char *smem_raw, int p, int i0, int j0, const int TX,
                                                   const int TY, const long long tile_id, const T *__restrict__ q, const T *__restrict__ gext,
                                                   const T *__restrict__ w1g, const T *__restrict__ Xg,
                                                   const T *__restrict__ t1w, const T *__restrict__ lep,
                                                   const T *__restrict__ lamL, T *__restrict__ tbuf, int N, int ne,
                                                   T omega, const FCoef<T> &fc, const T *__restrict__ ttw = nullptr) {
  constexpr int H = (K - 1) / 2, ME = (K + 1) / 2, NPOS = ME + 2;
  const int RW = TX + 2 * H, RH = TY + 2 * H, NT = blockDim.x;
  const int vx = min(TX, N - i0), vy = min(TY, N - j0);
  const int vw = vx + 2 * H, vh = vy + 2 * H;
  T *raw = reinterpret_cast<T *>(smem_raw);  // [3][RH][RW]
  T *xs = raw + 3 * RH * RW;                  // [3][NPOS][RH][TX]
  T *w1 = xs + 3 * NPOS * RH * TX;            // [NPOS][K]
  T *lcq = w1 + NPOS * K;                     // [3][ME*ME][NT] adjoint at cell points
  // phase 2's scratch: one stencil row's gradient per cell [3][K][TX*TY] and the tile's
  // gradient on its extended region [3][RH][RW]; it reuses the tile and x-pass region, which
  // nothing reads after phase 1, when that is large enough (every shape the library uses),
  // else it follows lcq
  const int ncap = TX * TY;
  const bool alias = 3 * K * ncap + 3 * RH * RW <= 3 * RH * RW + 3 * NPOS * RH * TX;
  T *gs = alias ? raw : lcq + 3 * ME * ME * NT;
  T *acc = gs + 3 * K * ncap;
  for (int t = threadIdx.x; t < NPOS * K; t += blockDim.x) w1[t] = w1g[t];
  {
    const size_t pn = (size_t)6 * N * N, pe = (size_t)6 * ne * ne;
    for (BoxWalk bw(vh, vw); bw.v < 3; bw.next()) {
      const int v = bw.v, r = bw.r, c = bw.c;
      const int i = i0 + c - H, j = j0 + r - H;
      T val = T(0);
      if (i >= 0 && i < N && j >= 0 && j < N)
        val = q[v * pn + ((size_t)p * N + j) * N + i];
      else if (i >= -H && i < N + H && j >= -H && j < N + H)
        val = gext[v * pe + ((size_t)p * ne + (j + H)) * ne + (i + H)];
      raw[(v * RH + r) * RW + c] = val;
    }
  }
  __syncthreads();
  for (BoxWalk bw(vh, vx); bw.v < 3; bw.next()) {
    const int v = bw.v, r = bw.r, c = bw.c;
    const T *row = raw + (v * RH + r) * RW + c;
#pragma unroll
    for (int t = 0; t < NPOS; ++t) {
      T s = 0;
#pragma unroll
      for (int b = 0; b < K; ++b) s = fma(w1[t * K + b], row[b], s);
      xs[((v * NPOS + t) * RH + r) * TX + c] = s;
    }
  }
  __syncthreads();
  const int tid = threadIdx.x;
  const int nc = vx * vy;
  const size_t pn = (size_t)6 * N * N;
  const bool own = tid < nc;
  const int ty = own ? tid / vx : 0, tx = own ? tid - ty * vx : 0;
  const int i = i0 + tx, j = j0 + ty;
  const size_t cell = ((size_t)p * N + j) * N + i;
  if (own) {
    const T fc0 = fc.c[3 * p], fc1 = fc.c[3 * p + 1], fc2 = fc.c[3 * p + 2];
    const T lS1 = lamL[pn + cell], lS2 = lamL[2 * pn + cell];
    // phase 1: adjoint at the cell points (recomputed values, source VJP)
#pragma unroll 1
    for (int g = 0; g < ME; ++g) {
      const T X = Xg[i * ME + g];
      T col[3][K];
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int b = 0; b < K; ++b) col[v][b] = xs[((v * NPOS + 2 + g) * RH + ty + b) * TX + tx];
#pragma unroll 1
      for (int h = 0; h < ME; ++h) {
        T qv[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          T s = 0;
#pragma unroll
          for (int b = 0; b < K; ++b) s = fma(w1[(2 + h) * K + b], col[v][b], s);
          qv[v] = s;
        }
        const T Y = Xg[j * ME + h];
        const T tw = t1w[(((size_t)j * N + i) * ME + h) * ME + g];
        const T os = omega * (fc0 + fc1 * X + fc2 * Y);
        T lq[3];
        source_vjp(qv, X, Y, os, tw, lS1, lS2, lq);
#pragma unroll
        for (int v = 0; v < 3; ++v) lcq[(v * ME * ME + h * ME + g) * NT + tid] = lq[v];
      }
    }
  }
  __syncthreads();  // the tile and x-pass are dead from here on (phase 2's scratch may alias them)
  T *tb = tbuf + (size_t)3 * RH * RW * tile_id;
  if (!ttw) {
    // phase 2, the transposes of the two passes: the transposed y-pass adds each cell's
    // point adjoints into the adjoints of its x-pass values (lxs, over the dead x-pass
    // region), stencil row by stencil row -- in row b the cells of a tile column add into
    // distinct x-pass rows ty + b, so no two threads update one value; then each location
    // of the extended region gathers its transposed x-pass terms (positions in order,
    // taps in order) and is written to the tile buffer
    T *lxs = xs;  // [3][NPOS][RH][TX]
    for (int t = threadIdx.x; t < 3 * NPOS * RH * TX; t += blockDim.x) lxs[t] = T(0);
    __syncthreads();
#pragma unroll 1
    for (int b = 0; b < K; ++b) {
      if (own) {
#pragma unroll 1
        for (int t = 0; t < NPOS; ++t) {
          T gt[3] = {0, 0, 0};
          if (t < 2) {
#pragma unroll
            for (int r = 0; r < ME; ++r) {
              const T w = w1[(2 + r) * K + b];
#pragma unroll
              for (int v = 0; v < 3; ++v) gt[v] = fma(w, lep[((size_t)(t * 3 + v) * ME + r) * pn + cell], gt[v]);
            }
          } else {
            const int g = t - 2;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
              const T w = w1[side * K + b];
#pragma unroll
              for (int v = 0; v < 3; ++v)
                gt[v] = fma(w, lep[((size_t)((2 + side) * 3 + v) * ME + g) * pn + cell], gt[v]);
            }
#pragma unroll
            for (int h = 0; h < ME; ++h) {
              const T w = w1[(2 + h) * K + b];
#pragma unroll
              for (int v = 0; v < 3; ++v) gt[v] = fma(w, lcq[(v * ME * ME + h * ME + g) * NT + tid], gt[v]);
            }
          }
#pragma unroll
          for (int v = 0; v < 3; ++v) lxs[((v * NPOS + t) * RH + ty + b) * TX + tx] += gt[v];
        }
      }
      __syncthreads();
    }
    for (BoxWalk bw(vh, vw); bw.v < 3; bw.next()) {
      const int v = bw.v, r = bw.r, c = bw.c;
      T sacc = T(0);
#pragma unroll
      for (int t = 0; t < NPOS; ++t) {
        const T *lrow = lxs + ((v * NPOS + t) * RH + r) * TX;
#pragma unroll
        for (int a = 0; a < K; ++a) {
          const int cx = c - a;
          if (cx >= 0 && cx < vx) sacc = fma(w1[t * K + a], lrow[cx], sacc);
        }
      }
      tb[(v * RH + r) * RW + c] = sacc;
    }
    __syncthreads();
    return;
  }
  for (int t = threadIdx.x; t < 3 * RH * RW; t += blockDim.x) acc[t] = T(0);
  // phase 2 over a surface (psi_B's transposed stencil map is not separable): per stencil
  // row b, gt[v][t] = sum over points at x-position t of w1[ty(pt)][b] lam(pt), then the
  // row's gradient g[v][a] = sum_t w1[t][a] gt[v][t] plus psi_B's terms for the mass
  // variable; the rows are added onto the tile's extended region: location (ty + b,
  // tx + a) gains the gradient of cell (tx, ty), summed over a in order, then over b in order
#pragma unroll 1
  for (int b = 0; b < K; ++b) {
    if (own) {
      T gacc[3][K];
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int a = 0; a < K; ++a) gacc[v][a] = T(0);
#pragma unroll 1
      for (int t = 0; t < NPOS; ++t) {
        T gt[3] = {0, 0, 0};
        if (t < 2) {
#pragma unroll
          for (int r = 0; r < ME; ++r) {
            const T w = w1[(2 + r) * K + b];
#pragma unroll
            for (int v = 0; v < 3; ++v) gt[v] = fma(w, lep[((size_t)(t * 3 + v) * ME + r) * pn + cell], gt[v]);
          }
        } else {
          const int g = t - 2;
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            const T w = w1[side * K + b];
#pragma unroll
            for (int v = 0; v < 3; ++v)
              gt[v] = fma(w, lep[((size_t)((2 + side) * 3 + v) * ME + g) * pn + cell], gt[v]);
          }
#pragma unroll
          for (int h = 0; h < ME; ++h) {
            const T w = w1[(2 + h) * K + b];
#pragma unroll
            for (int v = 0; v < 3; ++v) gt[v] = fma(w, lcq[(v * ME * ME + h * ME + g) * NT + tid], gt[v]);
          }
        }
#pragma unroll
        for (int a = 0; a < K; ++a) {
          const T w = w1[t * K + a];
#pragma unroll
          for (int v = 0; v < 3; ++v) gacc[v][a] = fma(w, gt[v], gacc[v][a]);
        }
      }
      if (ttw) {  // psi_B (eq. 2.14): its weights on the mass variable's stencil, transposed
        const T l1 = lamL[pn + cell], l2 = lamL[2 * pn + cell];
#pragma unroll
        for (int a = 0; a < K; ++a) {
          const size_t c = (size_t)b * K + a;
          gacc[0][a] += ttw[c * pn + cell] * l1 + ttw[((size_t)K * K + c) * pn + cell] * l2;
        }
      }
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int a = 0; a < K; ++a) gs[(v * K + a) * ncap + tid] = gacc[v][a];
    }
    __syncthreads();
    // extended rows b .. b + vy - 1: each location sums its K cells of this row
    for (int idx = threadIdx.x; idx < 3 * vy * vw; idx += blockDim.x) {
      const int v = idx / (vy * vw);
      const int rem = idx - v * vy * vw;
      const int rr = rem / vw, c = rem - rr * vw;
      T s = T(0);
#pragma unroll
      for (int a = 0; a < K; ++a) {
        const int cx = c - a;
        if (cx >= 0 && cx < vx) s += gs[(v * K + a) * ncap + rr * vx + cx];
      }
      acc[(v * RH + rr + b) * RW + c] += s;
    }
    __syncthreads();
  }
  // the tile's extended region [3][RH][RW] (valid part) to its slot of the tile buffer
  for (BoxWalk bw(vh, vw); bw.v < 3; bw.next()) {
    const int v = bw.v, r = bw.r, c = bw.c;
    tb[(v * RH + r) * RW + c] = acc[(v * RH + r) * RW + c];
  }
  __syncthreads();
}

// Shared memory of one reconstruction-adjoint tile of TX x TY cells with NT threads: the
// forward tile's, the cell-point adjoints, and phase 2's scratch unless it fits the tile and
// x-pass region it reuses.
template <typename T, int K>
__host__ __device__ constexpr size_t recon_adj_tile_smem_bytes(int TX, int TY, int NT) {
  return recon_tile_smem_bytes<T, K>(TX, TY) + sizeof(T) * 3 * ((K + 1) / 2) * ((K + 1) / 2) * NT +
         (3 * K * TX * TY <= 3 * ((K + 1) / 2 + 2) * (TY + K - 1) * TX
              ? 0
              : sizeof(T) * (3 * K * TX * TY + 3 * (TY + K - 1) * (TX + K - 1)));
}

// Elements of a member's tile buffer for TX x TY tiles.
__host__ __device__ constexpr long long tile_buf_elems(int N, int K, int TX, int TY) {
  return 6LL * ((N + TX - 1) / TX) * ((N + TY - 1) / TY) * 3 * (TY + K - 1) * (TX + K - 1);
}

template <typename T, int K>
__global__ void __launch_bounds__(REC_TX *REC_TY)
    k_recon_tpp_adj(const T *__restrict__ q, const T *__restrict__ gext, const T *__restrict__ w1g,
                    const T *__restrict__ Xg, const T *__restrict__ t1w, const T *__restrict__ lep,
                    const T *__restrict__ lamL, T *__restrict__ tbuf, int N, int ne, T omega, FCoef<T> fc,
                    const T *__restrict__ ttw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long tile = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  recon_tpp_adj_tile<T, K>(smem_raw, blockIdx.z, blockIdx.x * REC_TX, blockIdx.y * REC_TY, REC_TX, REC_TY, tile, q,
                           gext, w1g, Xg, t1w, lep, lamL, tbuf, N, ne, omega, fc, ttw);
}

template <typename T, int K>
__host__ __device__ constexpr size_t recon_adj_smem_bytes() {
  return recon_adj_tile_smem_bytes<T, K>(REC_TX, REC_TY, REC_TX * REC_TY);
}

// ---------------------------------------------------------------------------------
// Gather: lam at every extended cell (xi, yj) (interior coordinates in [-H, N+H)):
// sum over cells c = (xi + H - a, yj + H - b) of grad[c][b][a].  Interior cells go to
// lam_direct[3][6][N][N], ring cells to lam_ring[3][6][ne][ne].
// ---------------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void gather_adj_item(long long idx, const T *__restrict__ grad, T *__restrict__ lam_direct,
                                                T *__restrict__ lam_ring, int N) {
  constexpr int H = (K - 1) / 2;
  const int ne = N + 2 * H;
  const int ii = (int)(idx % ne);
  const long long pj = idx / ne;
  const int jj = (int)(pj % ne), p = (int)(pj / ne);
  const int xi = ii - H, yj = jj - H;
  const size_t pn = (size_t)6 * N * N, pe = (size_t)6 * ne * ne;
  T s[3] = {0, 0, 0};
#pragma unroll
  for (int b = 0; b < K; ++b) {
    const int cj = yj + H - b;
    if (cj < 0 || cj >= N) continue;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      const int ci = xi + H - a;
      if (ci < 0 || ci >= N) continue;
      const size_t cell = ((size_t)p * N + cj) * N + ci;
#pragma unroll
      for (int v = 0; v < 3; ++v) s[v] += grad[((size_t)v * K * K + b * K + a) * pn + cell];
    }
  }
  if (xi >= 0 && xi < N && yj >= 0 && yj < N) {
    const size_t cell = ((size_t)p * N + yj) * N + xi;
#pragma unroll
    for (int v = 0; v < 3; ++v) lam_direct[v * pn + cell] = s[v];
  } else {
#pragma unroll
    for (int v = 0; v < 3; ++v) lam_ring[v * pe + idx] = s[v];
  }
}

// Gather from a tile buffer (TPP): lam at every extended cell (xi, yj) of panel p is the sum,
// over the tiles whose extended regions cover it (ascending tile row, then column), of
// their contributions; TX x TY tiles, the last ones of a panel cut at its edge.
template <typename T, int K>
__device__ __forceinline__ void gather_tiles_item(long long idx, const T *__restrict__ tbuf, int TX, int TY,
                                                  T *__restrict__ lam_direct, T *__restrict__ lam_ring, int N) {
  constexpr int H = (K - 1) / 2;
  const int ne = N + 2 * H, RW = TX + 2 * H, RH = TY + 2 * H;
  const int ntx = (N + TX - 1) / TX, nty = (N + TY - 1) / TY;
  const int ii = (int)(idx % ne);
  const long long pj = idx / ne;
  const int jj = (int)(pj % ne), p = (int)(pj / ne);
  const int xi = ii - H, yj = jj - H;
  const size_t pn = (size_t)6 * N * N, pe = (size_t)6 * ne * ne;
  T s[3] = {0, 0, 0};
  const int ty_hi = min(nty - 1, (yj + H) / TY), tx_hi = min(ntx - 1, (xi + H) / TX);
  for (int ty = max(0, ty_hi - (2 * H + TY - 1) / TY - 1); ty <= ty_hi; ++ty) {
    const int y0 = ty * TY - H, vy = min(TY, N - ty * TY);
    if (yj < y0 || yj >= y0 + vy + 2 * H) continue;
    for (int tx = max(0, tx_hi - (2 * H + TX - 1) / TX - 1); tx <= tx_hi; ++tx) {
      const int x0 = tx * TX - H, vx = min(TX, N - tx * TX);
      if (xi < x0 || xi >= x0 + vx + 2 * H) continue;
      const T *tb = tbuf + (size_t)3 * RH * RW * (((size_t)p * nty + ty) * ntx + tx);
#pragma unroll
      for (int v = 0; v < 3; ++v) s[v] += tb[(v * RH + (yj - y0)) * RW + (xi - x0)];
    }
  }
  if (xi >= 0 && xi < N && yj >= 0 && yj < N) {
    const size_t cell = ((size_t)p * N + yj) * N + xi;
#pragma unroll
    for (int v = 0; v < 3; ++v) lam_direct[v * pn + cell] = s[v];
  } else {
#pragma unroll
    for (int v = 0; v < 3; ++v) lam_ring[v * pe + idx] = s[v];
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(256)
    k_gather_tiles(const T *__restrict__ tbuf, int TX, int TY, T *__restrict__ lam_direct, T *__restrict__ lam_ring,
                   int N) {
  const long long ne = N + K - 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 6LL * ne * ne) return;
  gather_tiles_item<T, K>(idx, tbuf, TX, TY, lam_direct, lam_ring, N);
}

template <typename T, int K>
__global__ void __launch_bounds__(256)
    k_gather_adj(const T *__restrict__ grad, T *__restrict__ lam_direct, T *__restrict__ lam_ring, int N) {
  const long long ne = N + K - 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 6LL * ne * ne) return;
  gather_adj_item<T, K>(idx, grad, lam_direct, lam_ring, N);
}

// Transposed ghost operator and Runge-Kutta combination: out = c (lam_direct + G^T lam_ring)
// + a x + b y + d z per interior cell (x, y, z may be null).  G^T is a CSR over the cells
// (gtp), each entry holding the ring position of its ghost row (gtr) and the row's 5
// weights (gtv); only the band of cells along the panel edges has entries.
template <typename T>
__device__ __forceinline__ void ghost_adj_finish(long long cid, T s0, T s1, T s2, const T *x, const T *y,
                                                 const T *z, T *out, T a, T b, T d, T c, long long ncell) {
  const T r3[3] = {s0, s1, s2};
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const long long k = v * ncell + cid;
    T o = c * r3[v];
    if (x) o += a * x[k];
    if (y) o += b * y[k];
    if (z) o += d * z[k];
    out[k] = o;
  }
}

// A cell that no ghost row reads: the combination alone (band cells are left to
// ghost_adj_band).
template <typename T>
__device__ __forceinline__ void ghost_adj_interior(long long cid, const T *__restrict__ lam_direct,
                                                   const int *__restrict__ gtp, const T *x, const T *y, const T *z,
                                                   T *out, T a, T b, T d, T c, int N) {
  if (gtp[cid + 1] > gtp[cid]) return;
  const long long ncell = 6LL * N * N;
  ghost_adj_finish(cid, lam_direct[cid], lam_direct[ncell + cid], lam_direct[2 * ncell + cid], x, y, z, out, a, b,
                   d, c, ncell);
}

// A band cell, by GADJ_LANES consecutive lanes of one warp (lane `sub` of the group):
// lane sub adds entries sub, sub + GADJ_LANES, ... in order (GADJ_UNROLL entries' loads in
// flight), the group sums its lanes by a fixed butterfly and lane 0, which started from the
// direct part, writes the cell.  `valid` false: the lane only joins the butterfly (every
// lane of the warp must reach the shuffles).
constexpr int GADJ_LANES = 8;
constexpr int GADJ_UNROLL = 4;
template <typename T>
__device__ __forceinline__ void ghost_adj_band(bool valid, long long band, int sub, const int *__restrict__ gband,
                                               const T *__restrict__ lam_direct, const T *__restrict__ lam_ring,
                                               const int *__restrict__ gtp, const int *__restrict__ gtr,
                                               const T *__restrict__ gtv, const T *x, const T *y, const T *z, T *out,
                                               T a, T b, T d, T c, int N, int ne) {
  const long long ncell = 6LL * N * N;
  const size_t pe = (size_t)6 * ne * ne;
  long long cid = 0;
  T s0 = 0, s1 = 0, s2 = 0;
  if (valid) {
    cid = gband[band];
    if (sub == 0) {
      s0 = lam_direct[cid];
      s1 = lam_direct[ncell + cid];
      s2 = lam_direct[2 * ncell + cid];
    }
    const int e0 = gtp[cid], e1 = gtp[cid + 1];
    constexpr int U = GADJ_UNROLL;
    for (int t0 = e0 + sub; t0 < e1; t0 += GADJ_LANES * U) {
      T g[U][3], w[U][5];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int t = t0 + GADJ_LANES * u;
        const bool ok = t < e1;
        const int dpos = ok ? gtr[t] : 0;
        g[u][0] = ok ? lam_ring[dpos] : T(0);
        g[u][1] = ok ? lam_ring[pe + dpos] : T(0);
        g[u][2] = ok ? lam_ring[2 * pe + dpos] : T(0);
#pragma unroll
        for (int k = 0; k < 5; ++k) w[u][k] = ok ? gtv[(size_t)t * 5 + k] : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        s0 += w[u][0] * g[u][0];
        s1 += w[u][1] * g[u][1] + w[u][3] * g[u][2];
        s2 += w[u][2] * g[u][1] + w[u][4] * g[u][2];
      }
    }
  }
#pragma unroll
  for (int o = GADJ_LANES / 2; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o, GADJ_LANES);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o, GADJ_LANES);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o, GADJ_LANES);
  }
  if (valid && sub == 0) ghost_adj_finish(cid, s0, s1, s2, x, y, z, out, a, b, d, c, ncell);
}

// Threads [0, nlanes) (nlanes: GADJ_LANES per band cell, rounded up to whole warps) take
// the band cells, the following ones a cell each.
template <typename T>
__global__ void __launch_bounds__(256)
    k_ghost_adj(const T *__restrict__ lam_direct, const T *__restrict__ lam_ring, const int *__restrict__ gtp,
                const int *__restrict__ gtr, const T *__restrict__ gtv, const int *__restrict__ gband, long long nband,
                long long nlanes, const T *x, const T *y, const T *z, T *out, T a, T b, T d, T c, int N, int ne) {
  const long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (it < nlanes) {
    const long long band = it / GADJ_LANES;
    ghost_adj_band(band < nband, band, (int)(it % GADJ_LANES), gband, lam_direct, lam_ring, gtp, gtr, gtv, x, y, z,
                   out, a, b, d, c, N, ne);
    return;
  }
  const long long cid = it - nlanes;
  if (cid >= 6LL * N * N) return;
  ghost_adj_interior(cid, lam_direct, gtp, x, y, z, out, a, b, d, c, N);
}

}  // namespace hope
