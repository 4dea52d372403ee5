// hope_weno1d.cuh -- the dimension-by-dimension WENO-Z reconstruction that section 5.5
// compares with the genuine two-dimensional one (the fifth-order "WENO-Z" of the dam-break
// experiment), with the cell-point sources, one thread per cell, for sm_103a.
//
// Section 5.5 names the scheme but prints no equations; it is read as the 1-D WENO-Z of
// Borges et al. (2008) applied along x on each of the k rows of a cell's stencil at the
// x position of a reconstruction point, and then along y on those k row values at the
// point's y position.  Per line of k cell averages v and position xi:
//   p_s      the l = (k+1)/2 sub-stencil values at xi (1-D cell-average weights),
//   beta_s   the Jiang-Shu indicator, sum over m = 1..l-1 of the integral of (p_s^(m))^2
//            over the target cell, a quadratic form v^T B_s v kept as its eigenpairs
//            (B_s = sum lam_k w_k w_k^T; the constant mode has lam = 0, so v - v_centre is
//            used, which keeps beta >= 0 and accurate in FP32),
//   tau      = |beta_0 - beta_2| (WENO-Z's tau5; fifth order only), f_s = 1 + tau / (beta_s + eps),
//   q(xi)    = sigma+ sum(gamma+ f p)/sum(gamma+ f) - sigma- sum(gamma- f p)/sum(gamma- f),
//            the 1-D linear weights gamma(xi) by the 1-D least squares of eqs. 3.16-3.19,
//            split with theta = 3 as in eq. 3.20 (sigma+ - sigma- = 1).
// beta, tau and f depend only on the line, not on xi, so each stencil row's (and each
// row-value column's) indicators are computed once and shared by all positions.
#pragma once
#include "hope_internal.h"
#include "hope_kernels.cuh"

namespace hope {

template <typename T, int K>
struct Weno1dShape {
  static constexpr int L = (K + 1) / 2;
  static constexpr int ME = L;
  static constexpr int NPOS = ME + 2;  // x / y positions: -1/2, +1/2, Gauss nodes
  static constexpr int NT = REC_TX * REC_TY;
  // tile + sub-stencil weights [NPOS][L][L] + split weights [NPOS][2][L] + sigma [NPOS][2]
  // + indicator eigenpairs [L][L*L + L] + cell-point values [3][ME*ME][NT]
  static constexpr size_t smem_elems() {
    return 3 * Shape<K>::RH * Shape<K>::RW + NPOS * L * L + NPOS * 2 * L + NPOS * 2 + L * (L * L + L) +
           3 * ME * ME * NT;
  }
};

// Indicators of one line of K values (stride `st`) and the factors f_s of eq. 3.23.
template <typename T, int K>
__device__ __forceinline__ void weno1d_factors(const T *v, int st, const T *bf, T eps, T f[(K + 1) / 2]) {
  constexpr int L = (K + 1) / 2, H = (K - 1) / 2;
  const T c = v[H * st];
  T beta[L];
#pragma unroll
  for (int s = 0; s < L; ++s) {
    const T *W = bf + s * (L * L + L);  // rows: eigenvectors; then the L eigenvalues
    T b = 0;
#pragma unroll
    for (int k = 0; k < L; ++k) {
      T z = 0;
#pragma unroll
      for (int a = 0; a < L; ++a) z = fma(W[k * L + a], v[(s + a) * st] - c, z);
      b = fma(W[L * L + k] * z, z, b);
    }
    beta[s] = b;
  }
  const T tau = fabs(beta[0] - beta[L - 1]);
#pragma unroll
  for (int s = 0; s < L; ++s) f[s] = T(1) + tau * rcp(beta[s] + eps);
}

// The WENO-Z value of a line at position `pos` from its factors.
template <typename T, int K>
__device__ __forceinline__ T weno1d_value(const T *v, int st, const T *f, int pos, const T *wsub, const T *gpm,
                                          const T *sig) {
  constexpr int L = (K + 1) / 2;
  T Ap = 0, Am = 0, Dp = 0, Dm = 0;
#pragma unroll
  for (int s = 0; s < L; ++s) {
    const T *w = wsub + (pos * L + s) * L;
    T p = 0;
#pragma unroll
    for (int a = 0; a < L; ++a) p = fma(w[a], v[(s + a) * st], p);
    const T gp = gpm[(pos * 2) * L + s] * f[s], gm = gpm[(pos * 2 + 1) * L + s] * f[s];
    Ap = fma(gp, p, Ap);
    Dp += gp;
    Am = fma(gm, p, Am);
    Dm += gm;
  }
  return sig[2 * pos] * Ap * rcp(Dp) - sig[2 * pos + 1] * Am * rcp(Dm);
}

// One block per 16 x 8 tile (blockIdx.z: panel); cells of a tile cut by the panel's edge
// are packed onto the first vx * vy threads.
template <typename T, int K>
__global__ void __launch_bounds__(REC_TX *REC_TY)
    k_recon_weno1d(const T *__restrict__ q, const T *__restrict__ gext, const T *__restrict__ wsub_g,
                   const T *__restrict__ gpm_g, const T *__restrict__ sig_g, const T *__restrict__ bf_g,
                   const T *__restrict__ Xg, const T *__restrict__ t1w, T *__restrict__ ep, T *__restrict__ sb,
                   int N, int ne, T omega, FCoef<T> fc, T eps) {
  using W = Weno1dShape<T, K>;
  using SH = Shape<K>;
  constexpr int L = W::L, ME = W::ME, NPOS = W::NPOS, NT = W::NT, H = (K - 1) / 2;
  constexpr int RW = SH::RW, RH = SH::RH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *raw = reinterpret_cast<T *>(smem_raw);  // [3][RH][RW]
  T *wsub = raw + 3 * RH * RW;               // [NPOS][L][L]
  T *gpm = wsub + NPOS * L * L;              // [NPOS][2][L]
  T *sig = gpm + NPOS * 2 * L;               // [NPOS][2]
  T *bf = sig + NPOS * 2;                    // [L][L*L + L]
  T *cq = bf + L * (L * L + L);              // [3][ME*ME][NT]
  const int p = blockIdx.z;
  const int i0 = blockIdx.x * REC_TX, j0 = blockIdx.y * REC_TY;
  const int vx = min(REC_TX, N - i0), vy = min(REC_TY, N - j0);
  for (int t = threadIdx.x; t < NPOS * L * L; t += blockDim.x) wsub[t] = wsub_g[t];
  for (int t = threadIdx.x; t < NPOS * 2 * L; t += blockDim.x) gpm[t] = gpm_g[t];
  for (int t = threadIdx.x; t < NPOS * 2; t += blockDim.x) sig[t] = sig_g[t];
  for (int t = threadIdx.x; t < L * (L * L + L); t += blockDim.x) bf[t] = bf_g[t];
  {
    // the valid part of the extended tile: interior cells from q, ring cells from gext
    const int vw = vx + 2 * H, vh = vy + 2 * H;
    const size_t pn = (size_t)6 * N * N, pe = (size_t)6 * ne * ne;
    for (int idx = threadIdx.x; idx < 3 * vh * vw; idx += blockDim.x) {
      const int v = idx / (vh * vw);
      const int rem = idx - v * vh * vw;
      const int r = rem / vw, c = rem - r * vw;
      const int ii = i0 + c - H, jj = j0 + r - H;
      T val = T(0);
      if (ii >= 0 && ii < N && jj >= 0 && jj < N)
        val = q[v * pn + ((size_t)p * N + jj) * N + ii];
      else if (ii >= -H && ii < N + H && jj >= -H && jj < N + H)
        val = gext[v * pe + ((size_t)p * ne + (jj + H)) * ne + (ii + H)];
      raw[(v * RH + r) * RW + c] = val;
    }
  }
  __syncthreads();
  const int tid = threadIdx.x;
  if (tid >= vx * vy) return;
  const int ty = tid / vx, tx = tid - ty * vx;
  const int i = i0 + tx, j = j0 + ty;
  const size_t pn = (size_t)6 * N * N;
  const size_t cell = ((size_t)p * N + j) * N + i;

#pragma unroll 1
  for (int v = 0; v < 3; ++v) {
    const T *Qv = raw + (v * RH + ty) * RW + tx;  // Q(r, c) = Qv[r * RW + c]
    // x pass: every stencil row at every x position
    T Lx[NPOS][K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
      T f[L];
      weno1d_factors<T, K>(Qv + r * RW, 1, bf, eps, f);
#pragma unroll
      for (int ix = 0; ix < NPOS; ++ix) Lx[ix][r] = weno1d_value<T, K>(Qv + r * RW, 1, f, ix, wsub, gpm, sig);
    }
    // y pass on each x position's column of row values
#pragma unroll
    for (int ix = 0; ix < NPOS; ++ix) {
      T f[L];
      weno1d_factors<T, K>(Lx[ix], 1, bf, eps, f);
      if (ix < 2) {
        // west (ix = 0) / east (ix = 1) edge points at the y Gauss nodes
#pragma unroll
        for (int r = 0; r < ME; ++r)
          ep[((size_t)(ix * 3 + v) * ME + r) * pn + cell] = weno1d_value<T, K>(Lx[ix], 1, f, 2 + r, wsub, gpm, sig);
      } else {
        const int g = ix - 2;
        // south / north edge points at x node g, then the cell points (g, h)
#pragma unroll
        for (int side = 0; side < 2; ++side)
          ep[((size_t)((2 + side) * 3 + v) * ME + g) * pn + cell] =
              weno1d_value<T, K>(Lx[ix], 1, f, side, wsub, gpm, sig);
#pragma unroll
        for (int h = 0; h < ME; ++h)
          cq[(v * ME * ME + h * ME + g) * NT + tid] = weno1d_value<T, K>(Lx[ix], 1, f, 2 + h, wsub, gpm, sig);
      }
    }
  }
  // ------------------------------------------------------------------ sources
  const T fc0 = fc.c[3 * p], fc1 = fc.c[3 * p + 1], fc2 = fc.c[3 * p + 2];
  T s1 = 0, s2 = 0;
#pragma unroll 1
  for (int h = 0; h < ME; ++h) {
    const T Y = Xg[j * ME + h];
#pragma unroll
    for (int g = 0; g < ME; ++g) {
      const T X = Xg[i * ME + g];
      const T q0 = cq[(0 * ME * ME + h * ME + g) * NT + tid];
      const T q1 = cq[(1 * ME * ME + h * ME + g) * NT + tid];
      const T q2 = cq[(2 * ME * ME + h * ME + g) * NT + tid];
      const T tw = t1w[(((size_t)j * N + i) * ME + h) * ME + g];
      const T os = omega * (fc0 + fc1 * X + fc2 * Y);
      const T rq = rcp(q0);
      const T XY = X * Y, X2 = X * X, Y2 = Y * Y;
      T a1 = (-XY * Y * q1 + Y * (T(1) + Y2) * q2) * q1 * rq + os * (-XY * q1 + (T(1) + Y2) * q2);
      T a2 = (X * (T(1) + X2) * q1 - X2 * Y * q2) * q2 * rq + os * (-(T(1) + X2) * q1 + XY * q2);
      s1 = fma(tw, a1, s1);
      s2 = fma(tw, a2, s2);
    }
  }
  sb[cell] = s1;
  sb[pn + cell] = s2;
}

}  // namespace hope
