// hope_weno.cuh -- genuine two-dimensional WENO-Z reconstruction (section 3.2) with the
// cell-point sources, one thread per cell, for sm_103a.
//
// Per cell and variable, with the k x k stencil Q staged in shared memory:
//   beta_i   smoothness indicator of each of the s = l^2 sub-stencils (eq. 3.25 read as
//            the sum of squared mixed derivatives), through the simultaneous
//            diagonalisation of the 1-D forms: beta = sum (lam_y lam_x - 1) Z^2 with
//            Z = Winv_y Q_i Winv_x^T, sum-factorised over the sub-stencil rows;
//   tau      eq. 3.24; f_i = 1 + tau / (beta_i + eps) (eq. 3.23);
//   p_i(pt)  the sub-stencil TPP values at every point, x-pass per sub-stencil column,
//            then y-pass per sub-stencil row;
//   q(pt)    = sigma+ sum(gamma+ f p)/sum(gamma+ f) - sigma- sum(gamma- f p)/sum(gamma- f)
//            (eqs. 3.20-3.23 with the sigma+- normalisation of the split weights).
// Edge points go to the edge-point buffer; the me^2 cell points of the three variables
// are staged in shared memory for the sources (eqs. 2.2, 2.3, 3.6).
#pragma once
#include "hope_internal.h"
#include "hope_kernels.cuh"
#include "hope_adjoint.cuh"

namespace hope {

template <typename T, int K>
struct WenoShape {
  static constexpr int L = (K + 1) / 2;
  static constexpr int S = L * L;
  static constexpr int ME = L;
  static constexpr int NPOS = ME + 2;
  static constexpr int NPOC = 4 * ME + ME * ME;
  static constexpr int NT = REC_TX * REC_TY;
  static constexpr size_t smem_elems() {
    return 3 * Shape<K>::RH * Shape<K>::RW + NPOS * L * L + NPOC * 2 * S + NPOC * 2 + L * (L * L + L) +
           S * S + 3 * ME * ME * NT;
  }
};

// Shared memory of the forward WENO kernel for a TX x TY tile and NT threads.
template <typename T, int K>
__host__ __device__ constexpr size_t weno_tile_smem_bytes(int TX, int TY, int NT) {
  using W = WenoShape<T, K>;
  return sizeof(T) * (3 * (TY + K - 1) * (TX + K - 1) + W::NPOS * W::L * W::L + W::NPOC * 2 * W::S + W::NPOC * 2 +
                      W::L * (W::L * W::L + W::L) + W::S * W::S + 3 * W::ME * W::ME * NT);
}

// Largest thread count of a forward WENO block (one thread per cell of the tile).
constexpr int WENO_MAX_THREADS = 256;

// One block per tile of TX x TY cells (blockIdx.z: panel); cells of a tile cut by the
// panel's edge are packed onto the first vx * vy threads.  RT = false compiles the
// default 16 x 8 tile with 128 threads as constants (the FP32 kernel is bound by its
// instruction count, and constant strides save the address arithmetic); RT = true takes
// the shape at run time (FP64 tiles chosen for balance).
// TOPO (bottom topography, eqs. 2.13-2.14, reading c26): the mass variable reconstructed is
// sqrtG phi_t = q0 + sqrtG phi_s (the surface's extended averages sext [6][ne][ne] added at
// the tile load), and the surface's own TPP values at the points (sep at the edge points,
// scp [me*me][6][N][N] at the cell points) are subtracted from it, leaving the depth.
template <typename T, int K, bool RT = false, bool TOPO = false>
__global__ void __launch_bounds__(RT ? WENO_MAX_THREADS : REC_TX * REC_TY)
    k_recon_weno(const T *__restrict__ q, const T *__restrict__ gext, const T *__restrict__ wsub_g,
                 const T *__restrict__ gpm_g, const T *__restrict__ sig_g, const T *__restrict__ bform_g,
                 const T *__restrict__ bcoef_g, const T *__restrict__ Xg, const T *__restrict__ t1w, T *__restrict__ ep, T *__restrict__ sb,
                 int N, int ne, int TXr, int TYr, T omega, FCoef<T> fc, T eps, const T *__restrict__ sext = nullptr,
                 const T *__restrict__ sep = nullptr, const T *__restrict__ scp = nullptr) {
  using W = WenoShape<T, K>;
  constexpr int L = W::L, S = W::S, ME = W::ME, NPOS = W::NPOS, NPOC = W::NPOC, H = (K - 1) / 2;
  const int TX = RT ? TXr : REC_TX, TY = RT ? TYr : REC_TY;
  const int NT = RT ? (int)blockDim.x : REC_TX * REC_TY, RW = TX + 2 * H, RH = TY + 2 * H;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *raw = reinterpret_cast<T *>(smem_raw);        // [3][RH][RW]
  T *wsub = raw + 3 * RH * RW;                     // [NPOS][L][L]
  T *gpm = wsub + NPOS * L * L;                    // [NPOC][2][S]
  T *sig = gpm + NPOC * 2 * S;                     // [NPOC][2]
  T *bform = sig + NPOC * 2;                       // [L][L*L + L] Winv, row sums
  T *bcoef = bform + L * (L * L + L);              // [L][L][L][L]
  T *cq = bcoef + S * S;                           // [3][ME*ME][NT]
  const int p = blockIdx.z;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int vx = min(TX, N - i0), vy = min(TY, N - j0);
  for (int t = threadIdx.x; t < NPOS * L * L; t += blockDim.x) wsub[t] = wsub_g[t];
  for (int t = threadIdx.x; t < NPOC * 2 * S; t += blockDim.x) gpm[t] = gpm_g[t];
  for (int t = threadIdx.x; t < NPOC * 2; t += blockDim.x) sig[t] = sig_g[t];
  for (int t = threadIdx.x; t < L * (L * L + L); t += blockDim.x) bform[t] = bform_g[t];
  for (int t = threadIdx.x; t < S * S; t += blockDim.x) bcoef[t] = bcoef_g[t];
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
      if constexpr (TOPO) {
        if (v == 0) val += sext[((size_t)p * ne + (jj + H)) * ne + (ii + H)];
      }
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
  const T tau_scale = T(2) / (T(S + 1) * T(S));

#pragma unroll 1
  for (int v = 0; v < 3; ++v) {
    const T *Qv = raw + (v * RH + ty) * RW + tx;  // Q(r, c) = Qv[r * RW + c]
    // ---------------------------------------------------------------- beta (eq. 3.25)
    // on Q - q_c (beta ignores constants): Zx = Winv_x (Q - q_c) row-wise, then Winv_y.
    const T qc = Qv[H * RW + H];
    T f[S];
#pragma unroll
    for (int t = 0; t < S; ++t) f[t] = T(0);
#pragma unroll
    for (int sx = 0; sx < L; ++sx) {
      const T *Wx = bform + sx * (L * L + L);
#pragma unroll 1
      for (int kp = 0; kp < L; ++kp) {
        T Zx[K];
        const T rs = Wx[L * L + kp];
#pragma unroll
        for (int r = 0; r < K; ++r) {
          T s = -qc * rs;
#pragma unroll
          for (int a = 0; a < L; ++a) s = fma(Wx[kp * L + a], Qv[r * RW + sx + a], s);
          Zx[r] = s;
        }
#pragma unroll
        for (int sy = 0; sy < L; ++sy) {
          const T *Wy = bform + sy * (L * L + L);
#pragma unroll
          for (int k = 0; k < L; ++k) {
            T z = 0;
#pragma unroll
            for (int b = 0; b < L; ++b) z = fma(Wy[k * L + b], Zx[sy + b], z);
            const T c = bcoef[((sy * L + k) * L + sx) * L + kp];
            f[sy * L + sx] = fma(c * z, z, f[sy * L + sx]);
          }
        }
      }
    }
    // ---------------------------------------------------------------- tau (eq. 3.24), f
    T tsum = 0;
#pragma unroll
    for (int e = 0; e < S - 1; ++e)
#pragma unroll
      for (int ps = e + 1; ps < S; ++ps) tsum += fabs(f[ps] - f[e]);
    const T tau = tsum * tau_scale;
#pragma unroll
    for (int t = 0; t < S; ++t) f[t] = T(1) + tau / (f[t] + eps);
    // ---------------------------------------------------------------- points
#pragma unroll 1
    for (int t = 0; t < NPOS; ++t) {
      const int npt = t < 2 ? ME : ME + 2;
      const int g = t - 2;
      T Ap[ME + 2], Am[ME + 2];
#pragma unroll
      for (int jj = 0; jj < ME + 2; ++jj) Ap[jj] = Am[jj] = T(0);
#pragma unroll
      for (int sx = 0; sx < L; ++sx) {
        T Xc[K];
        const T *wx = wsub + (t * L + sx) * L;
#pragma unroll
        for (int r = 0; r < K; ++r) {
          T s = 0;
#pragma unroll
          for (int a = 0; a < L; ++a) s = fma(wx[a], Qv[r * RW + sx + a], s);
          Xc[r] = s;
        }
#pragma unroll
        for (int jj = 0; jj < ME + 2; ++jj) {
          if (jj < npt) {
            const int tyi = t < 2 ? 2 + jj : jj;
            const int pt = t < 2 ? t * ME + jj : (jj == 0 ? 2 * ME + g : (jj == 1 ? 3 * ME + g : 4 * ME + (jj - 2) * ME + g));
            const T *gp = gpm + pt * 2 * S;
#pragma unroll
            for (int sy = 0; sy < L; ++sy) {
              const T *wy = wsub + (tyi * L + sy) * L;
              T pv = 0;
#pragma unroll
              for (int b = 0; b < L; ++b) pv = fma(wy[b], Xc[sy + b], pv);
              const int ii = sy * L + sx;
              const T fp = f[ii] * pv;
              Ap[jj] = fma(gp[ii], fp, Ap[jj]);
              Am[jj] = fma(gp[S + ii], fp, Am[jj]);
            }
          }
        }
      }
#pragma unroll
      for (int jj = 0; jj < ME + 2; ++jj) {
        if (jj < npt) {
          const int pt = t < 2 ? t * ME + jj : (jj == 0 ? 2 * ME + g : (jj == 1 ? 3 * ME + g : 4 * ME + (jj - 2) * ME + g));
          const T *gp = gpm + pt * 2 * S;
          T Dp = 0, Dm = 0;
#pragma unroll
          for (int ii = 0; ii < S; ++ii) {
            Dp = fma(gp[ii], f[ii], Dp);
            Dm = fma(gp[S + ii], f[ii], Dm);
          }
          T val = sig[2 * pt] * Ap[jj] / Dp - sig[2 * pt + 1] * Am[jj] / Dm;
          if constexpr (TOPO) {
            if (v == 0)  // the depth: sqrtG phi_t minus the surface's TPP value at the point
              val -= t < 2 ? sep[((size_t)t * ME + jj) * pn + cell]
                           : (jj < 2 ? sep[((size_t)(2 + jj) * ME + g) * pn + cell]
                                     : scp[((size_t)(jj - 2) * ME + g) * pn + cell]);
          }
          if (t < 2) {
            ep[((size_t)(t * 3 + v) * ME + jj) * pn + cell] = val;
          } else if (jj < 2) {
            ep[((size_t)((2 + jj) * 3 + v) * ME + g) * pn + cell] = val;
          } else {
            cq[(v * ME * ME + (jj - 2) * ME + g) * NT + tid] = val;
          }
        }
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
      const T sl = fc0 + fc1 * X + fc2 * Y;
      const T rq = rcp(q0);
      const T XY = X * Y, X2 = X * X, Y2 = Y * Y;
      const T os = omega * sl;
      T a1 = (-XY * Y * q1 + Y * (T(1) + Y2) * q2) * q1 * rq + os * (-XY * q1 + (T(1) + Y2) * q2);
      T a2 = (X * (T(1) + X2) * q1 - X2 * Y * q2) * q2 * rq + os * (-(T(1) + X2) * q1 + XY * q2);
      s1 = fma(tw, a1, s1);
      s2 = fma(tw, a2, s2);
    }
  }
  sb[cell] = s1;
  sb[pn + cell] = s2;
}

template <typename T, int K>
int launch_recon_weno(hope_ctx *ctx, Grid &g, const T *qs, cudaStream_t st);

template <typename T, int K>
int weno_set_smem_attr();

template <typename T, int K>
int launch_recon_weno_adj(hope_ctx *ctx, Grid &g, const T *qs, const T *lamL, cudaStream_t st);

}  // namespace hope

namespace hope {

// ---------------------------------------------------------------------------------
// WENO2D reconstruction + sources adjoint: per cell, recomputes the forward (indicators,
// nonlinear weights, cell-point values), applies the source VJP at the cell points, then
// back-propagates every point's adjoint through the WENO combination, the nonlinear
// weights (eqs. 3.22-3.24; d|x|/dx = sign(x), 0 at 0), the indicators (eq. 3.25) and the
// sub-stencil reconstructions into grad[v][b*K + a][cell] (the cell's own slice, no
// atomics).
// ---------------------------------------------------------------------------------
template <typename T, int K>
struct WenoAdjShape {
  static constexpr size_t smem_elems() {
    using W = WenoShape<T, K>;
    // + adjoint at the cell points + each thread's k x k stencil gradient
    return W::smem_elems() + 3 * W::ME * W::ME * W::NT + K * K * W::NT;
  }
};

template <typename T, int K>
__device__ __forceinline__ void weno_indicators(const T *Qv, const T *bform, const T *bcoef, T *beta) {
  constexpr int L = (K + 1) / 2, S = L * L, H = (K - 1) / 2, RW = Shape<K>::RW;
  const T qc = Qv[H * RW + H];
#pragma unroll
  for (int t = 0; t < S; ++t) beta[t] = T(0);
#pragma unroll
  for (int sx = 0; sx < L; ++sx) {
    const T *Wx = bform + sx * (L * L + L);
#pragma unroll 1
    for (int kp = 0; kp < L; ++kp) {
      T Zx[K];
      const T rs = Wx[L * L + kp];
#pragma unroll
      for (int r = 0; r < K; ++r) {
        T s = -qc * rs;
#pragma unroll
        for (int a = 0; a < L; ++a) s = fma(Wx[kp * L + a], Qv[r * RW + sx + a], s);
        Zx[r] = s;
      }
#pragma unroll
      for (int sy = 0; sy < L; ++sy) {
        const T *Wy = bform + sy * (L * L + L);
#pragma unroll
        for (int k = 0; k < L; ++k) {
          T z = 0;
#pragma unroll
          for (int b = 0; b < L; ++b) z = fma(Wy[k * L + b], Zx[sy + b], z);
          beta[sy * L + sx] = fma(bcoef[((sy * L + k) * L + sx) * L + kp] * z, z, beta[sy * L + sx]);
        }
      }
    }
  }
}

// TOPO: over a surface the forward reconstructed sqrtG phi_t (sext added to the mass
// variable's tile) and subtracted the surface's TPP values at the points; the recomputed
// cell-point depths do the same (scp), the derivatives are those at the shifted tile.
template <typename T, int K, bool TOPO = false>
__global__ void __launch_bounds__(REC_TX *REC_TY)
    k_recon_weno_adj(const T *__restrict__ q, const T *__restrict__ gext, const T *__restrict__ wsub_g,
                     const T *__restrict__ gpm_g, const T *__restrict__ sig_g, const T *__restrict__ bform_g,
                     const T *__restrict__ bcoef_g, const T *__restrict__ Xg, const T *__restrict__ t1w,
                     const T *__restrict__ lep, const T *__restrict__ lamL, T *__restrict__ grad, int N, int ne,
                     T omega, FCoef<T> fc, T eps, const T *__restrict__ sext = nullptr,
                     const T *__restrict__ scp = nullptr) {
  using W = WenoShape<T, K>;
  using SH = Shape<K>;
  constexpr int L = W::L, S = W::S, ME = W::ME, NPOS = W::NPOS, NPOC = W::NPOC, NT = W::NT, RW = SH::RW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *raw = reinterpret_cast<T *>(smem_raw);
  T *wsub = raw + 3 * SH::RH * SH::RW;
  T *gpm = wsub + NPOS * L * L;
  T *sig = gpm + NPOC * 2 * S;
  T *bform = sig + NPOC * 2;
  T *bcoef = bform + L * (L * L + L);
  T *cq = bcoef + S * S;       // [3][ME*ME][NT] forward values at the cell points
  T *lcq = cq + 3 * ME * ME * NT;  // [3][ME*ME][NT] adjoint at the cell points
  T *gsm = lcq + 3 * ME * ME * NT;  // [K*K][NT] stencil gradient of the current variable
  const int p = blockIdx.z;
  const int i0 = blockIdx.x * REC_TX, j0 = blockIdx.y * REC_TY;
  for (int t = threadIdx.x; t < NPOS * L * L; t += blockDim.x) wsub[t] = wsub_g[t];
  for (int t = threadIdx.x; t < NPOC * 2 * S; t += blockDim.x) gpm[t] = gpm_g[t];
  for (int t = threadIdx.x; t < NPOC * 2; t += blockDim.x) sig[t] = sig_g[t];
  for (int t = threadIdx.x; t < L * (L * L + L); t += blockDim.x) bform[t] = bform_g[t];
  for (int t = threadIdx.x; t < S * S; t += blockDim.x) bcoef[t] = bcoef_g[t];
  load_tile<T, K>(raw, q, gext, p, i0, j0, N, ne);
  if constexpr (TOPO) {
    __syncthreads();
    constexpr int H = (K - 1) / 2;
    for (int idx = threadIdx.x; idx < SH::RH * SH::RW; idx += blockDim.x) {
      const int r = idx / SH::RW, c = idx - r * SH::RW;
      const int ii = i0 + c - H, jj = j0 + r - H;
      if (ii >= -H && ii < N + H && jj >= -H && jj < N + H) raw[idx] += sext[((size_t)p * ne + (jj + H)) * ne + (ii + H)];
    }
  }
  __syncthreads();
  const int tid = threadIdx.x;
  const int tx = tid % REC_TX, ty = tid / REC_TX;
  const int i = i0 + tx, j = j0 + ty;
  if (i >= N || j >= N) return;
  const size_t pn = (size_t)6 * N * N;
  const size_t cell = ((size_t)p * N + j) * N + i;
  const T tau_scale = T(2) / (T(S + 1) * T(S));
  auto ptidx = [](int t, int jj) -> int {
    const int g = t - 2;
    return t < 2 ? t * ME + jj : (jj == 0 ? 2 * ME + g : (jj == 1 ? 3 * ME + g : 4 * ME + (jj - 2) * ME + g));
  };
  // ---------------- phase A: forward values at the cell points (all variables)
#pragma unroll 1
  for (int v = 0; v < 3; ++v) {
    const T *Qv = raw + (v * SH::RH + ty) * SH::RW + tx;
    T f[S];
    weno_indicators<T, K>(Qv, bform, bcoef, f);
    T tsum = 0;
#pragma unroll
    for (int e = 0; e < S - 1; ++e)
#pragma unroll
      for (int ps = e + 1; ps < S; ++ps) tsum += fabs(f[ps] - f[e]);
    const T tau = tsum * tau_scale;
#pragma unroll
    for (int t = 0; t < S; ++t) f[t] = T(1) + tau / (f[t] + eps);
#pragma unroll 1
    for (int g = 0; g < ME; ++g) {
      const int t = 2 + g;
      T Ap[ME], Am[ME];
#pragma unroll
      for (int h = 0; h < ME; ++h) Ap[h] = Am[h] = T(0);
#pragma unroll
      for (int sx = 0; sx < L; ++sx) {
        T Xc[K];
        const T *wx = wsub + (t * L + sx) * L;
#pragma unroll
        for (int r = 0; r < K; ++r) {
          T s = 0;
#pragma unroll
          for (int a = 0; a < L; ++a) s = fma(wx[a], Qv[r * RW + sx + a], s);
          Xc[r] = s;
        }
#pragma unroll
        for (int h = 0; h < ME; ++h) {
          const T *gp = gpm + (4 * ME + h * ME + g) * 2 * S;
#pragma unroll
          for (int sy = 0; sy < L; ++sy) {
            const T *wy = wsub + ((2 + h) * L + sy) * L;
            T pv = 0;
#pragma unroll
            for (int b = 0; b < L; ++b) pv = fma(wy[b], Xc[sy + b], pv);
            const int ii = sy * L + sx;
            const T fp = f[ii] * pv;
            Ap[h] = fma(gp[ii], fp, Ap[h]);
            Am[h] = fma(gp[S + ii], fp, Am[h]);
          }
        }
      }
#pragma unroll
      for (int h = 0; h < ME; ++h) {
        const int pt = 4 * ME + h * ME + g;
        const T *gp = gpm + pt * 2 * S;
        T Dp = 0, Dm = 0;
#pragma unroll
        for (int ii = 0; ii < S; ++ii) {
          Dp = fma(gp[ii], f[ii], Dp);
          Dm = fma(gp[S + ii], f[ii], Dm);
        }
        T val = sig[2 * pt] * Ap[h] / Dp - sig[2 * pt + 1] * Am[h] / Dm;
        if constexpr (TOPO) {
          if (v == 0) val -= scp[((size_t)h * ME + g) * pn + cell];
        }
        cq[(v * ME * ME + h * ME + g) * NT + tid] = val;
      }
    }
  }
  // ---------------- phase B: source adjoint at the cell points
  {
    const T fc0 = fc.c[3 * p], fc1 = fc.c[3 * p + 1], fc2 = fc.c[3 * p + 2];
    const T lS1 = lamL[pn + cell], lS2 = lamL[2 * pn + cell];
#pragma unroll 1
    for (int h = 0; h < ME; ++h) {
      const T Y = Xg[j * ME + h];
#pragma unroll 1
      for (int g = 0; g < ME; ++g) {
        const T X = Xg[i * ME + g];
        T qv[3], lq[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) qv[v] = cq[(v * ME * ME + h * ME + g) * NT + tid];
        const T tw = t1w[(((size_t)j * N + i) * ME + h) * ME + g];
        const T os = omega * (fc0 + fc1 * X + fc2 * Y);
        source_vjp(qv, X, Y, os, tw, lS1, lS2, lq);
#pragma unroll
        for (int v = 0; v < 3; ++v) lcq[(v * ME * ME + h * ME + g) * NT + tid] = lq[v];
      }
    }
  }
  // ---------------- phase C: per variable, back through WENO into the stencil gradient
  // (accumulated in the thread's shared-memory slice gs[t * NT], written out once)
  T *gs = gsm + tid;
#pragma unroll 1
  for (int v = 0; v < 3; ++v) {
    const T *Qv = raw + (v * SH::RH + ty) * SH::RW + tx;
    T *gv = grad + (size_t)v * K * K * pn + cell;  // gv[(b*K + a) * pn]
#pragma unroll 1
    for (int t = 0; t < K * K; ++t) gs[t * NT] = T(0);
    T beta[S], f[S], lf[S];
    weno_indicators<T, K>(Qv, bform, bcoef, beta);
    T tsum = 0;
#pragma unroll
    for (int e = 0; e < S - 1; ++e)
#pragma unroll
      for (int ps = e + 1; ps < S; ++ps) tsum += fabs(beta[ps] - beta[e]);
    const T tau = tsum * tau_scale;
#pragma unroll
    for (int t = 0; t < S; ++t) {
      f[t] = T(1) + tau / (beta[t] + eps);
      lf[t] = T(0);
    }
#pragma unroll 1
    for (int t = 0; t < NPOS; ++t) {
      const int npt = t < 2 ? ME : ME + 2;
      const int g = t - 2;
      // per point: denominators D+-, the point's adjoint lv and those of A+- (which need
      // no forward sums); A+- themselves are summed in the same sweep as their adjoints
      T Ap[ME + 2], Am[ME + 2], Dp[ME + 2], Dm[ME + 2], lAp[ME + 2], lAm[ME + 2], lv[ME + 2];
#pragma unroll
      for (int jj = 0; jj < ME + 2; ++jj) {
        Ap[jj] = Am[jj] = lAp[jj] = lAm[jj] = lv[jj] = T(0);
        Dp[jj] = Dm[jj] = T(1);
        if (jj < npt) {
          const int pt = ptidx(t, jj);
          const T *gp = gpm + pt * 2 * S;
          T dp = 0, dm = 0;
#pragma unroll
          for (int ii = 0; ii < S; ++ii) {
            dp = fma(gp[ii], f[ii], dp);
            dm = fma(gp[S + ii], f[ii], dm);
          }
          Dp[jj] = dp;
          Dm[jj] = dm;
          if (t < 2)
            lv[jj] = lep[((size_t)(t * 3 + v) * ME + jj) * pn + cell];
          else if (jj < 2)
            lv[jj] = lep[((size_t)((2 + jj) * 3 + v) * ME + g) * pn + cell];
          else
            lv[jj] = lcq[(v * ME * ME + (jj - 2) * ME + g) * NT + tid];
          lAp[jj] = sig[2 * pt] / dp * lv[jj];
          lAm[jj] = -sig[2 * pt + 1] / dm * lv[jj];
        }
      }
      // one sweep over the sub-stencil values p_i(pt): forward sums A+- and the
      // p-dependent adjoints (-> lf and the stencil gradient)
#pragma unroll
      for (int sx = 0; sx < L; ++sx) {
        T Xc[K], lXc[K];
        const T *wx = wsub + (t * L + sx) * L;
#pragma unroll
        for (int r = 0; r < K; ++r) {
          T s = 0;
#pragma unroll
          for (int a = 0; a < L; ++a) s = fma(wx[a], Qv[r * RW + sx + a], s);
          Xc[r] = s;
          lXc[r] = T(0);
        }
#pragma unroll
        for (int jj = 0; jj < ME + 2; ++jj) {
          if (jj < npt) {
            const int tyi = t < 2 ? 2 + jj : jj;
            const T *gp = gpm + ptidx(t, jj) * 2 * S;
#pragma unroll
            for (int sy = 0; sy < L; ++sy) {
              const T *wy = wsub + (tyi * L + sy) * L;
              T pv = 0;
#pragma unroll
              for (int b = 0; b < L; ++b) pv = fma(wy[b], Xc[sy + b], pv);
              const int ii = sy * L + sx;
              const T fp = f[ii] * pv;
              Ap[jj] = fma(gp[ii], fp, Ap[jj]);
              Am[jj] = fma(gp[S + ii], fp, Am[jj]);
              const T gl = gp[ii] * lAp[jj] + gp[S + ii] * lAm[jj];
              lf[ii] = fma(gl, pv, lf[ii]);
              const T lp = gl * f[ii];
#pragma unroll
              for (int b = 0; b < L; ++b) lXc[sy + b] = fma(wy[b], lp, lXc[sy + b]);
            }
          }
        }
#pragma unroll
        for (int r = 0; r < K; ++r)
#pragma unroll
          for (int a = 0; a < L; ++a) gs[(r * K + sx + a) * NT] += wx[a] * lXc[r];
      }
      // adjoints of D+- (they need A+-), through dD+-/df_i = gamma+-_i
#pragma unroll
      for (int jj = 0; jj < ME + 2; ++jj) {
        if (jj < npt) {
          const int pt = ptidx(t, jj);
          const T *gp = gpm + pt * 2 * S;
          const T lDp = -sig[2 * pt] * Ap[jj] / (Dp[jj] * Dp[jj]) * lv[jj];
          const T lDm = sig[2 * pt + 1] * Am[jj] / (Dm[jj] * Dm[jj]) * lv[jj];
#pragma unroll
          for (int ii = 0; ii < S; ++ii) lf[ii] = fma(gp[ii], lDp, fma(gp[S + ii], lDm, lf[ii]));
        }
      }
    }
    // f_i = 1 + tau / (beta_i + eps)
    T ltau = 0;
#pragma unroll
    for (int ii = 0; ii < S; ++ii) {
      const T ib = T(1) / (beta[ii] + eps);
      ltau = fma(lf[ii], ib, ltau);
      lf[ii] = -lf[ii] * tau * ib * ib;  // now d/d beta_i (direct part)
    }
    // tau = ts sum_{e<p} |beta_p - beta_e|
    const T lt = ltau * tau_scale;
#pragma unroll
    for (int e = 0; e < S - 1; ++e)
#pragma unroll
      for (int ps = e + 1; ps < S; ++ps) {
        const T d = beta[ps] - beta[e];
        const T sgn = d > T(0) ? T(1) : (d < T(0) ? T(-1) : T(0));
        lf[ps] += lt * sgn;
        lf[e] -= lt * sgn;
      }
    // beta = sum c z^2 on Q - q_c
    const T qc = Qv[SH::H * RW + SH::H];
    T lqc = 0;
#pragma unroll
    for (int sx = 0; sx < L; ++sx) {
      const T *Wx = bform + sx * (L * L + L);
#pragma unroll 1
      for (int kp = 0; kp < L; ++kp) {
        T Zx[K], lZx[K];
        const T rs = Wx[L * L + kp];
#pragma unroll
        for (int r = 0; r < K; ++r) {
          T s = -qc * rs;
#pragma unroll
          for (int a = 0; a < L; ++a) s = fma(Wx[kp * L + a], Qv[r * RW + sx + a], s);
          Zx[r] = s;
          lZx[r] = T(0);
        }
#pragma unroll
        for (int sy = 0; sy < L; ++sy) {
          const T *Wy = bform + sy * (L * L + L);
#pragma unroll
          for (int k = 0; k < L; ++k) {
            T z = 0;
#pragma unroll
            for (int b = 0; b < L; ++b) z = fma(Wy[k * L + b], Zx[sy + b], z);
            const T lz = T(2) * bcoef[((sy * L + k) * L + sx) * L + kp] * z * lf[sy * L + sx];
#pragma unroll
            for (int b = 0; b < L; ++b) lZx[sy + b] = fma(Wy[k * L + b], lz, lZx[sy + b]);
          }
        }
#pragma unroll
        for (int r = 0; r < K; ++r) {
          lqc -= rs * lZx[r];
#pragma unroll
          for (int a = 0; a < L; ++a) gs[(r * K + sx + a) * NT] += Wx[kp * L + a] * lZx[r];
        }
      }
    }
    gs[(SH::H * K + SH::H) * NT] += lqc;
#pragma unroll 1
    for (int t = 0; t < K * K; ++t) gv[(size_t)t * pn] = gs[t * NT];
  }
}

}  // namespace hope
