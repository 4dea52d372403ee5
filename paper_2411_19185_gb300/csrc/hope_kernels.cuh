// hope_kernels.cuh -- per-stage kernels of the HOPE cubed-sphere shallow-water core
// (arXiv 2411.19185) for sm_103a, templated on the element type T (double / float)
// and the stencil width K.
//
// One stage L(q) = dq/dt runs as
//   k_ghost      ghost ring = G q                       (appendix eq. 7.12)
//   k_recon_tpp  per tile: x-pass / y-pass sum-factorised TPP reconstruction at the
//                4 me edge points and me^2 cell points (eqs. 3.14-3.15, R = r_x (x) r_y),
//                edge points to global, cell-point sources quadrature (eqs. 2.2, 2.3, 3.6)
//   k_flux       LMARS at every edge Gauss point (eqs. 3.30-3.38) + edge quadrature
//                (eq. 3.5); panel-boundary edges once per cube edge with the
//                conversions of eqs. 3.26-3.29
//   k_update     flux difference + sources (eq. 3.1) fused with the RK stage combination
#pragma once
#include <cuda_runtime.h>

#include <cstring>
#include <stdint.h>

#include "../../include/hope.h"

namespace hope {

template <typename T>
struct Acc;  // edge/tendency accumulator: plain in FP64, compensated (TwoSum) in FP32

template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    float t = s + x;
    float bp = t - s;
    c += (s - (t - bp)) + (x - bp);  // Knuth TwoSum error term
    s = t;
  }
  __device__ __forceinline__ float value() const { return s + c; }
};

template <typename T>
__device__ __forceinline__ T rcp(T x) { return T(1) / x; }
// FP32 path: the PTX approximate reciprocal and square root (about 1 ulp) instead of the
// correctly rounded multi-instruction sequences; their error is of the order of the FP32
// rounding already in every value (inputs are normal, positive geopotentials and masses).
template <>
__device__ __forceinline__ float rcp<float>(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <typename T>
__device__ __forceinline__ T sqrt_pos(T x) { return sqrt(x); }
template <>
__device__ __forceinline__ float sqrt_pos<float>(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Programmatic dependent launch: the four per-grid stage kernels are launched with
// programmatic stream serialization, so each can be scheduled while its predecessor in the
// stream drains.  Each calls griddep_wait() before its first memory access; the wait returns
// once the preceding grid has completed and its writes are visible (at once when the kernel
// was launched without the attribute), so the kernels see exactly what a serial launch sees.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Coriolis coefficients per panel: sin(latitude about the rotation axis) * delta
// = c0 + c1 X + c2 Y (eq. 2.5 for an untilted axis: Y, 1 or -1).
template <typename T>
struct FCoef {
  T c[18];
};

// ---------------------------------------------------------------------------------
// Ghost fill: one warp per ghost cell, lanes stride over the row's nonzeros.
// ---------------------------------------------------------------------------------
// FP64 -> FP32 by truncating the significand with integer operations, so the FP32 tail
// of the ghost rows costs no FP64-pipe conversion.  Values outside the normal FP32 range
// become 0 (below it) or +-inf (above it, NaN included); the tail's weights are below
// 1e-9 of their row's largest, so truncation (2^-23 relative) is far below FP64 rounding.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int e = (int)((hi >> 20) & 0x7FFu) - (1023 - 127);
  const unsigned sign = hi & 0x80000000u;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

// (v, r, c) of the items threadIdx.x, threadIdx.x + blockDim.x, ... of a 3 x h x w box (c
// fastest), advanced by carries: the block stride is split once into (sv, sr, sc), and each
// component carries at most one into the next, so no item costs an integer division.
struct BoxWalk {
  int v, r, c, sv, sr, sc, h, w;
  __device__ __forceinline__ BoxWalk(int h_, int w_) : h(h_), w(w_) {
    const int hw = h * w, s = (int)threadIdx.x, d = (int)blockDim.x;
    v = s / hw;
    r = (s - v * hw) / w;
    c = s - v * hw - r * w;
    sv = d / hw;
    sr = (d - sv * hw) / w;
    sc = d - sv * hw - sr * w;
  }
  __device__ __forceinline__ void next() {
    c += sc;
    r += sr;
    v += sv;
    if (c >= w) {
      c -= w;
      ++r;
    }
    if (r >= h) {
      r -= h;
      ++v;
    }
  }
};

// Cube symmetry of the ghost operator (eq. 7.12 with the mean-at-tie reading): row r is
// the image of a panel-0 row under a rotation of the cube, so it reuses that row's weights
// (gsym[r] low bits) with its own columns.  Momentum components go through 2x2 signed
// permutations: each column carries the code of v = M^T u (bits 28-30: swap, negate the
// first, negate the second), the row the code of g = M s (gsym[r] bits 28-30).
// (integer selects and sign-bit flips: no FP64-pipe instruction)
__device__ __forceinline__ void sym_apply(int code, double &x, double &y) {
  const long long a = __double_as_longlong(x), b = __double_as_longlong(y);
  const long long s1 = (code & 1) ? b : a, s2 = (code & 1) ? a : b;
  x = __longlong_as_double(s1 ^ ((long long)((code >> 1) & 1) << 63));
  y = __longlong_as_double(s2 ^ ((long long)((code >> 2) & 1) << 63));
}
__device__ __forceinline__ void sym_apply(int code, float &x, float &y) {
  const int a = __float_as_int(x), b = __float_as_int(y);
  const int s1 = (code & 1) ? b : a, s2 = (code & 1) ? a : b;
  x = __int_as_float(s1 ^ (int)((unsigned)((code >> 1) & 1) << 31));
  y = __int_as_float(s2 ^ (int)((unsigned)((code >> 2) & 1) << 31));
}

// Layout of the ghost-operator weights: FP32 contexts store five planes [5][entries]
// (a warp's load of one weight over 32 consecutive entries reads one contiguous run, which
// relieves the L1 of the FP32 kernels); FP64 contexts keep [entries][5] for the head and
// the FP32 tail (their kernels wait on the FP64 pipe, and one base address per entry
// measured faster there).
template <typename T>
constexpr bool GHOST_PLANES = sizeof(T) == 4;

// End of a ghost row: a reduce-scatter of the lanes' partial sums s0, s1, s2.  The
// half-warps exchange the variables they do not keep (lanes 0-15 keep s0, s1; lanes 16-31
// keep s2 and a zero), the 8-lane groups likewise, and each group sums its variable: lanes
// 0, 8, 16 end with the row's s0, s1, s2 (6 additions a lane instead of 15 for three
// butterflies) and store them at ring position dst of the three variables.
template <typename T>
__device__ __forceinline__ void ghost_reduce_store(int lane, T s0, T s1, T s2, T *__restrict__ gext, size_t pe,
                                                   int dst) {
  const bool hi16 = lane & 16, hi8 = lane & 8;
  T ka = hi16 ? s2 : s0, kb = hi16 ? T(0) : s1;
  const T xa = hi16 ? s0 : s2, xb = hi16 ? s1 : T(0);
  ka += __shfl_xor_sync(0xffffffffu, xa, 16);
  kb += __shfl_xor_sync(0xffffffffu, xb, 16);
  T v = hi8 ? kb : ka;
  v += __shfl_xor_sync(0xffffffffu, hi8 ? ka : kb, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((lane & 7) == 0 && lane < 24) gext[(size_t)(lane >> 3) * pe + dst] = v;
}

// One ghost row: FP64/FP32 head sum in the context precision, plus (FP64 contexts) the
// FP32 tail of negligible weights.  SYM: weights of the row's representative with the
// symmetry transforms (the weights stay in L2); otherwise the row's own weights (every
// row holds the same values in its own order) and no transforms.
constexpr int GHOST_UNROLL = 4;

template <typename T, bool SYM = true>
__device__ __forceinline__ void ghost_row(int row, int lane, const T *__restrict__ q, T *__restrict__ gext,
                                          const int *__restrict__ grow, const int *__restrict__ gcol,
                                          const T *__restrict__ gval, const int *__restrict__ gdst,
                                          const int *__restrict__ gsym, const int *__restrict__ trow,
                                          const int *__restrict__ tcol, const float *__restrict__ tval, int N,
                                          int ne, size_t gs) {
  size_t pn = (size_t)6 * N * N, pe = (size_t)6 * ne * ne;
  const int info = SYM ? gsym[row] : row;
  const int wrow = info & 0x0FFFFFFF, ocode = info >> 28;
  // GHOST_UNROLL nonzeros per lane in flight: all their loads are issued before the FMAs,
  // so a lane waits for one round of (index, gather) latencies per GHOST_UNROLL entries.
  // Each lane still adds its entries in increasing order.
  constexpr int U = GHOST_UNROLL;
  const int b = grow[row], e = grow[row + 1];
  const int wb = grow[wrow];  // entry t of this row uses the weights of entry wb + (t - b)
  T s0 = 0, s1 = 0, s2 = 0;
  for (int t0 = b + lane; t0 < e; t0 += 32 * U) {
    int c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) c[u] = t0 + 32 * u < e ? gcol[t0 + 32 * u] : -1;
    T a[U][3], w[U][5];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = c[u] >= 0;
      const int cc = ok ? (c[u] & 0x0FFFFFFF) : 0;
      const size_t we = (size_t)(wb + (ok ? t0 + 32 * u - b : 0));
      const T *wp = gval + (GHOST_PLANES<T> ? we : 5 * we);
      a[u][0] = q[cc];
      a[u][1] = q[pn + cc];
      a[u][2] = q[2 * pn + cc];
      if (SYM) sym_apply(ok ? c[u] >> 28 : 0, a[u][1], a[u][2]);
#pragma unroll
      for (int k = 0; k < 5; ++k) w[u][k] = ok ? wp[GHOST_PLANES<T> ? k * gs : k] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      s0 = fma(w[u][0], a[u][0], s0);
      s1 = fma(w[u][1], a[u][1], fma(w[u][2], a[u][2], s1));
      s2 = fma(w[u][3], a[u][1], fma(w[u][4], a[u][2], s2));
    }
  }
  if constexpr (sizeof(T) == 8) {
    if (trow) {
      float f0 = 0.f, f1 = 0.f, f2 = 0.f;
      const int tb = trow[row], te = trow[row + 1];
      const int twb = trow[wrow];
      for (int t0 = tb + lane; t0 < te; t0 += 32 * U) {
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) c[u] = t0 + 32 * u < te ? tcol[t0 + 32 * u] : -1;
        float a[U][3], w[U][5];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool ok = c[u] >= 0;
          const int cc = ok ? (c[u] & 0x0FFFFFFF) : 0;
          const float *wp = tval + (size_t)(twb + (ok ? t0 + 32 * u - tb : 0)) * 5;
          a[u][0] = f64_to_f32_trunc(q[cc]);
          a[u][1] = f64_to_f32_trunc(q[pn + cc]);
          a[u][2] = f64_to_f32_trunc(q[2 * pn + cc]);
          if (SYM) sym_apply(ok ? c[u] >> 28 : 0, a[u][1], a[u][2]);
#pragma unroll
          for (int k = 0; k < 5; ++k) w[u][k] = ok ? wp[k] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          f0 = fmaf(w[u][0], a[u][0], f0);
          f1 = fmaf(w[u][1], a[u][1], fmaf(w[u][2], a[u][2], f1));
          f2 = fmaf(w[u][3], a[u][1], fmaf(w[u][4], a[u][2], f2));
        }
      }
      s0 += (T)f0;
      s1 += (T)f1;
      s2 += (T)f2;
    }
  }
  // the row's output transform is a signed permutation (exact), so it is applied to each
  // lane's partial sums
  if (SYM) sym_apply(ocode, s1, s2);
  ghost_reduce_store(lane, s0, s1, s2, gext, pe, gdst[row]);
}

template <typename T>
__global__ void __launch_bounds__(256, 4) k_ghost(const T *__restrict__ q, T *__restrict__ gext,
                                               const int *__restrict__ grow, const int *__restrict__ gcol,
                                               const T *__restrict__ gval, const int *__restrict__ gdst,
                                               const int *__restrict__ gsym, const int *__restrict__ trow,
                                               const int *__restrict__ tcol, const float *__restrict__ tval,
                                               int rows, int N, int ne, size_t gs) {
  griddep_wait();
  // grid of resident blocks; warps stride over the rows so every SM gets an equal share
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += nwarps)
    ghost_row(row, threadIdx.x & 31, q, gext, grow, gcol, gval, gdst, gsym, trow, tcol, tval, N, ne, gs);
}

// ---------------------------------------------------------------------------------
// TPP reconstruction + cell-point sources.  Block = TX x TY cells of one panel.
// ---------------------------------------------------------------------------------
constexpr int REC_TX = 16;
constexpr int REC_TY = 8;

template <int K, int TX = REC_TX, int TY = REC_TY>
struct Tile {
  static constexpr int H = (K - 1) / 2;
  static constexpr int ME = (K + 1) / 2;
  static constexpr int NPOS = ME + 2;  // x-pass evaluation positions
  static constexpr int RW = TX + 2 * H;
  static constexpr int RH = TY + 2 * H;
  static constexpr int NT = TX * TY;
};

template <int K>
using Shape = Tile<K, REC_TX, REC_TY>;

template <typename T, int K, int TX = REC_TX, int TY = REC_TY>
__host__ __device__ constexpr size_t recon_smem_bytes() {
  using S = Tile<K, TX, TY>;
  return sizeof(T) * (3 * S::RH * S::RW + 3 * S::NPOS * S::RH * TX + S::NPOS * K);
}

// Load the extended tile of the 3 variables: interior cells from q, ring cells from gext.
template <typename T, int K, int TX = REC_TX, int TY = REC_TY>
__device__ __forceinline__ void load_tile(T *raw, const T *__restrict__ q, const T *__restrict__ gext,
                                          int p, int i0, int j0, int N, int ne) {
  using S = Tile<K, TX, TY>;
  size_t pn = (size_t)6 * N * N, pe = (size_t)6 * ne * ne;
  for (int idx = threadIdx.x; idx < 3 * S::RH * S::RW; idx += blockDim.x) {
    int v = idx / (S::RH * S::RW);
    int rem = idx - v * S::RH * S::RW;
    int r = rem / S::RW, c = rem - r * S::RW;
    int i = i0 + c - S::H, j = j0 + r - S::H;
    T val = T(0);
    if (i >= 0 && i < N && j >= 0 && j < N)
      val = q[v * pn + ((size_t)p * N + j) * N + i];
    else if (i >= -S::H && i < N + S::H && j >= -S::H && j < N + S::H)
      val = gext[v * pe + ((size_t)p * ne + (j + S::H)) * ne + (i + S::H)];
    raw[idx] = val;
  }
}

// Shared memory of one TPP reconstruction tile of TX x TY cells (runtime shape).
template <typename T, int K>
__host__ __device__ constexpr size_t recon_tile_smem_bytes(int TX, int TY) {
  return sizeof(T) * (3 * (TY + K - 1) * (TX + K - 1) + 3 * ((K + 1) / 2 + 2) * (TY + K - 1) * TX + ((K + 1) / 2 + 2) * K);
}

// Largest thread count of a TPP reconstruction block (one thread per cell of the tile).
constexpr int REC_MAX_THREADS = 512;

// Mirror pairs of evaluation positions (t = 0: xi = -1/2, 1: +1/2, 2 + g: Gauss node g,
// ascending): pair 0 is the two edges, pair 1 + g (g < me/2) the nodes g and me-1-g, and
// for odd me the last pair is the middle node alone.  Their weights follow the point
// weights in the w1 table (see k_setup_order).
template <int K>
struct MirrorPairs {
  static constexpr int H = (K - 1) / 2, ME = (K + 1) / 2, NPOS = ME + 2;
  static constexpr int NPAIR = 1 + (ME + 1) / 2;
  static constexpr bool ODD = ME & 1;
  __host__ __device__ static constexpr int minus(int pi) { return pi == 0 ? 0 : 1 + pi; }
  __host__ __device__ static constexpr int plus(int pi) { return pi == 0 ? 1 : 2 + ME - pi; }
};

// Fold a line of K values in place: x[b] = x[b] + x[K-1-b], x[K-1-b] = x[b] - x[K-1-b].
template <typename T, int K>
__device__ __forceinline__ void mirror_fold(T *x) {
#pragma unroll
  for (int b = 0; b < (K - 1) / 2; ++b) {
    const T s = x[b] + x[K - 1 - b], d = x[b] - x[K - 1 - b];
    x[b] = s;
    x[K - 1 - b] = d;
  }
}

// Even and odd parts of one pair's value on a folded line: p(+xi) = E + O, p(-xi) = E - O.
template <typename T, int K>
__device__ __forceinline__ void mirror_eval(const T *w, const T *x, T &E, T &O) {
  constexpr int H = (K - 1) / 2;
  E = w[H] * x[H];
  O = w[H + 1] * x[H + 1];
#pragma unroll
  for (int b = 0; b < H; ++b) E = fma(w[b], x[b], E);
#pragma unroll
  for (int b = H + 2; b < K; ++b) O = fma(w[b], x[b], O);
}

// Mirror-pair weights of order K passed by value: a kernel parameter lives in the constant
// bank, so the reconstruction's multiply-adds take the weights as constant operands instead
// of loading each one from shared memory (the weights depend on k alone).
template <typename T, int K>
struct PairW {
  T w[MirrorPairs<K>::NPAIR * K];
};

// The mirror-pair rows of a host copy of the 1-D weight table (point rows first).
template <typename T, int K>
inline PairW<T, K> pair_weights(const unsigned char *w1_host) {
  PairW<T, K> pw;
  memcpy(pw.w, w1_host + sizeof(T) * MirrorPairs<K>::NPOS * K, sizeof(pw.w));
  return pw;
}

// One tile of at most TX x TY cells of panel p with its first cell at (i0, j0); called by
// all threads of a block of at least TX*TY threads; ends with a barrier so the shared
// memory can be reused for the next tile.  Tiles cut by the panel's edge only load,
// sweep and evaluate their vx x vy valid cells, and the cell phase packs those cells onto
// the first vx*vy threads so the idle warps of a ragged tile issue nothing.
// TOPO (bottom topography, single spheres): psi_B of eq. 2.14, an affine map of the cell's
// k x k depth stencil (weights ttw[2][k*k][cells], constants ttb[2][cells]), is added to the
// sources from the tile already in shared memory.
template <typename T, int K, bool TOPO = false>
__device__ __forceinline__ void recon_tpp_tile(unsigned char *smem_raw, int p, int i0, int j0, const int TX,
                                               const int TY, const T *__restrict__ q, const T *__restrict__ gext,
                                               const T *w1p, const T *__restrict__ Xg,
                                               const T *__restrict__ t1w, const T *__restrict__ src8,
                                               T *__restrict__ ep, T *__restrict__ sb, int N, int ne, T omega,
                                               const FCoef<T> &fc, const T *__restrict__ ttw = nullptr,
                                               const T *__restrict__ ttb = nullptr) {
  constexpr int H = (K - 1) / 2, ME = (K + 1) / 2, NPOS = ME + 2;
  const int RW = TX + 2 * H, RH = TY + 2 * H;
  const int vx = min(TX, N - i0), vy = min(TY, N - j0);
  const int vw = vx + 2 * H, vh = vy + 2 * H;
  using MP = MirrorPairs<K>;
  constexpr int NPAIR = MP::NPAIR;
  T *raw = reinterpret_cast<T *>(smem_raw);  // [3][RH][RW]
  T *xs = raw + 3 * RH * RW;                  // [3][NPOS][RH][TX]
  // FP32 multiplies by the weights of the parameter space directly; FP64 (bound by its FP64
  // pipe, where this measured faster) stages them in shared memory first
  const T *w1 = w1p;
  if constexpr (sizeof(T) == 8) {
    T *w1s = xs + 3 * NPOS * RH * TX;  // [NPAIR][K]
    for (int t = threadIdx.x; t < NPAIR * K; t += blockDim.x) w1s[t] = w1p[t];
    w1 = w1s;
  }
  {
    // extended tile of the 3 variables: interior cells from q, ring cells from gext
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
  // x-pass: every row of the extended tile, every valid tile column, the NPOS positions
  // as mirror pairs of the folded row
  for (BoxWalk bw(vh, vx); bw.v < 3; bw.next()) {
    const int v = bw.v, r = bw.r, c = bw.c;
    const T *row = raw + (v * RH + r) * RW + c;
    T a[K];
#pragma unroll
    for (int b = 0; b < K; ++b) a[b] = row[b];
    mirror_fold<T, K>(a);
    T *o = xs + ((size_t)v * NPOS * RH + r) * TX + c;
#pragma unroll
    for (int pi = 0; pi < NPAIR; ++pi) {
      T E, O;
      mirror_eval<T, K>(w1 + pi * K, a, E, O);
      o[MP::plus(pi) * RH * TX] = E + O;
      if (MP::minus(pi) != MP::plus(pi)) o[MP::minus(pi) * RH * TX] = E - O;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < vx * vy) {
    const int ty = threadIdx.x / vx, tx = threadIdx.x - ty * vx;
    const int i = i0 + tx, j = j0 + ty;
    const size_t pn = (size_t)6 * N * N;
    const size_t cell = ((size_t)p * N + j) * N + i;
    const T fc0 = fc.c[3 * p], fc1 = fc.c[3 * p + 1], fc2 = fc.c[3 * p + 2];
    T s1 = 0, s2 = 0;
    // metric (eq. 2.2) and Coriolis (eq. 2.3) sources at the cell point (g, h)
    auto source = [&](int g, int h, T X, const T qv[3]) {
      const T Y = Xg[j * ME + h];
      const size_t pt = (((size_t)j * N + i) * ME + h) * ME + g;
      const T os = omega * (fc0 + fc1 * X + fc2 * Y);  // Omega sin(latitude) delta, eq. 2.5
      const T rq = rcp(qv[0]);
      if constexpr (sizeof(T) == 8) {
        // FP64: the FP64 pipe is the bound, so the eight weighted polynomials are loaded
        const T *c8 = src8 + pt * 8;
        s1 += fma(c8[0], qv[1], c8[1] * qv[2]) * qv[1] * rq + os * fma(c8[4], qv[1], c8[5] * qv[2]);
        s2 += fma(c8[2], qv[1], c8[3] * qv[2]) * qv[2] * rq + os * fma(c8[6], qv[1], c8[7] * qv[2]);
      } else {
        // FP32: arithmetic is cheap next to load latency, so the polynomials are evaluated
        const T XY = X * Y, X2 = X * X, Y2 = Y * Y;
        const T a1 = (-XY * Y * qv[1] + Y * (T(1) + Y2) * qv[2]) * qv[1] * rq +
                     os * (-XY * qv[1] + (T(1) + Y2) * qv[2]);
        const T a2 = (X * (T(1) + X2) * qv[1] - X2 * Y * qv[2]) * qv[2] * rq +
                     os * (-(T(1) + X2) * qv[1] + XY * qv[2]);
        const T tw = t1w[pt];
        s1 = fma(tw, a1, s1);
        s2 = fma(tw, a2, s2);
      }
    };
#pragma unroll 1
    for (int t = 0; t < NPOS; ++t) {
      T col[3][K];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
#pragma unroll
        for (int b = 0; b < K; ++b) col[v][b] = xs[((v * NPOS + t) * RH + ty + b) * TX + tx];
        mirror_fold<T, K>(col[v]);
      }
      if (t < 2) {
        // west (t = 0) / east (t = 1) edge points at the Gauss nodes in y
#pragma unroll
        for (int pi = 1; pi < NPAIR; ++pi)
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            T E, O;
            mirror_eval<T, K>(w1 + pi * K, col[v], E, O);
            ep[((size_t)(t * 3 + v) * ME + (ME - pi)) * pn + cell] = E + O;
            if (MP::minus(pi) != MP::plus(pi)) ep[((size_t)(t * 3 + v) * ME + (pi - 1)) * pn + cell] = E - O;
          }
      } else {
        const int g = t - 2;
        // south / north edge points at x-node g
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          T E, O;
          mirror_eval<T, K>(w1, col[v], E, O);
          ep[((size_t)(2 * 3 + v) * ME + g) * pn + cell] = E - O;
          ep[((size_t)(3 * 3 + v) * ME + g) * pn + cell] = E + O;
        }
        // cell points (g, h) in mirror pairs of h
        const T X = Xg[i * ME + g];
#pragma unroll 1
        for (int pi = 1; pi < NPAIR; ++pi) {
          T qp[3], qm[3];
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            T E, O;
            mirror_eval<T, K>(w1 + pi * K, col[v], E, O);
            qp[v] = E + O;
            qm[v] = E - O;
          }
          source(g, ME - pi, X, qp);
          if (!(MP::ODD && pi == NPAIR - 1)) source(g, pi - 1, X, qm);
        }
      }
    }
    if constexpr (TOPO) {
      // psi_B from the depth stencil in shared memory (rows ty.., columns tx.. of variable 0)
      const T *st = raw + ty * RW + tx;
      T b1 = ttb[cell], b2 = ttb[pn + cell];
#pragma unroll 1
      for (int b = 0; b < K; ++b) {
#pragma unroll
        for (int a = 0; a < K; ++a) {
          const T v = st[b * RW + a];
          const size_t c = (size_t)(b * K + a);
          b1 = fma(ttw[c * pn + cell], v, b1);
          b2 = fma(ttw[((size_t)K * K + c) * pn + cell], v, b2);
        }
      }
      s1 += b1;
      s2 += b2;
    }
    sb[cell] = s1;
    sb[pn + cell] = s2;
  }
  __syncthreads();
}

// One block per tile of TX x TY cells (blockIdx.x, blockIdx.y: tile column and row,
// blockIdx.z: panel); TX*TY <= blockDim.x <= REC_MAX_THREADS.
template <typename T, int K, bool TOPO = false>
__global__ void __launch_bounds__(REC_MAX_THREADS)
    k_recon_tpp(const T *__restrict__ q, const T *__restrict__ gext, const T *__restrict__ Xg,
                const T *__restrict__ t1w, const T *__restrict__ src8, T *__restrict__ ep, T *__restrict__ sb,
                int N, int ne, int TX, int TY, T omega, FCoef<T> fc, const T *__restrict__ ttw,
                const T *__restrict__ ttb, const __grid_constant__ PairW<T, K> pw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  griddep_wait();
  recon_tpp_tile<T, K, TOPO>(smem_raw, blockIdx.z, blockIdx.x * TX, blockIdx.y * TY, TX, TY, q, gext, pw.w, Xg, t1w,
                             src8, ep, sb, N, ne, omega, fc, ttw, ttb);
}

// ---------------------------------------------------------------------------------
// Metric terms of the edge points (k_setup_grid): five planes {1/sqrtG, sqrt(G^nn),
// 1/sqrt(G^nn), sqrtG G^nn/2, sqrtG G^nc/2} (true metric) of me x N x (N+1) values each,
// stored twice: with the edge-line index e fastest (x-edges, whose consecutive items take
// consecutive lines) and then with the position a along the line fastest (y-edges and
// cube edges, whose consecutive items take consecutive positions), so that each of the
// five loads of a warp reads one contiguous run.  The planes are metric_plane() apart.
// ---------------------------------------------------------------------------------
__host__ __device__ __forceinline__ size_t metric_plane(int N, int ME) { return (size_t)ME * N * (N + 1); }
__device__ __forceinline__ size_t metric_x(int N, int e, int a, int g) { return ((size_t)g * N + a) * (N + 1) + e; }
__device__ __forceinline__ size_t metric_y(int N, int ME, int e, int a, int g) {
  return 5 * metric_plane(N, ME) + ((size_t)g * (N + 1) + e) * N + a;
}

// ---------------------------------------------------------------------------------
// LMARS flux at one edge point (eqs. 3.31-3.38) from table metric terms m5[c * mstr],
// c = 0..4 as listed above.  dir 0: x-edge (normal momentum var 1), 1: y-edge (var 2).
// ---------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void lmars(const T qL[3], const T qR[3], const T *m5, size_t mstr, int dir, T F[3],
                                      unsigned *status) {
  const T isg = m5[0], s11 = m5[mstr], is11 = m5[2 * mstr], pn = m5[3 * mstr], pc = m5[4 * mstr];
  const T phL = qL[0] * isg, phR = qR[0] * isg;
  if (!(phL > T(0)) || !(phR > T(0))) atomicOr(status, HOPE_STATUS_NONPHYS_PHI);
  // normal momentum component (selects, not a runtime index, keep the arrays in registers)
  const T qnL = dir ? qL[2] : qL[1], qnR = dir ? qR[2] : qR[1];
  const T rLR = rcp(qL[0] * qR[0]);  // one reciprocal for both states
  const T uL = qnL * (qR[0] * rLR) * is11, uR = qnR * (qL[0] * rLR) * is11;
  const T sL = sqrt_pos(phL), sR = sqrt_pos(phR);
  const T c = T(0.5) * (sL + sR);
  // (phR - phL) / (2 c) = sR - sL exactly, so the interface velocity needs no division
  const T ms = T(0.5) * (uL + uR) - (sR - sL);
  const T ph = T(0.5) * (phL + phR - c * (uR - uL));
  const T m = ms * s11;
  // 1/2 [m (qL + qR) - |m| (qR - qL)] is the upwind state times m: qL for m >= 0, else qR
  // (a select instead of the cancelling terms)
  const bool up = m >= T(0);
#pragma unroll
  for (int v = 0; v < 3; ++v) F[v] = m * (up ? qL[v] : qR[v]);
  const T p2 = ph * ph;
  F[1] += (dir ? pc : pn) * p2;
  F[2] += (dir ? pn : pc) * p2;
}

// LMARS over bottom topography (eqs. 2.13, 3.32-3.38): q holds the depth sqrtG phi, and
// sL, sR are sqrtG phi_s at the point.  The wave speed and the upwinded q come from the
// depth; the pressure jump and the interface value used by P from phi_t = phi + phi_s:
// (phi_t,R - phi_t,L)/(2c) = (cR - cL) + (phi_s,R - phi_s,L)/(2c).  With sL = sR = 0 the
// result is lmars()'s exactly.
template <typename T>
__device__ __forceinline__ void lmars_topo(const T qL[3], const T qR[3], T sL, T sR, const T *m5, size_t mstr,
                                           int dir, T F[3], unsigned *status) {
  const T isg = m5[0], s11 = m5[mstr], is11 = m5[2 * mstr], pn = m5[3 * mstr], pc = m5[4 * mstr];
  const T phL = qL[0] * isg, phR = qR[0] * isg;
  if (!(phL > T(0)) || !(phR > T(0))) atomicOr(status, HOPE_STATUS_NONPHYS_PHI);
  const T fsL = sL * isg, fsR = sR * isg;
  const T qnL = dir ? qL[2] : qL[1], qnR = dir ? qR[2] : qR[1];
  const T rLR = rcp(qL[0] * qR[0]);
  const T uL = qnL * (qR[0] * rLR) * is11, uR = qnR * (qL[0] * rLR) * is11;
  const T cL = sqrt_pos(phL), cR = sqrt_pos(phR);
  const T c = T(0.5) * (cL + cR);
  const T ms = T(0.5) * (uL + uR) - (cR - cL) - (fsR - fsL) * rcp(c + c);
  const T ph = T(0.5) * ((phL + fsL) + (phR + fsR) - c * (uR - uL));
  const T m = ms * s11;
  // 1/2 [m (qL + qR) - |m| (qR - qL)] is the upwind state times m: qL for m >= 0, else qR
  // (a select instead of the cancelling terms)
  const bool up = m >= T(0);
#pragma unroll
  for (int v = 0; v < 3; ++v) F[v] = m * (up ? qL[v] : qR[v]);
  const T p2 = ph * ph;
  F[1] += (dir ? pc : pn) * p2;
  F[2] += (dir ? pn : pc) * p2;
}

// ---------------------------------------------------------------------------------
// Edge fluxes: interior x-edges, interior y-edges, then the 12 cube edges x N cells.
// TOPO: bottom topography, with sep[4][me][6][N][N] = sqrtG phi_s at the edge points
// (same side and node order as ep).
// ---------------------------------------------------------------------------------
// Panel-boundary edge item r (cube edge r / N, cell r % N along it): the flux in panel A's
// frame and its conversion to panel B's (eqs. 3.26-3.29, reading c10).
template <typename T, int ME, bool TOPO>
__device__ __forceinline__ void flux_cube_item(int r, const T *__restrict__ ep, const T *__restrict__ mx,
                                            const T *__restrict__ gwg, const int *__restrict__ bedge,
                                            const T *__restrict__ bconv, T *__restrict__ fx, T *__restrict__ fy,
                                            int N, unsigned *status, const T *__restrict__ sep) {
  const size_t pn = (size_t)6 * N * N;
  const size_t fe = (size_t)6 * N * (N + 1);
  const size_t ms = metric_plane(N, ME);
  T gw[ME];
#pragma unroll
  for (int g = 0; g < ME; ++g) gw[g] = gwg[g];
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
  const int dirA = sA >> 1, dirB = sB >> 1;
  const T sgA = (sA & 1) ? T(1) : T(-1), sgB = (sB & 1) ? T(1) : T(-1);
  const T sg = -sgA * sgB;
  const int eA = (sA & 1) ? N : 0;
  Acc<T> accA[3], accB[3];
#pragma unroll
  for (int g = 0; g < ME; ++g) {
    const int gB = flip ? ME - 1 - g : g;
    const T *cv = bconv + (((size_t)ce * N + t) * ME + g) * 9;
    T qin[3], qb[3], qo[3], F[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      qin[v] = ep[((size_t)(sA * 3 + v) * ME + g) * pn + cA];
      qb[v] = ep[((size_t)(sB * 3 + v) * ME + gB) * pn + cB];
    }
    qo[0] = cv[0] * qb[0];
    qo[1] = cv[1] * qb[1] + cv[2] * qb[2];
    qo[2] = cv[3] * qb[1] + cv[4] * qb[2];
    const T *m5 = mx + metric_y(N, ME, eA, t, g);
    if constexpr (TOPO) {
      const T sin_ = sep[((size_t)sA * ME + g) * pn + cA];
      const T so = cv[0] * sep[((size_t)sB * ME + gB) * pn + cB];
      if (sA & 1)
        lmars_topo(qin, qo, sin_, so, m5, ms, dirA, F, status);
      else
        lmars_topo(qo, qin, so, sin_, m5, ms, dirA, F, status);
    } else {
      if (sA & 1)
        lmars(qin, qo, m5, ms, dirA, F, status);
      else
        lmars(qo, qin, m5, ms, dirA, F, status);
    }
#pragma unroll
    for (int v = 0; v < 3; ++v) accA[v].add(gw[g] * F[v]);
    accB[1].add(gw[gB] * sg * (cv[5] * F[1] + cv[6] * F[2]));
    accB[2].add(gw[gB] * sg * (cv[7] * F[1] + cv[8] * F[2]));
  }
  const T fA0 = accA[0].value();
  const T outA[3] = {fA0, accA[1].value(), accA[2].value()};
  const T outB[3] = {sg * fA0, accB[1].value(), accB[2].value()};
  const int eB = (sB & 1) ? N : 0;
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    if (dirA == 0)
      fx[v * fe + ((size_t)A * N + t) * (N + 1) + eA] = outA[v];
    else
      fy[v * fe + ((size_t)A * (N + 1) + eA) * N + t] = outA[v];
    if (dirB == 0)
      fx[v * fe + ((size_t)B * N + tB) * (N + 1) + eB] = outB[v];
    else
      fy[v * fe + ((size_t)B * (N + 1) + eB) * N + tB] = outB[v];
  }
}

// The same item out of line, for the FP32 persistent stage: inlined, its register demand
// (both panels' sums and the conversions) sets the allocation of the whole edge loop, which
// then spills under the persistent kernel's register cap.
template <typename T, int ME, bool TOPO>
__device__ __noinline__ void flux_cube_item_outline(int r, const T *__restrict__ ep, const T *__restrict__ mx,
                                                    const T *__restrict__ gwg, const int *__restrict__ bedge,
                                                    const T *__restrict__ bconv, T *__restrict__ fx,
                                                    T *__restrict__ fy, int N, unsigned *status,
                                                    const T *__restrict__ sep) {
  flux_cube_item<T, ME, TOPO>(r, ep, mx, gwg, bedge, bconv, fx, fy, N, status, sep);
}

template <typename T, int ME, bool TOPO = false, bool OUTLINE = false>
__device__ __forceinline__ void flux_item(int idx, const T *__restrict__ ep, const T *__restrict__ mx,
                                          const T *__restrict__ gwg, const int *__restrict__ bedge,
                                          const T *__restrict__ bconv, T *__restrict__ fx, T *__restrict__ fy,
                                          int N, unsigned *status, const T *__restrict__ sep = nullptr) {
  // 32-bit item arithmetic: 12 N (N + 1) < 2^31 for N <= 8192
  const int nx = 6 * N * (N - 1), ny = nx;
  const size_t pn = (size_t)6 * N * N;
  const size_t fe = (size_t)6 * N * (N + 1);
  const size_t ms = metric_plane(N, ME);
  T gw[ME];
#pragma unroll
  for (int g = 0; g < ME; ++g) gw[g] = gwg[g];
  if (idx < nx + ny) {
    const int dir = idx < nx ? 0 : 1;
    const unsigned r = (unsigned)(dir ? idx - nx : idx);
    // x-edge: (p, j, e=1..N-1), e fastest; y-edge: (p, e=1..N-1, i), i fastest
    int p, a, e;  // a = row j (x) / column i (y)
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
    size_t cl, cr;  // left / right (below / above) cells
    if (dir == 0) {
      cl = ((size_t)p * N + a) * N + (e - 1);
      cr = cl + 1;
    } else {
      cl = ((size_t)p * N + (e - 1)) * N + a;
      cr = cl + N;
    }
    const int sl = dir ? 3 : 1, sr = dir ? 2 : 0;
    Acc<T> acc[3];
#pragma unroll
    for (int g = 0; g < ME; ++g) {
      T qL[3], qR[3], F[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        qL[v] = ep[((size_t)(sl * 3 + v) * ME + g) * pn + cl];
        qR[v] = ep[((size_t)(sr * 3 + v) * ME + g) * pn + cr];
      }
      const T *m5 = mx + (dir ? metric_y(N, ME, e, a, g) : metric_x(N, e, a, g));
      if constexpr (TOPO)
        lmars_topo(qL, qR, sep[((size_t)sl * ME + g) * pn + cl], sep[((size_t)sr * ME + g) * pn + cr], m5, ms, dir,
                   F, status);
      else
        lmars(qL, qR, m5, ms, dir, F, status);
#pragma unroll
      for (int v = 0; v < 3; ++v) acc[v].add(gw[g] * F[v]);
    }
    if (dir == 0) {
#pragma unroll
      for (int v = 0; v < 3; ++v) fx[v * fe + ((size_t)p * N + a) * (N + 1) + e] = acc[v].value();
    } else {
#pragma unroll
      for (int v = 0; v < 3; ++v) fy[v * fe + ((size_t)p * (N + 1) + e) * N + a] = acc[v].value();
    }
    return;
  }
  // panel-boundary edge: cube edge ce, cell t along it
  if constexpr (OUTLINE)
    flux_cube_item_outline<T, ME, TOPO>(idx - nx - ny, ep, mx, gwg, bedge, bconv, fx, fy, N, status, sep);
  else
    flux_cube_item<T, ME, TOPO>(idx - nx - ny, ep, mx, gwg, bedge, bconv, fx, fy, N, status, sep);
}

template <typename T, int ME>
__global__ void __launch_bounds__(256)
    k_flux(const T *__restrict__ ep, const T *__restrict__ mx, const T *__restrict__ gwg,
           const int *__restrict__ bedge, const T *__restrict__ bconv, T *__restrict__ fx,
           T *__restrict__ fy, int N, unsigned *status) {
  griddep_wait();
  const long long n = 12LL * N * (N - 1) + 12LL * N;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    flux_item<T, ME>((int)idx, ep, mx, gwg, bedge, bconv, fx, fy, N, status);
}

template <typename T, int ME>
__global__ void __launch_bounds__(256)
    k_flux_topo(const T *__restrict__ ep, const T *__restrict__ mx, const T *__restrict__ gwg,
                const int *__restrict__ bedge, const T *__restrict__ bconv, T *__restrict__ fx,
                T *__restrict__ fy, int N, unsigned *status, const T *__restrict__ sep) {
  const long long n = 12LL * N * (N - 1) + 12LL * N;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    flux_item<T, ME, true>((int)idx, ep, mx, gwg, bedge, bconv, fx, fy, N, status, sep);
}

// ---------------------------------------------------------------------------------
// psi_B of eq. 2.14, cell-averaged, added to the sources.  For a fixed surface the
// gradient of phi_t = (P_depth + P_s)/sqrtG at the cell Gauss points is affine in the
// cell's k x k depth stencil (P the TPP polynomials of section 3.1), so the cell average
// of sqrtG phi_s G^ij d_j phi_t is sum_c w[v][c] * stencil_c + b[v], with the weights
// w[2][k*k][6][N][N] and constants b[2][6][N][N] built in FP64 at set-up.  One thread
// per cell; the stencil's ring cells come from the ghost ring of the mass variable.
// ---------------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(256)
    k_topo_src(const T *__restrict__ q, const T *__restrict__ gext, const T *__restrict__ tw,
               const T *__restrict__ tb, T *__restrict__ sb, int N, int ne) {
  constexpr int H = (K - 1) / 2;
  const long long n = 6LL * N * N;
  const long long cid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cid >= n) return;
  const int i = (int)(cid % N), j = (int)((cid / N) % N), p = (int)(cid / ((long long)N * N));
  T s1 = tb[cid], s2 = tb[n + cid];
#pragma unroll 1
  for (int b = 0; b < K; ++b) {
    const int jj = j + b - H;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      const int ii = i + a - H;
      const T v = (ii >= 0 && ii < N && jj >= 0 && jj < N)
                      ? q[((size_t)p * N + jj) * N + ii]
                      : gext[((size_t)p * ne + (jj + H)) * ne + (ii + H)];
      const size_t c = (size_t)(b * K + a);
      s1 = fma(tw[c * n + cid], v, s1);
      s2 = fma(tw[((size_t)K * K + c) * n + cid], v, s2);
    }
  }
  sb[cid] += s1;
  sb[n + cid] += s2;
}

// ---------------------------------------------------------------------------------
// Tendency (eq. 3.1) and the Runge-Kutta stage combination:
//   mode 0: out = L
//   mode 1: out = a*q0 + b*qs + c*L
// With low-word pointers (FP32 contexts) every state is the unevaluated sum hi + lo of two
// floats, and the combination is formed with error-free transformations (TwoProd by
// fma, TwoSum), so the FP32 state keeps the low-order part of each stage increment.
// ---------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
  s = a + b;
  T bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// Rounding residual of a stage coefficient in precision T (zero in FP64).
template <typename T>
inline T coef_lo(double x) {
  return (T)(x - (double)(T)x);
}

// The stage coefficients are split too (a = a + alo with alo the rounding residual of
// the double coefficient): 1/3 and 2/3 round up in FP32, and without their residuals the
// third SSP-RK3 stage would scale the state by 1 + 3e-8 every step.
template <typename T>
__device__ __forceinline__ T combine(T a, T q0, T b, T qs, T c, T L, T alo, T blo, T clo, const T *q0l,
                                     const T *qsl, T *outl, long long idx) {
  if (q0l == nullptr) return a * q0 + b * qs + c * L;
  const T p1 = a * q0, e1 = fma(a, q0, -p1);
  const T p2 = b * qs, e2 = fma(b, qs, -p2);
  const T p3 = c * L, e3 = fma(c, L, -p3);
  T s, r1, s2, r2;
  two_sum(p1, p2, s, r1);
  two_sum(s, p3, s2, r2);
  T lo = ((r1 + r2) + (e1 + e2 + e3)) + (a * q0l[idx] + b * qsl[idx]) + (alo * q0 + blo * qs + clo * L);
  T hi = s2 + lo;
  outl[idx] = lo - (hi - s2);
  return hi;
}

template <typename T>
__device__ __forceinline__ void update_cell(int cid, const T *__restrict__ fx, const T *__restrict__ fy,
                                            const T *__restrict__ sb, const T *q0, const T *qs, T *out, int N,
                                            T inv_dx, int mode, T a, T b, T c, T alo, T blo, T clo, const T *q0l,
                                            const T *qsl, T *outl, unsigned *status) {
  // 32-bit cell arithmetic: 3 * 6 N^2 < 2^31 for N <= 8192
  const int ncell = 6 * N * N;
  const int pj = (int)((unsigned)cid / (unsigned)N);  // p*N + j
  const int i = cid - pj * N;
  const int p = (int)((unsigned)pj / (unsigned)N), j = pj - p * N;
  const size_t fe = (size_t)6 * N * (N + 1);
  bool bad = false;
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const T *fxv = fx + v * fe + (size_t)pj * (N + 1);
    const T *fyv = fy + v * fe + ((size_t)p * (N + 1) + j) * N + i;
    Acc<T> acc;
    acc.add(-(fxv[i + 1] - fxv[i]) * inv_dx);
    acc.add(-(fyv[N] - fyv[0]) * inv_dx);
    if (v > 0) acc.add(sb[(v - 1) * ncell + cid]);
    T L = acc.value();
    T r;
    if (mode == 0) {
      r = L;
    } else {
      const int idx = v * ncell + cid;
      r = combine(a, q0[idx], b, qs[idx], c, L, alo, blo, clo, q0l, qsl, outl, idx);
    }
    bad |= !isfinite(r);
    out[v * ncell + cid] = r;
  }
  if (bad) atomicOr(status, HOPE_STATUS_NAN);
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_update(const T *__restrict__ fx, const T *__restrict__ fy, const T *__restrict__ sb,
             const T *q0, const T *qs, T *out, int N, T inv_dx, int mode, T a, T b, T c, T alo, T blo,
             T clo, const T *q0l, const T *qsl, T *outl, unsigned *status) {
  const int cid = blockIdx.x * blockDim.x + threadIdx.x;
  if (cid >= 6 * N * N) return;
  griddep_wait();
  update_cell(cid, fx, fy, sb, q0, qs, out, N, inv_dx, mode, a, b, c, alo, blo, clo, q0l, qsl, outl, status);
}

// ---------------------------------------------------------------------------------
// Deterministic FP64 mass sum: fixed per-block ranges, then an ordered final pass.
// ---------------------------------------------------------------------------------
constexpr int MASS_BLOCKS = 152;
constexpr int MASS_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(MASS_THREADS) k_mass_partial(const T *__restrict__ q, long long n,
                                                               double *__restrict__ part) {
  __shared__ double red[MASS_THREADS];
  long long chunk = (n + gridDim.x - 1) / gridDim.x;
  long long b = blockIdx.x * chunk, e = b + chunk < n ? b + chunk : n;
  double s = 0.0;
  for (long long t = b + threadIdx.x; t < e; t += blockDim.x) s += (double)q[t];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = MASS_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_mass_final(const double *__restrict__ part, int nparts, double scale, double *out);

}  // namespace hope
