// hope_ensemble.cu -- one persistent launch per Runge-Kutta stage for an ensemble of
// cubed spheres at uneven resolutions (TPP reconstruction).
//
// The four phases of a stage (ghost fill, reconstruction + sources, edge fluxes, tendency
// + stage combination) become work lists over all members, walked by a cooperative grid
// of resident blocks and separated by grid-wide barriers.  Every barrier wait is bounded:
// a block that waits longer than the limit sets HOPE_STATUS_TIMEOUT and the launch
// returns instead of hanging.  The tile shape (TX x TY cells per work item, a run-time
// argument) and the block size (128 or 256 threads, compiled) are chosen by timing a list
// of candidates (hope_autotune).
#include <cuda_runtime.h>

#include <algorithm>

#include <string>
#include <vector>

#include "hope_adjoint.cuh"
#include "hope_ensemble.h"
#include "hope_kernels.cuh"
#include "hope_setup_math.cuh"

namespace hope {

template <typename T>
struct MemberDev {
  int N, ne;
  long long off;  // element offset of the member in ensemble states
  const int *grow, *gcol, *gdst, *gsym;
  const T *gval;
  const int *trow, *tcol;
  const float *tval;
  size_t gs;  // plane stride of gval (FP32 contexts)
  T *gext;
  const T *Xg, *t1w, *src8, *mx, *bconv;
  const int *bedge;
  T *ep, *sb, *fx, *fy;
  long long b_ghost, b_tile, b_flux, b_cell;  // first global item of each phase
  int tiles_x, tiles_y;
  T inv_dx;  // 2N / pi, computed on the host (no FP64 division per cell)
  // adjoint (filled once the context's adjoint scratch exists): edge-point adjoints,
  // stencil gradients, ring and interior adjoints, the transposed ghost operator, the
  // first item of the gather phase (6 ne^2 per member), and the member's block in a step
  // tape (element offset; ghost-ring and edge-point elements of one stage)
  T *lep, *tbuf, *lring, *ldir;
  const int *gtp, *gtr, *gband;
  const T *gtv;
  long long nband;
  long long b_gather, b_band;  // first item of the gather phase and of the band lanes
  long long tape_off, tape_ge, tape_ee;
};

// Ghost-fill work of the members that share one ghost operator (equal N): one item per
// (operator row, chunk of up to GHOST_GROUP_CHUNK members), chunks fastest; one warp
// applies the row to the whole chunk (ghost_row_members), and the chunks of a row run back
// to back on one SM, where they find the row's weights in L1.  The rows use their own
// weights (no cube-symmetry transforms: this reuse already keeps the weights on chip).
constexpr int GHOST_GROUP_CHUNK = 4;
struct GhostGroup {
  long long b_item;  // first item
  int rows, nchunk, first, nmem;  // operator rows; member chunks; members gmem[first ...]
};

// One ghost row applied at once to the MB members of a chunk (unused slots repeat the
// first member and are not stored): each lane loads an entry's column and five weights
// once and applies them to every member, so the weights stay in registers instead of being
// read again per member.  Every member's sums take the entries in ghost_row's order (lane
// l: entries b + l, b + l + 32, ...), then the same reduce-scatter, so each member's ring
// equals ghost_row<T, false>'s bit for bit (ghost_row's padding lanes add zero products,
// which can only change the sign of a zero sum).  q[m]: member m's state; ring[m]: its
// ghost ring.
template <typename T, int MB>
__device__ __forceinline__ void ghost_row_members(int row, int lane, const T *const (&q)[MB], T *const (&ring)[MB],
                                                  int nm, const int *__restrict__ grow,
                                                  const int *__restrict__ gcol, const T *__restrict__ gval,
                                                  const int *__restrict__ gdst, const int *__restrict__ trow,
                                                  const int *__restrict__ tcol, const float *__restrict__ tval,
                                                  int N, int ne, size_t gs) {
  const size_t pn = (size_t)6 * N * N, pe = (size_t)6 * ne * ne;
  T s[MB][3];
#pragma unroll
  for (int m = 0; m < MB; ++m) s[m][0] = s[m][1] = s[m][2] = T(0);
  const int b = grow[row], e = grow[row + 1];
  for (int t = b + lane; t < e; t += 32) {
    const int cc = gcol[t] & 0x0FFFFFFF;
    T w[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) w[k] = gval[GHOST_PLANES<T> ? k * gs + t : 5 * (size_t)t + k];
#pragma unroll
    for (int m = 0; m < MB; ++m) {
      const T a0 = q[m][cc], a1 = q[m][pn + cc], a2 = q[m][2 * pn + cc];
      s[m][0] = fma(w[0], a0, s[m][0]);
      s[m][1] = fma(w[1], a1, fma(w[2], a2, s[m][1]));
      s[m][2] = fma(w[3], a1, fma(w[4], a2, s[m][2]));
    }
  }
  if constexpr (sizeof(T) == 8) {
    if (trow) {
      // FP64 contexts: the FP32 tail of negligible weights, as ghost_row evaluates it
      float f[MB][3];
#pragma unroll
      for (int m = 0; m < MB; ++m) f[m][0] = f[m][1] = f[m][2] = 0.f;
      const int tb = trow[row], te = trow[row + 1];
      for (int t = tb + lane; t < te; t += 32) {
        const int cc = tcol[t] & 0x0FFFFFFF;
        float w[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) w[k] = tval[5 * (size_t)t + k];
#pragma unroll
        for (int m = 0; m < MB; ++m) {
          const float a0 = f64_to_f32_trunc(q[m][cc]), a1 = f64_to_f32_trunc(q[m][pn + cc]),
                      a2 = f64_to_f32_trunc(q[m][2 * pn + cc]);
          f[m][0] = fmaf(w[0], a0, f[m][0]);
          f[m][1] = fmaf(w[1], a1, fmaf(w[2], a2, f[m][1]));
          f[m][2] = fmaf(w[3], a1, fmaf(w[4], a2, f[m][2]));
        }
      }
#pragma unroll
      for (int m = 0; m < MB; ++m) {
        s[m][0] += (T)f[m][0];
        s[m][1] += (T)f[m][1];
        s[m][2] += (T)f[m][2];
      }
    }
  }
  const int dst = gdst[row];
#pragma unroll
  for (int m = 0; m < MB; ++m)
    if (m < nm) ghost_reduce_store(lane, s[m][0], s[m][1], s[m][2], ring[m], pe, dst);
}

// Ghost-fill item `it` (a row of a group's operator and a chunk of its members), for every
// thread of a warp.
template <typename T>
__device__ __forceinline__ void ghost_item(long long it, int lane, const GhostGroup *__restrict__ ggrp, int ngrp,
                                           const int *__restrict__ gmem, const MemberDev<T> *__restrict__ mem,
                                           const T *__restrict__ qs) {
  int lo = 0, hi = ngrp - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ggrp[mid].b_item <= it)
      lo = mid;
    else
      hi = mid - 1;
  }
  const GhostGroup &G = ggrp[lo];
  const long long local = it - G.b_item;
  const int r = (int)(local / G.nchunk), c = (int)(local - (long long)r * G.nchunk);
  const int k0 = c * GHOST_GROUP_CHUNK, nm = min(G.nmem - k0, GHOST_GROUP_CHUNK);
  const T *q[GHOST_GROUP_CHUNK];
  T *ring[GHOST_GROUP_CHUNK];
#pragma unroll
  for (int k = 0; k < GHOST_GROUP_CHUNK; ++k) {
    const MemberDev<T> &m = mem[gmem[G.first + k0 + (k < nm ? k : 0)]];
    q[k] = qs + m.off;
    ring[k] = m.gext;
  }
  const MemberDev<T> &m0 = mem[gmem[G.first + k0]];
  ghost_row_members<T, GHOST_GROUP_CHUNK>(r, lane, q, ring, nm, m0.grow, m0.gcol, m0.gval, m0.gdst, m0.trow, m0.tcol,
                                          m0.tval, m0.N, m0.ne, m0.gs);
}

template <typename T>
struct StageArgs {
  const T *qs, *q0;
  T *out;
  const T *q0l, *qsl;
  T *outl;
  T a, b, c, alo, blo, clo;  // stage coefficients and their rounding residuals
  int mode;
  T omega;
  FCoef<T> fc;
  const T *gw;
  unsigned long long *stamp;  // profiling: [start, 3 phase ends, end] or null
  const GhostGroup *ggrp;     // ghost-fill groups
  const int *gmem;            // member indices of the groups
  int ngrp;
  int tx, ty;                 // reconstruction tile (cells)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr long long BARRIER_WAIT_CYCLES = 2000000000ll;  // about one second of SM clock

// Grid-wide barrier over the co-resident blocks of a cooperative launch.  bar[0] counts
// arrivals, bar[1] is the generation.  Returns false (and sets the timeout bit) if the
// wait exceeded the limit or another block already timed out.
// `extra` raises the expected arrival count (fault injection for the timeout path: no
// block releases the barrier, every block gives up after the bounded wait).
__device__ __forceinline__ bool grid_sync(unsigned *bar, unsigned *status, unsigned extra) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned *vgen = bar + 1;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == gridDim.x + extra) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > BARRIER_WAIT_CYCLES) {
          atomicOr(status, HOPE_STATUS_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
    if (*(volatile unsigned *)status & HOPE_STATUS_TIMEOUT) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// Begin offsets of one phase's work lists, staged in shared memory at the start of the
// phase (ensembles of at most MEMBER_CACHE members; larger ones search the member table
// in global memory), so that the per-item member lookup reads no global memory.
constexpr int MEMBER_CACHE = 128;

template <typename T>
__device__ __forceinline__ long long phase_begin(const MemberDev<T> &m, int phase) {
  return phase == 0 ? m.b_ghost
         : phase == 1 ? m.b_tile
         : phase == 2 ? m.b_flux
         : phase == 3 ? m.b_cell
         : phase == 4 ? m.b_gather
                      : m.b_band;
}

// Called by every thread of the block between two block-wide barriers.
template <typename T>
__device__ __forceinline__ void stage_member_begins(long long *sbeg, const MemberDev<T> *mem, int nmem, int phase) {
  if (nmem > MEMBER_CACHE) return;
  __syncthreads();
  for (int i = threadIdx.x; i < nmem; i += blockDim.x) sbeg[i] = phase_begin(mem[i], phase);
  __syncthreads();
}

// member owning global item `it` of a phase: binary search over the staged begin offsets
__device__ __forceinline__ int find_member_cached(const long long *sbeg, int nmem, long long it) {
  int lo = 0, hi = nmem - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sbeg[mid] <= it)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// member owning global item `it` of a phase (begin offsets ascending by member)
template <typename T>
__device__ __forceinline__ int find_member(const MemberDev<T> *mem, int nmem, long long it, int phase) {
  int lo = 0, hi = nmem - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    const long long b = phase_begin(mem[mid], phase);
    if (b <= it)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// FP32: 128-thread blocks are capped at 64 registers (8 resident blocks), 256-thread
// blocks at 80 (3 resident blocks); the autotuner times both kinds.  FP64 is uncapped.
template <typename T, int K, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? (NT == 128 ? 8 : 3) : 1)
    k_stage_persistent(const MemberDev<T> *__restrict__ mem, int nmem, long long n_ghost, long long n_tile,
                       long long n_flux, long long n_cell, StageArgs<T> sa, unsigned *bar, unsigned *status,
                       unsigned inject, const __grid_constant__ PairW<T, K> pw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ME = (K + 1) / 2;
  constexpr int WPB = NT / 32;
  const int TX = sa.tx, TY = sa.ty;
  __shared__ long long sbeg[MEMBER_CACHE];
  auto lookup = [&](long long it, int phase) {
    return nmem <= MEMBER_CACHE ? find_member_cached(sbeg, nmem, it) : find_member(mem, nmem, it, phase);
  };
  const bool stamper = sa.stamp && blockIdx.x == 0 && threadIdx.x == 0;
  if (stamper) sa.stamp[0] = global_ns();
  // phase 1: ghost rows, one warp per (row, member chunk) item
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (long long it = (long long)blockIdx.x * WPB + warp; it < n_ghost; it += (long long)gridDim.x * WPB)
      ghost_item(it, lane, sa.ggrp, sa.ngrp, sa.gmem, mem, sa.qs);
  }
  if (!grid_sync(bar, status, inject)) return;
  if (stamper) sa.stamp[1] = global_ns();
  // phase 2: reconstruction tiles, one block each
  stage_member_begins(sbeg, mem, nmem, 1);
  for (long long it = blockIdx.x; it < n_tile; it += gridDim.x) {
    const MemberDev<T> &m = mem[lookup(it, 1)];
    const int local = int(it - m.b_tile);
    const int p = local / (m.tiles_x * m.tiles_y);
    const int rem = local - p * m.tiles_x * m.tiles_y;
    const int ty = rem / m.tiles_x, tx = rem - ty * m.tiles_x;
    recon_tpp_tile<T, K>(smem_raw, p, tx * TX, ty * TY, TX, TY, sa.qs + m.off, m.gext, pw.w, m.Xg, m.t1w, m.src8, m.ep,
                                 m.sb, m.N, m.ne, sa.omega, sa.fc);
  }
  if (!grid_sync(bar, status, inject)) return;
  if (stamper) sa.stamp[2] = global_ns();
  // phase 3: edge fluxes, one thread per edge
  stage_member_begins(sbeg, mem, nmem, 2);
  for (long long it = (long long)blockIdx.x * NT + threadIdx.x; it < n_flux; it += (long long)gridDim.x * NT) {
    const MemberDev<T> &m = mem[lookup(it, 2)];
    flux_item<T, ME, false, sizeof(T) == 4>((int)(it - m.b_flux), m.ep, m.mx, sa.gw, m.bedge, m.bconv, m.fx, m.fy,
                                            m.N, status);
  }
  if (!grid_sync(bar, status, inject)) return;
  if (stamper) sa.stamp[3] = global_ns();
  // phase 4: tendency and stage combination, one thread per cell
  stage_member_begins(sbeg, mem, nmem, 3);
  for (long long it = (long long)blockIdx.x * NT + threadIdx.x; it < n_cell; it += (long long)gridDim.x * NT) {
    const MemberDev<T> &m = mem[lookup(it, 3)];
    auto off = [&](const T *p) -> const T * { return p ? p + m.off : nullptr; };
    update_cell((int)(it - m.b_cell), m.fx, m.fy, m.sb, off(sa.q0), sa.qs + m.off, sa.out + m.off, m.N,
                m.inv_dx, sa.mode, sa.a, sa.b, sa.c, sa.alo, sa.blo, sa.clo, off(sa.q0l), off(sa.qsl),
                sa.outl ? sa.outl + m.off : nullptr, status);
  }
  if (sa.stamp) {
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(sa.stamp + 4, global_ns());
  }
}

// -------------------------------------------------------------------------------------
// One stage VJP of the whole ensemble (the reverse of a stage, section 4's autograd
// replaced by hand-written adjoints): out = a x + b y + d z + c (dL/dq at qs)^T lamL for
// every member, as one cooperative launch whose phases walk all members' work lists:
//   [forward recompute of the ghost rings and edge points, unless a step tape holds them]
//   flux adjoint per edge | reconstruction + source adjoint per tile | stencil-gradient
//   gather per extended cell | transposed ghost operator + combination per cell,
// separated by the same bounded grid barriers as the forward stage.
// -------------------------------------------------------------------------------------
template <typename T>
struct VjpArgs {
  const T *qs, *lamL;
  const T *x, *y, *z;
  T *out;
  T a, b, d, c;
  int have_fwd;
  const T *tape;   // step tape holding the stage's ghost rings and edge points, or null
  int tape_stage;  // its stage slot
  T omega;
  FCoef<T> fc;
  const T *gw, *w1;
  const GhostGroup *ggrp;
  const int *gmem;
  int ngrp;
  unsigned long long *stamp;  // profiling: 7 phase stamps, or null
  int tx, ty;                 // reconstruction tile (cells)
};

// FP32: registers capped for five resident 128-thread blocks (the phases are latency-bound;
// the shared memory of a 16 x 8 tile allows five), FP64 uncapped (it would spill)
template <typename T, int K, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 640 / NT : 1)
    k_vjp_persistent(const MemberDev<T> *__restrict__ mem, int nmem, long long n_ghost, long long n_tile,
                     long long n_flux, long long n_cell, long long n_gather, long long n_band, VjpArgs<T> va,
                     unsigned *bar, unsigned *status, unsigned inject,
                     const __grid_constant__ PairW<T, K> pw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ME = (K + 1) / 2;
  constexpr int WPB = NT / 32;
  const int TX = va.tx, TY = va.ty;
  __shared__ long long sbeg[MEMBER_CACHE];
  auto lookup = [&](long long it, int phase) {
    return nmem <= MEMBER_CACHE ? find_member_cached(sbeg, nmem, it) : find_member(mem, nmem, it, phase);
  };
  const bool stamper = va.stamp && blockIdx.x == 0 && threadIdx.x == 0;
  if (stamper) va.stamp[0] = va.stamp[1] = va.stamp[2] = global_ns();
  // ghost ring and edge points of member m at this stage
  auto gext_of = [&](const MemberDev<T> &m) -> const T * {
    return va.tape ? va.tape + m.tape_off + (long long)va.tape_stage * (m.tape_ge + m.tape_ee) : m.gext;
  };
  auto ep_of = [&](const MemberDev<T> &m) -> const T * {
    return va.tape ? va.tape + m.tape_off + (long long)va.tape_stage * (m.tape_ge + m.tape_ee) + m.tape_ge : m.ep;
  };
  if (!va.have_fwd) {
    // forward recompute: ghost rows (as the forward stage's first phase), then tiles
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (long long it = (long long)blockIdx.x * WPB + warp; it < n_ghost; it += (long long)gridDim.x * WPB)
      ghost_item(it, lane, va.ggrp, va.ngrp, va.gmem, mem, va.qs);
    if (!grid_sync(bar, status, inject)) return;
    if (stamper) va.stamp[1] = global_ns();
    stage_member_begins(sbeg, mem, nmem, 1);
    for (long long it = blockIdx.x; it < n_tile; it += gridDim.x) {
      const MemberDev<T> &m = mem[lookup(it, 1)];
      const int local = int(it - m.b_tile);
      const int p = local / (m.tiles_x * m.tiles_y);
      const int rem = local - p * m.tiles_x * m.tiles_y;
      const int ty = rem / m.tiles_x, tx = rem - ty * m.tiles_x;
      recon_tpp_tile<T, K>(smem_raw, p, tx * TX, ty * TY, TX, TY, va.qs + m.off, m.gext, pw.w, m.Xg, m.t1w, m.src8,
                           m.ep, m.sb, m.N, m.ne, va.omega, va.fc);
    }
    if (!grid_sync(bar, status, inject)) return;
    if (stamper) va.stamp[2] = global_ns();
  }
  // edge quadrature and LMARS adjoints, one thread per edge
  stage_member_begins(sbeg, mem, nmem, 2);
  for (long long it = (long long)blockIdx.x * NT + threadIdx.x; it < n_flux; it += (long long)gridDim.x * NT) {
    const MemberDev<T> &m = mem[lookup(it, 2)];
    flux_adj_item<T, ME>((int)(it - m.b_flux), ep_of(m), m.mx, va.gw, m.bedge, m.bconv, va.lamL + m.off, m.lep, m.N,
                         m.inv_dx);
  }
  if (!grid_sync(bar, status, inject)) return;
  if (stamper) va.stamp[3] = global_ns();
  // reconstruction and source adjoints, one block per tile
  stage_member_begins(sbeg, mem, nmem, 1);
  for (long long it = blockIdx.x; it < n_tile; it += gridDim.x) {
    const MemberDev<T> &m = mem[lookup(it, 1)];
    const int local = int(it - m.b_tile);
    const int p = local / (m.tiles_x * m.tiles_y);
    const int rem = local - p * m.tiles_x * m.tiles_y;
    const int ty = rem / m.tiles_x, tx = rem - ty * m.tiles_x;
    recon_tpp_adj_tile<T, K>(smem_raw, p, tx * TX, ty * TY, TX, TY, local, va.qs + m.off, gext_of(m), va.w1, m.Xg,
                             m.t1w, m.lep, va.lamL + m.off, m.tbuf, m.N, m.ne, va.omega, va.fc);
  }
  if (!grid_sync(bar, status, inject)) return;
  if (stamper) va.stamp[4] = global_ns();
  // gather of the tiles' extended regions, one thread per extended cell
  stage_member_begins(sbeg, mem, nmem, 4);
  for (long long it = (long long)blockIdx.x * NT + threadIdx.x; it < n_gather; it += (long long)gridDim.x * NT) {
    const MemberDev<T> &m = mem[lookup(it, 4)];
    gather_tiles_item<T, K>(it - m.b_gather, m.tbuf, TX, TY, m.ldir, m.lring, m.N);
  }
  if (!grid_sync(bar, status, inject)) return;
  if (stamper) va.stamp[5] = global_ns();
  // transposed ghost operator and the Runge-Kutta combination: a thread per cell that no
  // ghost row reads, then GADJ_LANES lanes per band cell (the lane items padded to whole
  // warps: every lane of a warp reaches the group's shuffles; a member's lanes start at a
  // multiple of GADJ_LANES, so no group straddles two members or two warps)
  stage_member_begins(sbeg, mem, nmem, 3);
  for (long long it = (long long)blockIdx.x * NT + threadIdx.x; it < n_cell; it += (long long)gridDim.x * NT) {
    const MemberDev<T> &m = mem[lookup(it, 3)];
    auto off = [&](const T *p) -> const T * { return p ? p + m.off : nullptr; };
    ghost_adj_interior(it - m.b_cell, m.ldir, m.gtp, off(va.x), off(va.y), off(va.z), va.out + m.off, va.a, va.b,
                       va.d, va.c, m.N);
  }
  stage_member_begins(sbeg, mem, nmem, 5);
  const long long n_band_pad = (n_band + 31) / 32 * 32;
  for (long long it = (long long)blockIdx.x * NT + threadIdx.x; it < n_band_pad; it += (long long)gridDim.x * NT) {
    const bool valid = it < n_band;
    const MemberDev<T> &m = mem[lookup(valid ? it : n_band - 1, 5)];
    const long long local = (valid ? it : n_band - 1) - m.b_band;
    auto off = [&](const T *p) -> const T * { return p ? p + m.off : nullptr; };
    ghost_adj_band(valid, local / GADJ_LANES, (int)(local % GADJ_LANES), m.gband, m.ldir, m.lring, m.gtp, m.gtr,
                   m.gtv, off(va.x), off(va.y), off(va.z), va.out + m.off, va.a, va.b, va.d, va.c, m.N, m.ne);
  }
  if (va.stamp) {
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(va.stamp + 6, global_ns());
  }
}

// -------------------------------------------------------------------------------------
// host side
// -------------------------------------------------------------------------------------
template <typename T>
static int build_members(hope_ctx *ctx, int TX, int TY, std::vector<MemberDev<T>> &out, long long n[6]) {
  out.clear();
  long long bg = 0, bt = 0, bf = 0, bc = 0, bgat = 0, bband = 0, tape_acc = 0;
  for (auto &g : ctx->grids) {
    MemberDev<T> m{};
    m.N = g.N;
    m.inv_dx = (T)(2.0 * g.N / HOPE_PI);
    m.ne = g.ne;
    m.off = (long long)g.off;
    m.grow = g.grow;
    m.gcol = g.gcol;
    m.gsym = g.gsym;
    m.gdst = g.gdst;
    m.gval = (const T *)g.gval;
    m.trow = g.trow;
    m.tcol = g.tcol;
    m.tval = g.tval;
    m.gs = (size_t)g.gstride;
    m.gext = (T *)g.gext;
    m.Xg = (const T *)g.Xg;
    m.t1w = (const T *)g.t1w;
    m.src8 = (const T *)g.src8;
    m.mx = (const T *)g.mx;
    m.bconv = (const T *)g.bconv;
    m.bedge = g.bedge;
    m.ep = (T *)g.ep;
    m.sb = (T *)g.sb;
    m.fx = (T *)g.fx;
    m.fy = (T *)g.fy;
    m.tiles_x = (g.N + TX - 1) / TX;
    m.tiles_y = (g.N + TY - 1) / TY;
    m.lep = (T *)g.lep;
    m.tbuf = (T *)g.tbuf;
    m.lring = (T *)g.lring;
    m.ldir = (T *)g.ldir;
    m.gtp = g.gtp;
    m.gtr = g.gtr;
    m.gtv = (const T *)g.gtv;
    m.gband = g.gband;
    m.nband = g.nband;
    m.b_band = bband;
    bband += g.nband * GADJ_LANES;
    m.tape_ge = 3LL * 6 * g.ne * g.ne;
    m.tape_ee = 4LL * 3 * ctx->me * 6 * g.N * g.N;
    m.tape_off = 2LL * (long long)ctx->total + tape_acc;
    tape_acc += 3 * (m.tape_ge + m.tape_ee);
    m.b_gather = bgat;
    bgat += 6LL * g.ne * g.ne;
    m.b_ghost = bg;
    m.b_tile = bt;
    m.b_flux = bf;
    m.b_cell = bc;
    bg += g.rows;
    bt += 6LL * m.tiles_x * m.tiles_y;
    bf += 12LL * g.N * (g.N - 1) + 12LL * g.N;
    bc += 6LL * g.N * g.N;
    out.push_back(m);
  }
  n[0] = bg;
  n[1] = bt;
  n[2] = bf;
  n[3] = bc;
  n[4] = bgat;
  n[5] = bband;
  return HOPE_OK;
}

// Candidate shapes: tiles of 32 to 256 cells on 128- and 256-thread blocks.
static const EnsembleShape kCandidates[] = {
    {16, 8, 128}, {8, 16, 128}, {32, 4, 128}, {16, 4, 128}, {12, 10, 128}, {24, 5, 128}, {8, 8, 128},
    {16, 16, 256}, {32, 8, 256}, {16, 12, 256}, {24, 10, 256}, {12, 20, 256}};

template <typename T, int K>
static size_t stage_smem(const EnsembleShape &c) {
  return recon_tile_smem_bytes<T, K>(c.tx, c.ty);
}

template <typename T, int K>
static size_t vjp_smem(const EnsembleShape &c) {
  const size_t f = recon_tile_smem_bytes<T, K>(c.tx, c.ty), a = recon_adj_tile_smem_bytes<T, K>(c.tx, c.ty, c.nt);
  return f > a ? f : a;
}

// Cooperative launch of a persistent kernel with every block resident; *grid caches the
// resident grid of this (kernel, shape).
template <typename Kern, typename... Args>
static int launch_coop(hope_ctx *ctx, Kern kern, int nt, size_t smem, int *grid, const char *what, cudaStream_t st,
                       Args... args) {
  if (*grid == 0) {
    // opt in to the largest dynamic size the kernel can have (the block's limit less its
    // static shared memory), so every candidate's tile fits
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
      set_error(std::string(what) + ": kernel attributes unavailable");
      return HOPE_ECUDA;
    }
    const int dyn_max = optin - (int)fa.sharedSizeBytes;
    if ((long long)smem > dyn_max ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess) {
      set_error(std::string(what) + ": shared-memory attribute failed");
      return HOPE_ECUDA;
    }
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (per_sm < 1) {
      set_error(std::string(what) + ": no resident block fits");
      return HOPE_EUNSUPPORTED;
    }
    *grid = per_sm * sms;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(*grid);
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
  if (e != cudaSuccess) {
    set_error(std::string(what) + " launch: " + cudaGetErrorString(e));
    return HOPE_ECUDA;
  }
  return HOPE_OK;
}

template <typename T, int K>
static int launch_any(hope_ctx *ctx, EnsembleState &es, const StageArgs<T> &sa, cudaStream_t st) {
  const EnsembleShape &c = es.cand[es.shape];
  const MemberDev<T> *mem = (const MemberDev<T> *)es.members;
  const long long *n = es.items;
  const unsigned inject = es.inject_timeout ? 1u : 0u;
  es.inject_timeout = 0;
  const int nmem = (int)ctx->grids.size();
  const size_t smem = stage_smem<T, K>(c);
  const PairW<T, K> pw = pair_weights<T, K>(ctx->w1_host.data());
  if (c.nt == 256)
    return launch_coop(ctx, k_stage_persistent<T, K, 256>, 256, smem, &es.grid[es.shape], "persistent stage", st, mem,
                       nmem, n[0], n[1], n[2], n[3], sa, es.barrier, ctx->status, inject, pw);
  return launch_coop(ctx, k_stage_persistent<T, K, 128>, 128, smem, &es.grid[es.shape], "persistent stage", st, mem,
                     nmem, n[0], n[1], n[2], n[3], sa, es.barrier, ctx->status, inject, pw);
}

template <typename T>
static int stage_persistent_t(hope_ctx *ctx, const void *qs, const void *q0, void *out, int mode, double a, double b,
                              double c, const void *q0l, const void *qsl, void *outl, cudaStream_t st) {
  EnsembleState &es = *ctx->ens;
  StageArgs<T> sa;
  sa.qs = (const T *)qs;
  sa.q0 = (const T *)q0;
  sa.out = (T *)out;
  sa.q0l = (const T *)q0l;
  sa.qsl = (const T *)qsl;
  sa.outl = (T *)outl;
  sa.a = (T)a;
  sa.b = (T)b;
  sa.c = (T)c;
  sa.alo = coef_lo<T>(a);
  sa.blo = coef_lo<T>(b);
  sa.clo = coef_lo<T>(c);
  sa.mode = mode;
  sa.omega = (T)ctx->omega;
  for (int t = 0; t < 18; ++t) sa.fc.c[t] = (T)ctx->fcoef[t];
  sa.gw = (const T *)ctx->gw;
  sa.stamp = ctx->profiling && ctx->prof_stage >= 0 ? es.stamps + 5 * ctx->prof_stage : nullptr;
  sa.ggrp = (const GhostGroup *)es.ggrp;
  sa.gmem = es.gmem;
  sa.ngrp = es.ngrp;
  sa.tx = es.cand[es.shape].tx;
  sa.ty = es.cand[es.shape].ty;
  if (sa.stamp && cudaMemsetAsync(sa.stamp + 4, 0, sizeof(unsigned long long), st) != cudaSuccess) return HOPE_ECUDA;
  switch (ctx->k) {
    case 3: return launch_any<T, 3>(ctx, es, sa, st);
    case 5: return launch_any<T, 5>(ctx, es, sa, st);
    case 7: return launch_any<T, 7>(ctx, es, sa, st);
    case 9: return launch_any<T, 9>(ctx, es, sa, st);
    case 11: return launch_any<T, 11>(ctx, es, sa, st);
  }
  return HOPE_EINVAL;
}

int stage_persistent(hope_ctx *ctx, const void *qs, const void *q0, void *out, int mode, double a, double b,
                     double c, const void *q0l, const void *qsl, void *outl, cudaStream_t st) {
  if (ctx->prec == HOPE_FP64)
    return stage_persistent_t<double>(ctx, qs, q0, out, mode, a, b, c, q0l, qsl, outl, st);
  return stage_persistent_t<float>(ctx, qs, q0, out, mode, a, b, c, q0l, qsl, outl, st);
}

template <typename T, int K>
static int launch_vjp_any(hope_ctx *ctx, EnsembleState &es, const VjpArgs<T> &va, cudaStream_t st) {
  const EnsembleShape &c = es.cand[es.shape];
  const MemberDev<T> *mem = (const MemberDev<T> *)es.members;
  const long long *n = es.items;
  const unsigned inject = es.inject_timeout ? 1u : 0u;
  es.inject_timeout = 0;
  const int nmem = (int)ctx->grids.size();
  const size_t smem = vjp_smem<T, K>(c);
  const PairW<T, K> pw = pair_weights<T, K>(ctx->w1_host.data());
  if (c.nt == 256)
    return launch_coop(ctx, k_vjp_persistent<T, K, 256>, 256, smem, &es.vgrid[es.shape], "persistent stage VJP", st,
                       mem, nmem, n[0], n[1], n[2], n[3], n[4], n[5], va, es.barrier, ctx->status, inject, pw);
  return launch_coop(ctx, k_vjp_persistent<T, K, 128>, 128, smem, &es.vgrid[es.shape], "persistent stage VJP", st,
                     mem, nmem, n[0], n[1], n[2], n[3], n[4], n[5], va, es.barrier, ctx->status, inject, pw);
}

// The member table of the current shape (with the adjoint scratch pointers once they
// exist), uploaded into the context's one device array: captured graphs keep pointing at it,
// but a change of shape makes them stale (the caller drops them).
template <typename T>
static int upload_members_t(hope_ctx *ctx) {
  EnsembleState &es = *ctx->ens;
  const EnsembleShape &c = es.cand[es.shape];
  std::vector<MemberDev<T>> mv;
  const long long ghost_items = es.items[0];
  build_members<T>(ctx, c.tx, c.ty, mv, es.items);
  if (es.ngrp) es.items[0] = ghost_items;  // ghost work is itemised by operator groups
  if (!es.members && cudaMalloc(&es.members, sizeof(MemberDev<T>) * mv.size()) != cudaSuccess) return HOPE_ENOMEM;
  if (cudaMemcpy(es.members, mv.data(), sizeof(MemberDev<T>) * mv.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("persistent stage: member table upload failed");
    return HOPE_ECUDA;
  }
  es.adj_ready = ctx->grids[0].lep != nullptr;
  return HOPE_OK;
}

static int upload_members(hope_ctx *ctx) {
  return ctx->prec == HOPE_FP64 ? upload_members_t<double>(ctx) : upload_members_t<float>(ctx);
}

template <typename T>
static int vjp_persistent_t(hope_ctx *ctx, const void *qs, const void *lamL, void *out, const void *x, const void *y,
                            const void *z, double a, double b, double d, double c, int have_fwd, const void *tape,
                            int tape_stage, cudaStream_t st) {
  EnsembleState &es = *ctx->ens;
  if (!es.adj_ready) {
    int rc = upload_members_t<T>(ctx);
    if (rc) return rc;
  }
  VjpArgs<T> va;
  va.qs = (const T *)qs;
  va.lamL = (const T *)lamL;
  va.x = (const T *)x;
  va.y = (const T *)y;
  va.z = (const T *)z;
  va.out = (T *)out;
  va.a = (T)a;
  va.b = (T)b;
  va.d = (T)d;
  va.c = (T)c;
  va.have_fwd = have_fwd;
  va.tape = (const T *)tape;
  va.tape_stage = tape_stage;
  va.omega = (T)ctx->omega;
  for (int t = 0; t < 18; ++t) va.fc.c[t] = (T)ctx->fcoef[t];
  va.gw = (const T *)ctx->gw;
  va.w1 = (const T *)ctx->w1;
  va.ggrp = (const GhostGroup *)es.ggrp;
  va.gmem = es.gmem;
  va.ngrp = es.ngrp;
  va.stamp = ctx->profiling ? es.vstamps : nullptr;
  va.tx = es.cand[es.shape].tx;
  va.ty = es.cand[es.shape].ty;
  if (va.stamp && cudaMemsetAsync(va.stamp + 6, 0, sizeof(unsigned long long), st) != cudaSuccess) return HOPE_ECUDA;
  switch (ctx->k) {
    case 3: return launch_vjp_any<T, 3>(ctx, es, va, st);
    case 5: return launch_vjp_any<T, 5>(ctx, es, va, st);
    case 7: return launch_vjp_any<T, 7>(ctx, es, va, st);
    case 9: return launch_vjp_any<T, 9>(ctx, es, va, st);
    case 11: return launch_vjp_any<T, 11>(ctx, es, va, st);
  }
  return HOPE_EINVAL;
}

int vjp_persistent(hope_ctx *ctx, const void *qs, const void *lamL, void *out, const void *x, const void *y,
                   const void *z, double a, double b, double d, double c, int have_fwd, const void *tape,
                   int tape_stage, cudaStream_t st) {
  if (ctx->prec == HOPE_FP64)
    return vjp_persistent_t<double>(ctx, qs, lamL, out, x, y, z, a, b, d, c, have_fwd, tape, tape_stage, st);
  return vjp_persistent_t<float>(ctx, qs, lamL, out, x, y, z, a, b, d, c, have_fwd, tape, tape_stage, st);
}

template <typename T>
static int ensemble_init_t(hope_ctx *ctx) {
  EnsembleState *es = new EnsembleState();
  ctx->ens = es;
  for (const EnsembleShape &c : kCandidates) {
    // a candidate whose tile needs more shared memory than a block may have is left out
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    size_t need = 0;
    switch (ctx->k) {
      case 3: need = vjp_smem<T, 3>(c); break;
      case 5: need = vjp_smem<T, 5>(c); break;
      case 7: need = vjp_smem<T, 7>(c); break;
      case 9: need = vjp_smem<T, 9>(c); break;
      default: need = vjp_smem<T, 11>(c); break;
    }
    const size_t static_smem = sizeof(long long) * MEMBER_CACHE + 64;  // the kernels' own shared arrays
    if (need + static_smem <= (size_t)optin && es->ncand < ENS_MAX_SHAPES) es->cand[es->ncand++] = c;
  }
  if (es->ncand == 0) {
    set_error("persistent stage: no tile shape fits the shared memory");
    return HOPE_EUNSUPPORTED;
  }
  es->shape = 0;
  {
    // ghost-fill groups: members that share an operator (the same table pointers)
    std::vector<const int *> tables;
    std::vector<std::vector<int>> members;
    for (int i = 0; i < (int)ctx->grids.size(); ++i) {
      const int *t = ctx->grids[i].grow;
      size_t g = 0;
      while (g < tables.size() && tables[g] != t) ++g;
      if (g == tables.size()) {
        tables.push_back(t);
        members.emplace_back();
      }
      members[g].push_back(i);
    }
    std::vector<GhostGroup> groups;
    std::vector<int> gm;
    long long b = 0;
    for (size_t g = 0; g < tables.size(); ++g) {
      GhostGroup G;
      G.b_item = b;
      G.rows = (int)ctx->grids[members[g][0]].rows;
      G.nmem = (int)members[g].size();
      G.nchunk = (G.nmem + GHOST_GROUP_CHUNK - 1) / GHOST_GROUP_CHUNK;
      G.first = (int)gm.size();
      gm.insert(gm.end(), members[g].begin(), members[g].end());
      b += (long long)G.rows * G.nchunk;
      groups.push_back(G);
    }
    es->items[0] = b;
    es->ngrp = (int)groups.size();
    if (cudaMalloc(&es->ggrp, sizeof(GhostGroup) * groups.size()) != cudaSuccess ||
        cudaMalloc(&es->gmem, sizeof(int) * gm.size()) != cudaSuccess)
      return HOPE_ENOMEM;
    cudaMemcpy(es->ggrp, groups.data(), sizeof(GhostGroup) * groups.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(es->gmem, gm.data(), sizeof(int) * gm.size(), cudaMemcpyHostToDevice);
  }
  if (cudaMalloc(&es->barrier, 2 * sizeof(unsigned)) != cudaSuccess) return HOPE_ENOMEM;
  if (cudaMalloc(&es->stamps, 5 * PROF_STAGES * sizeof(unsigned long long)) != cudaSuccess) return HOPE_ENOMEM;
  if (cudaMalloc(&es->vstamps, 7 * sizeof(unsigned long long)) != cudaSuccess) return HOPE_ENOMEM;
  cudaMemset(es->vstamps, 0, 7 * sizeof(unsigned long long));
  cudaMemset(es->stamps, 0, 5 * PROF_STAGES * sizeof(unsigned long long));
  cudaMemset(es->barrier, 0, 2 * sizeof(unsigned));
  return upload_members_t<T>(ctx);
}

int ensemble_init(hope_ctx *ctx) {
  return ctx->prec == HOPE_FP64 ? ensemble_init_t<double>(ctx) : ensemble_init_t<float>(ctx);
}

void ensemble_free(hope_ctx *ctx) {
  if (!ctx->ens) return;
  if (ctx->ens->members) cudaFree(ctx->ens->members);
  if (ctx->ens->barrier) cudaFree(ctx->ens->barrier);
  if (ctx->ens->stamps) cudaFree(ctx->ens->stamps);
  if (ctx->ens->vstamps) cudaFree(ctx->ens->vstamps);
  if (ctx->ens->ggrp) cudaFree(ctx->ens->ggrp);
  if (ctx->ens->gmem) cudaFree(ctx->ens->gmem);
  delete ctx->ens;
  ctx->ens = nullptr;
}

void ensemble_reset_barrier(hope_ctx *ctx) {
  if (ctx->ens && ctx->ens->barrier) cudaMemset(ctx->ens->barrier, 0, 2 * sizeof(unsigned));
}

// Time `reps` tendency stages of every candidate shape on the scratch buffers and keep
// the fastest.  ms_out (may be null, ENS_MAX_SHAPES floats) receives the per-shape times
// (-1 for a shape that failed to launch and past the candidates).
int ensemble_autotune(hope_ctx *ctx, const void *qs, void *out, int reps, float *ms_out, cudaStream_t st) {
  EnsembleState &es = *ctx->ens;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_s = 0;
  if (ms_out)
    for (int s = 0; s < ENS_MAX_SHAPES; ++s) ms_out[s] = -1.0f;
  int rc = HOPE_OK;
  for (int s = 0; s < es.ncand; ++s) {
    es.shape = s;
    if ((rc = upload_members(ctx))) break;
    if (stage_persistent(ctx, qs, nullptr, out, 0, 0, 0, 0, nullptr, nullptr, nullptr, st)) continue;
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) stage_persistent(ctx, qs, nullptr, out, 0, 0, 0, 0, nullptr, nullptr, nullptr, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms_out) ms_out[s] = ms;
    if (ms < best) {
      best = ms;
      best_s = s;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  es.shape = best_s;
  es.tuned = 1;
  if (rc == HOPE_OK) rc = upload_members(ctx);
  if (rc) return rc;
  return cudaGetLastError() == cudaSuccess ? HOPE_OK : HOPE_ECUDA;
}

void ensemble_shape(const hope_ctx *ctx, int *tx, int *ty, int *grid) {
  const EnsembleState &es = *ctx->ens;
  *tx = es.cand[es.shape].tx;
  *ty = es.cand[es.shape].ty;
  *grid = es.grid[es.shape];
}

int ensemble_num_shapes(const hope_ctx *ctx) { return ctx->ens ? ctx->ens->ncand : 0; }

size_t ensemble_tile_buf_elems(const hope_ctx *ctx, int N) {
  size_t m = 0;
  for (int s = 0; ctx->ens && s < ctx->ens->ncand; ++s)
    m = std::max(m, (size_t)tile_buf_elems(N, ctx->k, ctx->ens->cand[s].tx, ctx->ens->cand[s].ty));
  return m;
}

}  // namespace hope
