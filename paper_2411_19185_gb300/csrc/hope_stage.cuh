// hope_stage.cuh -- per-stage launch sequences (forward stage, stage VJP) of the HOPE
// GB300 library, templated on precision and order; instantiated per (precision, order
// group) in hope_stage_*.cu so the heavy kernels compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <utility>

#include "hope_adjoint.cuh"
#include "hope_internal.h"
#include "hope_kernels.cuh"
#include "hope_setup_math.cuh"
#include "hope_weno.cuh"
#include "hope_weno1d.cuh"

namespace hope {

#define HOPE_CUDA_TRY(expr)                                                              \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess) {                                                             \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                     \
      return HOPE_ECUDA;                                                                 \
    }                                                                                    \
  } while (0)

// Launch shape of a grid-strided kernel over n equal items: every block resident from
// the start (at most nsm x the kernel's resident blocks per SM at that block size) and
// every SM given the same number of items, so that an FP64-bound kernel neither ends with
// some SMs running one block more than the others nor with a partial second wave.  Tries
// 1, 2, ... items per thread and block sizes that are multiples of 32 up to max_tpb, and
// keeps the shape that wastes the fewest thread slots.
template <typename Kern>
inline void balanced_grid(Kern kern, long long n, int nsm, int max_tpb, int *blocks, int *tpb) {
  double best = -1.0;
  *tpb = max_tpb;
  *blocks = (int)((n + max_tpb - 1) / max_tpb);
  for (int k = 1; k <= 4 && best < 0.97; ++k) {
    const long long nt = (n + k - 1) / k;  // threads
    for (int m = 1; m <= 32; ++m) {
      const long long t = 32 * ((nt + 32LL * nsm * m - 1) / (32LL * nsm * m));
      if (t > max_tpb) continue;
      if (t < 64) break;
      int resident = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kern, (int)t, 0) != cudaSuccess) resident = 1;
      if (m > resident) continue;
      const long long b = (nt + t - 1) / t;
      const double eff = (double)n / ((double)nsm * ((b + nsm - 1) / nsm) * t * k);
      if (eff > best + 1e-3) {
        best = eff;
        *tpb = (int)t;
        *blocks = (int)b;
      }
    }
  }
}

// Resident-grid size of a row-strided kernel with 256-thread blocks.
template <typename Kern>
inline int resident_blocks(Kern kern, const hope_ctx *ctx, long long rows_x32) {
  int resident = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kern, 256, 0) != cudaSuccess || resident < 1)
    resident = 1;
  const long long need = (rows_x32 + 255) / 256;
  const long long cap = (long long)resident * ctx->nsm;
  return (int)(need < cap ? need : cap);
}

template <typename T>
inline FCoef<T> fcoef(const hope_ctx *ctx) {
  FCoef<T> f;
  for (int t = 0; t < 18; ++t) f.c[t] = (T)ctx->fcoef[t];
  return f;
}

template <typename T, int K>
int launch_recon_weno(hope_ctx *ctx, Grid &g, const T *qs, cudaStream_t st) {
  if constexpr (K > HOPE_WENO_MAXK) {
    (void)ctx; (void)g; (void)qs; (void)st;
    set_error("WENO2D supports orders up to 9");
    return HOPE_EUNSUPPORTED;
  } else {
  const int N = g.N, TX = g.wtx, TY = g.wty;
  dim3 grid((N + TX - 1) / TX, (N + TY - 1) / TY, 6);
  const int threads = (TX * TY + 31) / 32 * 32;
  const size_t smem = weno_tile_smem_bytes<T, K>(TX, TY, threads);
  auto args = [&](auto kern) {
    kern<<<grid, threads, smem, st>>>(qs, (const T *)g.gext, (const T *)ctx->wsub, (const T *)ctx->gpm,
                                      (const T *)ctx->sig, (const T *)ctx->bform, (const T *)ctx->bcoef,
                                      (const T *)g.Xg, (const T *)g.t1w, (T *)g.ep, (T *)g.sb, N, g.ne, TX, TY,
                                      (T)ctx->omega, fcoef<T>(ctx), (T)ctx->eps, (const T *)g.tsext,
                                      (const T *)g.tsep, (const T *)g.tscp);
  };
  if (g.tsext) {
    // over a surface: FP64 takes the runtime-tile form (any shape), FP32 the 16 x 8 form
    args(k_recon_weno<T, K, sizeof(T) == 8, true>);
    return HOPE_OK;
  }
  if constexpr (sizeof(T) == 8) {
    if (TX != REC_TX || TY != REC_TY) {
      args(k_recon_weno<T, K, true>);
      return HOPE_OK;
    }
  }
  args(k_recon_weno<T, K, false>);
  return HOPE_OK;
  }
}

template <typename T, int K>
int launch_recon_weno1d(hope_ctx *ctx, Grid &g, const T *qs, cudaStream_t st) {
  if constexpr (K != 5) {
    (void)ctx; (void)g; (void)qs; (void)st;
    set_error("WENO1D is fifth order only");
    return HOPE_EUNSUPPORTED;
  } else {
    const int N = g.N;
    dim3 grid((N + REC_TX - 1) / REC_TX, (N + REC_TY - 1) / REC_TY, 6);
    k_recon_weno1d<T, K><<<grid, REC_TX * REC_TY, sizeof(T) * Weno1dShape<T, K>::smem_elems(), st>>>(
        qs, (const T *)g.gext, (const T *)ctx->wsub, (const T *)ctx->w1gpm, (const T *)ctx->w1sig,
        (const T *)ctx->w1bf, (const T *)g.Xg, (const T *)g.t1w, (T *)g.ep, (T *)g.sb, N, g.ne, (T)ctx->omega,
        fcoef<T>(ctx), (T)ctx->eps);
    return HOPE_OK;
  }
}

template <typename T, int K>
int weno_set_smem_attr() {
  if constexpr (K > HOPE_WENO_MAXK) {
    return HOPE_OK;
  } else {
  size_t smem = sizeof(T) * WenoShape<T, K>::smem_elems();
  size_t smem_adj = sizeof(T) * WenoAdjShape<T, K>::smem_elems();
  if (K <= HOPE_WENO_ADJ_MAXK && smem_adj <= 227 * 1024) {
    cudaError_t e2 = cudaFuncSetAttribute(k_recon_weno_adj<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem_adj);
    if (e2 == cudaSuccess)
      e2 = cudaFuncSetAttribute(k_recon_weno_adj<T, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_adj);
    if (e2 != cudaSuccess) {
      set_error(std::string("WENO adjoint shared memory attribute: ") + cudaGetErrorString(e2));
      return HOPE_ECUDA;
    }
  }
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  (void)smem;
  cudaError_t e = cudaFuncSetAttribute(k_recon_weno<T, K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if constexpr (K == 5) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_recon_weno1d<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(sizeof(T) * Weno1dShape<T, K>::smem_elems()));
  }
  if constexpr (sizeof(T) == 8) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_recon_weno<T, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  }
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_recon_weno<T, K, sizeof(T) == 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin);
  if (e != cudaSuccess) {
    set_error(std::string("WENO shared memory attribute: ") + cudaGetErrorString(e));
    return HOPE_ECUDA;
  }
  return HOPE_OK;
  }
}

template <typename T, int K>
int launch_recon_weno_adj(hope_ctx *ctx, Grid &g, const T *qs, const T *lamL, cudaStream_t st) {
  if constexpr (K > HOPE_WENO_ADJ_MAXK) {
    (void)ctx; (void)g; (void)qs; (void)lamL; (void)st;
    set_error("the WENO2D adjoint supports orders up to 7");
    return HOPE_EUNSUPPORTED;
  } else {
  const int N = g.N;
  dim3 grid((N + REC_TX - 1) / REC_TX, (N + REC_TY - 1) / REC_TY, 6);
  size_t smem = sizeof(T) * WenoAdjShape<T, K>::smem_elems();
  if (smem > 227 * 1024) {
    set_error("WENO adjoint: order too high for the per-cell shared-memory staging");
    return HOPE_EUNSUPPORTED;
  }
  auto kern = g.tsext ? k_recon_weno_adj<T, K, true> : k_recon_weno_adj<T, K, false>;
  kern<<<grid, REC_TX * REC_TY, smem, st>>>(
      qs, (const T *)g.gext, (const T *)ctx->wsub, (const T *)ctx->gpm, (const T *)ctx->sig, (const T *)ctx->bform,
      (const T *)ctx->bcoef, (const T *)g.Xg, (const T *)g.t1w, (const T *)g.lep, lamL, (T *)g.grad, N, g.ne,
      (T)ctx->omega, fcoef<T>(ctx), (T)ctx->eps, (const T *)g.tsext, (const T *)g.tscp);
  return HOPE_OK;
  }
}

// Launch of a stage kernel with programmatic stream serialization (the kernel calls
// griddep_wait() before touching memory; see hope_kernels.cuh).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// -------------------------------------------------------------------------------
// One stage on one grid: out = L(qs) (mode 0) or a*q0 + b*qs + c*L(qs) (mode 1).
// -------------------------------------------------------------------------------
// TPP reconstruction + sources of one grid with the grid's tile shape.
template <typename T, int K>
inline cudaError_t launch_recon_tpp(hope_ctx *ctx, Grid &g, const T *qs, cudaStream_t st) {
  const int N = g.N, TX = g.rtx, TY = g.rty;
  dim3 grid((N + TX - 1) / TX, (N + TY - 1) / TY, 6);
  const int threads = (TX * TY + 31) / 32 * 32;
  // over a surface psi_B (eq. 2.14) is added in the tile's epilogue
  auto kern = g.tsep ? k_recon_tpp<T, K, true> : k_recon_tpp<T, K, false>;
  return launch_pdl(kern, grid, dim3(threads), recon_tile_smem_bytes<T, K>(TX, TY), st, qs, (const T *)g.gext,
                    (const T *)g.Xg, (const T *)g.t1w, (const T *)g.src8, (T *)g.ep, (T *)g.sb, N, g.ne, TX, TY,
                    (T)ctx->omega, fcoef<T>(ctx), (const T *)g.ttw, (const T *)g.ttb,
                    pair_weights<T, K>(ctx->w1_host.data()));
}

template <typename T, int K>
inline int stage_grid(hope_ctx *ctx, Grid &g, const T *qs, const T *q0, T *out, int mode, double a,
                      double b, double c, const T *q0l, const T *qsl, T *outl, cudaStream_t st) {
  constexpr int ME = (K + 1) / 2;
  const int N = g.N, ne = g.ne;
  const bool prof = ctx->prof_stage >= 0 && &g == &ctx->grids[0];
  auto mark = [&](int t) {
    if (prof) cudaEventRecordWithFlags(ctx->prof_ev[ctx->prof_stage][t], st, cudaEventRecordExternal);
  };
  mark(0);
  // ghost ring
  if (g.rows > 0) {
    if (!g.ghost_grid) g.ghost_grid = resident_blocks(k_ghost<T>, ctx, g.rows * 32);
    HOPE_CUDA_TRY(launch_pdl(k_ghost<T>, dim3(g.ghost_grid), dim3(256), 0, st, qs, (T *)g.gext, g.grow, g.gcol,
                             (const T *)g.gval, g.gdst, g.gsym, g.trow, g.tcol, g.tval, (int)g.rows, N, ne,
                             (size_t)g.gstride));
  }
  mark(1);
  // reconstruction + sources
  if (ctx->scheme == HOPE_TPP) {
    HOPE_CUDA_TRY((launch_recon_tpp<T, K>(ctx, g, qs, st)));
  } else if (ctx->scheme == HOPE_WENO1D) {
    int rc = launch_recon_weno1d<T, K>(ctx, g, qs, st);
    if (rc) return rc;
  } else {
    int rc = launch_recon_weno<T, K>(ctx, g, qs, st);
    if (rc) return rc;
  }
  // bottom topography: psi_B (eq. 2.14) added to the sources (TPP: in the reconstruction)
  if (g.tsep && ctx->scheme != HOPE_TPP) {
    const long long cells = 6LL * N * N;
    k_topo_src<T, K><<<(int)((cells + 255) / 256), 256, 0, st>>>(qs, (const T *)g.gext, (const T *)g.ttw,
                                                                 (const T *)g.ttb, (T *)g.sb, N, ne);
  }
  mark(2);
  // fluxes
  {
    long long items = 12LL * N * (N - 1) + 12LL * N;
    if (g.tsep) {
      k_flux_topo<T, ME><<<(int)((items + 255) / 256), 256, 0, st>>>(
          (const T *)g.ep, (const T *)g.mx, (const T *)ctx->gw, g.bedge, (const T *)g.bconv, (T *)g.fx, (T *)g.fy, N,
          ctx->status, (const T *)g.tsep);
    } else {
      if (!g.flux_tpb) balanced_grid(k_flux<T, ME>, items, ctx->nsm, 256, &g.flux_grid, &g.flux_tpb);
      HOPE_CUDA_TRY(launch_pdl(k_flux<T, ME>, dim3(g.flux_grid), dim3(g.flux_tpb), 0, st, (const T *)g.ep,
                               (const T *)g.mx, (const T *)ctx->gw, g.bedge, (const T *)g.bconv, (T *)g.fx,
                               (T *)g.fy, N, ctx->status));
    }
  }
  mark(3);
  // tendency + stage combination
  {
    long long cells = 6LL * N * N;
    int blocks = (int)((cells + 255) / 256);
    HOPE_CUDA_TRY(launch_pdl(k_update<T>, dim3(blocks), dim3(256), 0, st, (const T *)g.fx, (const T *)g.fy,
                             (const T *)g.sb, q0, qs, out, N, (T)(2.0 * N / HOPE_PI), mode, (T)a, (T)b, (T)c,
                             coef_lo<T>(a), coef_lo<T>(b), coef_lo<T>(c), q0l, qsl, outl, ctx->status));
  }
  mark(4);
  HOPE_CUDA_TRY(cudaGetLastError());
  return HOPE_OK;
}

// Low words of the three stage states for compensated FP32 stepping (all null in FP64).
struct LoWords {
  const void *q0l = nullptr, *qsl = nullptr;
  void *outl = nullptr;
};

template <typename T, int K>
inline int stage_all(hope_ctx *ctx, const void *qs, const void *q0, void *out, int mode, double a, double b,
                     double c, LoWords lw, cudaStream_t st) {
  for (auto &g : ctx->grids) {
    auto off = [&](const void *p) -> const T * { return p ? (const T *)p + g.off : nullptr; };
    int rc = stage_grid<T, K>(ctx, g, (const T *)qs + g.off, off(q0), (T *)out + g.off, mode, a, b, c,
                              off(lw.q0l), off(lw.qsl), lw.outl ? (T *)lw.outl + g.off : nullptr, st);
    if (rc) return rc;
  }
  return HOPE_OK;
}

typedef int (*stage_fn)(hope_ctx *, const void *, const void *, void *, int, double, double, double, LoWords,
                        cudaStream_t);

template <typename T, int K>
inline int set_smem_attr() {
  int optin = 0, dev = 0;
  HOPE_CUDA_TRY(cudaGetDevice(&dev));
  HOPE_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  HOPE_CUDA_TRY(cudaFuncSetAttribute(k_recon_tpp<T, K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  HOPE_CUDA_TRY(cudaFuncSetAttribute(k_recon_tpp<T, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  HOPE_CUDA_TRY(cudaFuncSetAttribute(k_recon_tpp_adj<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)recon_adj_smem_bytes<T, K>()));
  return weno_set_smem_attr<T, K>();
}

// -------------------------------------------------------------------------------
// One stage VJP on one grid:  out = a*x + b*y + d*z + c*(dL/dq at qs)^T lamL.
// -------------------------------------------------------------------------------
struct VjpComb {
  const void *x = nullptr, *y = nullptr, *z = nullptr;
  double a = 0, b = 0, d = 0, c = 1;
  int have_fwd = 0;  // the grids' ghost rings and edge points already hold the forward at qs
  // ensembles: with have_fwd, the ghost rings and edge points are read from this step tape's
  // stage slot instead (no copies); ignored by the per-grid path
  const void *tape = nullptr;
  int tape_stage = 0;
};

template <typename T, int K>
inline int stage_vjp_grid(hope_ctx *ctx, Grid &g, const T *qs, const T *lamL, const T *x, const T *y, const T *z,
                          T *out, const VjpComb &cb, cudaStream_t st) {
  constexpr int ME = (K + 1) / 2;
  const int N = g.N, ne = g.ne;
  if (g.rows > 0 && !cb.have_fwd) {
    if (!g.ghost_grid) g.ghost_grid = resident_blocks(k_ghost<T>, ctx, g.rows * 32);
    k_ghost<T><<<g.ghost_grid, 256, 0, st>>>(qs, (T *)g.gext, g.grow, g.gcol, (const T *)g.gval, g.gdst, g.gsym, g.trow, g.tcol,
                                       g.tval, (int)g.rows, N, ne, (size_t)g.gstride);
  }
  dim3 grid((N + REC_TX - 1) / REC_TX, (N + REC_TY - 1) / REC_TY, 6);
  if (cb.have_fwd) {
    // ghost ring and edge points restored from a step tape
  } else if (ctx->scheme == HOPE_TPP) {
    HOPE_CUDA_TRY((launch_recon_tpp<T, K>(ctx, g, qs, st)));
  } else {
    int rc = launch_recon_weno<T, K>(ctx, g, qs, st);
    if (rc) return rc;
  }
  const T inv_dx = (T)(2.0 * N / HOPE_PI);
  {
    long long items = 12LL * N * (N - 1) + 12LL * N;
    auto kern = g.tsep ? k_flux_adj<T, ME, true> : k_flux_adj<T, ME, false>;
    kern<<<(int)((items + 255) / 256), 256, 0, st>>>((const T *)g.ep, (const T *)g.mx, (const T *)ctx->gw, g.bedge,
                                                      (const T *)g.bconv, lamL, (T *)g.lep, N, inv_dx,
                                                      (const T *)g.tsep);
  }
  const long long ext_cells = 6LL * ne * ne;
  if (ctx->scheme == HOPE_TPP) {
    // per tile, the gradients added up on the tile's extended region (psi_B's transposed
    // stencil map included over a surface), then gathered per extended cell
    k_recon_tpp_adj<T, K><<<grid, REC_TX * REC_TY, recon_adj_smem_bytes<T, K>(), st>>>(
        qs, (const T *)g.gext, (const T *)ctx->w1, (const T *)g.Xg, (const T *)g.t1w, (const T *)g.lep, lamL,
        (T *)g.tbuf, N, ne, (T)ctx->omega, fcoef<T>(ctx), (const T *)g.ttw);
    k_gather_tiles<T, K><<<(int)((ext_cells + 255) / 256), 256, 0, st>>>((const T *)g.tbuf, REC_TX, REC_TY,
                                                                        (T *)g.ldir, (T *)g.lring, N);
  } else {
    int rc = launch_recon_weno_adj<T, K>(ctx, g, qs, lamL, st);
    if (rc) return rc;
    if (g.tsep) {
      // psi_B's stencil map, transposed, into the mass variable's stencil gradient
      const long long cells = 6LL * N * N;
      k_topo_src_adj<T, K><<<(int)((cells + 255) / 256), 256, 0, st>>>(lamL, (const T *)g.ttw, (T *)g.grad, N);
    }
    k_gather_adj<T, K><<<(int)((ext_cells + 255) / 256), 256, 0, st>>>((const T *)g.grad, (T *)g.ldir,
                                                                      (T *)g.lring, N);
  }
  {
    const long long cells = 6LL * N * N, nlanes = (g.nband * GADJ_LANES + 31) / 32 * 32;
    k_ghost_adj<T><<<(int)((nlanes + cells + 255) / 256), 256, 0, st>>>(
        (const T *)g.ldir, (const T *)g.lring, g.gtp, g.gtr, (const T *)g.gtv, g.gband, g.nband, nlanes, x, y, z, out,
        (T)cb.a, (T)cb.b, (T)cb.d, (T)cb.c, N, ne);
  }
  HOPE_CUDA_TRY(cudaGetLastError());
  return HOPE_OK;
}

template <typename T, int K>
inline int stage_vjp_all(hope_ctx *ctx, const void *qs, const void *lamL, void *out, const VjpComb &cb,
                         cudaStream_t st) {
  for (auto &g : ctx->grids) {
    auto off = [&](const void *p) -> const T * { return p ? (const T *)p + g.off : nullptr; };
    int rc = stage_vjp_grid<T, K>(ctx, g, off(qs), off(lamL), off(cb.x), off(cb.y), off(cb.z), (T *)out + g.off,
                                  cb, st);
    if (rc) return rc;
  }
  return HOPE_OK;
}

typedef int (*vjp_fn)(hope_ctx *, const void *, const void *, void *, const VjpComb &, cudaStream_t);





// Per-(precision, order) entry points, defined in hope_stage_<tag>.cu.
stage_fn stage_entry(int prec, int k);
vjp_fn vjp_entry(int prec, int k);
int smem_attr_entry(int prec, int k);

}  // namespace hope
