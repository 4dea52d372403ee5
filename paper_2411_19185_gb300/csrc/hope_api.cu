// hope_api.cu -- the C ABI of include/hope.h: context construction, per-stage launch
// sequences, Runge-Kutta steps (CUDA-graph replay), initial conditions, the FP64 mass
// diagnostic and the ALU-peak microbenchmark.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <queue>
#include <string>
#include <vector>

#include "hope_ensemble.h"
#include "hope_internal.h"
#include "hope_setup.h"
#include "hope_stage.cuh"

namespace hope {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }


__global__ void k_mass_final(const double *__restrict__ part, int nparts, double scale, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[b];
    *out = s * scale;
  }
}

static stage_fn pick_stage(const hope_ctx *ctx) { return stage_entry(ctx->prec, ctx->k); }

// One stage of any context: TPP ensembles as one persistent launch, else per grid.
static int run_stage(hope_ctx *ctx, const void *qs, const void *q0, void *out, int mode, double a, double b,
                     double c, LoWords lw, cudaStream_t st) {
  if (ctx->ens) return stage_persistent(ctx, qs, q0, out, mode, a, b, c, lw.q0l, lw.qsl, lw.outl, st);
  return pick_stage(ctx)(ctx, qs, q0, out, mode, a, b, c, lw, st);
}

// One stage VJP of a TPP ensemble as one persistent launch over all members.
static int vjp_ensemble(hope_ctx *ctx, const void *qs, const void *lamL, void *out, const VjpComb &cb,
                        cudaStream_t st) {
  return vjp_persistent(ctx, qs, lamL, out, cb.x, cb.y, cb.z, cb.a, cb.b, cb.d, cb.c, cb.have_fwd, cb.tape,
                        cb.tape_stage, st);
}
static vjp_fn pick_vjp(const hope_ctx *ctx) { return ctx->ens ? vjp_ensemble : vjp_entry(ctx->prec, ctx->k); }
static int set_attrs(const hope_ctx *ctx) { return smem_attr_entry(ctx->prec, ctx->k); }

// Modelled FP64-pipe time (in warp instructions of the most loaded SM) of the TPP
// reconstruction with TX x TY tiles on an N x N panel: a tile's x-pass issues NPOS*K FMAs
// per (variable, extended row, valid column) item, its cell phase a fixed count per
// 32 valid cells (the edge- and cell-point y-pass and the sources), plus its loads; tiles
// go in launch order to the least loaded SM.
static double recon_tile_cost(int N, int K, int TX, int TY, int nsm) {
  const int H = (K - 1) / 2, me = (K + 1) / 2, npos = me + 2;
  const int threads = (TX * TY + 31) / 32 * 32;
  const double per_item = (double)npos * K;
  const double per_warp_cells = (double)(4 * me + me * me) * 3 * K + (double)me * me * 22;
  const int nbx = (N + TX - 1) / TX, nby = (N + TY - 1) / TY;
  std::vector<double> load(nsm, 0.0);
  std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>, std::greater<>> heap;
  for (int s = 0; s < nsm; ++s) heap.push({0.0, s});
  double worst = 0.0;
  for (int p = 0; p < 6; ++p)
    for (int by = 0; by < nby; ++by)
      for (int bx = 0; bx < nbx; ++bx) {
        const int vx = std::min(TX, N - bx * TX), vy = std::min(TY, N - by * TY);
        const int items = 3 * (vy + 2 * H) * vx;
        const int loads = 3 * (vy + 2 * H) * (vx + 2 * H);
        const double xw = (double)(items / threads) * (threads / 32) + (items % threads + 31) / 32;
        const double cost = xw * per_item + ((vx * vy + 31) / 32) * per_warp_cells +
                            50.0 * ((loads + threads - 1) / threads);
        auto top = heap.top();
        heap.pop();
        top.first += cost;
        worst = std::max(worst, top.first);
        heap.push(top);
      }
  return worst;
}

// Tile shape of the per-kernel TPP reconstruction that minimises recon_tile_cost over
// tiles of 64..512 cells that fit the shared memory.
static void model_recon_tile(const hope_ctx *ctx, int N, int *tx, int *ty) {
  *tx = REC_TX;
  *ty = REC_TY;
  int nsm = 0, optin = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  if (nsm < 1) return;
  const int K = ctx->k;
  const int me = (K + 1) / 2, npos = me + 2;
  double best = recon_tile_cost(N, K, *tx, *ty, nsm);
  for (int TY = 4; TY <= 32; ++TY)
    for (int TX = 8; TX <= 32; ++TX) {
      if (TX * TY < 64 || TX * TY > REC_MAX_THREADS) continue;
      const size_t smem =
          (size_t)ctx->esize * (3 * (TY + K - 1) * (TX + K - 1) + 3 * npos * (TY + K - 1) * TX + npos * K);
      if (smem > (size_t)optin) continue;
      const double c = recon_tile_cost(N, K, TX, TY, nsm);
      if (c < best * 0.999) {
        best = c;
        *tx = TX;
        *ty = TY;
      }
    }
}

// Tile of the forward WENO2D kernel (one thread per cell, ~1e5 FP64 flops per cell at
// k = 9): FP64 contexts deal tiles of 96..256 cells (whole warps of work each) to the least
// loaded SM and keep the shape with the smallest most-loaded SM that fits the shared
// memory; FP32 keeps 16 x 8.
static void choose_weno_tile(const hope_ctx *ctx, Grid &g) {
  g.wtx = REC_TX;
  g.wty = REC_TY;
  if (ctx->scheme != HOPE_WENO2D || ctx->prec != HOPE_FP64) return;
  int nsm = 0, optin = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  if (nsm < 1) return;
  const int N = g.N, K = ctx->k, L = (K + 1) / 2, S = L * L, npos = L + 2, npoc = 4 * L + L * L;
  auto cost = [&](int TX, int TY) {
    std::priority_queue<double, std::vector<double>, std::greater<double>> heap;
    for (int s = 0; s < nsm; ++s) heap.push(0.0);
    double worst = 0.0;
    for (int p = 0; p < 6; ++p)
      for (int by = 0; by < (N + TY - 1) / TY; ++by)
        for (int bx = 0; bx < (N + TX - 1) / TX; ++bx) {
          const int cells = std::min(TX, N - bx * TX) * std::min(TY, N - by * TY);
          double l = heap.top() + (cells + 31) / 32;
          heap.pop();
          heap.push(l);
          worst = std::max(worst, l);
        }
    return worst;
  };
  double best = cost(g.wtx, g.wty);
  for (int TY = 2; TY <= 32; ++TY)
    for (int TX = 4; TX <= 32; ++TX) {
      const int T = TX * TY, threads = (T + 31) / 32 * 32;
      if (T < 96 || threads > 256) continue;  // at least three warps per block
      const size_t smem = sizeof(double) * (3 * (TY + K - 1) * (TX + K - 1) + npos * L * L + npoc * 2 * S +
                                            npoc * 2 + L * (L * L + L) + S * S + 3 * L * L * threads);
      if (smem > (size_t)optin) continue;
      const double c = cost(TX, TY);
      if (c < best * 0.999) {
        best = c;
        g.wtx = TX;
        g.wty = TY;
      }
    }
}

// Set-up choice: the FP64 kernel is bound by the FP64 pipe, so it takes the model's shape;
// the FP32 kernel is latency-bound and starts from 16 x 8 (hope_init_grid then times the
// candidates, tune_recon_tile).
static void choose_recon_tile(const hope_ctx *ctx, Grid &g) {
  g.rtx = REC_TX;
  g.rty = REC_TY;
  if (ctx->scheme != HOPE_TPP || ctx->prec != HOPE_FP64) return;
  model_recon_tile(ctx, g.N, &g.rtx, &g.rty);
}

static int ensure_adjoint_scratch(hope_ctx *ctx) {
  for (auto &g : ctx->grids) {
    if (g.lep) continue;
    const size_t N = g.N, ne = g.ne, es = ctx->esize, me = ctx->me, K = ctx->k;
    // TPP: one extended region per reconstruction tile, for the largest tile buffer of the
    // per-kernel tiles and of the persistent launch's candidate shapes; WENO2D: the per-cell
    // stencil gradients
    size_t tiles = (size_t)tile_buf_elems(g.N, ctx->k, REC_TX, REC_TY);
    if (ctx->ens) tiles = std::max(tiles, ensemble_tile_buf_elems(ctx, g.N));
    const bool tpp = ctx->scheme == HOPE_TPP;
    if (cudaMalloc(&g.lep, es * 4 * 3 * me * 6 * N * N) != cudaSuccess ||
        (tpp ? cudaMalloc(&g.tbuf, es * tiles) : cudaMalloc(&g.grad, es * 3 * K * K * 6 * N * N)) != cudaSuccess ||
        cudaMalloc(&g.lring, es * 3 * 6 * ne * ne) != cudaSuccess ||
        cudaMalloc(&g.ldir, es * 3 * 6 * N * N) != cudaSuccess) {
      set_error("adjoint scratch allocation failed");
      return HOPE_ENOMEM;
    }
    cudaMemset(g.lring, 0, es * 3 * 6 * ne * ne);
  }
  if (!ctx->lam_a) {
    if (cudaMalloc(&ctx->lam_a, ctx->esize * ctx->total) != cudaSuccess ||
        cudaMalloc(&ctx->lam_b, ctx->esize * ctx->total) != cudaSuccess) {
      set_error("adjoint scratch allocation failed");
      return HOPE_ENOMEM;
    }
  }
  return HOPE_OK;
}

// RK step sequence (3 stages) on stream st
static int step_sequence(hope_ctx *ctx, void *q, double dt, int rk, bool prof, cudaStream_t st) {
  stage_fn f = pick_stage(ctx);
  int rc = HOPE_OK;
  double A[3], B[3], C[3];
  const void *qs[3] = {q, ctx->q1, ctx->q2};
  void *out[3] = {ctx->q1, ctx->q2, q};
  if (rk == HOPE_WSRK3) {
    double a[3] = {1.0, 1.0, 1.0}, b[3] = {0.0, 0.0, 0.0}, c[3] = {dt / 3.0, dt / 2.0, dt};
    for (int s = 0; s < 3; ++s) { A[s] = a[s]; B[s] = b[s]; C[s] = c[s]; }
  } else {
    double a[3] = {0.0, 0.75, 1.0 / 3.0}, b[3] = {1.0, 0.25, 2.0 / 3.0}, c[3] = {dt, 0.25 * dt, 2.0 / 3.0 * dt};
    for (int s = 0; s < 3; ++s) { A[s] = a[s]; B[s] = b[s]; C[s] = c[s]; }
  }
  // FP32: compensated state words (the context's carry belongs to q)
  const bool comp = ctx->prec == HOPE_FP32;
  const void *qsl[3] = {ctx->carry, ctx->q1l, ctx->q2l};
  void *outl[3] = {ctx->q1l, ctx->q2l, ctx->carry};
  for (int s = 0; s < 3 && rc == HOPE_OK; ++s) {
    ctx->prof_stage = prof ? s : -1;
    LoWords lw;
    if (comp) {
      lw.q0l = ctx->carry;
      lw.qsl = qsl[s];
      lw.outl = outl[s];
    }
    if (ctx->ens)
      rc = stage_persistent(ctx, qs[s], q, out[s], 1, A[s], B[s], C[s], lw.q0l, lw.qsl, lw.outl, st);
    else
      rc = f(ctx, qs[s], q, out[s], 1, A[s], B[s], C[s], lw, st);
  }
  ctx->prof_stage = -1;
  return rc;
}

// -------------------------------------------------------------------------------
// Initial conditions on the device (cell averages by the me x me Gauss rule).
// -------------------------------------------------------------------------------
struct ICParams {
  double v[8];
};

// phi_s = g hs0 (1 - r/R) of eq. 5.8, M = (hs0, R, lon_c, lat_c); the longitude
// difference is taken modulo 2 pi.
__device__ inline double mountain_phis(const double *M, double g, double lam, double th) {
  const double dl = remainder(lam - M[2], 2.0 * HOPE_PI), dt = th - M[3];
  const double r = sqrt(fmin(M[1] * M[1], dl * dl + dt * dt));
  return g * M[0] * (1.0 - r / M[1]);
}

// Perturbed jet of section 5.4 (Galewsky et al. 2004), P = (umax, theta0, theta1, theta2,
// alpha, beta, hhat, phi0): u(theta) of eq. 5.16, zero outside (theta0, theta1).
__host__ __device__ inline double jet_u(const double *P, double th) {
  if (th <= P[1] || th >= P[2]) return 0.0;
  const double en = exp(-4.0 / ((P[2] - P[1]) * (P[2] - P[1])));
  return P[0] / en * exp(1.0 / ((th - P[1]) * (th - P[2])));
}

// The balance integral of eq. 5.17 from the south pole to theta, a u (2 Omega sin t +
// tan(t) u / a) over (theta0, min(theta, theta1)) by composite Gauss-Legendre: 16 panels of
// the 8-point rule xw = (nodes on [-1/2, 1/2], weights summing to 1).
__host__ __device__ inline double jet_balance(const double *P, const double *xw, double a, double Om, double th) {
  const double hi = th < P[2] ? th : P[2];
  if (hi <= P[1]) return 0.0;
  const double h = (hi - P[1]) / 16.0;
  double s = 0.0;
  for (int pnl = 0; pnl < 16; ++pnl)
    for (int q = 0; q < 8; ++q) {
      const double t = P[1] + (pnl + 0.5 + xw[q]) * h, u = jet_u(P, t);
      s += xw[8 + q] * h * a * u * (2.0 * Om * sin(t) + tan(t) * u / a);
    }
  return s;
}

__device__ inline void ic_field(int cs, const ICParams &P, const double *ex, int nex, double a, double g,
                                double Om, double lam, double th, double *phi, double *us, double *vs) {
  double ct = cos(th), st = sin(th);
  if (cs == 11) {
    // eqs. 5.16-5.18, lambda in (-pi, pi]; ex holds the 8-point rule of jet_balance
    const double d2 = (lam / P.v[4]) * (lam / P.v[4]) + ((P.v[3] - th) / P.v[5]) * ((P.v[3] - th) / P.v[5]);
    *phi = P.v[7] + g * P.v[6] * ct * exp(-d2) - jet_balance(P.v, ex, a, Om, th);
    *us = jet_u(P.v, th);
    *vs = 0.0;
    (void)nex;
  } else if (cs == 5) {
    *phi = mountain_phis(P.v, g, lam, th);
    *us = 0.0;
    *vs = 0.0;
  } else if (cs == 2 || cs == 8 || cs == 10) {
    double al = P.v[0], u0 = P.v[1], phi0 = P.v[2];
    double t = -cos(lam) * ct * sin(al) + st * cos(al);
    *phi = phi0 - (a * Om * u0 + 0.5 * u0 * u0) * t * t;
    *us = u0 * (ct * cos(al) + cos(lam) * st * sin(al));
    *vs = -u0 * sin(lam) * sin(al);
    if (cs == 8) {
      for (int b = 0; b < nex / 2; ++b) {
        double l2 = ex[2 * b], t2 = ex[2 * b + 1];
        double cd = st * sin(t2) + ct * cos(t2) * cos(lam - l2);
        cd = cd > 1.0 ? 1.0 : (cd < -1.0 ? -1.0 : cd);
        double d = acos(cd) / P.v[4];
        *phi += g * P.v[3] * exp(-d * d);
      }
    }
    if (cs == 10) *phi -= mountain_phis(P.v + 3, g, lam, th);  // phi of eq. 5.1 is the free surface
  } else if (cs == 6) {
    double w = P.v[0], K = P.v[1], R = P.v[2], h0 = P.v[3];
    double c2 = ct * ct;
    double cR = pow(ct, R), c2R = cR * cR;
    double A = 0.5 * w * (2.0 * Om + w) * c2 + 0.25 * K * K * c2R * ((R + 1) * c2 + 2 * R * R - R - 2 - 2 * R * R / c2);
    double B = 2.0 * (Om + w) * K / ((R + 1) * (R + 2)) * cR * (R * R + 2 * R + 2 - (R + 1) * (R + 1) * c2);
    double C = 0.25 * K * K * c2R * ((R + 1) * c2 - R - 2);
    *phi = g * h0 + a * a * (A + B * cos(R * lam) + C * cos(2 * R * lam));
    double cR1 = pow(ct, R - 1);
    *us = a * w * ct + a * K * cR1 * (R * st * st - c2) * cos(R * lam);
    *vs = -a * K * R * cR1 * st * sin(R * lam);
  } else {
    double cd = st * sin(P.v[1]) + ct * cos(P.v[1]) * cos(lam - P.v[0]);
    cd = cd > 1.0 ? 1.0 : (cd < -1.0 ? -1.0 : cd);
    *phi = g * (acos(cd) < P.v[2] ? P.v[3] : P.v[4]);
    *us = 0.0;
    *vs = 0.0;
  }
}

template <typename T>
__global__ void k_initial(int N, int me, const double *__restrict__ nw, int cs, ICParams P,
                          const double *__restrict__ ex, int nex, double radius, double gravity, double omega,
                          T *q) {
  long long ncell = 6LL * N * N;
  long long cid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cid >= ncell) return;
  int i = (int)(cid % N), j = (int)((cid / N) % N), p = (int)(cid / ((long long)N * N));
  double dx = HOPE_PI / (2.0 * N);
  double acc0 = 0, acc1 = 0, acc2 = 0;
  for (int h = 0; h < me; ++h)
    for (int g = 0; g < me; ++g) {
      double X = tan(-HOPE_QPI + (i + 0.5 + nw[g]) * dx), Y = tan(-HOPE_QPI + (j + 0.5 + nw[h]) * dx);
      double Pt[3], ax[3], ay[3];
      panel_point(p, X, Y, Pt);
      tangent_basis(p, X, Y, ax, ay);
      double lam = atan2(Pt[1], Pt[0]);
      double th = atan2(Pt[2], sqrt(Pt[0] * Pt[0] + Pt[1] * Pt[1]));
      double phi, us, vs;
      ic_field(cs, P, ex, nex, radius, gravity, omega, lam, th, &phi, &us, &vs);
      // spherical wind -> contravariant components through the dual basis
      double el[3] = {-sin(lam), cos(lam), 0.0};
      double et[3] = {-sin(th) * cos(lam), -sin(th) * sin(lam), cos(th)};
      double V[3];
      for (int c = 0; c < 3; ++c) V[c] = (us * el[c] + vs * et[c]) / radius;
      double g11 = dot3(ax, ax), g12 = dot3(ax, ay), g22 = dot3(ay, ay);
      double det = g11 * g22 - g12 * g12;
      double b1 = dot3(ax, V), b2 = dot3(ay, V);
      double u = (g22 * b1 - g12 * b2) / det, v = (g11 * b2 - g12 * b1) / det;
      double sg = sqrtg_unit(X, Y), W = nw[me + g] * nw[me + h];
      acc0 += W * sg * phi;
      acc1 += W * sg * phi * u;
      acc2 += W * sg * phi * v;
    }
  q[cid] = (T)acc0;
  q[ncell + cid] = (T)acc1;
  q[2 * ncell + cid] = (T)acc2;
}

// -------------------------------------------------------------------------------
// Plain-ALU FMA peak: 8 independent FMA chains per thread.
// -------------------------------------------------------------------------------
template <typename T>
__global__ void k_fma_peak(T *out, int iters, T x, unsigned long long *stamps) {
  // stamps (optional): per block, SM clock cycles and global-timer nanoseconds that its
  // thread 0 spent in the loop, so the host can tell the clock the loop ran at
  unsigned long long c0 = 0, t0 = 0;
  if (stamps && threadIdx.x == 0) {
    c0 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  T a0 = x, a1 = x + T(1), a2 = x + T(2), a3 = x + T(3), a4 = x + T(4), a5 = x + T(5), a6 = x + T(6),
    a7 = x + T(7);
  const T m = T(0.999999), c = T(1e-7);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
      a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
    }
  }
  T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == T(-12345.0)) out[0] = s;  // keeps the loop live
  if (stamps && threadIdx.x == 0) {
    unsigned long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    stamps[2 * blockIdx.x] = clock64() - c0;
    stamps[2 * blockIdx.x + 1] = t1 - t0;
  }
}

}  // namespace hope

using namespace hope;

template <typename T>
static std::vector<T> convert(const std::vector<double> &v) {
  std::vector<T> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
  return o;
}

// ===============================================================================
// C ABI
// ===============================================================================
extern "C" {

void hope_default_params(hope_params *p) {
  if (!p) return;
  p->radius = 6.37122e6;
  p->gravity = 9.80616;
  p->omega = 7.292e-5;
  p->n_gauss = 0;
  p->precision = HOPE_FP64;
  p->rk = HOPE_SSPRK3;
  p->ghost_iters = 10;
  p->weno_eps = 0.0;
  p->coriolis_tilt = 0.0;
}

const char *hope_strerror(int code) {
  switch (code) {
    case HOPE_OK: return "ok";
    case HOPE_EINVAL: return "invalid argument";
    case HOPE_ECUDA: return "CUDA error";
    case HOPE_ENOMEM: return "out of memory";
    case HOPE_ENONPHYS: return "non-physical state";
    case HOPE_ETIMEOUT: return "device wait timed out";
    case HOPE_EUNSUPPORTED: return "unsupported configuration";
  }
  return "unknown error";
}

const char *hope_last_error_message(void) { return g_err.c_str(); }

static void free_grid(Grid &g) {
  if (g.owns_tables) {
    void *tables[] = {g.Xg, g.t1w, g.mx, g.src8, g.gval, g.grow, g.gcol, g.gdst, g.gsym, g.bedge, g.bconv, g.gtp, g.gtr, g.gtv,
                      g.trow, g.tcol, g.tval, g.gband};
    for (void *p : tables)
      if (p) cudaFree(p);
  }
  void *scratch[] = {g.gext, g.ep, g.fx, g.fy, g.sb, g.lep, g.grad, g.tbuf, g.lring, g.ldir, g.tsep, g.ttw, g.ttb,
                     g.tsext, g.tscp};
  for (void *p : scratch)
    if (p) cudaFree(p);
  g = Grid();
}

void hope_destroy(hope_t ctx) {
  if (!ctx) return;
  for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  for (auto &g : ctx->grids) free_grid(g);
  void *ptrs[] = {ctx->w1, ctx->gw, ctx->wsub, ctx->gpm, ctx->sig, ctx->bform, ctx->bcoef, ctx->w1gpm,
                  ctx->w1sig, ctx->w1bf, ctx->state,
                  ctx->q1, ctx->q2, ctx->lbuf, ctx->status, ctx->mass_part, ctx->mass_out,
                  ctx->carry, ctx->q1l, ctx->q2l, ctx->lam_a, ctx->lam_b};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  ensemble_free(ctx);
  for (int s = 0; s < PROF_STAGES; ++s)
    for (int t = 0; t <= PROF_KERNELS; ++t)
      if (ctx->prof_ev[s][t]) cudaEventDestroy(ctx->prof_ev[s][t]);
  delete ctx;
}

static int alloc(void **p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    set_error("cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    return HOPE_ENOMEM;
  }
  return HOPE_OK;
}

// Ghost-operator weights from [entry][5] to five planes [5][entry], so that a warp's load
// of one weight over 32 consecutive entries reads one contiguous run.
extern "C++" {
template <typename V>
std::vector<V> weight_planes(const std::vector<V> &v) {
  const size_t n = v.size() / 5;
  std::vector<V> t(v.size());
  for (size_t e = 0; e < n; ++e)
    for (int k = 0; k < 5; ++k) t[k * n + e] = v[e * 5 + k];
  return t;
}
}

static int upload(void **dst, const std::vector<double> &v, int esize) {
  size_t bytes = (size_t)esize * (v.empty() ? 1 : v.size());
  int rc = alloc(dst, bytes);
  if (rc) return rc;
  if (v.empty()) return HOPE_OK;
  cudaError_t e;
  if (esize == 8) {
    e = cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice);
  } else {
    std::vector<float> f = convert<float>(v);
    e = cudaMemcpy(*dst, f.data(), bytes, cudaMemcpyHostToDevice);
  }
  return e == cudaSuccess ? HOPE_OK : HOPE_ECUDA;
}

static int upload_int(int **dst, const std::vector<int> &v) {
  size_t bytes = sizeof(int) * (v.empty() ? 1 : v.size());
  int rc = alloc((void **)dst, bytes);
  if (rc) return rc;
  if (v.empty()) return HOPE_OK;
  return cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess ? HOPE_OK : HOPE_ECUDA;
}

static int tune_recon_tile(hope_ctx *ctx, int reps, float *ms_out, cudaStream_t st);

static int init_impl(int n_members, const int *Ns, int order, int scheme, const hope_params *params,
                     hope_t *out) {
  if (!out) {
    set_error("null output pointer");
    return HOPE_EINVAL;
  }
  *out = nullptr;
  hope_params prm;
  hope_default_params(&prm);
  if (params) prm = *params;
  if (n_members < 1 || !Ns || order < 3 || order > HOPE_MAXK || order % 2 == 0 ||
      (scheme != HOPE_TPP && scheme != HOPE_WENO2D && scheme != HOPE_WENO1D) ||
      (prm.precision != HOPE_FP64 && prm.precision != HOPE_FP32) ||
      (prm.rk != HOPE_SSPRK3 && prm.rk != HOPE_WSRK3) || prm.ghost_iters < 1 ||
      (prm.n_gauss != 0 && prm.n_gauss != (order + 1) / 2) || !(prm.radius > 0)) {
    set_error("invalid order/scheme/precision/params");
    return HOPE_EINVAL;
  }
  if (scheme == HOPE_WENO2D && order > HOPE_WENO_MAXK) {
    set_error("WENO2D supports orders 3..9");
    return HOPE_EUNSUPPORTED;
  }
  if (scheme == HOPE_WENO1D && order != 5) {
    set_error("the dimension-by-dimension WENO-Z comparator is fifth order (order 5) only");
    return HOPE_EUNSUPPORTED;
  }
  for (int m = 0; m < n_members; ++m)
    if (Ns[m] < order || Ns[m] > 8192) {
      set_error("N must satisfy order <= N <= 8192");
      return HOPE_EINVAL;
    }
  hope_ctx *ctx = new hope_ctx();
  ctx->k = order;
  ctx->H = (order - 1) / 2;
  ctx->me = (order + 1) / 2;
  ctx->npoc = 4 * ctx->me + ctx->me * ctx->me;
  ctx->scheme = scheme;
  ctx->prec = prm.precision;
  ctx->esize = prm.precision == HOPE_FP64 ? 8 : 4;
  ctx->rk = prm.rk;
  ctx->ghost_iters = prm.ghost_iters;
  ctx->radius = prm.radius;
  ctx->gravity = prm.gravity;
  ctx->omega = prm.omega;
  ctx->tilt = prm.coriolis_tilt;
  {
    // rotation axis (-sin(alpha_c), 0, cos(alpha_c)); per panel, axis . (n + X e1 + Y e2)
    double ax[3] = {-sin(prm.coriolis_tilt), 0.0, cos(prm.coriolis_tilt)};
    for (int p = 0; p < 6; ++p) {
      double n[3], e1[3], e2[3];
      panel_frame(p, n, e1, e2);
      ctx->fcoef[3 * p] = dot3(ax, n);
      ctx->fcoef[3 * p + 1] = dot3(ax, e1);
      ctx->fcoef[3 * p + 2] = dot3(ax, e2);
    }
  }
  ctx->eps = prm.weno_eps != 0.0 ? prm.weno_eps : (prm.precision == HOPE_FP64 ? 1e-40 : 1e-12);
  cudaGetDevice(&ctx->device);
  cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  if (ctx->nsm < 1) ctx->nsm = 1;
  int rc;
  std::vector<double> nodes, weights;
#define TRY(x)          \
  do {                  \
    rc = (x);           \
    if (rc) {           \
      hope_destroy(ctx); \
      return rc;        \
    }                   \
  } while (0)
  TRY(set_attrs(ctx));
  TRY(setup_order_tables(ctx, nodes, weights));
  if (scheme != HOPE_TPP) TRY(setup_weno_tables(ctx, nodes));
  size_t off = 0;
  std::map<int, int> first_of_N;  // members with equal N share one set of tables
  for (int m = 0; m < n_members; ++m) {
    Grid g;
    g.N = Ns[m];
    g.ne = Ns[m] + 2 * ctx->H;
    g.off = off;
    off += (size_t)3 * 6 * Ns[m] * Ns[m];
    auto it = first_of_N.find(Ns[m]);
    if (it != first_of_N.end()) {
      const Grid &src = ctx->grids[it->second];
      g.Xg = src.Xg; g.t1w = src.t1w; g.mx = src.mx; g.src8 = src.src8;
      g.gval = src.gval; g.grow = src.grow; g.gcol = src.gcol; g.gdst = src.gdst; g.gsym = src.gsym;
      g.ghost_symmetric = src.ghost_symmetric;
      g.trow = src.trow; g.tcol = src.tcol; g.tval = src.tval; g.tnnz = src.tnnz; g.gstride = src.gstride;
      g.rows = src.rows; g.nnz = src.nnz;
      g.bedge = src.bedge; g.bconv = src.bconv;
      g.gtp = src.gtp; g.gtr = src.gtr; g.gtv = src.gtv; g.gband = src.gband; g.nband = src.nband;
      for (int e = 0; e < 12; ++e) g.edges[e] = src.edges[e];
      g.owns_tables = false;
      ctx->grids.push_back(g);
    } else {
      first_of_N[Ns[m]] = (int)ctx->grids.size();
      ctx->grids.push_back(g);
      Grid &gr = ctx->grids.back();
      TRY(setup_grid_tables(ctx, gr, nodes, weights));
      std::vector<int> rowptr, cols, dst;
      std::vector<double> vals;
      GhostSplit split;
      GhostSym sym;
      TRY(build_ghost_operator(ctx, gr.N, nodes, weights, rowptr, cols, vals, dst,
                               ctx->prec == HOPE_FP64 ? &split : nullptr, &sym));
      gr.rows = (long long)dst.size();
      gr.nnz = rowptr.back();
      gr.ghost_symmetric = sym.symmetric;
      TRY(upload_int(&gr.gdst, dst));
      TRY(upload_int(&gr.gsym, sym.finfo));
      if (ctx->prec == HOPE_FP64) {
        TRY(upload_int(&gr.grow, split.head_ptr));
        TRY(upload_int(&gr.gcol, split.head_col));
        // FP64 contexts keep [entry][5] (GHOST_PLANES)
        gr.gstride = (long long)split.head_col.size();
        TRY(upload(&gr.gval, split.head_val, ctx->esize));
        TRY(upload_int(&gr.trow, split.tail_ptr));
        TRY(upload_int(&gr.tcol, split.tail_col));
        gr.tnnz = (long long)split.tail_col.size();
        TRY(alloc((void **)&gr.tval, sizeof(float) * (split.tail_val.empty() ? 1 : split.tail_val.size())));
        if (!split.tail_val.empty())
          cudaMemcpy(gr.tval, split.tail_val.data(), sizeof(float) * split.tail_val.size(), cudaMemcpyHostToDevice);
      } else {
        std::vector<int> tagged(cols.size());
        for (size_t e = 0; e < cols.size(); ++e) tagged[e] = cols[e] | (sym.ccode[e] << 28);
        TRY(upload_int(&gr.grow, rowptr));
        TRY(upload_int(&gr.gcol, tagged));
        // FP32 contexts store five weight planes (GHOST_PLANES)
        gr.gstride = (long long)cols.size();
        TRY(upload(&gr.gval, weight_planes(vals), ctx->esize));
      }
      {
        // transposed ghost operator for the adjoint: CSR over interior cells, each entry
        // holding the ring position its ghost row writes; and the list of the cells that
        // have entries (the band along the panel edges)
        const int ncell = 6 * gr.N * gr.N;
        std::vector<int> tp(ncell + 1, 0), tr(cols.size());
        std::vector<double> tv(vals.size());
        for (size_t t = 0; t < cols.size(); ++t) tp[cols[t] + 1]++;
        for (int c = 0; c < ncell; ++c) tp[c + 1] += tp[c];
        std::vector<int> fill(tp.begin(), tp.end() - 1);
        for (int r = 0; r + 1 < (int)rowptr.size(); ++r)
          for (int t = rowptr[r]; t < rowptr[r + 1]; ++t) {
            int o = fill[cols[t]]++;
            tr[o] = dst[r];
            for (int u = 0; u < 5; ++u) tv[(size_t)5 * o + u] = vals[(size_t)5 * t + u];
          }
        std::vector<int> band;
        for (int c = 0; c < ncell; ++c)
          if (tp[c + 1] > tp[c]) band.push_back(c);
        gr.nband = (long long)band.size();
        if (band.empty()) band.push_back(0);
        TRY(upload_int(&gr.gtp, tp));
        TRY(upload_int(&gr.gtr, tr));
        TRY(upload_int(&gr.gband, band));
        TRY(upload(&gr.gtv, tv, ctx->esize));
      }
      std::vector<double> conv;
      TRY(build_cube_edges(ctx, gr.N, nodes, gr.edges, conv));
      std::vector<int> be;
      for (int e = 0; e < 12; ++e) {
        be.push_back(gr.edges[e].A);
        be.push_back(gr.edges[e].sideA);
        be.push_back(gr.edges[e].B);
        be.push_back(gr.edges[e].sideB);
        be.push_back(gr.edges[e].flip);
      }
      TRY(upload_int(&gr.bedge, be));
      TRY(upload(&gr.bconv, conv, ctx->esize));
    }
    Grid &gr = ctx->grids.back();
    const size_t N = gr.N, ne = gr.ne, es = ctx->esize, me = ctx->me;
    TRY(alloc(&gr.gext, es * 3 * 6 * ne * ne));
    cudaMemset(gr.gext, 0, es * 3 * 6 * ne * ne);
    TRY(alloc(&gr.ep, es * 4 * 3 * me * 6 * N * N));
    TRY(alloc(&gr.fx, es * 3 * 6 * N * (N + 1)));
    TRY(alloc(&gr.fy, es * 3 * 6 * (N + 1) * N));
    TRY(alloc(&gr.sb, es * 2 * 6 * N * N));
    choose_recon_tile(ctx, gr);
    choose_weno_tile(ctx, gr);
  }
  ctx->total = off;
  const size_t es = ctx->esize;
  TRY(alloc(&ctx->state, es * off));
  TRY(alloc(&ctx->q1, es * off));
  TRY(alloc(&ctx->q2, es * off));
  TRY(alloc(&ctx->lbuf, es * off));
  if (ctx->prec == HOPE_FP32) {
    TRY(alloc(&ctx->carry, es * off));
    TRY(alloc(&ctx->q1l, es * off));
    TRY(alloc(&ctx->q2l, es * off));
    cudaMemset(ctx->carry, 0, es * off);
  }
  TRY(alloc((void **)&ctx->status, sizeof(unsigned)));
  cudaMemset(ctx->status, 0, sizeof(unsigned));
  TRY(alloc((void **)&ctx->mass_part, sizeof(double) * MASS_BLOCKS));
  TRY(alloc((void **)&ctx->mass_out, sizeof(double) * n_members));
  if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    hope_destroy(ctx);
    set_error("cudaStreamCreate failed");
    return HOPE_ECUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error(std::string("setup: ") + cudaGetErrorString(cudaGetLastError()));
    hope_destroy(ctx);
    return HOPE_ECUDA;
  }
  if (n_members > 1 && scheme == HOPE_TPP) {
    TRY(ensemble_init(ctx));
    // tune the tile shape on a benign state (steady geostrophic flow) in the scratch buffers
    const double u0 = 2.0 * HOPE_PI * ctx->radius / (12.0 * 86400.0);
    const double prm[3] = {0.0, u0, 2.94e4};
    TRY(hope_initial_state(ctx, 2, prm, 3, nullptr, 0, ctx->q1, nullptr));
    TRY(ensemble_autotune(ctx, ctx->q1, ctx->lbuf, 3, nullptr, nullptr));
    if (cudaDeviceSynchronize() != cudaSuccess) {
      set_error(std::string("ensemble autotune: ") + cudaGetErrorString(cudaGetLastError()));
      hope_destroy(ctx);
      return HOPE_ECUDA;
    }
    cudaMemset(ctx->status, 0, sizeof(unsigned));
  }
  if (n_members == 1 && scheme == HOPE_TPP && ctx->prec == HOPE_FP32) TRY(tune_recon_tile(ctx, 3, nullptr, nullptr));
#undef TRY
  *out = ctx;
  return HOPE_OK;
}

int hope_init_grid(int N, int order, int scheme, const hope_params *params, hope_t *out) {
  return init_impl(1, &N, order, scheme, params, out);
}

int hope_init_ensemble(int n_members, const int *N, int order, int scheme, const hope_params *params,
                       hope_t *out) {
  return init_impl(n_members, N, order, scheme, params, out);
}

size_t hope_state_elems(hope_t ctx) { return ctx ? ctx->total : 0; }
int hope_elem_size(hope_t ctx) { return ctx ? ctx->esize : 0; }

int hope_initial_state(hope_t ctx, int ic_case, const double *params, int n_params, const double *extra_host,
                       int n_extra, void *q_dev, hope_stream_t stream) {
  if (!ctx || !q_dev ||
      (ic_case != 2 && ic_case != 5 && ic_case != 6 && ic_case != 7 && ic_case != 8 && ic_case != 10 &&
       ic_case != 11) ||
      n_params < 0 ||
      n_params > 8 || (n_params > 0 && !params) || n_extra < 0 || (n_extra > 0 && !extra_host)) {
    set_error("hope_initial_state: invalid argument");
    return HOPE_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  ICParams P;
  for (int t = 0; t < 8; ++t) P.v[t] = t < n_params ? params[t] : 0.0;
  std::vector<double> jet_rule;
  if (ic_case == 11) {
    // the quadrature rule of the jet's balance integral travels in the extra array
    jet_rule.resize(16);
    gauss_legendre(8, jet_rule.data(), jet_rule.data() + 8);
    if (P.v[7] == 0.0) {
      // phi0 = 0 asks for Galewsky's constant: the area mean of the balanced phi (without
      // the bump) is g x 10 km, phi0 = g 1e4 + 1/2 int I(theta) cos(theta) d theta
      const double h = (P.v[2] - P.v[1]) / 16.0;
      double s = 0.0;
      for (int pnl = 0; pnl < 16; ++pnl)
        for (int q = 0; q < 8; ++q) {
          const double t = P.v[1] + (pnl + 0.5 + jet_rule[q]) * h;
          s += jet_rule[8 + q] * h * jet_balance(P.v, jet_rule.data(), ctx->radius, ctx->omega, t) * cos(t);
        }
      s += jet_balance(P.v, jet_rule.data(), ctx->radius, ctx->omega, P.v[2]) * (1.0 - sin(P.v[2]));
      P.v[7] = ctx->gravity * 1.0e4 + 0.5 * s;
    }
    extra_host = jet_rule.data();
    n_extra = 16;
  }
  double *d_ex = nullptr, *d_nw = nullptr;
  HOPE_CUDA_TRY(cudaMalloc(&d_ex, sizeof(double) * (n_extra > 0 ? n_extra : 1)));
  if (n_extra > 0) HOPE_CUDA_TRY(cudaMemcpy(d_ex, extra_host, sizeof(double) * n_extra, cudaMemcpyHostToDevice));
  std::vector<double> nw(2 * ctx->me);
  gauss_legendre(ctx->me, nw.data(), nw.data() + ctx->me);
  HOPE_CUDA_TRY(cudaMalloc(&d_nw, sizeof(double) * 2 * ctx->me));
  HOPE_CUDA_TRY(cudaMemcpy(d_nw, nw.data(), sizeof(double) * 2 * ctx->me, cudaMemcpyHostToDevice));
  for (auto &g : ctx->grids) {
    long long cells = 6LL * g.N * g.N;
    int blocks = (int)((cells + 127) / 128);
    if (ctx->prec == HOPE_FP64)
      k_initial<double><<<blocks, 128, 0, st>>>(g.N, ctx->me, d_nw, ic_case, P, d_ex, n_extra, ctx->radius,
                                                ctx->gravity, ctx->omega, (double *)q_dev + g.off);
    else
      k_initial<float><<<blocks, 128, 0, st>>>(g.N, ctx->me, d_nw, ic_case, P, d_ex, n_extra, ctx->radius,
                                               ctx->gravity, ctx->omega, (float *)q_dev + g.off);
  }
  HOPE_CUDA_TRY(cudaGetLastError());
  HOPE_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFree(d_ex);
  cudaFree(d_nw);
  return HOPE_OK;
}

int hope_set_state(hope_t ctx, const void *q_dev, hope_stream_t stream) {
  if (!ctx || !q_dev) return HOPE_EINVAL;
  if (ctx->carry_owner == ctx->state) ctx->carry_owner = nullptr;  // new contents: fresh carry
  HOPE_CUDA_TRY(cudaMemcpyAsync(ctx->state, q_dev, ctx->esize * ctx->total, cudaMemcpyDeviceToDevice,
                                (cudaStream_t)stream));
  return HOPE_OK;
}

int hope_get_state(hope_t ctx, void *q_dev, hope_stream_t stream) {
  if (!ctx || !q_dev) return HOPE_EINVAL;
  HOPE_CUDA_TRY(cudaMemcpyAsync(q_dev, ctx->state, ctx->esize * ctx->total, cudaMemcpyDeviceToDevice,
                                (cudaStream_t)stream));
  return HOPE_OK;
}

int hope_tendency(hope_t ctx, const void *q_dev, void *dqdt_dev, hope_stream_t stream) {
  if (!ctx || !dqdt_dev) {
    set_error("hope_tendency: null argument");
    return HOPE_EINVAL;
  }
  const void *q = q_dev ? q_dev : ctx->state;
  if (q == dqdt_dev) {
    set_error("hope_tendency: q and dqdt must not overlap");
    return HOPE_EINVAL;
  }
  if (ctx->ens)
    return stage_persistent(ctx, q, nullptr, dqdt_dev, 0, 0.0, 0.0, 0.0, nullptr, nullptr, nullptr,
                            (cudaStream_t)stream);
  return pick_stage(ctx)(ctx, q, nullptr, dqdt_dev, 0, 0.0, 0.0, 0.0, LoWords(), (cudaStream_t)stream);
}

static int step_impl(hope_t ctx, void *q_dev, double dt, int nsteps, int rk, cudaStream_t st) {
  if (!ctx || nsteps < 0 || !(dt == dt)) {
    set_error("hope_step: invalid argument");
    return HOPE_EINVAL;
  }
  void *q = q_dev ? q_dev : ctx->state;
  if (ctx->prec == HOPE_FP32 && ctx->carry_owner != q) {
    // a new state buffer: its compensation word starts at zero
    HOPE_CUDA_TRY(cudaMemsetAsync(ctx->carry, 0, ctx->esize * ctx->total, st));
    ctx->carry_owner = q;
  }
  GraphKey key{q, dt, rk, ctx->profiling};
  auto it = ctx->graphs.find(key);
  cudaGraphExec_t exec = nullptr;
  if (it == ctx->graphs.end()) {
    cudaGraph_t graph = nullptr;
    HOPE_CUDA_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = step_sequence(ctx, q, dt, rk, ctx->profiling != 0, ctx->cap_stream);
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) {
      set_error(std::string("graph capture: ") + cudaGetErrorString(e));
      return HOPE_ECUDA;
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      set_error(std::string("graph instantiate: ") + cudaGetErrorString(e));
      return HOPE_ECUDA;
    }
    if (ctx->graphs.size() > 64) {
      for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
      ctx->graphs.clear();
    }
    ctx->graphs[key] = exec;
  } else {
    exec = it->second;
  }
  for (int s = 0; s < nsteps; ++s) HOPE_CUDA_TRY(cudaGraphLaunch(exec, st));
  return HOPE_OK;
}

int hope_step(hope_t ctx, void *q_dev, double dt, int nsteps, hope_stream_t stream) {
  if (!ctx) return HOPE_EINVAL;
  return step_impl(ctx, q_dev, dt, nsteps, ctx->rk, (cudaStream_t)stream);
}

int hope_step_ssprk3(hope_t ctx, void *q_dev, double dt, hope_stream_t stream) {
  return step_impl(ctx, q_dev, dt, 1, HOPE_SSPRK3, (cudaStream_t)stream);
}

int hope_step_host(hope_t ctx, const void *q_host_in, void *q_host_out, double dt, int nsteps,
                   hope_stream_t stream) {
  if (!ctx || !q_host_in || !q_host_out) return HOPE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  size_t bytes = ctx->esize * ctx->total;
  HOPE_CUDA_TRY(cudaMemcpyAsync(ctx->state, q_host_in, bytes, cudaMemcpyHostToDevice, st));
  if (ctx->carry_owner == ctx->state) ctx->carry_owner = nullptr;  // new contents: fresh carry
  int rc = step_impl(ctx, ctx->state, dt, nsteps, ctx->rk, st);
  if (rc) return rc;
  HOPE_CUDA_TRY(cudaMemcpyAsync(q_host_out, ctx->state, bytes, cudaMemcpyDeviceToHost, st));
  HOPE_CUDA_TRY(cudaStreamSynchronize(st));
  return HOPE_OK;
}

int hope_total_mass(hope_t ctx, const void *q_dev, double *mass_host, hope_stream_t stream) {
  if (!ctx || !mass_host) return HOPE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const void *q = q_dev ? q_dev : ctx->state;
  for (size_t m = 0; m < ctx->grids.size(); ++m) {
    Grid &g = ctx->grids[m];
    long long n = 6LL * g.N * g.N;
    if (ctx->prec == HOPE_FP64)
      k_mass_partial<double><<<MASS_BLOCKS, MASS_THREADS, 0, st>>>((const double *)q + g.off, n, ctx->mass_part);
    else
      k_mass_partial<float><<<MASS_BLOCKS, MASS_THREADS, 0, st>>>((const float *)q + g.off, n, ctx->mass_part);
    double dx = HOPE_PI / (2.0 * g.N);
    k_mass_final<<<1, 32, 0, st>>>(ctx->mass_part, MASS_BLOCKS, dx * dx, ctx->mass_out + m);
  }
  HOPE_CUDA_TRY(cudaGetLastError());
  HOPE_CUDA_TRY(cudaMemcpyAsync(mass_host, ctx->mass_out, sizeof(double) * ctx->grids.size(),
                                cudaMemcpyDeviceToHost, st));
  HOPE_CUDA_TRY(cudaStreamSynchronize(st));
  return HOPE_OK;
}

int hope_status(hope_t ctx, unsigned *device_status) {
  if (!ctx || !device_status) return HOPE_EINVAL;
  HOPE_CUDA_TRY(cudaDeviceSynchronize());
  HOPE_CUDA_TRY(cudaMemcpy(device_status, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  HOPE_CUDA_TRY(cudaMemset(ctx->status, 0, sizeof(unsigned)));
  if (*device_status & HOPE_STATUS_TIMEOUT) ensemble_reset_barrier(ctx);
  return HOPE_OK;
}

int hope_ghost_selfcheck(int N, int order, int precision, int *symmetric, double *max_dev_sym,
                         double *max_dev_apply) {
  if (N < 1 || order < 3 || order > HOPE_MAXK || order % 2 == 0 ||
      (precision != HOPE_FP64 && precision != HOPE_FP32) || !symmetric || !max_dev_sym || !max_dev_apply) {
    set_error("hope_ghost_selfcheck: invalid argument");
    return HOPE_EINVAL;
  }
  hope_ctx ctx;
  ctx.k = order;
  ctx.H = (order - 1) / 2;
  ctx.me = (order + 1) / 2;
  ctx.prec = precision;
  ctx.scheme = HOPE_TPP;
  ctx.ghost_iters = 10;
  std::vector<double> nodes(ctx.me), weights(ctx.me);
  gauss_legendre(ctx.me, nodes.data(), weights.data());
  std::vector<int> rowptr, cols, dst;
  std::vector<double> vals;
  GhostSplit split;
  GhostSym sym;
  const bool fp64 = precision == HOPE_FP64;
  int rc = build_ghost_operator(&ctx, N, nodes, weights, rowptr, cols, vals, dst, fp64 ? &split : nullptr, &sym);
  if (rc) return rc;
  *symmetric = sym.symmetric ? 1 : 0;
  *max_dev_sym = sym.max_dev;
  // the stored form as the ghost kernel reads it (row's columns with their input codes,
  // the representative's weights, the row's output code) against the full operator, on a
  // seeded state
  const size_t pn = (size_t)6 * N * N;
  std::vector<double> q(3 * pn);
  unsigned long long st = 0x9E3779B97F4A7C15ull;
  for (auto &v : q) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    v = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
  auto apply_code = [](int code, double &x, double &y) {
    const double a = (code & 1) ? y : x, b = (code & 1) ? x : y;
    x = (code & 2) ? -a : a;
    y = (code & 4) ? -b : b;
  };
  const int rows = (int)dst.size();
  std::vector<int> tagged(cols.size());
  for (size_t e = 0; e < cols.size(); ++e) tagged[e] = cols[e] | (sym.ccode[e] << 28);
  double worst = 0.0, scale = 0.0;
  for (int r = 0; r < rows; ++r) {
    double f[3] = {0, 0, 0}, g3[3] = {0, 0, 0};
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
      const int c = cols[e];
      const double *v = &vals[(size_t)5 * e];
      f[0] += v[0] * q[c];
      f[1] += v[1] * q[pn + c] + v[2] * q[2 * pn + c];
      f[2] += v[3] * q[pn + c] + v[4] * q[2 * pn + c];
    }
    const int info = sym.finfo[r], wrow = info & 0x0FFFFFFF, oc = info >> 28;
    for (int part = 0; part < (fp64 ? 2 : 1); ++part) {
      const std::vector<int> &ptr = !fp64 ? rowptr : (part ? split.tail_ptr : split.head_ptr);
      const std::vector<int> &col = !fp64 ? tagged : (part ? split.tail_col : split.head_col);
      for (int t = ptr[r]; t < ptr[r + 1]; ++t) {
        const int c = col[t] & 0x0FFFFFFF, code = col[t] >> 28, wi = ptr[wrow] + (t - ptr[r]);
        double w[5];
        for (int k = 0; k < 5; ++k)
          w[k] = !fp64 ? vals[(size_t)5 * wi + k]
                       : (part ? (double)split.tail_val[(size_t)5 * wi + k] : split.head_val[(size_t)5 * wi + k]);
        double a1 = q[pn + c], a2 = q[2 * pn + c];
        apply_code(code, a1, a2);
        g3[0] += w[0] * q[c];
        g3[1] += w[1] * a1 + w[2] * a2;
        g3[2] += w[3] * a1 + w[4] * a2;
      }
    }
    apply_code(oc, g3[1], g3[2]);
    for (int v = 0; v < 3; ++v) {
      worst = fmax(worst, fabs(g3[v] - f[v]));
      scale = fmax(scale, fabs(f[v]));
    }
  }
  *max_dev_apply = scale > 0.0 ? worst / scale : worst;
  return HOPE_OK;
}

int hope_ghost_nnz(hope_t ctx, long long *nnz, long long *rows) {
  if (!ctx || !nnz || !rows) return HOPE_EINVAL;
  *nnz = 0;
  *rows = 0;
  for (auto &g : ctx->grids) {
    *nnz += g.nnz;
    *rows += g.rows;
  }
  return HOPE_OK;
}

int hope_launches_per_stage(hope_t ctx, int *launches) {
  if (!ctx || !launches) return HOPE_EINVAL;
  *launches = ctx->ens ? 1 : 4 * (int)ctx->grids.size();
  if (!ctx->ens)
    for (auto &g : ctx->grids) *launches += (g.tsep && ctx->scheme != HOPE_TPP) ? 1 : 0;  // TPP: psi_B in recon
  return HOPE_OK;
}

// Forms without a hand-written adjoint: the WENO1D comparator.
static int adjoint_guard(const hope_ctx *ctx) {
  if (ctx->scheme == HOPE_WENO1D) {
    set_error("the dimension-by-dimension WENO comparator has no adjoint");
    return HOPE_EUNSUPPORTED;
  }
  return HOPE_OK;
}

int hope_tendency_vjp(hope_t ctx, const void *q_dev, const void *lam_dqdt_dev, void *lam_q_dev,
                      hope_stream_t stream) {
  if (!ctx || !q_dev || !lam_dqdt_dev || !lam_q_dev || lam_q_dev == q_dev || lam_q_dev == lam_dqdt_dev) {
    set_error("hope_tendency_vjp: invalid or overlapping arguments");
    return HOPE_EINVAL;
  }
  if (int ge = adjoint_guard(ctx)) return ge;
  int rc = ensure_adjoint_scratch(ctx);
  if (rc) return rc;
  VjpComb cb;
  return pick_vjp(ctx)(ctx, q_dev, lam_dqdt_dev, lam_q_dev, cb, (cudaStream_t)stream);
}

static int step_vjp_impl(hope_t ctx, int rk, const void *qn_dev, const void *lam_np1_dev, void *lam_n_dev,
                         double dt, hope_stream_t stream);

int hope_step_vjp(hope_t ctx, const void *qn_dev, const void *lam_np1_dev, void *lam_n_dev, double dt,
                  hope_stream_t stream) {
  return ctx ? step_vjp_impl(ctx, ctx->rk, qn_dev, lam_np1_dev, lam_n_dev, dt, stream) : HOPE_EINVAL;
}

int hope_step_ssprk3_vjp(hope_t ctx, const void *qn_dev, const void *lam_np1_dev, void *lam_n_dev, double dt,
                         hope_stream_t stream) {
  return step_vjp_impl(ctx, HOPE_SSPRK3, qn_dev, lam_np1_dev, lam_n_dev, dt, stream);
}

static int step_vjp_impl(hope_t ctx, int rk, const void *qn_dev, const void *lam_np1_dev, void *lam_n_dev,
                         double dt, hope_stream_t stream) {
  if (!ctx || !qn_dev || !lam_np1_dev || !lam_n_dev || lam_n_dev == qn_dev || lam_n_dev == lam_np1_dev ||
      !(dt == dt)) {
    set_error("hope_step_vjp: invalid or overlapping arguments");
    return HOPE_EINVAL;
  }
  if (int ge = adjoint_guard(ctx)) return ge;
  int rc = ensure_adjoint_scratch(ctx);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  stage_fn f = run_stage;
  vjp_fn v = pick_vjp(ctx);
  // recompute the stage states q1, q2 from q^n
  if (rk == HOPE_WSRK3) {
    if ((rc = f(ctx, qn_dev, qn_dev, ctx->q1, 1, 1.0, 0.0, dt / 3.0, LoWords(), st))) return rc;
    if ((rc = f(ctx, ctx->q1, qn_dev, ctx->q2, 1, 1.0, 0.0, dt / 2.0, LoWords(), st))) return rc;
    VjpComb c3;  // lam** = dt L^T(q**) lam
    c3.c = dt;
    if ((rc = v(ctx, ctx->q2, lam_np1_dev, ctx->lam_b, c3, st))) return rc;
    VjpComb c2;  // lam* = dt/2 L^T(q*) lam**
    c2.c = dt / 2.0;
    if ((rc = v(ctx, ctx->q1, ctx->lam_b, ctx->lam_a, c2, st))) return rc;
    VjpComb c1;  // lam_n = lam + lam** + lam* + dt/3 L^T(q) lam*
    c1.x = lam_np1_dev; c1.a = 1.0;
    c1.y = ctx->lam_b; c1.b = 1.0;
    c1.z = ctx->lam_a; c1.d = 1.0;
    c1.c = dt / 3.0;
    return v(ctx, qn_dev, ctx->lam_a, lam_n_dev, c1, st);
  }
  if ((rc = f(ctx, qn_dev, qn_dev, ctx->q1, 1, 0.0, 1.0, dt, LoWords(), st))) return rc;
  if ((rc = f(ctx, ctx->q1, qn_dev, ctx->q2, 1, 0.75, 0.25, 0.25 * dt, LoWords(), st))) return rc;
  VjpComb c3;  // lam2 = 2/3 lam + 2/3 dt L^T(q2) lam
  c3.x = lam_np1_dev; c3.a = 2.0 / 3.0;
  c3.c = 2.0 / 3.0 * dt;
  if ((rc = v(ctx, ctx->q2, lam_np1_dev, ctx->lam_b, c3, st))) return rc;
  VjpComb c2;  // lam1 = 1/4 lam2 + 1/4 dt L^T(q1) lam2
  c2.x = ctx->lam_b; c2.a = 0.25;
  c2.c = 0.25 * dt;
  if ((rc = v(ctx, ctx->q1, ctx->lam_b, ctx->lam_a, c2, st))) return rc;
  VjpComb c1;  // lam_n = 1/3 lam + 3/4 lam2 + lam1 + dt L^T(q) lam1
  c1.x = lam_np1_dev; c1.a = 1.0 / 3.0;
  c1.y = ctx->lam_b; c1.b = 0.75;
  c1.z = ctx->lam_a; c1.d = 1.0;
  c1.c = dt;
  return v(ctx, qn_dev, ctx->lam_a, lam_n_dev, c1, st);
}

// ---------------------------------------------------------------------------------
// Step tapes: one RK step's stage states and each stage's ghost ring and edge points,
// so that a reverse sweep over recomputed steps needs no further forward work.
// Layout (bytes): q1, q2 (one state each), then per grid and stage s = 0, 1, 2: the
// ghost ring, then the edge points, of the stage whose input is q^n, q1, q2.
// ---------------------------------------------------------------------------------
static size_t gext_bytes(const hope_ctx *ctx, const Grid &g) { return ctx->esize * 3 * 6 * (size_t)g.ne * g.ne; }
static size_t ep_bytes(const hope_ctx *ctx, const Grid &g) {
  return ctx->esize * 4 * 3 * (size_t)ctx->me * 6 * g.N * g.N;
}

static size_t tape_size(const hope_ctx *ctx) {
  size_t b = 2 * ctx->esize * ctx->total;
  for (auto &g : ctx->grids) b += 3 * (gext_bytes(ctx, g) + ep_bytes(ctx, g));
  return b;
}

// copy the grids' ghost rings and edge points to (save) or from (!save) a tape's stage s
static int tape_io(hope_ctx *ctx, unsigned char *tape, int s, bool save, cudaStream_t st) {
  size_t off = 2 * ctx->esize * ctx->total;
  for (auto &g : ctx->grids) {
    const size_t gb = gext_bytes(ctx, g), eb = ep_bytes(ctx, g);
    unsigned char *t = tape + off + (size_t)s * (gb + eb);
    cudaError_t e1 = save ? cudaMemcpyAsync(t, g.gext, gb, cudaMemcpyDeviceToDevice, st)
                          : cudaMemcpyAsync(g.gext, t, gb, cudaMemcpyDeviceToDevice, st);
    cudaError_t e2 = save ? cudaMemcpyAsync(t + gb, g.ep, eb, cudaMemcpyDeviceToDevice, st)
                          : cudaMemcpyAsync(g.ep, t + gb, eb, cudaMemcpyDeviceToDevice, st);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      set_error("step tape copy failed");
      return HOPE_ECUDA;
    }
    off += 3 * (gb + eb);
  }
  return HOPE_OK;
}

int hope_tape_bytes(hope_t ctx, size_t *bytes) {
  if (!ctx || !bytes) return HOPE_EINVAL;
  *bytes = tape_size(ctx);
  return HOPE_OK;
}

int hope_step_record(hope_t ctx, void *q_dev, double dt, void *tape_dev, hope_stream_t stream) {
  if (!ctx || !q_dev || !tape_dev || !(dt == dt)) {
    set_error("hope_step_record: invalid argument");
    return HOPE_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  stage_fn f = run_stage;
  unsigned char *tape = (unsigned char *)tape_dev;
  void *q1 = tape, *q2 = tape + ctx->esize * ctx->total;
  int rc;
  if (ctx->rk == HOPE_WSRK3) {
    if ((rc = f(ctx, q_dev, q_dev, q1, 1, 1.0, 0.0, dt / 3.0, LoWords(), st)) || (rc = tape_io(ctx, tape, 0, true, st)))
      return rc;
    if ((rc = f(ctx, q1, q_dev, q2, 1, 1.0, 0.0, dt / 2.0, LoWords(), st)) || (rc = tape_io(ctx, tape, 1, true, st)))
      return rc;
    if ((rc = f(ctx, q2, q_dev, q_dev, 1, 1.0, 0.0, dt, LoWords(), st))) return rc;
    return tape_io(ctx, tape, 2, true, st);
  }
  if ((rc = f(ctx, q_dev, q_dev, q1, 1, 0.0, 1.0, dt, LoWords(), st)) || (rc = tape_io(ctx, tape, 0, true, st)))
    return rc;
  if ((rc = f(ctx, q1, q_dev, q2, 1, 0.75, 0.25, 0.25 * dt, LoWords(), st)) ||
      (rc = tape_io(ctx, tape, 1, true, st)))
    return rc;
  if ((rc = f(ctx, q2, q_dev, q_dev, 1, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0 * dt, LoWords(), st))) return rc;
  return tape_io(ctx, tape, 2, true, st);
}

int hope_step_vjp_tape(hope_t ctx, const void *qn_dev, const void *tape_dev, const void *lam_np1_dev,
                       void *lam_n_dev, double dt, hope_stream_t stream) {
  if (!ctx || !qn_dev || !tape_dev || !lam_np1_dev || !lam_n_dev || lam_n_dev == qn_dev ||
      lam_n_dev == lam_np1_dev || !(dt == dt)) {
    set_error("hope_step_vjp_tape: invalid or overlapping arguments");
    return HOPE_EINVAL;
  }
  if (int ge = adjoint_guard(ctx)) return ge;
  int rc = ensure_adjoint_scratch(ctx);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  vjp_fn v = pick_vjp(ctx);
  unsigned char *tape = (unsigned char *)tape_dev;
  const void *q1 = tape, *q2 = tape + ctx->esize * ctx->total;
  // the stage's ghost rings and edge points: ensembles read them from the tape in the
  // persistent launch, single spheres copy them back into the grid buffers
  auto restore = [&](int s, VjpComb &cb) -> int {
    if (ctx->ens) {
      cb.tape = tape;
      cb.tape_stage = s;
      return HOPE_OK;
    }
    return tape_io(ctx, tape, s, false, st);
  };
  if (ctx->rk == HOPE_WSRK3) {
    VjpComb c3;
    c3.c = dt;
    c3.have_fwd = 1;
    if ((rc = restore(2, c3)) || (rc = v(ctx, q2, lam_np1_dev, ctx->lam_b, c3, st))) return rc;
    VjpComb c2;
    c2.c = dt / 2.0;
    c2.have_fwd = 1;
    if ((rc = restore(1, c2)) || (rc = v(ctx, q1, ctx->lam_b, ctx->lam_a, c2, st))) return rc;
    VjpComb c1;
    c1.x = lam_np1_dev; c1.a = 1.0;
    c1.y = ctx->lam_b; c1.b = 1.0;
    c1.z = ctx->lam_a; c1.d = 1.0;
    c1.c = dt / 3.0;
    c1.have_fwd = 1;
    if ((rc = restore(0, c1))) return rc;
    return v(ctx, qn_dev, ctx->lam_a, lam_n_dev, c1, st);
  }
  VjpComb c3;  // lam2 = 2/3 lam + 2/3 dt L^T(q2) lam
  c3.x = lam_np1_dev; c3.a = 2.0 / 3.0;
  c3.c = 2.0 / 3.0 * dt;
  c3.have_fwd = 1;
  if ((rc = restore(2, c3)) || (rc = v(ctx, q2, lam_np1_dev, ctx->lam_b, c3, st))) return rc;
  VjpComb c2;  // lam1 = 1/4 lam2 + 1/4 dt L^T(q1) lam2
  c2.x = ctx->lam_b; c2.a = 0.25;
  c2.c = 0.25 * dt;
  c2.have_fwd = 1;
  if ((rc = restore(1, c2)) || (rc = v(ctx, q1, ctx->lam_b, ctx->lam_a, c2, st))) return rc;
  VjpComb c1;  // lam_n = 1/3 lam + 3/4 lam2 + lam1 + dt L^T(q) lam1
  c1.x = lam_np1_dev; c1.a = 1.0 / 3.0;
  c1.y = ctx->lam_b; c1.b = 0.75;
  c1.z = ctx->lam_a; c1.d = 1.0;
  c1.c = dt;
  c1.have_fwd = 1;
  if ((rc = restore(0, c1))) return rc;
  return v(ctx, qn_dev, ctx->lam_a, lam_n_dev, c1, st);
}

static void drop_graphs(hope_ctx *ctx) {
  for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
}

// Times `reps` tendency stages of a single TPP sphere with each candidate tile shape --
// 16 x 8, the model's shape, 12 x 12 -- on a benign state in the context's scratch
// buffers and keeps the fastest.  ms_out (3 floats, may be null) gets the times (-1 for a
// candidate equal to an earlier one).
static int tune_recon_tile(hope_ctx *ctx, int reps, float *ms_out, cudaStream_t st) {
  Grid &g = ctx->grids[0];
  int cand[3][2] = {{REC_TX, REC_TY}, {0, 0}, {12, 12}};
  model_recon_tile(ctx, g.N, &cand[1][0], &cand[1][1]);
  const double u0 = 2.0 * HOPE_PI * ctx->radius / (12.0 * 86400.0);
  const double prm[3] = {0.0, u0, 2.94e4};
  int rc = hope_initial_state(ctx, 2, prm, 3, nullptr, 0, ctx->q1, st);
  if (rc) return rc;
  stage_fn f = pick_stage(ctx);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bx = g.rtx, by = g.rty;
  for (int c = 0; c < 3; ++c) {
    bool dup = false;
    for (int d = 0; d < c; ++d) dup |= cand[d][0] == cand[c][0] && cand[d][1] == cand[c][1];
    if (dup) {
      if (ms_out) ms_out[c] = -1.0f;
      continue;
    }
    g.rtx = cand[c][0];
    g.rty = cand[c][1];
    if ((rc = f(ctx, ctx->q1, nullptr, ctx->lbuf, 0, 0, 0, 0, LoWords(), st))) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && !rc; ++r) rc = f(ctx, ctx->q1, nullptr, ctx->lbuf, 0, 0, 0, 0, LoWords(), st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms_out) ms_out[c] = ms;
    if (ms < best) {
      best = ms;
      bx = cand[c][0];
      by = cand[c][1];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g.rtx = bx;
  g.rty = by;
  drop_graphs(ctx);
  cudaMemsetAsync(ctx->status, 0, sizeof(unsigned), st);
  if (rc) return rc;
  return cudaStreamSynchronize(st) == cudaSuccess ? HOPE_OK : HOPE_ECUDA;
}

int hope_set_recon_tile(hope_t ctx, int tx, int ty) {
  if (!ctx || ctx->scheme != HOPE_TPP || tx < 1 || ty < 1 || tx * ty > REC_MAX_THREADS) {
    set_error("hope_set_recon_tile: needs a TPP context and 1 <= tx*ty <= 512");
    return HOPE_EINVAL;
  }
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  const int K = ctx->k, npos = (K + 1) / 2 + 2;
  const size_t smem = (size_t)ctx->esize * (3 * (ty + K - 1) * (tx + K - 1) + 3 * npos * (ty + K - 1) * tx + npos * K);
  if (smem > (size_t)optin) {
    set_error("hope_set_recon_tile: the tile's shared memory exceeds the per-block limit");
    return HOPE_EINVAL;
  }
  for (auto &g : ctx->grids) {
    g.rtx = tx;
    g.rty = ty;
  }
  drop_graphs(ctx);
  return HOPE_OK;
}

int hope_recon_tile(hope_t ctx, int *tx, int *ty) {
  if (!ctx || !tx || !ty) return HOPE_EINVAL;
  *tx = ctx->grids[0].rtx;
  *ty = ctx->grids[0].rty;
  return HOPE_OK;
}

int hope_autotune(hope_t ctx, int reps, float *ms_out, int *tx, int *ty, int *grid) {
  if (!ctx || reps < 1) return HOPE_EINVAL;
  if (!ctx->ens) {
    if (ctx->scheme != HOPE_TPP || ctx->grids.size() != 1) {
      set_error("hope_autotune: needs a TPP sphere or a TPP ensemble");
      return HOPE_EUNSUPPORTED;
    }
    int rc = tune_recon_tile(ctx, reps, ms_out, nullptr);
    if (rc) return rc;
    const Grid &g = ctx->grids[0];
    if (tx) *tx = g.rtx;
    if (ty) *ty = g.rty;
    if (grid) *grid = 6 * ((g.N + g.rtx - 1) / g.rtx) * ((g.N + g.rty - 1) / g.rty);
    return HOPE_OK;
  }
  HOPE_CUDA_TRY(cudaDeviceSynchronize());  // queued stages may still use the member table
  drop_graphs(ctx);  // captured stages bake in the tile shape and block size
  int rc = ensemble_autotune(ctx, ctx->q1, ctx->lbuf, reps, ms_out, nullptr);
  if (rc) return rc;
  HOPE_CUDA_TRY(cudaDeviceSynchronize());
  int a = 0, b = 0, c = 0;
  ensemble_shape(ctx, &a, &b, &c);
  if (tx) *tx = a;
  if (ty) *ty = b;
  if (grid) *grid = c;
  return HOPE_OK;
}

int hope_autotune_candidates(hope_t ctx) {
  if (!ctx) return 0;
  return ctx->ens ? ensemble_num_shapes(ctx) : (ctx->scheme == HOPE_TPP ? 3 : 0);
}

int hope_inject_fault(hope_t ctx, int what) {
  if (!ctx || what != HOPE_INJECT_BARRIER_TIMEOUT) return HOPE_EINVAL;
  if (!ctx->ens) {
    set_error("hope_inject_fault: only the persistent ensemble stage has grid barriers");
    return HOPE_EUNSUPPORTED;
  }
  ctx->ens->inject_timeout = 1;
  return HOPE_OK;
}

int hope_set_profiling(hope_t ctx, int enable) {
  if (!ctx) return HOPE_EINVAL;
  if (enable && !ctx->prof_ev[0][0]) {
    for (int s = 0; s < PROF_STAGES; ++s)
      for (int t = 0; t <= PROF_KERNELS; ++t) HOPE_CUDA_TRY(cudaEventCreate(&ctx->prof_ev[s][t]));
  }
  ctx->profiling = enable ? 1 : 0;
  return HOPE_OK;
}

int hope_kernel_times(hope_t ctx, float *ms_out, int max_entries, int *n_entries) {
  if (!ctx || !ms_out || !n_entries || !ctx->prof_ev[0][0]) return HOPE_EINVAL;
  if (ctx->ens) {
    // persistent stage: the phases' global-timer stamps (block 0 after each grid barrier)
    unsigned long long t[5 * PROF_STAGES];
    HOPE_CUDA_TRY(cudaDeviceSynchronize());
    HOPE_CUDA_TRY(cudaMemcpy(t, ctx->ens->stamps, sizeof(t), cudaMemcpyDeviceToHost));
    int n = 0;
    for (int s = 0; s < PROF_STAGES; ++s)
      for (int k = 0; k < PROF_KERNELS && n < max_entries; ++k)
        ms_out[n++] = (float)((double)(t[5 * s + k + 1] - t[5 * s + k]) * 1e-6);
    *n_entries = n;
    return HOPE_OK;
  }
  HOPE_CUDA_TRY(cudaEventSynchronize(ctx->prof_ev[PROF_STAGES - 1][PROF_KERNELS]));
  int n = 0;
  for (int s = 0; s < PROF_STAGES; ++s)
    for (int t = 0; t < PROF_KERNELS; ++t) {
      if (n >= max_entries) break;
      float ms = 0.0f;
      HOPE_CUDA_TRY(cudaEventElapsedTime(&ms, ctx->prof_ev[s][t], ctx->prof_ev[s][t + 1]));
      ms_out[n++] = ms;
    }
  *n_entries = n;
  return HOPE_OK;
}

int hope_vjp_phase_times(hope_t ctx, float *ms_out) {
  if (!ctx || !ms_out || !ctx->ens) {
    set_error("hope_vjp_phase_times: needs a TPP ensemble context");
    return HOPE_EINVAL;
  }
  unsigned long long t[7];
  HOPE_CUDA_TRY(cudaDeviceSynchronize());
  HOPE_CUDA_TRY(cudaMemcpy(t, ctx->ens->vstamps, sizeof(t), cudaMemcpyDeviceToHost));
  for (int k = 0; k < 6; ++k) ms_out[k] = (float)((double)(t[k + 1] - t[k]) * 1e-6);
  return HOPE_OK;
}

// -------------------------------------------------------------------------------
// Bottom topography (eqs. 2.13-2.14).  The state keeps the depth sqrtG phi; the library
// reconstructs it as it is and adds the surface's part of phi_t from static tables built
// here in FP64 from the cell averages of sqrtG phi_s: its ghost ring (the composed ghost
// operator of eq. 7.12 applied on the host), its TPP values at the edge points (for
// LMARS's phi_t), and psi_B's cell average as an affine map of the depth stencil.  For
// the linear TPP reconstruction this is the same operator as reconstructing
// sqrtG phi_t = sqrtG phi + sqrtG phi_s and subtracting the surface's reconstruction.
// -------------------------------------------------------------------------------
static void free_topography(Grid &g) {
  void *ptrs[] = {g.tsep, g.ttw, g.ttb, g.tsext, g.tscp};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  g.tsep = g.ttw = g.ttb = g.tsext = g.tscp = nullptr;
}

int hope_set_topography(hope_t ctx, const double *phis_avg_host) {
  if (!ctx) {
    set_error("hope_set_topography: null context");
    return HOPE_EINVAL;
  }
  if (ctx->grids.size() != 1 || ctx->ens || ctx->scheme == HOPE_WENO1D) {
    set_error("hope_set_topography: bottom topography is built for single TPP and WENO2D spheres");
    return HOPE_EUNSUPPORTED;
  }
  Grid &g = ctx->grids[0];
  const int N = g.N;
  const size_t pn = (size_t)6 * N * N;
  if (phis_avg_host)
    for (size_t c = 0; c < pn; ++c)
      if (!std::isfinite(phis_avg_host[c])) {
        set_error("hope_set_topography: non-finite surface value");
        return HOPE_EINVAL;
      }
  HOPE_CUDA_TRY(cudaDeviceSynchronize());  // queued stages may still read the old tables
  drop_graphs(ctx);
  free_topography(g);
  if (!phis_avg_host) return HOPE_OK;
  std::vector<double> sep, tw, tb, sext, scp;
  const bool weno = ctx->scheme == HOPE_WENO2D;
  int rc = build_topography_tables(ctx, N, phis_avg_host, sep, tw, tb, weno ? &sext : nullptr,
                                   weno ? &scp : nullptr);
  if (rc) return rc;
  if ((rc = upload(&g.tsep, sep, ctx->esize)) || (rc = upload(&g.ttw, tw, ctx->esize)) ||
      (rc = upload(&g.ttb, tb, ctx->esize)) || (weno && (rc = upload(&g.tsext, sext, ctx->esize))) ||
      (weno && (rc = upload(&g.tscp, scp, ctx->esize)))) {
    free_topography(g);
    return rc;
  }
  return HOPE_OK;
}

int hope_topography_tables(int N, int order, double radius, const double *phis_avg_host, double *sep_out,
                           double *w_out, double *b_out) {
  if (N < order || order < 3 || order > HOPE_MAXK || order % 2 == 0 || !(radius > 0) || !phis_avg_host) {
    set_error("hope_topography_tables: invalid argument");
    return HOPE_EINVAL;
  }
  hope_ctx ctx;
  ctx.k = order;
  ctx.H = (order - 1) / 2;
  ctx.me = (order + 1) / 2;
  ctx.prec = HOPE_FP64;
  ctx.scheme = HOPE_TPP;
  ctx.ghost_iters = 10;
  ctx.radius = radius;
  std::vector<double> sep, tw, tb;
  int rc = build_topography_tables(&ctx, N, phis_avg_host, sep, tw, tb);
  if (rc) return rc;
  if (sep_out) memcpy(sep_out, sep.data(), sizeof(double) * sep.size());
  if (w_out) memcpy(w_out, tw.data(), sizeof(double) * tw.size());
  if (b_out) memcpy(b_out, tb.data(), sizeof(double) * tb.size());
  return HOPE_OK;
}

int hope_measure_fma_peak(int precision, double *flops_per_s) {
  return hope_measure_fma_peak_clock(precision, 4, flops_per_s, nullptr, nullptr);
}

int hope_measure_fma_peak_clock(int precision, int reps, double *flops_per_s, double *sm_mhz,
                                double *flops_per_sm_clock) {
  if (!flops_per_s || (precision != HOPE_FP64 && precision != HOPE_FP32) || reps < 2) return HOPE_EINVAL;
  int dev, sms;
  HOPE_CUDA_TRY(cudaGetDevice(&dev));
  HOPE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8;
  void *out;
  HOPE_CUDA_TRY(cudaMalloc(&out, 16 + sizeof(unsigned long long) * 2 * blocks));
  unsigned long long *stamps = (unsigned long long *)((char *)out + 16);
  const int iters = precision == HOPE_FP64 ? 256 : 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  double best_mhz = 0.0, best_cyc = 0.0;
  std::vector<unsigned long long> h(2 * (size_t)blocks);
  for (int rep = 0; rep < reps; ++rep) {
    cudaEventRecord(e0);
    if (precision == HOPE_FP64)
      k_fma_peak<double><<<blocks, threads>>>((double *)out, iters, 1.0, stamps);
    else
      k_fma_peak<float><<<blocks, threads>>>((float *)out, iters, 1.0f, stamps);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) {
      best = ms;
      if (cudaMemcpy(h.data(), stamps, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost) ==
          cudaSuccess) {
        // clock = cycles / time, summed over blocks; cycles per SM = the slowest block's
        double cyc = 0.0, ns = 0.0, cmax = 0.0;
        for (int b = 0; b < blocks; ++b) {
          cyc += (double)h[2 * b];
          ns += (double)h[2 * b + 1];
          if ((double)h[2 * b] > cmax) cmax = (double)h[2 * b];
        }
        best_mhz = ns > 0 ? 1e3 * cyc / ns : 0.0;
        best_cyc = cmax;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  HOPE_CUDA_TRY(cudaGetLastError());
  double flops = 2.0 * 8 * 16 * (double)iters * threads * blocks;
  *flops_per_s = flops / (best * 1e-3);
  if (sm_mhz) *sm_mhz = best_mhz;
  if (flops_per_sm_clock) *flops_per_sm_clock = best_cyc > 0 ? flops / sms / best_cyc : 0.0;
  return HOPE_OK;
}

}  // extern "C"
