// hope_ensemble.h -- persistent per-stage launch for ensembles (hope_ensemble.cu).
#pragma once
#include <cuda_runtime.h>

#include "hope_internal.h"

namespace hope {

// Candidate shapes of the persistent launch: tx x ty cells per reconstruction work item,
// nt threads per block (the x-pass, flux, update and gather items stride over the block).
constexpr int ENS_MAX_SHAPES = 16;
struct EnsembleShape {
  int tx, ty, nt;
};

struct EnsembleState {
  void *members = nullptr;   // MemberDev<T>[n] for the current shape
  long long items[6] = {};   // ghost items, tiles, edges, cells, extended cells, band lanes (current shape)
  EnsembleShape cand[ENS_MAX_SHAPES] = {};
  int ncand = 0;
  int grid[ENS_MAX_SHAPES] = {};   // resident blocks of the forward launch per candidate
  int vgrid[ENS_MAX_SHAPES] = {};  // resident blocks of the VJP launch per candidate
  int adj_ready = 0;  // member tables carry the adjoint scratch pointers
  int shape = 0;      // current candidate
  int tuned = 0;
  int inject_timeout = 0;  // the next launch's barriers expect one block more (test hook)
  unsigned *barrier = nullptr;  // [count, generation]
  unsigned long long *stamps = nullptr;  // profiling: per stage [start, 3 phase ends, end] (ns)
  // profiling: the last VJP launch's [start, forward ghost end, forward tiles end, flux end,
  // reconstruction end, gather end, end] (ns; the forward entries equal the start when the
  // stage's forward came from a tape)
  unsigned long long *vstamps = nullptr;
  void *ggrp = nullptr;  // GhostGroup[ngrp]: ghost-fill work grouped by shared operator
  int *gmem = nullptr;   // member indices of the groups
  int ngrp = 0;
};

int ensemble_init(hope_ctx *ctx);
void ensemble_free(hope_ctx *ctx);
void ensemble_reset_barrier(hope_ctx *ctx);
int stage_persistent(hope_ctx *ctx, const void *qs, const void *q0, void *out, int mode, double a, double b,
                     double c, const void *q0l, const void *qsl, void *outl, cudaStream_t st);
// Times every candidate shape (ms_out: ENS_MAX_SHAPES floats, -1 past the candidates) and
// keeps the fastest; captured step graphs of the context must be dropped by the caller.
int ensemble_autotune(hope_ctx *ctx, const void *qs, void *out, int reps, float *ms_out, cudaStream_t st);
// One stage VJP of every member in one persistent launch: out = a x + b y + d z + c L^T lamL
// at qs (x, y, z may be null).  have_fwd: the ghost rings and edge points at qs are in the
// members' buffers, or in `tape` (a step tape, stage slot tape_stage) when tape is not null.
int vjp_persistent(hope_ctx *ctx, const void *qs, const void *lamL, void *out, const void *x, const void *y,
                   const void *z, double a, double b, double d, double c, int have_fwd, const void *tape,
                   int tape_stage, cudaStream_t st);
void ensemble_shape(const hope_ctx *ctx, int *tx, int *ty, int *grid);
int ensemble_num_shapes(const hope_ctx *ctx);
// Largest tile buffer (elements) of a member of N cells over the candidate shapes.
size_t ensemble_tile_buf_elems(const hope_ctx *ctx, int N);

}  // namespace hope
