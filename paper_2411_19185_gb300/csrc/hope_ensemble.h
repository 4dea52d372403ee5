// hope_ensemble.h -- persistent per-stage launch for ensembles (hope_ensemble.cu).
#pragma once
#include <cuda_runtime.h>

#include "hope_internal.h"

namespace hope {

struct EnsembleState {
  void *members[3] = {nullptr, nullptr, nullptr};  // MemberDev<T>[n] per tile shape
  long long items[3][4] = {};                       // ghost rows, tiles, edges, cells
  int grid[3] = {0, 0, 0};                          // resident blocks per shape
  int shape = 0;
  int tuned = 0;
  int inject_timeout = 0;  // the next launch's barriers expect one block more (test hook)
  unsigned *barrier = nullptr;  // [count, generation]
  unsigned long long *stamps = nullptr;  // profiling: per stage [start, 3 phase ends, end] (ns)
  void *ggrp = nullptr;  // GhostGroup[ngrp]: ghost-fill work grouped by shared operator
  int *gmem = nullptr;   // member indices of the groups
  int ngrp = 0;
};

int ensemble_init(hope_ctx *ctx);
void ensemble_free(hope_ctx *ctx);
void ensemble_reset_barrier(hope_ctx *ctx);
int stage_persistent(hope_ctx *ctx, const void *qs, const void *q0, void *out, int mode, double a, double b,
                     double c, const void *q0l, const void *qsl, void *outl, cudaStream_t st);
int ensemble_autotune(hope_ctx *ctx, const void *qs, void *out, int reps, float *ms_out, cudaStream_t st);
void ensemble_shape(const hope_ctx *ctx, int *tx, int *ty, int *grid);

}  // namespace hope
