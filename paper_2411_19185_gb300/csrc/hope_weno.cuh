// hope_weno.cuh -- genuine-2D WENO-Z reconstruction kernels (section 3.2).
#pragma once
#include "hope_internal.h"

namespace hope {

template <typename T, int K>
int launch_recon_weno(hope_ctx *ctx, Grid &g, const T *qs, cudaStream_t st) {
  (void)ctx; (void)g; (void)qs; (void)st;
  set_error("WENO2D reconstruction is not available in this build");
  return HOPE_EUNSUPPORTED;
}

template <typename T, int K>
int weno_set_smem_attr() {
  return HOPE_OK;
}

}  // namespace hope
