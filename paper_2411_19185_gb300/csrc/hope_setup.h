// hope_setup.h -- setup entry points shared between the library's translation units.
#pragma once
#include <vector>

#include "hope_internal.h"

namespace hope {
int setup_order_tables(hope_ctx *ctx, std::vector<double> &nodes, std::vector<double> &weights);
int setup_grid_tables(hope_ctx *ctx, Grid &gr, const std::vector<double> &nodes,
                      const std::vector<double> &weights);
struct GhostSplit {
  // columns carry the input transform code of the cube symmetry in bits 28-30
  std::vector<int> head_ptr, head_col, tail_ptr, tail_col;
  std::vector<double> head_val;
  std::vector<float> tail_val;
};
// Cube symmetry of the ghost operator: every row is the image of a row on panel 0 under
// one of the cube's 24 rotations, so its weights are read from that row's.  Per row:
// finfo = (row holding the weights) | output code << 28; per nonzero: code << 28 of the
// input transform (see GHOST_SYM_* in hope_kernels.cuh).  Identity codes when the
// operator is not symmetric (it always is for the central-stencil ghost scheme).
struct GhostSym {
  std::vector<int> finfo;  // [rows]
  std::vector<int> ccode;  // [nnz] input code of each nonzero, row order
  bool symmetric = false;
  double max_dev = 0.0;    // largest relative deviation of a row from its symmetric image
};
int build_ghost_operator(const hope_ctx *ctx, int N, const std::vector<double> &nodes,
                         const std::vector<double> &weights, std::vector<int> &rowptr,
                         std::vector<int> &cols, std::vector<double> &vals, std::vector<int> &dst,
                         GhostSplit *split = nullptr, GhostSym *sym = nullptr);
int build_cube_edges(const hope_ctx *ctx, int N, const std::vector<double> &nodes, CubeEdge edges[12],
                     std::vector<double> &conv);
int setup_weno_tables(hope_ctx *ctx, const std::vector<double> &nodes);
// Static tables of a bottom surface from the cell averages of sqrtG phi_s (FP64).
// Optional outputs for the WENO2D reconstruction of sqrtG phi_t: the surface's extended
// averages sext [6][ne][ne] (interior and ghost ring) and its TPP values at the cell points
// scp [me*me][6][N][N] (y node major).
int build_topography_tables(const hope_ctx *ctx, int N, const double *phis_avg_host, std::vector<double> &sep,
                            std::vector<double> &tw, std::vector<double> &tb, std::vector<double> *sext = nullptr,
                            std::vector<double> *scp = nullptr);
}  // namespace hope
