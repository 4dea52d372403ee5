// hope_setup.h -- setup entry points shared between the library's translation units.
#pragma once
#include <vector>

#include "hope_internal.h"

namespace hope {
int setup_order_tables(hope_ctx *ctx, std::vector<double> &nodes, std::vector<double> &weights);
int setup_grid_tables(hope_ctx *ctx, Grid &gr, const std::vector<double> &nodes,
                      const std::vector<double> &weights);
struct GhostSplit {
  std::vector<int> head_ptr, head_col, tail_ptr, tail_col;
  std::vector<double> head_val;
  std::vector<float> tail_val;
};
int build_ghost_operator(const hope_ctx *ctx, int N, const std::vector<double> &nodes,
                         const std::vector<double> &weights, std::vector<int> &rowptr,
                         std::vector<int> &cols, std::vector<double> &vals, std::vector<int> &dst,
                         GhostSplit *split = nullptr);
int build_cube_edges(const hope_ctx *ctx, int N, const std::vector<double> &nodes, CubeEdge edges[12],
                     std::vector<double> &conv);
int setup_weno_tables(hope_ctx *ctx, const std::vector<double> &nodes);
}  // namespace hope
