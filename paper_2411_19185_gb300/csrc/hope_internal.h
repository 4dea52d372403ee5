// hope_internal.h -- context layout and launch helpers of the HOPE GB300 library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/hope.h"

#define HOPE_WENO_MAXK 9      // highest WENO2D order compiled
#define HOPE_WENO_ADJ_MAXK 7  // highest WENO2D order with a compiled adjoint

namespace hope {

struct EnsembleState;

// One cube edge shared by panels A < B: A's side sideA meets B's side sideB
// (0 west x=-pi/4, 1 east, 2 south y=-pi/4, 3 north); along the edge, A's cell t and
// Gauss node g coincide with B's cell (flip ? N-1-t : t) and node (flip ? me-1-g : g).
struct CubeEdge {
  int A, sideA, B, sideB, flip;
};

// Device tables and scratch of one sphere (one member of an ensemble).
struct Grid {
  int N = 0, ne = 0;
  int rtx = 16, rty = 8;  // TPP reconstruction tile (cells) of the per-kernel path
  int wtx = 16, wty = 8;  // forward WENO2D tile (cells)
  int ghost_grid = 0, flux_grid = 0, flux_tpb = 0;  // launch shapes, set on first use
  size_t off = 0;   // element offset of this member in ensemble states
  bool owns_tables = true;  // false: tables shared with an earlier member of equal N
  // tables (element type = context precision)
  void *Xg = nullptr;    // [N][me]  tan of the cell Gauss-node coordinates
  void *t1w = nullptr;   // [N][N][me][me]  2/delta^2 * W_gh at the cell points
  void *mx = nullptr;    // edge-point metric terms: [2 orders][5][me][...] (metric_x / metric_y)
  void *src8 = nullptr;  // [N][N][me][me][8] source polynomials times the cell-point weight
  // ghost operator weights (mass, C00, C01, C10, C11): [5][gstride] planes in FP32 contexts,
  // [gstride][5] in FP64 contexts (GHOST_PLANES)
  void *gval = nullptr;
  long long gstride = 0;  // entries of grow/gcol/gval
  int *grow = nullptr;   // [rows+1]
  int *gcol = nullptr;   // [nnz]  source cell p*N*N + j*N + i
  int *gdst = nullptr;   // [rows] destination p*ne*ne + jj*ne + ii
  // [rows] cube symmetry: row whose weights this row uses | output transform code << 28
  // (gcol/tcol carry each nonzero's input transform code in bits 28-30)
  int *gsym = nullptr;
  bool ghost_symmetric = false;
  long long rows = 0, nnz = 0;
  // FP64 contexts: grow/gcol/gval hold the FP64 head of each row, these the FP32 tail
  int *trow = nullptr, *tcol = nullptr;
  float *tval = nullptr;  // [tnnz][5]
  long long tnnz = 0;
  int *bedge = nullptr;  // [12][5] CubeEdge
  void *bconv = nullptr; // [12][N][me][9] ratio_BA, C_BA[4], C_AB[4]
  // scratch
  void *gext = nullptr;  // [3][6][ne][ne] ghost ring (interior unused)
  void *ep = nullptr;    // [4][3][me][6][N][N] edge-point reconstructions
  void *fx = nullptr;    // [3][6][N][N+1]
  void *fy = nullptr;    // [3][6][N+1][N]
  void *sb = nullptr;    // [2][6][N][N] cell-averaged sources
  // bottom topography (eqs. 2.13-2.14), null without: sqrtG phi_s at the edge points
  // [4][me][6][N][N], and psi_B's cell average as an affine map of the depth stencil,
  // weights [2][k*k][6][N][N] and constants [2][6][N][N]
  void *tsep = nullptr, *ttw = nullptr, *ttb = nullptr;
  // WENO2D over a surface: the surface's extended averages [6][ne][ne] (added to the mass
  // variable before the nonlinear reconstruction) and its TPP values at the cell points
  // [me*me][6][N][N] (subtracted after it)
  void *tsext = nullptr, *tscp = nullptr;
  CubeEdge edges[12];
  // transposed ghost operator (adjoint): CSR over interior cells
  int *gtp = nullptr;    // [6*N*N + 1]
  int *gtr = nullptr;    // [nnz] ring position of the entry's ghost row (its gdst)
  int *gband = nullptr;  // [nband] cells that some ghost row reads (ascending)
  long long nband = 0;
  void *gtv = nullptr;   // [nnz][5]
  // adjoint scratch (allocated on the first VJP call)
  void *lep = nullptr;    // like ep
  void *grad = nullptr;   // [3][k*k][6][N][N] (WENO2D; TPP adds the gradients up per tile)
  void *tbuf = nullptr;   // TPP: per reconstruction tile, its gradient on its extended region
  void *lring = nullptr;  // like gext
  void *ldir = nullptr;   // [3][6][N][N]
};

struct GraphKey {
  const void *q;
  double dt;
  int rk;
  int prof;
  bool operator<(const GraphKey &o) const {
    if (q != o.q) return q < o.q;
    if (dt != o.dt) return dt < o.dt;
    if (rk != o.rk) return rk < o.rk;
    return prof < o.prof;
  }
};

constexpr int PROF_STAGES = 3;
constexpr int PROF_KERNELS = 4;

}  // namespace hope

struct hope_ctx {
  int k = 0, H = 0, me = 0, npoc = 0, scheme = 0, prec = 0, rk = 0, ghost_iters = 10;
  double radius = 0, gravity = 0, omega = 0, eps = 0, tilt = 0;
  double fcoef[18] = {0};  // per panel (c0, c1, c2): f*delta/(2 Omega) = c0 + c1 X + c2 Y
  int device = 0;
  int nsm = 1;  // streaming multiprocessors of the device (launch balancing)
  int esize = 8;
  size_t total = 0;  // elements of one (ensemble) state
  std::vector<hope::Grid> grids;
  // order-dependent tables (element type = precision)
  void *w1 = nullptr;   // [me+2][k] 1-D TPP weights at xi = -1/2, +1/2, g_0..g_{me-1}, then [1+(me+1)/2][k] mirror pairs
  void *gw = nullptr;   // [me] Gauss weights
  std::vector<unsigned char> w1_host;  // host copy of w1 (context precision), for by-value kernel arguments
  // WENO tables
  void *wsub = nullptr;   // [me+2][l][l]  1-D sub-stencil weights at the same positions
  void *gpm = nullptr;    // [npoc][2][s] normalised gamma+/sigma+, gamma-/sigma-
  void *sig = nullptr;    // [npoc][2] sigma+, sigma-
  void *bform = nullptr;  // [l][l*l + l] Winv and its row sums per sub-stencil offset
  void *bcoef = nullptr;  // [l][l][l][l] indicator mode weights
  // dimension-by-dimension WENO-Z (HOPE_WENO1D): 1-D split linear weights gamma+-
  // [me+2][2][l], sigma+- [me+2][2], indicator eigenpairs per sub-stencil [l][l*l + l]
  void *w1gpm = nullptr, *w1sig = nullptr, *w1bf = nullptr;
  // buffers
  void *state = nullptr;  // context-owned state
  void *q1 = nullptr, *q2 = nullptr, *lbuf = nullptr;
  // FP32 compensated stepping: low words of the caller's state (carry) and of q1, q2
  void *carry = nullptr, *q1l = nullptr, *q2l = nullptr;
  // adjoint stage states
  void *lam_a = nullptr, *lam_b = nullptr;
  const void *carry_owner = nullptr;
  unsigned *status = nullptr;
  double *mass_part = nullptr;
  double *mass_out = nullptr;
  cudaStream_t cap_stream = nullptr;
  // profiling: events around the first sphere's kernels of each stage of a step
  hope::EnsembleState *ens = nullptr;  // persistent per-stage launch (TPP ensembles)
  int profiling = 0;
  int prof_stage = -1;  // stage being captured (-1: no events)
  cudaEvent_t prof_ev[hope::PROF_STAGES][hope::PROF_KERNELS + 1] = {};
  std::map<hope::GraphKey, cudaGraphExec_t> graphs;
};

namespace hope {
void set_error(const std::string &msg);
}
