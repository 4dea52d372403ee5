/*
 * hope.h -- C ABI of the GB300 (sm_103a) implementation of the per-Runge-Kutta-stage
 * tendency of HOPE's cubed-sphere shallow-water core (Zhou, arXiv 2411.19185).
 *
 * The operation
 *   L(q) = dq/dt  (eq. 3.1): ghost-cell fill across the six panel boundaries
 *   (section 3.3.1 and appendix eq. 7.12), reconstruction of the three state variables
 *   at the Gauss points of every cell by tensor-product polynomials (section 3.1,
 *   eqs. 3.7-3.15) or genuine-2D WENO-Z (section 3.2, eqs. 3.16-3.25), panel conversion
 *   of boundary states (section 3.3.2, eqs. 3.26-3.29), the LMARS flux at every edge
 *   Gauss point (section 3.4, eqs. 3.30-3.38), Gauss quadrature of edge fluxes
 *   (eq. 3.5) and of the metric and Coriolis sources (eqs. 2.2, 2.3, 3.6).
 *
 * State layout and units (every state, tendency and adjoint buffer):
 *   q[var][panel][j][i], var = 0..2, panel = 0..5 (the paper's panels 1..6),
 *   j, i = 0..N-1 with i (the panel's x direction) fastest; element type double
 *   (HOPE_FP64) or float (HOPE_FP32) as chosen at init.
 *   var 0 = sqrtG*phi, var 1 = sqrtG*phi*u, var 2 = sqrtG*phi*v: cell averages, where
 *   sqrtG = (1+X^2)(1+Y^2)/delta^3 is the unit-sphere metric Jacobian (eq. 2.8 divided by
 *   r^2), phi = g*h in m^2/s^2 and (u, v) the contravariant wind in rad/s.
 *   Panel p maps (X, Y) = (tan x, tan y), x, y in [-pi/4, pi/4], to the unit vector
 *   (n_p + X e1_p + Y e2_p)/delta with (n, e1, e2) =
 *     p0 ((1,0,0),(0,1,0),(0,0,1))   p1 ((0,1,0),(-1,0,0),(0,0,1))
 *     p2 ((-1,0,0),(0,-1,0),(0,0,1)) p3 ((0,-1,0),(1,0,0),(0,0,1))
 *     p4 ((0,0,1),(0,1,0),(-1,0,0))  p5 ((0,0,-1),(0,1,0),(1,0,0)),
 *   the convention under which the paper's J (eqs. 2.10-2.11) and sin(latitude)
 *   (eq. 2.5) hold.  Cell (i, j) spans x in [-pi/4 + i dx, -pi/4 + (i+1) dx], dx = pi/(2N).
 *
 * Ownership: the caller owns every state/tendency/adjoint buffer (device memory on
 * the context's device, unless a name ends in _host).  The context owns its tables and
 * scratch.  Buffers passed to one call must not overlap unless stated.
 *
 * Errors: every call returns HOPE_OK (0) or a negative HOPE_E* code; nothing throws or
 * aborts across the ABI.  hope_strerror() names a code; hope_last_error_message() gives
 * the detail of the last failure on the calling thread.  Device-side problems (a
 * non-positive or non-finite phi met by the flux, a non-finite result) set a sticky
 * status word read and cleared by hope_status().
 *
 * Streams: calls taking a stream enqueue work on it and return without synchronising,
 * except where stated (hope_total_mass and the *_host calls synchronise).  One context
 * must not be used from two streams at once: its scratch is shared by all its calls.
 */
#ifndef HOPE_H
#define HOPE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hope_ctx *hope_t;
typedef void *hope_stream_t; /* a cudaStream_t; NULL = the legacy default stream */

/* return codes */
#define HOPE_OK 0
#define HOPE_EINVAL -1      /* bad argument (size, order, null pointer, ...) */
#define HOPE_ECUDA -2       /* a CUDA runtime call failed */
#define HOPE_ENOMEM -3      /* device or host allocation failed */
#define HOPE_ENONPHYS -4    /* non-physical state reported by the device */
#define HOPE_ETIMEOUT -5    /* a bounded device-side wait gave up */
#define HOPE_EUNSUPPORTED -6

/* schemes, precisions, time steppers */
#define HOPE_TPP 0     /* tensor-product polynomial reconstruction, section 3.1 */
#define HOPE_WENO2D 1  /* genuine two-dimensional WENO-Z, section 3.2            */
#define HOPE_WENO1D 2  /* dimension-by-dimension WENO-Z, the comparator of section 5.5: the 1-D
                          WENO-Z of Borges et al. (2008) along x on each stencil row at a point's
                          x position, then along y on the row values; 1-D linear weights by the
                          least squares of eqs. 3.16-3.19 split as eq. 3.20, Jiang-Shu indicators,
                          tau5 = |beta_0 - beta_2|; fifth order only (order 5, the paper's;
                          WENO-Z's tau is order-specific); forward only (the VJP calls return
                          HOPE_EUNSUPPORTED) */
#define HOPE_FP64 0
#define HOPE_FP32 1
#define HOPE_SSPRK3 0  /* strong-stability-preserving RK3 (Shu-Osher form) */
#define HOPE_WSRK3 1   /* Wicker-Skamarock RK3 of eqs. 3.39-3.41 */

/* sticky device status bits (hope_status) */
#define HOPE_STATUS_NONPHYS_PHI 1u /* phi <= 0 where the LMARS flux takes sqrt(phi), eq. 3.35 */
#define HOPE_STATUS_NAN 2u         /* a non-finite value in a computed tendency or state   */
#define HOPE_STATUS_TIMEOUT 4u     /* a bounded grid-wide wait of the persistent ensemble stage gave up */

typedef struct {
  double radius;   /* sphere radius a (m), default 6.37122e6 (section 5.1) */
  double gravity;  /* g (m/s^2), default 9.80616 */
  double omega;    /* rotation rate Omega (1/s), default 7.292e-5; 0 disables Coriolis */
  int n_gauss;     /* Gauss points per edge m_e; 0 => (order+1)/2, the only value supported */
  int precision;   /* HOPE_FP64 (default) or HOPE_FP32 */
  int rk;          /* HOPE_SSPRK3 (default) or HOPE_WSRK3 */
  int ghost_iters; /* sweeps of the ghost-cell iteration (section 3.3.1), default 10 */
  double weno_eps; /* epsilon of eq. 3.23; 0 => 1e-40 (FP64) / 1e-12 (FP32) */
  double coriolis_tilt; /* tilt alpha_c of the rotation axis, default 0: f = 2 Omega sin(theta)
                           (eq. 2.5); alpha_c != 0 gives f = 2 Omega (-cos(lambda) cos(theta)
                           sin(alpha_c) + sin(theta) cos(alpha_c)), the Coriolis parameter
                           under which the geostrophic case rotated by alpha = alpha_c
                           (eqs. 5.1-5.3) is steady (Williamson et al. 1992, case 2) */
} hope_params;

/* Fill *p with the defaults above. */
void hope_default_params(hope_params *p);

/*
 * Create a context for one cubed sphere with N cells per panel edge, stencil width
 * `order` (odd; 3..11 for TPP, the design order of section 3.1; 3..9 for WENO2D, whose
 * adjoint is available up to 7; 5 for WENO1D) and `scheme`.  All tables
 * (reconstruction weights eqs. 3.14-3.15, WENO linear weights eqs. 3.19-3.20 and
 * smoothness forms eq. 3.25, the ghost operator G of eq. 7.12, per-point metric terms
 * eqs. 2.2-2.8) are built in FP64 and stored on the current CUDA device.  Requires
 * N >= order.  On failure *out is NULL.
 */
int hope_init_grid(int N, int order, int scheme, const hope_params *params, hope_t *out);

/*
 * Create one context for an ensemble of n_members independent spheres with
 * N[m] cells per edge (uneven resolutions allowed), sharing order, scheme and params.
 * Ensemble states concatenate the members' (3,6,N[m],N[m]) blocks in member order;
 * hope_state_elems() gives the total length.  A stage of the whole ensemble runs as
 * one persistent launch (work list over all members' tiles).
 */
int hope_init_ensemble(int n_members, const int *N, int order, int scheme,
                       const hope_params *params, hope_t *out);

void hope_destroy(hope_t ctx);

/* Number of elements of one state (3*6*N^2 summed over members). */
size_t hope_state_elems(hope_t ctx);

/* Element size in bytes of the context's precision (8 or 4). */
int hope_elem_size(hope_t ctx);

/*
 * Cell averages of an analytic initial condition (section 5), computed on the device
 * with the me x me Gauss rule of sqrtG times the field, written to q_dev.
 *   case 2  steady geostrophic flow, eqs. 5.1-5.3     params: alpha, u0, phi0
 *   case 6  Rossby-Haurwitz wave, eqs. 5.10-5.15       params: omega_rh, K, R, h0
 *   case 7  dam break: h_in inside a great-circle cap  params: lon, lat, radius, h_in, h_out
 *   case 8  case 2 plus Gaussian bumps of phi          params: alpha, u0, phi0, amp_m, radius;
 *           extra_host: n_extra/2 (lon, lat) centres
 *   case 5  the isolated mountain of eq. 5.8 as a surface: sqrtG phi_s in variable 0,
 *           zero momentum (the input of hope_set_topography)
 *                                                      params: hs0_m, R_rad, lon_c, lat_c
 *   case 10 section 5.2's flow over that mountain: case 2 with its phi read as the free
 *           surface phi_t, stored as the depth phi_t - phi_s
 *                                                      params: alpha, u0, phi0, hs0_m, R_rad,
 *                                                              lon_c, lat_c
 *           (the mountain's longitude difference is taken modulo 2 pi)
 *   case 11 perturbed jet of section 5.4, eqs. 5.16-5.18 (balance integral by composite
 *           Gauss-Legendre)                            params: umax, theta0, theta1, theta2,
 *                                                              alpha, beta, hhat_m, phi0
 *           (phi0 = 0: the constant giving a mean depth of 10 km without the bump);
 *           extra_host is not used
 * For an ensemble every member gets the same case.
 */
int hope_initial_state(hope_t ctx, int ic_case, const double *params, int n_params,
                       const double *extra_host, int n_extra, void *q_dev, hope_stream_t stream);

/*
 * Bottom topography (section 2, eqs. 2.13-2.14; the mountain of section 5.2 is one such
 * surface).  phis_avg_host: HOST array (6, N, N), i fastest, of the cell averages of
 * sqrtG * phi_s (unit-sphere sqrtG as for the state, phi_s = g h_s in m^2/s^2), FP64
 * whatever the context's precision; copied, so the caller keeps ownership.  NULL removes
 * the surface.  The state keeps the fluid depth (q0 = sqrtG phi); the reconstruction acts
 * on sqrtG phi_t = sqrtG (phi + phi_s), LMARS takes its wave speed and upwinded state from
 * the depth and its pressure jump and interface value (eqs. 3.32, 3.33, 3.38) from phi_t,
 * and psi_B = sqrtG phi_s G^ij d phi_t/dx^j (eq. 2.14) joins the cell sources, with the
 * gradient taken from the TPP polynomial of sqrtG phi_t at the cell Gauss points.
 * Builds the surface's tables in FP64 on the host (its ghost ring, its edge-point values
 * and psi_B's weights: 2 k^2 + 4 me + 2 values per cell) after synchronising the device;
 * captured step graphs are dropped.  Single TPP and WENO2D spheres (HOPE_EUNSUPPORTED for
 * ensembles and WENO1D).  With WENO2D the nonlinear reconstruction acts on sqrtG phi_t
 * (the surface's extended averages added to the depth's) and the surface's own TPP values
 * at the points are subtracted, leaving the depth (two more tables: (N+k-1)^2 and me^2 per
 * cell and panel).  The VJP and tape-adjoint calls include the surface's terms (the
 * LMARS adjoint with phi_t, psi_B's stencil map transposed; WENO2D's adjoint recomputes
 * its forward on sqrtG phi_t).  HOPE_EINVAL for a null context or a non-finite value.
 */
int hope_set_topography(hope_t ctx, const double *phis_avg_host);

/* Copy a caller state into / out of the context's own state buffer (device to device). */
int hope_set_state(hope_t ctx, const void *q_dev, hope_stream_t stream);
int hope_get_state(hope_t ctx, void *q_dev, hope_stream_t stream);

/*
 * dqdt_dev = L(q_dev) for one stage (eq. 3.1).  q_dev and dqdt_dev are caller-owned
 * device buffers of hope_state_elems() elements and must not overlap.  q_dev == NULL
 * uses the context's own state.
 */
int hope_tendency(hope_t ctx, const void *q_dev, void *dqdt_dev, hope_stream_t stream);

/*
 * nsteps Runge-Kutta steps of size dt (seconds) in place on q_dev (NULL = the context's
 * own state), with the context's stepper (SSP-RK3 by default).  Each stage fuses the
 * stage combination into the tendency's final kernel.  Steps are replayed from a CUDA
 * graph captured on first use for a given (q_dev, dt).
 * FP32 contexts step compensated: the context keeps an FP32 low word for the most recently
 * stepped buffer (zeroed when another buffer is stepped or hope_set_state / hope_step_host
 * load new contents), and every stage combination is formed with error-free FP32
 * transformations, so rounding of the FP32 state does not accumulate over long runs.
 * A caller that overwrites q_dev between calls should step another buffer or call
 * hope_set_state so that the low word restarts from zero.
 */
int hope_step(hope_t ctx, void *q_dev, double dt, int nsteps, hope_stream_t stream);

/* hope_step with SSP-RK3 regardless of the context's default stepper. */
int hope_step_ssprk3(hope_t ctx, void *q_dev, double dt, hope_stream_t stream);

/*
 * End-to-end form of hope_step for callers holding HOST memory: copies q_host_in
 * (hope_state_elems() elements, ideally pinned) to the device, runs nsteps steps,
 * copies the result to q_host_out (may equal q_host_in) and synchronises the stream.
 */
int hope_step_host(hope_t ctx, const void *q_host_in, void *q_host_out, double dt,
                   int nsteps, hope_stream_t stream);

/*
 * Vector-Jacobian products (hand-written adjoints, no tracing).
 *   hope_tendency_vjp:  lam_q = (dL/dq)^T lam_dqdt at q_dev.
 *   hope_step_vjp:      lam_n = (dS/dq)^T lam_np1 for one RK step S of size dt taken from
 *                       qn_dev (the stage states are recomputed).
 * Output buffers are overwritten; none may overlap an input.
 */
int hope_tendency_vjp(hope_t ctx, const void *q_dev, const void *lam_dqdt_dev, void *lam_q_dev,
                      hope_stream_t stream);
int hope_step_vjp(hope_t ctx, const void *qn_dev, const void *lam_np1_dev, void *lam_n_dev,
                  double dt, hope_stream_t stream);
/* hope_step_vjp of an SSP-RK3 step regardless of the context's default stepper (the
   adjoint of hope_step_ssprk3). */
int hope_step_ssprk3_vjp(hope_t ctx, const void *qn_dev, const void *lam_np1_dev, void *lam_n_dev,
                         double dt, hope_stream_t stream);

/*
 * Step tapes for reverse sweeps over recomputed steps (the checkpointed recompute of the
 * differentiation form, section 4's autograd replaced by hand-written adjoints).
 *   hope_tape_bytes:    bytes of one step's tape: the stage states q1, q2 and, per sphere
 *                       and stage, the ghost ring and the edge-point reconstructions
 *                       (C180 WENO5 FP64: 188 MB).
 *   hope_step_record:   one RK step of q_dev in place (plain stage combinations, also in
 *                       FP32), writing its tape to tape_dev (caller-owned device memory of
 *                       hope_tape_bytes() bytes, alignment 256 B).
 *   hope_step_vjp_tape: hope_step_vjp for the step recorded in tape_dev from qn_dev: the
 *                       stage states, ghost rings and edge points come from the tape, so
 *                       only the adjoint kernels run.  Results equal hope_step_vjp's up to
 *                       rounding.  Output may not overlap an input.
 * Errors: HOPE_EINVAL for null or overlapping arguments, HOPE_ECUDA for failed copies.
 */
int hope_tape_bytes(hope_t ctx, size_t *bytes);
int hope_step_record(hope_t ctx, void *q_dev, double dt, void *tape_dev, hope_stream_t stream);
int hope_step_vjp_tape(hope_t ctx, const void *qn_dev, const void *tape_dev, const void *lam_np1_dev,
                       void *lam_n_dev, double dt, hope_stream_t stream);

/*
 * Total mass M = dx*dy*sum(q[0]) (the I() sum of eq. 5.7 times the cell area) of q_dev,
 * accumulated in FP64 in a fixed order on the device (bitwise reproducible).  For an
 * ensemble, mass_host receives one value per member.  Synchronises the stream.
 */
int hope_total_mass(hope_t ctx, const void *q_dev, double *mass_host, hope_stream_t stream);

/*
 * hope_total_mass_noalloc -- the mass diagnostic of hope_total_mass for one sphere,
 * without a context and without allocating device memory.  (The paper has no
 * counterpart: this is an interface for callers that cannot allocate.)
 *
 * Who needs it: code that must not call cudaMalloc when it wants the diagnostic -- for
 * example a host framework that fixes its device-memory budget after start-up and owns
 * every allocation, a monitoring thread that must not change the device's allocation
 * state, or a time-stepping loop that cannot afford the device-wide synchronisation an
 * allocation may cause.
 * Creating a context allocates its tables, so these callers cannot use hope_total_mass.
 *
 *   q_dev      state (3, 6, N, N) of one sphere on the current device, element type
 *              double (precision HOPE_FP64) or float (HOPE_FP32); caller-owned input.
 *   mass_dev   device pointer to one double; receives dx*dy*sum(q[0]) (FP64 sum in a fixed
 *              order); caller-owned output.  Nothing is copied to the host and the call
 *              does not synchronise.
 *
 * Scratch: the per-block partial sums live in a file-scope device array of
 * HOPE_NOALLOC_MASS_PARTIALS doubles (32 KiB), which every GPU that loads the library holds
 * until the process exits.  Each partial sums HOPE_NOALLOC_MASS_CHUNK elements, so
 * N <= HOPE_NOALLOC_MASS_MAX_N; larger N returns HOPE_EINVAL with a message.  Every used
 * slot is written before it is read, so no clearing is needed between calls.  All calls on
 * a device share the array, which keeps the last call's partials: calls that overlap on
 * the GPU (two streams, or two host threads on one device) race and must be serialised by
 * the caller.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before any stream
 * capture.  No cudaMalloc, cudaFree or allocating library routine is called.
 */
#define HOPE_NOALLOC_MASS_PARTIALS 4096
#define HOPE_NOALLOC_MASS_CHUNK 2048
#define HOPE_NOALLOC_MASS_MAX_N 1182
int hope_total_mass_noalloc(const void *q_dev, int precision, int N, double *mass_dev,
                            hope_stream_t stream);

/* Read and clear the sticky device status (HOPE_STATUS_* bits).  Synchronises. */
int hope_status(hope_t ctx, unsigned *device_status);

/*
 * Ensembles (hope_init_ensemble, TPP): each stage is one persistent cooperative launch over
 * all members' work lists.  hope_autotune times the candidate shapes of that launch -- a
 * tile of TX x TY cells per reconstruction work item (a run-time argument) on blocks of 128
 * or 256 threads: 16x8, 8x16, 32x4, 16x4, 12x10, 24x5, 8x8 on 128 threads, 16x16, 32x8,
 * 16x12, 24x10, 12x20 on 256, less those whose tile does not fit the shared memory -- for
 * reps stages on the context's scratch buffers and keeps the fastest; it runs once at
 * hope_init_ensemble and drops captured step graphs when called again.  ms_out (may be
 * NULL; HOPE_AUTOTUNE_MAX floats) gets one stage time per candidate, -1 after the last
 * (hope_autotune_candidates gives their number); tx/ty/grid the chosen shape and resident
 * grid size.  For a single TPP sphere it times the reconstruction tile candidates 16 x 8, the
 * model's shape and 12 x 12 (3 entries, -1 for a repeated candidate), keeps the fastest (as
 * hope_set_recon_tile) and returns the tile count in grid; it runs at hope_init_grid for
 * FP32.  Returns HOPE_EUNSUPPORTED for WENO2D contexts.
 */
#define HOPE_AUTOTUNE_MAX 16
int hope_autotune(hope_t ctx, int reps, float *ms_out, int *tx, int *ty, int *grid);
/* Number of autotuner candidates of the context (0 for contexts without a tuner). */
int hope_autotune_candidates(hope_t ctx);

/*
 * Tile shape of the per-kernel TPP reconstruction (single spheres; Section 4 describes the
 * reconstruction, the tiling is this library's).  One block reconstructs tx x ty cells of
 * one panel: it stages the tile with its (k-1)/2 halo in shared memory, runs the x-pass
 * over the tile's extended rows and one thread per cell runs the y-pass and the sources.
 * hope_init_grid picks the shape: for FP64 the one that minimises a model of the FP64-pipe
 * time of the most loaded SM (tiles of 64..512 cells); for FP32 (latency-bound) the fastest
 * of 16 x 8, the model's shape and 12 x 12, timed at set-up (hope_autotune).  The results do
 * not depend on the shape (every point value is the same sum in the same order).
 * hope_set_recon_tile overrides it (1 <= tx*ty <= 512 and the tile's shared memory,
 * 8 (FP64) or 4 (FP32) bytes x (3 (ty+k-1)(tx+k-1) + 3 ((k+1)/2+2)(ty+k-1) tx + ((k+1)/2+2) k),
 * within the device's per-block limit; else HOPE_EINVAL) and drops the captured step graphs;
 * HOPE_EINVAL for WENO2D contexts.  hope_recon_tile reads the current shape.
 */
int hope_set_recon_tile(hope_t ctx, int tx, int ty);
int hope_recon_tile(hope_t ctx, int *tx, int *ty);

/*
 * Failure-path hook for tests: HOPE_INJECT_BARRIER_TIMEOUT makes the next persistent stage
 * launch of an ensemble expect one block more at its grid barriers than it launches, so
 * no block is released; every block gives up after the bounded wait (about one second),
 * HOPE_STATUS_TIMEOUT is set and the launch returns.  The context stays usable: the next
 * hope_status() reads and clears the bit and resets the barrier.  No GPU fault is made.
 */
#define HOPE_INJECT_BARRIER_TIMEOUT 1
int hope_inject_fault(hope_t ctx, int what);

/* Total nonzeros of the ghost operator G (eq. 7.12) and its row count. */
int hope_ghost_nnz(hope_t ctx, long long *nnz, long long *rows);

/*
 * Host-only check of the ghost operator's storage (eq. 7.12; needs no GPU): builds the
 * operator for (N, order, precision) on the host as hope_init_grid does and reports
 * whether every row is stored as the rotated copy of a panel-0 representative
 * (symmetric), the largest relative deviation of a directly composed row from its
 * representative's image (max_dev_sym), and the largest relative difference between the
 * stored form as the ghost kernel applies it (the row's columns with their symmetry codes,
 * the representative's weights) and the full operator on a seeded state
 * (max_dev_apply).  HOPE_EINVAL for N < 1, an unsupported order or precision, or null
 * outputs.
 */
int hope_ghost_selfcheck(int N, int order, int precision, int *symmetric, double *max_dev_sym,
                         double *max_dev_apply);

/*
 * Host-only construction, in FP64, of the bottom-surface tables that hope_set_topography
 * uploads (no device is touched), for checks on machines without a GPU.  N >= order,
 * order odd in 3..11, radius > 0 (m).  phis_avg_host: (6, N, N) cell averages of
 * sqrtG phi_s.  Outputs are caller-owned host arrays, each may be NULL:
 *   sep_out [4][me][6][N][N]  sqrtG phi_s at the edge points (west and east at the
 *                             y-nodes, south and north at the x-nodes)
 *   w_out   [2][k*k][6][N][N] weights of psi_B's cell average (eq. 2.14, momentum x and y)
 *                             on the k x k stencil of the depth (cell (a, b) of the
 *                             stencil at index b*k + a, offsets -H..H)
 *   b_out   [2][6][N][N]      its constant part
 * so that the cell average of psi_B is b + sum_c w[c] * stencil_c.  HOPE_EINVAL on bad
 * arguments.
 */
int hope_topography_tables(int N, int order, double radius, const double *phis_avg_host, double *sep_out,
                           double *w_out, double *b_out);

/* Launch configuration introspection for profiling: number of kernel launches one
   tendency enqueues. */
int hope_launches_per_stage(hope_t ctx, int *launches);

/*
 * Per-kernel timing for profiling.  hope_set_profiling(ctx, 1) makes the graphs that
 * hope_step captures from then on record a CUDA event before and after every kernel of
 * the first sphere's stages; hope_kernel_times() then returns, for the most recent step,
 * the elapsed milliseconds of each kernel in launch order: stage-major, and within a
 * stage [ghost fill, reconstruction, flux, update] (HOPE_KERNELS_PER_STAGE entries).
 * It synchronises on the last event.  n_entries receives the number written.  For TPP
 * ensembles (one persistent launch per stage over all members) the four entries are the
 * launch's phases, from GPU global-timer stamps that block 0 takes at the grid barriers
 * (the last entry ends when the last block finishes); the call synchronises the device.
 */
#define HOPE_KERNELS_PER_STAGE 4
int hope_set_profiling(hope_t ctx, int enable);
int hope_kernel_times(hope_t ctx, float *ms_out, int max_entries, int *n_entries);
/* Phases of the most recent stage VJP of a TPP ensemble (one persistent launch) while
 * profiling is enabled: ms_out[6] = forward ghost fill, forward reconstruction (both 0 when
 * the stage's forward came from a step tape), flux adjoint, reconstruction and source
 * adjoint, stencil-gradient gather, transposed ghost operator; from global-timer stamps of
 * block 0 at the grid barriers (the last ends when the last block finishes).  Synchronises
 * the device.  HOPE_EINVAL for a context that is not a TPP ensemble. */
int hope_vjp_phase_times(hope_t ctx, float *ms_out);

const char *hope_strerror(int code);
const char *hope_last_error_message(void);

/*
 * Microbenchmark of the device's plain-ALU peak (no tensor cores): dependent-chain-free
 * fused multiply-add loops in FP64 (precision HOPE_FP64) or FP32 on every SM, timed with
 * CUDA events.  *flops_per_s receives the measured rate (2 flops per FMA).
 */
int hope_measure_fma_peak(int precision, double *flops_per_s);
/*
 * hope_measure_fma_peak with the clock it ran at: reps launches (>= 2; the first is a
 * warm-up), the fastest kept.  sm_mhz (may be NULL) receives the SM clock during that
 * launch (SM cycle counter over the global timer, summed over blocks), flops_per_sm_clock
 * (may be NULL) the flops per SM per clock cycle, i.e. the rate independent of the clock
 * (the FP64 pipe's nominal 2 FMA per SM per cycle give 4).
 */
int hope_measure_fma_peak_clock(int precision, int reps, double *flops_per_s, double *sm_mhz,
                                double *flops_per_sm_clock);

#ifdef __cplusplus
}
#endif
#endif
