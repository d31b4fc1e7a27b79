/*
 * gks.h -- C ABI of the GB300 (sm_103a) implementation of the hot path of the
 * compact third-order gas-kinetic scheme of Pan & Xu ("A compact third-order
 * gas-kinetic scheme for compressible Euler and Navier-Stokes equations",
 * arXiv:1412.4489) on 2D structured grids.
 *
 * One call of gks_step is one time step of the scheme:
 *   (a) compact reconstruction of every cell from its cell average, the four
 *       neighbouring averages and the tracked point values at the Gauss points
 *       of its four faces (Section 3.2: Eq. over-sys, Eq. limiter, Eq. average);
 *   (b) the third-order gas evolution model at every face centre (Section 2.2:
 *       Eq. compatibility2 for g0, the equilibrium polynomial of Section 3.3,
 *       the coefficient systems after Eq. dis3, the collision time of Section 4);
 *   (c) the analytically time-integrated flux (Eq. dis1 + Eq. dis2 integrated in
 *       time and along the face), the face point values W(t^{n+1}) (Eq. point),
 *       the conservative update (Eq. finite) and the CFL time step reduction.
 *
 * Conventions
 *   Grid: nx by ny cells on [0, Lx] x [0, Ly], cell (i, j) centred at
 *   ((i+1/2) Lx/nx, (j+1/2) Ly/ny).  A 1D problem is nx by 1 with periodic y.
 *   Conservative variables (rho, rho U, rho V, rho E), p = (gamma-1)(rho E - rho|U|^2/2).
 *   Host state arrays are FP64, structure of arrays, x fastest:
 *     U [4][ny][nx]           cell averages
 *     Wx[4][2][ny][nx+1]      x-face point values at y_j - g dy (g index 0) and
 *                             y_j + g dy (index 1), g = sqrt(3)/6
 *     Wy[4][2][ny+1][nx]      y-face point values at x_i - g dx, x_i + g dx
 *   Face i of Wx lies between cells i-1 and i; on a periodic side faces 0 and
 *   nx (0 and ny) are the same face and must carry equal values.
 *   Boundary sides are ordered x-low, x-high, y-low, y-high.
 *
 * Ownership: the library allocates and owns all device memory of a handle
 * (cudaMalloc in gks_create, cudaFree in gks_destroy).  Host pointers passed in
 * are read (set) or written (get) during the call only.  Device pointers passed
 * to the *_device calls must hold FP64 arrays of the layouts above on the
 * handle's device.
 *
 * Positivity fallback (the paper is silent on positivity): when the update
 * makes a cell non-physical (rho <= 0, p <= 0 or not finite), every face of
 * that cell is evolved again with the collisionless first-order flux of the two
 * cell averages (the tau -> infinity limit of the scheme) and the update is
 * redone; if a cell is still non-physical, every face of the grid gets that
 * flux for this step.
 *
 * Errors are returned as gks_status, never by aborting; gks_last_error gives a
 * message.  A step whose new state is still not physical after the fallback is
 * not taken: the state stays the one before the step and GKS_ENONPHYSICAL is
 * reported (by gks_step, or by the next gks_sync / gks_get_state after
 * gks_advance).
 */
#ifndef GKS_H
#define GKS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GKS_OK = 0,
  GKS_EINVAL = 1,        /* invalid argument */
  GKS_ENOMEM = 2,        /* device allocation failed */
  GKS_ECUDA = 3,         /* a CUDA call failed (message in gks_last_error) */
  GKS_ENONPHYSICAL = 4,  /* a step produced a non-physical state; state rolled back */
  GKS_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
  GKS_EUNSUPPORTED = 6
} gks_status;

/* Boundary conditions.  The paper names its boundary conditions (periodic,
 * non-reflecting / outflow, reflective, isothermal no-slip) without defining
 * them; this library uses: periodic = index wrap; outflow = the inside
 * polynomial continued across the boundary face (equal states and
 * derivatives), ghost averages copied; slip wall = mirror image with the normal
 * momentum negated; isothermal no-slip = mirror image with velocity
 * 2 u_wall - u, temperature 2 T_wall - T and equal density (images of the
 * derivatives by the chain rule of that map); adiabatic no-slip = mirror image
 * with velocity 2 u_wall - u, equal temperature and density (no heat flux
 * through the wall; T_wall unused). */
typedef enum {
  GKS_BC_PERIODIC = 0,
  GKS_BC_OUTFLOW = 1,
  GKS_BC_SLIPWALL = 2,
  GKS_BC_NOSLIP_ISOTHERMAL = 3,
  GKS_BC_NOSLIP_ADIABATIC = 4,
  GKS_BC_EXCHANGE = 5  /* y sides only: the handle is one row slab of a larger grid and the
                          neighbouring slab's cells across this side are supplied by the
                          caller (partitioned step, below) */
} gks_bc_kind;

typedef struct {
  int kind;        /* gks_bc_kind */
  double u_wall;   /* wall velocity (x component), no-slip only */
  double v_wall;   /* wall velocity (y component), no-slip only */
  double T_wall;   /* wall temperature p/rho, no-slip only */
} gks_bc;

typedef enum {
  GKS_FP64 = 0,      /* every step in FP64 */
  GKS_FP32_BULK = 1  /* everything in FP32; the cell averages are kept as
                        double-float pairs (hi + lo FP32) updated with compensated
                        (error-free) arithmetic; host transfers in FP64 */
} gks_precision;

typedef struct {
  int precision;     /* gks_precision */
  double weno_eps;   /* epsilon of the nonlinear weights, Eq. average (paper: unstated; default 1e-6) */
  double weno_C;     /* C of I(U1) = C dx dy, Section 3.1 (paper: unstated; default 10: the
                        central stencil must win on smooth data, see the design notes) */
  double tau_eps;    /* epsilon of the inviscid collision time, Section 4 (default 0.05) */
  double tau_C;      /* C of the inviscid collision time, Section 4 (default 1) */
  int viscous_dt;    /* 1: also bound dt by CFL rho h^2 / (2 mu max(4/3, gamma/Pr)) */
  int characteristic;  /* 1: reconstruct in characteristic variables (Section 4: the paper's
                          choice for flows with discontinuities): x-derivatives from the
                          variables projected on the eigenvectors of the x-flux Jacobian of
                          the cell average, y-derivatives likewise, the cross derivative the
                          mean of both; 0 (default): conservative variables */
} gks_options;

typedef struct gks_handle gks_handle;

/* Fills *opt with the defaults listed above. */
void gks_default_options(gks_options* opt);

/* Creates a solver for an nx by ny grid on [0,Lx] x [0,Ly] (nx, ny >= 1;
 * ny = 1 requires periodic y, and likewise nx = 1 periodic x).  gamma > 1 is
 * the ratio of specific heats (K = (4-2 gamma)/(gamma-1) internal degrees of
 * freedom, Section 2.1); mu >= 0 the dynamic viscosity (mu = 0 selects the
 * Euler model f_G = g and the inviscid collision time, Section 2.2 / 4); Pr > 0
 * the Prandtl number (the energy flux gets (1/Pr - 1) times the face heat flux
 * when Pr != 1).  bc[4] may be NULL for all-periodic.  opt may be NULL for the
 * defaults.  cuda_stream is a cudaStream_t (NULL = the legacy default stream)
 * on which all work of the handle is queued.  The state is zero until
 * gks_set_state.  Returns GKS_EINVAL, GKS_ENOMEM or GKS_ECUDA on failure and
 * leaves *out NULL. */
gks_status gks_create(int nx, int ny, double Lx, double Ly, double gamma, double Pr, double mu,
                      const gks_bc* bc, const gks_options* opt, void* cuda_stream,
                      gks_handle** out);

/* Copies a state from host memory (layouts above; Wx/Wy may be NULL, which
 * sets every face point value to the mean of the two adjacent cell averages, a
 * second-order start).  t is the simulation time.  Computes the first CFL
 * bound.  Synchronous.  Clears a pending GKS_ENONPHYSICAL.
 * Page-locked arrays mapped into the device's address space (cudaHostAlloc,
 * cudaHostRegister with the mapped flag, or any page-locked memory on a system
 * with unified addressing) are read in place by the kernels over the host link;
 * other host memory goes through a device staging buffer.  Either way each array
 * must hold the full size given above. */
gks_status gks_set_state(gks_handle* h, const double* U, const double* Wx, const double* Wy,
                         double t);

/* Same, from device memory of the handle's device (FP64 arrays).  The reads are
 * ordered on the handle's stream only: the caller must have finished writing the
 * arrays with respect to that stream (create the handle on the caller's stream,
 * or synchronise first).  Synchronous on return. */
gks_status gks_set_state_device(gks_handle* h, const double* dU, const double* dWx,
                                const double* dWy, double t);

/* One time step with dt = min(CFL * dt_cfl, dt_max) where dt_cfl =
 * min over cells of min(dx/(|U|+c), dy/(|V|+c)) (and the viscous bound if
 * enabled) of the current state.  Synchronous: returns the status of this step
 * and, if dt_taken != NULL, the dt used (0 if no step was taken). */
gks_status gks_step(gks_handle* h, double CFL, double dt_max, double* dt_taken);

/* Queues nsteps steps on the handle's stream without synchronising, each with
 * dt = min(CFL * dt_cfl, t_end - t); steps once t >= t_end are skipped.  The
 * sequence is captured once into a CUDA graph and replayed.  Errors of the
 * queued steps are reported by gks_sync or gks_get_state. */
gks_status gks_advance(gks_handle* h, int nsteps, double CFL, double t_end);

/* Waits for queued work; returns the pending status.  t and steps (either may
 * be NULL) receive the simulation time and the number of steps taken. */
gks_status gks_sync(gks_handle* h, double* t, long long* steps);

/* Copies the state to host memory (any of U, Wx, Wy, t may be NULL); mapped
 * page-locked arrays are written in place by the kernels, as in gks_set_state.
 * Synchronous; returns the pending status (the state is the last good one). */
gks_status gks_get_state(gks_handle* h, double* U, double* Wx, double* Wy, double* t);

/* Same, into device memory (FP64 arrays).  The writes are ordered on the handle's
 * stream and complete on return; the arrays must not be in use by other streams
 * meanwhile. */
gks_status gks_get_state_device(gks_handle* h, double* dU, double* dWx, double* dWy, double* t);

/* Frees the handle and its device memory.  NULL is ignored. */
void gks_destroy(gks_handle* h);

/* Message of the last failed call on h (h may be NULL for create failures). */
const char* gks_last_error(const gks_handle* h);

/* Number of kernel launches one step issues (for launch accounting). */
int gks_launches_per_step(const gks_handle* h);

/* Takes one step like gks_step(h, CFL, +inf, NULL) with CUDA events recorded on
 * the handle's stream between its kernels, and writes the duration in ms of
 * each of the seven kernels to ms[0..6], in launch order: reconstruction (which
 * also opens the step), x-face evolution, y-face evolution, update (which also
 * refreshes the ghost ring), the two update passes of the positivity fallback
 * (no work unless a cell needed it), end.
 * Synchronous; returns the status of the step. */
gks_status gks_profile_step(gks_handle* h, double CFL, float* ms);

/* ---- partitioned step: one grid split into row slabs (domain decomposition) ----
 *
 * A grid of nx by NY cells is split into row slabs, slab r holding global rows
 * [j_r, j_r + ny_r).  Each slab is a handle of nx by ny_r cells on [0, Lx] x
 * [0, ny_r dy] whose y-sides are GKS_BC_EXCHANGE where another slab lies beyond
 * (on a periodic y-axis every y-side of every slab is; with a single slab its own
 * copy), and the grid's own boundary condition where the grid ends.  Its state
 * is the slab's rows of U and Wx and the ny_r + 1 rows of Wy from j_r to
 * j_r + ny_r (both partition faces).  The scheme's step (Eq. finite over the whole
 * grid) is then taken as:
 *   1. bound_r = gks_part_bound(slab r); dt = min(CFL * min_r bound_r, dt_max)
 *      (a min-reduction over all slabs);
 *   2. gks_part_recon(slab r, dt) on every slab: the reconstruction of its cells;
 *   3. the edge rows of reconstruction records (what = GKS_PART_RECORDS) go to
 *      the neighbours: slab r's low edge (gks_part_get_edge(r, 2, ...)) becomes the
 *      high halo of the slab below (gks_part_set_halo(r - 1, 3, ...)), its high
 *      edge the low halo of the slab above;
 *   4. gks_part_finish(slab r): the face evolution of its faces -- the partition
 *      faces are evaluated by both slabs from the same inputs, so neither has to
 *      send its fluxes -- and the update of its cells;
 *   5. the edge rows of the new cell averages (what = GKS_PART_STATE) go to the
 *      neighbours' halos in the same way (also once after gks_set_state, before
 *      the first step).
 * Every cell and face then sees exactly the inputs of the single-grid step, and
 * the slabs' states equal the single-grid state bit for bit.  The positivity
 * fallback is per slab: a step in which a cell next to a partition needs it
 * differs from the single-grid step there (see the design notes).
 * The edge and halo buffers hold raw compute-type data of gks_part_halo_bytes
 * bytes (host or device memory: copies use cudaMemcpyDefault); the calls are
 * synchronous.  Nothing here uses more than the handle's own GPU: the exchange
 * between slabs is the caller's (copies, NCCL or a host transport). */
#define GKS_PART_STATE 0
#define GKS_PART_RECORDS 1

/* Bytes of one edge row of averages (what = GKS_PART_STATE) or of reconstruction
 * records (GKS_PART_RECORDS), ghost columns included. */
gks_status gks_part_halo_bytes(const gks_handle* h, int what, size_t* bytes);

/* CFL bound of the slab's current state (its cells' minimum; see gks_step). */
gks_status gks_part_bound(gks_handle* h, double* bound);

/* Opens a step of the given (global) dt and reconstructs the slab's cells. */
gks_status gks_part_recon(gks_handle* h, double dt);

/* Evolves the slab's faces and updates its cells; closes the step.  Returns
 * GKS_ENONPHYSICAL (state kept) like gks_step. */
gks_status gks_part_finish(gks_handle* h);

/* Copies the slab's edge row on y-side `side` (2: low, 3: high) into dst, or the
 * neighbour's row from src into the slab's halo on that side; `side` must be an
 * exchange side. */
gks_status gks_part_get_edge(gks_handle* h, int side, int what, void* dst);
gks_status gks_part_set_halo(gks_handle* h, int side, int what, const void* src);

/* ---- batched form: many independent grids in one persistent launch ----
 *
 * Grids of uneven sizes, each with its own gamma, mu, Pr, boundary conditions,
 * time step and time, advance together: gks_batch_step queues ONE cooperative
 * kernel that runs nsteps steps of every grid (the phases of Section 2-3 over
 * flat work lists of 128-element tiles from all grids, separated by device-wide
 * barriers), captured once into a CUDA graph and replayed.  Each grid takes
 * dt = CFL * (its own CFL bound), as gks_step does.  Every barrier wait is
 * bounded in time: a wait that runs out abandons the call and gks_batch_sync
 * returns GKS_ETIMEOUT (the batch must then be set up again with
 * gks_batch_set_state).  A grid whose new state is not physical stops (its
 * last good state is kept) and gks_batch_sync returns GKS_ENONPHYSICAL.
 * Host arrays are FP64 in the per-grid layouts of the single-grid API. */
typedef struct {
  int nx, ny;                /* >= 2 */
  double Lx, Ly, gamma, Pr, mu;
  gks_bc bc[4];              /* x-low, x-high, y-low, y-high */
} gks_grid_desc;

typedef struct gks_batch gks_batch;

/* Creates a batch of n grids (device memory for all of them is allocated here).
 * opt may be NULL; its precision selects FP64 or FP32-bulk for every grid. */
gks_status gks_batch_create(int n, const gks_grid_desc* grids, const gks_options* opt,
                            void* cuda_stream, gks_batch** out);

/* Copies grid g's state from host memory (all three arrays required); t is
 * its time.  Synchronous. */
gks_status gks_batch_set_state(gks_batch* b, int g, const double* U, const double* Wx,
                               const double* Wy, double t);

/* Copies grid g's state to host memory (any pointer may be NULL).  Synchronous;
 * returns the grid's status. */
gks_status gks_batch_get_state(gks_batch* b, int g, double* U, double* Wx, double* Wy, double* t,
                               long long* steps);

/* Queues nsteps steps of every grid as one persistent launch (graph replay). */
gks_status gks_batch_step(gks_batch* b, int nsteps, double CFL);

/* Waits; steps_min/steps_max (may be NULL) receive the range of per-grid step
 * counts.  Returns GKS_ETIMEOUT, GKS_ENONPHYSICAL or GKS_OK. */
gks_status gks_batch_sync(gks_batch* b, long long* steps_min, long long* steps_max);

/* Time, step count and status of grid g (synchronous). */
gks_status gks_batch_grid_info(gks_batch* b, int g, double* t, long long* steps, int* status);

/* Sets the face-phase tile widths of x-faces and y-faces (4, 8, 16, 32, 64 or 128
 * faces per row of a 128-face tile: a grid has nx + 1 x-faces per row and ny + 1 rows
 * of y-faces, so narrow tiles waste least on x-faces and wide ones on y-faces) and the
 * resident blocks per SM of the persistent kernel.  gks_batch_configure sets one width
 * for both. */
gks_status gks_batch_configure_tiles(gks_batch* b, int face_tile_width_x, int face_tile_width_y,
                                     int blocks_per_sm);
gks_status gks_batch_configure(gks_batch* b, int face_tile_width, int blocks_per_sm);

/* Autotuner: on the batch itself (the state is saved and restored) times trial_steps
 * steps per trial, searching the x-face tile width, then the y-face tile width, then
 * the resident blocks per SM, keeping the fastest of each; reports the result (any
 * output may be NULL; best_ms per step). */
gks_status gks_batch_autotune(gks_batch* b, double CFL, int trial_steps, int* face_tile_width_x,
                              int* face_tile_width_y, int* blocks_per_sm, float* best_ms);

/* Limit of every device barrier wait, in seconds (default 2).
 * test_skip_block >= 0 makes that block of the persistent kernel skip its
 * barrier arrivals -- a test hook that makes every other wait run out, so that
 * the timeout path can be exercised; -1 disables it. */
gks_status gks_batch_set_wait_limit(gks_batch* b, double seconds, int test_skip_block);

/* Measurement: advances the batch nsteps steps in one (uncaptured) persistent launch
 * in which one block stamps the device clock at each device-wide barrier, and writes
 * the mean time per step of each phase to ms[6], in milliseconds: opening the step
 * (dt per grid), reconstruction, face evolution, update passes 1, 2 and 3 (the last two
 * are 0 unless some grid needed the positivity fallback).  The grids advance as with
 * gks_batch_step.  Synchronous; allocates nsteps * 48 bytes of device memory for the
 * stamps. */
gks_status gks_batch_profile(gks_batch* b, int nsteps, double CFL, double* ms);

/* Total cells of all grids; kernel launches per gks_batch_step call. */
long long gks_batch_cells(const gks_batch* b);
int gks_batch_launches_per_call(const gks_batch* b);
void gks_batch_destroy(gks_batch* b);
const char* gks_batch_last_error(const gks_batch* b);

/* ---- measurement helpers ---- */

/* Counts the arithmetic of one evaluation of the face routine (the gas
 * evolution of Section 2.2 at one face centre, as the kernels compute it) by
 * running it once on the host with a counting number type, for the given
 * face-frame inputs: L, R = [6][4] value and (dn, dt, dnn, dnt, dtt)
 * derivatives of the two sides, avg = [2][3][4] the six cell averages of
 * Section 3.3, cell sizes dn (normal) and dtan (along the face), time step dt.
 * precision selects the branch thresholds of GKS_FP64 or GKS_FP32_BULK.
 * counts[9] receives: additions/subtractions, multiplications, divisions,
 * comparisons, sqrt, rsqrt, exp, expm1, erfc.  Host only; needs no GPU. */
gks_status gks_face_op_count(const double* L, const double* R, const double* avg, double dn,
                             double dtan, double dt, double gamma, double mu, double Pr,
                             double tau_eps, double tau_C, int precision, long long* counts);

/* Measures the FMA throughput of the current device in FP32 (GKS_FP32_BULK) or
 * FP64 (GKS_FP64) with independent FMA chains on every SM; writes TFLOP/s
 * (an FMA = 2 flops).  Synchronous; allocates 64 bytes of device memory. */
gks_status gks_measure_alu_peak(int precision, double* tflops);

/* ---- allocation-free single step ----
 *
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory themselves -- code that runs under another runtime's
 * memory manager or a hard memory cap, and latency-critical loops in which a
 * cudaMalloc/cudaFree would synchronise the device -- and so cannot hold a
 * gks_handle (gks_create allocates).
 *
 * One FP64 time step (the same kernels as gks_step) from the caller's device
 * arrays dU, dWx, dWy (state layouts above, FP64, on the current device) into
 * the caller's device arrays dU_out, dWx_out, dWy_out, with dt = min(CFL *
 * dt_cfl, dt_max) written to *dt_taken (may be NULL).  An output that overlaps
 * an input or another output is rejected with GKS_EINVAL.  The other arguments
 * mean what they mean for gks_create (opt may be NULL; its precision must be
 * GKS_FP64).  The call is synchronous: its work is queued on cuda_stream (NULL =
 * the legacy default stream) and it returns after that work has finished.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine: its scratch
 * (cell averages before and after, reconstruction coefficients, face fluxes and
 * a control block) is one static 60 MiB device array inside this library, which
 * every GPU that loads the library holds until the process exits.  Every grid
 * of up to 65,536 cells fits; larger grids are rejected with GKS_EINVAL and a
 * message in gks_last_error(NULL).  Every call shares that array and leaves its contents
 * behind; the control block is cleared at the start of each call.  Calls whose
 * work overlaps on the GPU (from several threads or streams) race on the array
 * and must be serialised by the caller.  The first call on a device looks up the
 * array's device address (once per device, with that device current); make that
 * first call before any stream capture.  The address is kept for the life of the
 * process, so the device's primary context must not be reset (cudaDeviceReset)
 * between calls.  Returns GKS_ENONPHYSICAL (outputs not
 * valid) if the new state is not physical, GKS_EINVAL if dt would be 0. */
gks_status gks_step_noalloc(int nx, int ny, double Lx, double Ly, double gamma, double Pr, double mu,
                            const gks_bc* bc, const gks_options* opt, const double* dU,
                            const double* dWx, const double* dWy, double CFL, double dt_max,
                            double* dU_out, double* dWx_out, double* dWy_out, double* dt_taken,
                            void* cuda_stream);

/* ---- unit-level entry points used for per-kernel parity checks ---- */

/* Runs only the reconstruction of the current state and copies the
 * coefficients (Ubar, a2, a3, a4, a5, a6) of every cell to host memory in the
 * layout coef[4][6][ny][nx] (FP64).  Synchronous. */
gks_status gks_debug_recon(gks_handle* h, double* coef);

/* Runs reconstruction and the face evolution of the current state with the
 * given dt and copies the face fluxes Fx[4][ny][nx+1], Fy[4][ny+1][nx] and new
 * face values (state layout) to host memory, without updating the state. */
gks_status gks_debug_flux(gks_handle* h, double dt, double* Fx, double* Fy, double* Wx_new,
                          double* Wy_new);

#ifdef __cplusplus
}
#endif
#endif /* GKS_H */
