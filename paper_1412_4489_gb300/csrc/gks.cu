// GB300 (sm_103a) kernels and C ABI of the compact third-order gas-kinetic
// scheme (Pan & Xu, arXiv:1412.4489).  See include/gks.h for the interface.
//
// One step = seven launches on the handle's stream, all reading a device-resident
// control block so that the sequence can be captured once in a CUDA graph:
//   k_recon    dt = min(CFL * dt_cfl, dt_max, t_end - t) from the running min
//              (block 0), and the compact reconstruction of every cell (Section 3.2)
//   k_flux<0>  gas evolution at every x-face (Section 2.2, 3.3, 4)
//   k_flux<1>  gas evolution at every y-face (frame rotated: n = y, t = x)
//   k_update   conservative update (Eq. finite) into FP64 averages, or in
//              FP32-bulk mode into double-float (hi + lo FP32) averages, the
//              ghost cells that are images of the updated cells, the next CFL
//              bound (warp-shuffle / block / atomic min) and the physical check;
//              three passes, the second and third only for the positivity fallback
//   k_end      advance t and the step counter
// The ghost ring of a newly set state is filled by k_ghost.
// Cell averages and face values are double-buffered; the buffer in use is the
// parity of the device step counter, so a failed step leaves the last good
// state in place.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <string>

#include "../../include/gks.h"
#include "gks_device.cuh"
#include "gks_grid.cuh"

using namespace gks;

namespace {

constexpr int kLaunchesPerStep = 7;

template <class T> struct Store;
template <> struct Store<double> { static __device__ __forceinline__ double to(double x) { return x; } };
template <> struct Store<float> { static __device__ __forceinline__ float to(double x) { return (float)x; } };

// ---------------------------------------------------------------------------
// control kernels
// ---------------------------------------------------------------------------
__global__ void k_end(Ctrl* c) {
  pdl_enter();
  ctrl_end(c);
}

// ---------------------------------------------------------------------------
// ghost ring: perimeter of the padded cell array of the current buffer
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_ghost(Geo g, Cells<R> U0, Cells<R> U1, const Ctrl* c, int force) {
  if (!force && c->skip) return;
  const int par = (int)(c->steps & 1);
  ghost_at<R>(g, par ? U1 : U0, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// reconstruction; U is the padded cell-average array in the compute type
// ---------------------------------------------------------------------------
// begin = 1: block 0 also opens the step (ctrl_begin); the other blocks then do
// not look at the skip flag it sets (coefficients of a skipped step go unused).
// CHAR: reconstruction in characteristic variables.
// resident 256-thread blocks per SM the reconstruction is compiled for: FP32 conservative 4
// (64 registers; the kernel is latency-bound, so occupancy pays), FP64 characteristic 1
// (it needs more than 128 registers), the others 2 (128)
template <class R, bool CHAR> struct ReconBlocks { static constexpr int value = 2; };
template <> struct ReconBlocks<float, false> { static constexpr int value = 4; };
template <> struct ReconBlocks<double, true> { static constexpr int value = 1; };

template <class R, class TW, bool CHAR>
__global__ void __launch_bounds__(256, ReconBlocks<R, CHAR>::value) k_recon(Geo g, const R* U0, const R* U1, const TW* Wx0, const TW* Wx1,
                                               const TW* Wy0, const TW* Wy1, R* __restrict__ rec, R dx, R dy,
                                               R weps, R wC, Ctrl* c, int force, int begin, double cfl,
                                               double dt_max, double t_end) {
  pdl_enter();
  if (begin) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) ctrl_begin(c, cfl, dt_max, t_end);
  } else if (!force && c->skip) {
    return;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const int par = (int)(c->steps & 1);
  recon_cell<R, TW, CHAR>(g, par ? U1 : U0, par ? Wx1 : Wx0, par ? Wy1 : Wy0, rec, i, j, dx, dy, weps, wC);
}

// ---------------------------------------------------------------------------
// face evolution
// ---------------------------------------------------------------------------
// resident 128-thread blocks per SM the face kernel is compiled for (register cap).
// FP32: 4 blocks = 16 warps per SM at 128 registers (registers are allocated per SM
// quarter, so more than 12 warps means at most 128); the Euler routine fits without
// spilling, and the extra warps hide more of its latency than 3 blocks at 168 registers.
#ifndef GKS_FLUX_MINB_F32
#define GKS_FLUX_MINB_F32 4
#endif
template <class R> struct FluxBlocks;
template <> struct FluxBlocks<double> { static constexpr int value = 1; };
template <> struct FluxBlocks<float> { static constexpr int value = GKS_FLUX_MINB_F32; };

// NS: Navier-Stokes (1) or Euler (0) face routine, chosen per grid by flux_kernel
template <int AX, class R, class TW, int NS>
__global__ void __launch_bounds__(128, FluxBlocks<R>::value) k_flux(Geo g, FaceConst<R> C, const R* __restrict__ rec,
                                                                    TW* Wn0, TW* Wn1, R* __restrict__ F,
                                                                    const Ctrl* c, int force) {
  pdl_enter();
  if (!force && c->skip) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (AX == 0 && (g.nx & 31) == 0 && blockIdx.x == gridDim.x - 1) {
    // the column of blocks past a row of nx = 32 k x-faces holds only the last face of
    // each row: it takes those faces 128 rows to a block, in whole warps, instead of one
    // busy lane per warp
    i = g.nx;
    j = blockIdx.y * 128 + threadIdx.y * 32 + threadIdx.x;
  }
  const int fx = AX == 0 ? g.nx + 1 : g.nx, fy = AX == 0 ? g.ny : g.ny + 1;
  if (i >= fx || j >= fy) return;
  const int par = (int)(c->steps & 1);
  // new face values go to the other buffer
  flux_face<AX, R, TW, NS>(g, C, rec, par ? Wn0 : Wn1, F, i, j, step_dt<R>(c));
}

template <int AX, class R, class TW>
auto flux_kernel(const Geo& g) -> decltype(&k_flux<AX, R, TW, 1>) {
  return g.mu > 0.0 ? &k_flux<AX, R, TW, 1> : &k_flux<AX, R, TW, 0>;
}

// ---------------------------------------------------------------------------
// update, CFL bound of the new state, physical check
// ---------------------------------------------------------------------------
// Update pass 1, 2 or 3 (see update_cell): pass 1 marks the cells it leaves
// non-physical; pass 2 runs only if pass 1 marked cells, pass 3 only if pass 2
// still left one; a cell non-physical after pass 3 fails the step.  Each pass
// keeps its own running minimum of the CFL bound.  Blocks walk the grid's
// 32 x 8 tiles with a stride of the launch grid: pass 1 is launched with one block
// per tile, passes 2 and 3 (usually no work) with a few blocks per SM.
// Resident blocks per SM the update is compiled for: the rarely taken fallback path
// must not raise the register count of the common one (FP32: 64 registers).
template <class R> struct UpdateBlocks;
template <> struct UpdateBlocks<double> { static constexpr int value = 2; };
template <> struct UpdateBlocks<float> { static constexpr int value = 4; };

template <class R, class TW>
__global__ void __launch_bounds__(256, UpdateBlocks<R>::value) k_update(Geo g, Cells<R> U0, Cells<R> U1, const R* __restrict__ Fx,
                                                const R* __restrict__ Fy, TW* Wx0, TW* Wx1, TW* Wy0, TW* Wy1,
                                                unsigned char* __restrict__ bad, Ctrl* c, int pass) {
  pdl_enter();
  if (c->skip || (pass == 2 && !c->bad_found[0]) || (pass == 3 && !c->bad_found[1])) return;
  const int par = (int)(c->steps & 1);
  R inv_max = R(0);  // over the block's tiles: one block reduction per block
  for (int j0 = blockIdx.y * blockDim.y; j0 < g.ny; j0 += gridDim.y * blockDim.y) {
    for (int i0 = blockIdx.x * blockDim.x; i0 < g.nx; i0 += gridDim.x * blockDim.x) {
      const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
      R inv = R(0);
      if (i < g.nx && j < g.ny) {
        bool b;
        inv = update_cell<R, TW>(g, par ? U1 : U0, par ? U0 : U1, Fx, Fy, par ? Wx0 : Wx1, par ? Wy0 : Wy1, bad, pass,
                                 step_dt<R>(c), i, j, b);
        if (pass == 1) {
          bad[(size_t)j * g.nx + i] = b ? 1 : 0;
          if (b) atomicOr(&c->bad_found[0], 1);
        } else if (pass == 2) {
          if (b) atomicOr(&c->bad_found[1], 1);
        } else if (b && atomicCAS(&c->status, GKS_OK, GKS_ENONPHYSICAL) == GKS_OK) {
          c->fail_step = c->steps;
        }
      }
      inv_max = fmax(inv_max, inv);
    }
  }
  block_bound_to<R>(inv_max, &c->dtb[pass - 1]);
}

// launch grid of an update pass (32 x 8 tiles): pass 1 takes one wave of resident
// blocks (blocks_per_sm per SM), each walking ceil(tiles / wave) tiles along y, so
// that the per-block work (control reads, the CFL reduction) is shared by its tiles;
// the fallback passes at most 8 x (SMs / 2) blocks (usually no work)
dim3 update_grid(const Geo& g, int pass, int sms, int blocks_per_sm) {
  unsigned tx = (unsigned)((g.nx + 31) / 32), ty = (unsigned)((g.ny + 7) / 8);
  if (pass == 1 && sms > 0) {
    const unsigned wave = (unsigned)sms * (unsigned)blocks_per_sm;
    const unsigned rows = wave / tx > 0 ? wave / tx : 1;  // block rows that fit in one wave
    const unsigned k = (ty + rows - 1) / rows;            // tiles per block
    ty = (ty + k - 1) / k;
  }
  if (pass > 1) {
    const unsigned cy = (unsigned)(sms > 1 ? sms / 2 : 76);
    if (tx > 8) tx = 8;
    if (ty > cy) ty = cy;
  }
  return dim3(tx, ty);
}

// CFL bound of the current state (after set_state), in FP64
template <class R>
__global__ void k_dtbound(Geo g, Cells<R> U0, Cells<R> U1, Ctrl* c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int par = (int)(c->steps & 1);
  const Cells<R> U = par ? U1 : U0;
  double inv = 0.0;
  if (i < g.nx && j < g.ny) {
    double w[4];
    for (int v = 0; v < 4; ++v) w[v] = U.get(g, v, i, j);
    bool ok;
    inv = inv_bound<double>(g, w, ok);
    if (!ok || !(inv < INFINITY)) {
      atomicCAS(&c->status, GKS_OK, GKS_ENONPHYSICAL);
      inv = 0.0;
    }
  }
  block_bound_to<double>(inv, &c->bound);
}

// ---------------------------------------------------------------------------
// state transfer
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_scatter_U(Geo g, const double* __restrict__ src, Cells<R> U0, Cells<R> U1, const Ctrl* c,
                            int to_dev) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const Cells<R> U = (c->steps & 1) ? U1 : U0;
  for (int v = 0; v < 4; ++v) {
    const size_t o = ((size_t)v * g.ny + j) * g.nx + i;
    if (to_dev) U.set(g, v, i, j, src[o]);
    else const_cast<double*>(src)[o] = U.get(g, v, i, j);
  }
}

template <class TW>
__global__ void k_copy_W(const double* __restrict__ src, TW* W0, TW* W1, size_t n, const Ctrl* c, int to_dev) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  TW* W = (c->steps & 1) ? W1 : W0;
  if (to_dev) W[k] = Store<TW>::to(src[k]);
  else const_cast<double*>(src)[k] = (double)W[k];
}

// face values = mean of the two adjacent averages (ghosts included)
template <int AX, class TW>
__global__ void k_init_W(Geo g, Cells<TW> U0, Cells<TW> U1, TW* W0, TW* W1, const Ctrl* c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int fx = AX == 0 ? g.nx + 1 : g.nx, fy = AX == 0 ? g.ny : g.ny + 1;
  if (i >= fx || j >= fy) return;
  const int par = (int)(c->steps & 1);
  const Cells<TW> U = par ? U1 : U0;
  TW* W = par ? W1 : W0;
  const size_t n = (size_t)fx * fy, o = (size_t)j * fx + i;
  for (int v = 0; v < 4; ++v) {
    const double a = U.get(g, v, AX == 0 ? i - 1 : i, AX == 0 ? j : j - 1);
    const double b = U.get(g, v, i, j);
    W[(size_t)(v * 2) * n + o] = Store<TW>::to(0.5 * (a + b));
    W[(size_t)(v * 2 + 1) * n + o] = Store<TW>::to(0.5 * (a + b));
  }
}

template <class R>
__global__ void k_coef_out(Geo g, Cells<R> U0, Cells<R> U1, const R* rec, double* out, const Ctrl* c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const Cells<R> U = (c->steps & 1) ? U1 : U0;
  const size_t N = (size_t)g.nx * g.ny, o = (size_t)j * g.nx + i;
  const R* r = rec + ri(g, i, j);
  for (int v = 0; v < 4; ++v) {
    out[(size_t)(v * 6) * N + o] = U.get(g, v, i, j);
    for (int k = 0; k < 5; ++k) out[(size_t)(v * 6 + k + 1) * N + o] = (double)r[4 + 4 * k + v];
  }
}

template <class R>
__global__ void k_to_double(const R* src, double* dst, size_t n) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) dst[k] = (double)src[k];
}

// opens a step of the partitioned form with the dt the caller reduced over all slabs
__global__ void k_part_begin(Ctrl* c, double dt) {
  c->dt = dt;
  c->dt_f = (float)dt;
  c->skip = (c->status != GKS_OK || !(dt > 0.0)) ? 1 : 0;
  c->dtb[0] = c->dtb[1] = c->dtb[2] = dbits(INFINITY);
  c->bad_found[0] = c->bad_found[1] = 0;
}

__global__ void k_set_dt(Ctrl* c, double dt) {
  c->dt = dt;
  c->dt_f = (float)dt;
  c->skip = 0;
}

}  // namespace

// ===========================================================================
// host side
// ===========================================================================
struct gks_handle {
  Geo g;
  int prec;
  cudaStream_t stream;
  bool own_stream;
  cudaStream_t side;              // the y-face evolution runs here, beside the x-faces
  cudaEvent_t fork, join;         // recon -> y-faces, y-faces -> update
  int device;
  int sms;  // multiprocessors of the device
  double* U[2];      // cell averages (Cells<R>: FP64, or FP32 hi / lo planes), 4 * plane doubles each
  void* Wx[2];
  void* Wy[2];
  void* rec;  // reconstruction records (rec_count(g) values of the compute type)
  void* Fx;
  void* Fy;
  unsigned char* bad;  // cells whose first update failed (positivity fallback)
  Ctrl* ctrl;
  Ctrl* hctrl;       // pinned mirror
  double* staging;   // device FP64 scratch for host transfers
  size_t staging_n;
  cudaGraphExec_t graph1, graph16;
  double graph_cfl, graph_tend;
  std::string err;
};

static thread_local std::string g_create_err;

namespace {

size_t n_wx(const Geo& g) { return (size_t)8 * g.ny * (g.nx + 1); }
size_t n_wy(const Geo& g) { return (size_t)8 * (g.ny + 1) * g.nx; }
size_t n_u(const Geo& g) { return (size_t)4 * g.nx * g.ny; }

gks_status fail(gks_handle* h, gks_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(h, GKS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

dim3 grid2(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

// launch of a step kernel; pdl: with programmatic stream serialisation (see pdl_enter)
template <typename... KArgs, typename... Args>
cudaError_t launch(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ev (optional, 10 events): recorded before each of the nine kernels and after the last
template <class R>
FaceConst<R> fconst(const Geo& g, int axis) {
  return grid_face_const<R>(g, axis);
}

// cell-average buffer b, and the compute-type array of its averages
template <class R> Cells<R> cellbuf(const gks_handle* h, int b) { return Cells<R>{(R*)h->U[b]}; }
template <class R> const R* cells(const gks_handle* h, int b) { return (const R*)h->U[b]; }

template <class R>
void launch_ghost(gks_handle* h, int force) {
  const Geo& g = h->g;
  k_ghost<R><<<(perimeter(g) + 127) / 128, 128, 0, h->stream>>>(g, cellbuf<R>(h, 0), cellbuf<R>(h, 1), h->ctrl, force);
}

template <class R, class TW>
cudaError_t launch_recon(gks_handle* h, int force, int begin = 0, double cfl = 0, double dt_max = 0,
                         double t_end = 0, bool pdl = false) {
  const Geo& g = h->g;
  const dim3 b2(32, 8);
  return launch(pdl, g.characteristic ? k_recon<R, TW, true> : k_recon<R, TW, false>, grid2(g.nx, g.ny, b2), b2,
                h->stream, g, cells<R>(h, 0), cells<R>(h, 1),
         (const TW*)h->Wx[0], (const TW*)h->Wx[1], (const TW*)h->Wy[0], (const TW*)h->Wy[1], (R*)h->rec, R(g.dx),
         R(g.dy), R(g.weno_eps), R(g.weno_C), h->ctrl, force, begin, cfl, dt_max, t_end);
}

// ev (optional, kLaunchesPerStep + 1 events): recorded before each kernel and after the last.
// with_begin_end = false (face evaluation of the current state for gks_debug_flux):
// the ghost ring is refreshed first and the step is neither opened nor closed.
template <class R, class TW>
gks_status launch_step_kernels(gks_handle* h, double cfl, double dt_max, double t_end, bool with_begin_end,
                               bool do_update, int force, cudaEvent_t* ev = nullptr, bool do_recon = true) {
  const Geo& g = h->g;
  cudaStream_t s = h->stream;
  auto mark = [&](int k) {
    if (ev) cudaEventRecord(ev[k], s);
  };
  if (!with_begin_end && do_recon) launch_ghost<R>(h, force);
  // programmatic dependent launch between the step's kernels, except when events
  // are recorded between them (per-kernel timing)
  const bool pdl = ev == nullptr;
  cudaError_t le = cudaSuccess;
  auto keep = [&](cudaError_t e) {
    if (le == cudaSuccess) le = e;
  };
  mark(0);
  if (do_recon) keep(launch_recon<R, TW>(h, force, with_begin_end ? 1 : 0, cfl, dt_max, t_end, pdl));
  mark(1);
  const dim3 b2(32, 8), bf(32, 4);
  // the x- and y-face evolutions are independent: without per-kernel timing the y-faces run
  // on a side stream (fork after the reconstruction, join before the update), so that each
  // fills the other's tail wave
  const bool fork = ev == nullptr;
  if (fork) {
    keep(cudaEventRecord(h->fork, s));
    keep(cudaStreamWaitEvent(h->side, h->fork, 0));
    keep(launch(false, flux_kernel<1, R, TW>(g), grid2(g.nx, g.ny + 1, bf), bf, h->side, g, fconst<R>(g, 1),
                (const R*)h->rec, (TW*)h->Wy[0], (TW*)h->Wy[1], (R*)h->Fy, (const Ctrl*)h->ctrl, force));
    keep(cudaEventRecord(h->join, h->side));
  }
  keep(launch(pdl, flux_kernel<0, R, TW>(g), grid2(g.nx + 1, g.ny, bf), bf, s, g, fconst<R>(g, 0), (const R*)h->rec,
              (TW*)h->Wx[0], (TW*)h->Wx[1], (R*)h->Fx, (const Ctrl*)h->ctrl, force));
  mark(2);
  if (fork) {
    keep(cudaStreamWaitEvent(s, h->join, 0));
  } else {
    keep(launch(pdl, flux_kernel<1, R, TW>(g), grid2(g.nx, g.ny + 1, bf), bf, s, g, fconst<R>(g, 1),
                (const R*)h->rec, (TW*)h->Wy[0], (TW*)h->Wy[1], (R*)h->Fy, (const Ctrl*)h->ctrl, force));
  }
  mark(3);
  for (int pass = 1; pass <= 3; ++pass) {
    if (do_update)
      // pass 1 follows the join (two predecessors): an ordinary launch
      keep(launch(pdl && !(fork && pass == 1), k_update<R, TW>, update_grid(g, pass, h->sms, UpdateBlocks<R>::value), b2, s, g,
                  cellbuf<R>(h, 0), cellbuf<R>(h, 1),
                  (const R*)h->Fx, (const R*)h->Fy, (TW*)h->Wx[0], (TW*)h->Wx[1], (TW*)h->Wy[0], (TW*)h->Wy[1],
                  h->bad, h->ctrl, pass));
    mark(3 + pass);
  }
  if (with_begin_end) keep(launch(pdl, k_end, dim3(1), dim3(1), s, h->ctrl));
  mark(7);
  CK(le);
  CK(cudaGetLastError());
  return GKS_OK;
}

gks_status launch_step(gks_handle* h, double cfl, double dt_max, double t_end) {
  if (h->prec == GKS_FP64) return launch_step_kernels<double, double>(h, cfl, dt_max, t_end, true, true, 0);
  return launch_step_kernels<float, float>(h, cfl, dt_max, t_end, true, true, 0);
}

gks_status read_ctrl(gks_handle* h) {
  CK(cudaMemcpyAsync(h->hctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return GKS_OK;
}

void destroy_graphs(gks_handle* h) {
  if (h->graph1) cudaGraphExecDestroy(h->graph1);
  if (h->graph16) cudaGraphExecDestroy(h->graph16);
  h->graph1 = h->graph16 = nullptr;
}

gks_status capture(gks_handle* h, int nsteps, double cfl, double t_end, cudaGraphExec_t* out) {
  cudaGraph_t graph;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  gks_status st = GKS_OK;
  for (int k = 0; k < nsteps && st == GKS_OK; ++k) st = launch_step(h, cfl, INFINITY, t_end);
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (st != GKS_OK) return st;
  if (e != cudaSuccess) return fail(h, GKS_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(h, GKS_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  return GKS_OK;
}

gks_status reset_ctrl(gks_handle* h, double t) {
  memset(h->hctrl, 0, sizeof(Ctrl));
  const double inf = INFINITY;
  uint64_t b;
  memcpy(&b, &inf, 8);
  h->hctrl->bound = b;
  h->hctrl->dtb[0] = h->hctrl->dtb[1] = h->hctrl->dtb[2] = b;
  h->hctrl->t = t;
  CK(cudaMemcpyAsync(h->ctrl, h->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return GKS_OK;
}

// Loads a state from device FP64 arrays.  With stage_w set, dWx /
// dWy are host arrays copied in turn through the staging buffer (which must
// then not hold dU).
// The device address of a page-locked host array mapped into the device's address
// space (cudaHostAlloc, cudaHostRegister): kernels then read or write it in place over
// the host link.  nullptr for any other pointer (pageable host memory goes through
// the staging buffer).
const double* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // an unknown pointer: clear the error it left
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost && a.devicePointer ? (const double*)a.devicePointer : nullptr;
}

// dU, dWx, dWy: device-accessible arrays, except that a face-value array flagged in
// stage_x / stage_y is a host array copied through the staging buffer first
template <class TW>
gks_status load_state(gks_handle* h, const double* dU, const double* dWx, const double* dWy, bool stage_x = false,
                      bool stage_y = false) {
  const Geo& g = h->g;
  cudaStream_t s = h->stream;
  const dim3 b2(32, 8);
  const Cells<TW> U0 = cellbuf<TW>(h, 0), U1 = cellbuf<TW>(h, 1);
  k_scatter_U<TW><<<grid2(g.nx, g.ny, b2), b2, 0, s>>>(g, dU, U0, U1, h->ctrl, 1);
  launch_ghost<TW>(h, 1);
  for (int axis = 0; axis < 2; ++axis) {
    const double* src = axis == 0 ? dWx : dWy;
    const size_t n = axis == 0 ? n_wx(g) : n_wy(g);
    TW* W0 = (TW*)(axis == 0 ? h->Wx[0] : h->Wy[0]);
    TW* W1 = (TW*)(axis == 0 ? h->Wx[1] : h->Wy[1]);
    if (src) {
      if (axis == 0 ? stage_x : stage_y) {
        CK(cudaMemcpyAsync(h->staging, src, n * sizeof(double), cudaMemcpyHostToDevice, s));
        src = h->staging;
      }
      k_copy_W<TW><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, W0, W1, n, h->ctrl, 1);
    } else if (axis == 0) {
      k_init_W<0, TW><<<grid2(g.nx + 1, g.ny, b2), b2, 0, s>>>(g, U0, U1, W0, W1, h->ctrl);
    } else {
      k_init_W<1, TW><<<grid2(g.nx, g.ny + 1, b2), b2, 0, s>>>(g, U0, U1, W0, W1, h->ctrl);
    }
  }
  k_dtbound<TW><<<grid2(g.nx, g.ny, b2), b2, 0, s>>>(g, U0, U1, h->ctrl);
  CK(cudaGetLastError());
  return GKS_OK;
}

template <class TW>
gks_status store_state(gks_handle* h, double* dU, double* dWx, double* dWy) {
  const Geo& g = h->g;
  cudaStream_t s = h->stream;
  const dim3 b2(32, 8);
  if (dU) k_scatter_U<TW><<<grid2(g.nx, g.ny, b2), b2, 0, s>>>(g, dU, cellbuf<TW>(h, 0), cellbuf<TW>(h, 1), h->ctrl, 0);
  if (dWx)
    k_copy_W<TW><<<(unsigned)((n_wx(g) + 255) / 256), 256, 0, s>>>(dWx, (TW*)h->Wx[0], (TW*)h->Wx[1], n_wx(g), h->ctrl, 0);
  if (dWy)
    k_copy_W<TW><<<(unsigned)((n_wy(g) + 255) / 256), 256, 0, s>>>(dWy, (TW*)h->Wy[0], (TW*)h->Wy[1], n_wy(g), h->ctrl, 0);
  CK(cudaGetLastError());
  return GKS_OK;
}

void make_geo(Geo& g, int nx, int ny, double Lx, double Ly, double gamma, double Pr, double mu, const gks_bc* bc,
              const gks_options& o) {
  memset(&g, 0, sizeof(g));
  g.nx = nx; g.ny = ny;
  g.dx = Lx / nx; g.dy = Ly / ny;
  g.gamma = gamma; g.mu = mu; g.Pr = Pr;
  g.weno_eps = o.weno_eps; g.weno_C = o.weno_C; g.tau_eps = o.tau_eps; g.tau_C = o.tau_C;
  g.viscous_dt = o.viscous_dt;
  g.characteristic = o.characteristic;
  for (int k = 0; k < 4; ++k) {
    g.bc.kind[k] = bc ? bc[k].kind : GKS_BC_PERIODIC;
    g.bc.uw[k] = bc ? bc[k].u_wall : 0.0;
    g.bc.vw[k] = bc ? bc[k].v_wall : 0.0;
    g.bc.Tw[k] = bc ? bc[k].T_wall : 1.0;
  }
  geo_finish(g);
}

gks_status check_args(int nx, int ny, double Lx, double Ly, double gamma, double Pr, double mu, const gks_bc* bc,
                      const gks_options* o, std::string& why) {
  if (nx < 1 || ny < 1 || (long long)nx * ny > (1LL << 31)) { why = "nx, ny >= 1 and nx * ny <= 2^31 required"; return GKS_EINVAL; }
  // launch grids: the face kernels cover ny + 1 rows with 4-row blocks (grid y <= 65535)
  if (ny > 4 * 65535 - 1) { why = "ny must be < 262140"; return GKS_EINVAL; }
  if (!(Lx > 0) || !(Ly > 0)) { why = "Lx, Ly must be > 0"; return GKS_EINVAL; }
  if (!(gamma > 1.0) || !(gamma < 3.0)) { why = "gamma must lie in (1, 3)"; return GKS_EINVAL; }
  if (!(Pr > 0)) { why = "Pr must be > 0"; return GKS_EINVAL; }
  if (!(mu >= 0)) { why = "mu must be >= 0"; return GKS_EINVAL; }
  if (o->precision != GKS_FP64 && o->precision != GKS_FP32_BULK) { why = "unknown precision"; return GKS_EINVAL; }
  if (o->characteristic != 0 && o->characteristic != 1) { why = "characteristic must be 0 or 1"; return GKS_EINVAL; }
  if (!(o->weno_eps >= 0) || !(o->weno_C > 0) || !(o->tau_eps >= 0) || !(o->tau_C >= 0)) {
    why = "invalid scheme constants"; return GKS_EINVAL;
  }
  if (bc) {
    for (int k = 0; k < 4; ++k) {
      if (bc[k].kind < 0 || bc[k].kind > GKS_BC_EXCHANGE) { why = "unknown boundary kind"; return GKS_EINVAL; }
      if (bc[k].kind == GKS_BC_EXCHANGE && k < 2) { why = "exchange sides are y sides"; return GKS_EINVAL; }
      if (bc[k].kind == GKS_BC_NOSLIP_ISOTHERMAL && !(bc[k].T_wall > 0)) { why = "T_wall must be > 0"; return GKS_EINVAL; }
    }
    if ((bc[0].kind == GKS_BC_PERIODIC) != (bc[1].kind == GKS_BC_PERIODIC) ||
        (bc[2].kind == GKS_BC_PERIODIC) != (bc[3].kind == GKS_BC_PERIODIC)) {
      why = "periodic must be set on both sides of an axis"; return GKS_EINVAL;
    }
    if ((nx == 1 && bc[0].kind != GKS_BC_PERIODIC) ||
        (ny == 1 && bc[2].kind != GKS_BC_PERIODIC && (bc[2].kind != GKS_BC_EXCHANGE || bc[3].kind != GKS_BC_EXCHANGE))) {
      why = "a single cell across needs periodic sides"; return GKS_EINVAL;
    }
  }
  return GKS_OK;
}

}  // namespace

extern "C" {

void gks_default_options(gks_options* o) {
  if (!o) return;
  o->precision = GKS_FP64;
  o->weno_eps = 1e-6;
  o->weno_C = 10.0;
  o->tau_eps = 0.05;
  o->tau_C = 1.0;
  o->viscous_dt = 0;
  o->characteristic = 0;
}

gks_status gks_create(int nx, int ny, double Lx, double Ly, double gamma, double Pr, double mu, const gks_bc* bc,
                      const gks_options* opt, void* cuda_stream, gks_handle** out) {
  if (!out) { g_create_err = "out is NULL"; return GKS_EINVAL; }
  *out = nullptr;
  gks_options o;
  gks_default_options(&o);
  if (opt) o = *opt;
  std::string why;
  if (check_args(nx, ny, Lx, Ly, gamma, Pr, mu, bc, &o, why) != GKS_OK) { g_create_err = why; return GKS_EINVAL; }
  gks_handle* h = new gks_handle();
  Geo& g = h->g;
  make_geo(g, nx, ny, Lx, Ly, gamma, Pr, mu, bc, o);
  h->prec = o.precision;
  const size_t wsz = h->prec == GKS_FP64 ? 8 : 4;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) {
    if (cuda_stream) { h->stream = (cudaStream_t)cuda_stream; h->own_stream = false; }
    else { e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking); h->own_stream = true; }
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming);
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  for (int b = 0; b < 2; ++b) {
    alloc((void**)&h->U[b], 4 * g.plane * sizeof(double));
    alloc(&h->Wx[b], n_wx(g) * wsz);
    alloc(&h->Wy[b], n_wy(g) * wsz);
  }
  alloc(&h->rec, rec_count(g) * wsz);
  alloc(&h->Fx, (size_t)4 * ny * (nx + 1) * wsz);
  alloc(&h->Fy, (size_t)4 * (ny + 1) * nx * wsz);
  alloc((void**)&h->bad, (size_t)nx * ny);
  alloc((void**)&h->ctrl, sizeof(Ctrl));
  h->staging_n = n_u(g);
  if (n_wx(g) > h->staging_n) h->staging_n = n_wx(g);
  if (n_wy(g) > h->staging_n) h->staging_n = n_wy(g);
  if (h->staging_n < (size_t)24 * nx * ny) h->staging_n = (size_t)24 * nx * ny;
  alloc((void**)&h->staging, h->staging_n * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->hctrl, sizeof(Ctrl));
  if (e == cudaSuccess)
    for (int b = 0; b < 2; ++b) {
      if (e == cudaSuccess) e = cudaMemsetAsync(h->U[b], 0, 4 * g.plane * sizeof(double), h->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->Wx[b], 0, n_wx(g) * wsz, h->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->Wy[b], 0, n_wy(g) * wsz, h->stream);
    }
  if (e != cudaSuccess) {
    g_create_err = std::string("gks_create: ") + cudaGetErrorString(e);
    const gks_status st = e == cudaErrorMemoryAllocation ? GKS_ENOMEM : GKS_ECUDA;
    gks_destroy(h);
    return st;
  }
  if (reset_ctrl(h, 0.0) != GKS_OK) {
    g_create_err = h->err;
    gks_destroy(h);
    return GKS_ECUDA;
  }
  *out = h;
  return GKS_OK;
}

gks_status gks_set_state_device(gks_handle* h, const double* dU, const double* dWx, const double* dWy, double t) {
  if (!h || !dU) return fail(h, GKS_EINVAL, "gks_set_state: U is required");
  CK(cudaSetDevice(h->device));
  gks_status st = reset_ctrl(h, t);
  if (st != GKS_OK) return st;
  st = h->prec == GKS_FP64 ? load_state<double>(h, dU, dWx, dWy) : load_state<float>(h, dU, dWx, dWy);
  if (st != GKS_OK) return st;
  st = read_ctrl(h);
  if (st != GKS_OK) return st;
  if (h->hctrl->status != GKS_OK) return fail(h, GKS_ENONPHYSICAL, "gks_set_state: state has rho <= 0 or p <= 0");
  return GKS_OK;
}

gks_status gks_set_state(gks_handle* h, const double* U, const double* Wx, const double* Wy, double t) {
  if (!h || !U) return fail(h, GKS_EINVAL, "gks_set_state: U is required");
  CK(cudaSetDevice(h->device));
  const Geo& g = h->g;
  gks_status st = reset_ctrl(h, t);
  if (st != GKS_OK) return st;
  // page-locked host arrays are read in place by the kernels; the others go through
  // the staging buffer in turn (U first: the scatter reads it before the face values
  // reuse the buffer, same stream)
  const double* dU = mapped_host(U);
  const double* dWx = Wx ? mapped_host(Wx) : nullptr;
  const double* dWy = Wy ? mapped_host(Wy) : nullptr;
  if (!dU) {
    CK(cudaMemcpyAsync(h->staging, U, n_u(g) * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    dU = h->staging;
  }
  const bool sx = Wx && !dWx, sy = Wy && !dWy;
  if (sx) dWx = Wx;
  if (sy) dWy = Wy;
  st = h->prec == GKS_FP64 ? load_state<double>(h, dU, dWx, dWy, sx, sy)
                           : load_state<float>(h, dU, dWx, dWy, sx, sy);
  if (st != GKS_OK) return st;
  st = read_ctrl(h);
  if (st != GKS_OK) return st;
  if (h->hctrl->status != GKS_OK) return fail(h, GKS_ENONPHYSICAL, "gks_set_state: state has rho <= 0 or p <= 0");
  return GKS_OK;
}

gks_status gks_step(gks_handle* h, double CFL, double dt_max, double* dt_taken) {
  if (!h) return GKS_EINVAL;
  if (!(CFL > 0) || !(dt_max > 0)) return fail(h, GKS_EINVAL, "gks_step: CFL and dt_max must be > 0");
  CK(cudaSetDevice(h->device));
  gks_status st = launch_step(h, CFL, dt_max, INFINITY);
  if (st != GKS_OK) return st;
  st = read_ctrl(h);
  if (st != GKS_OK) return st;
  if (dt_taken) *dt_taken = h->hctrl->skip ? 0.0 : h->hctrl->dt;
  if (h->hctrl->status != GKS_OK) return fail(h, (gks_status)h->hctrl->status, "step produced a non-physical state; state kept");
  return GKS_OK;
}

gks_status gks_advance(gks_handle* h, int nsteps, double CFL, double t_end) {
  if (!h) return GKS_EINVAL;
  if (nsteps < 0 || !(CFL > 0)) return fail(h, GKS_EINVAL, "gks_advance: nsteps >= 0 and CFL > 0 required");
  CK(cudaSetDevice(h->device));
  if (!h->graph1 || h->graph_cfl != CFL || h->graph_tend != t_end) {
    destroy_graphs(h);
    gks_status st = capture(h, 1, CFL, t_end, &h->graph1);
    if (st == GKS_OK) st = capture(h, 16, CFL, t_end, &h->graph16);
    if (st != GKS_OK) { destroy_graphs(h); return st; }
    h->graph_cfl = CFL;
    h->graph_tend = t_end;
  }
  int left = nsteps;
  while (left >= 16) { CK(cudaGraphLaunch(h->graph16, h->stream)); left -= 16; }
  while (left > 0) { CK(cudaGraphLaunch(h->graph1, h->stream)); --left; }
  return GKS_OK;
}

gks_status gks_sync(gks_handle* h, double* t, long long* steps) {
  if (!h) return GKS_EINVAL;
  CK(cudaSetDevice(h->device));
  gks_status st = read_ctrl(h);
  if (st != GKS_OK) return st;
  if (t) *t = h->hctrl->t;
  if (steps) *steps = h->hctrl->steps;
  if (h->hctrl->status != GKS_OK) return fail(h, (gks_status)h->hctrl->status, "a queued step produced a non-physical state; state kept");
  return GKS_OK;
}

gks_status gks_get_state_device(gks_handle* h, double* dU, double* dWx, double* dWy, double* t) {
  if (!h) return GKS_EINVAL;
  CK(cudaSetDevice(h->device));
  gks_status st = h->prec == GKS_FP64 ? store_state<double>(h, dU, dWx, dWy) : store_state<float>(h, dU, dWx, dWy);
  if (st != GKS_OK) return st;
  st = read_ctrl(h);
  if (st != GKS_OK) return st;
  if (t) *t = h->hctrl->t;
  if (h->hctrl->status != GKS_OK) return fail(h, (gks_status)h->hctrl->status, "a step produced a non-physical state; state kept");
  return GKS_OK;
}

gks_status gks_get_state(gks_handle* h, double* U, double* Wx, double* Wy, double* t) {
  if (!h) return GKS_EINVAL;
  CK(cudaSetDevice(h->device));
  const Geo& g = h->g;
  struct { double* host; size_t n; int which; } parts[3] = {{U, n_u(g), 0}, {Wx, n_wx(g), 1}, {Wy, n_wy(g), 2}};
  for (auto& p : parts) {
    if (!p.host) continue;
    // page-locked host arrays are written in place by the kernels; the others through
    // the staging buffer in turn
    double* direct = const_cast<double*>(mapped_host(p.host));
    double* dst = direct ? direct : h->staging;
    gks_status st = h->prec == GKS_FP64
                        ? store_state<double>(h, p.which == 0 ? dst : nullptr, p.which == 1 ? dst : nullptr,
                                              p.which == 2 ? dst : nullptr)
                        : store_state<float>(h, p.which == 0 ? dst : nullptr, p.which == 1 ? dst : nullptr,
                                             p.which == 2 ? dst : nullptr);
    if (st != GKS_OK) return st;
    if (!direct) CK(cudaMemcpyAsync(p.host, h->staging, p.n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  gks_status st = read_ctrl(h);
  if (st != GKS_OK) return st;
  if (t) *t = h->hctrl->t;
  if (h->hctrl->status != GKS_OK) return fail(h, (gks_status)h->hctrl->status, "a step produced a non-physical state; state kept");
  return GKS_OK;
}

void gks_destroy(gks_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  destroy_graphs(h);
  for (int b = 0; b < 2; ++b) {
    cudaFree(h->U[b]);
    cudaFree(h->Wx[b]);
    cudaFree(h->Wy[b]);
  }
  cudaFree(h->rec);
  cudaFree(h->Fx);
  cudaFree(h->Fy);
  cudaFree(h->bad);
  cudaFree(h->ctrl);
  cudaFree(h->staging);
  if (h->hctrl) cudaFreeHost(h->hctrl);
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->fork) cudaEventDestroy(h->fork);
  if (h->join) cudaEventDestroy(h->join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

const char* gks_last_error(const gks_handle* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

gks_status gks_profile_step(gks_handle* h, double CFL, float* ms) {
  if (!h || !ms || !(CFL > 0)) return fail(h, GKS_EINVAL, "gks_profile_step: CFL > 0 and ms[7] required");
  CK(cudaSetDevice(h->device));
  cudaEvent_t ev[kLaunchesPerStep + 1];
  for (int k = 0; k <= kLaunchesPerStep; ++k) CK(cudaEventCreate(&ev[k]));
  gks_status st = h->prec == GKS_FP64 ? launch_step_kernels<double, double>(h, CFL, INFINITY, INFINITY, true, true, 0, ev)
                                      : launch_step_kernels<float, float>(h, CFL, INFINITY, INFINITY, true, true, 0, ev);
  if (st == GKS_OK) {
    cudaError_t e = cudaEventSynchronize(ev[kLaunchesPerStep]);
    for (int k = 0; k < kLaunchesPerStep && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]);
    if (e != cudaSuccess) st = fail(h, GKS_ECUDA, std::string("gks_profile_step: ") + cudaGetErrorString(e));
  }
  for (int k = 0; k <= kLaunchesPerStep; ++k) cudaEventDestroy(ev[k]);
  if (st != GKS_OK) return st;
  st = read_ctrl(h);
  if (st != GKS_OK) return st;
  if (h->hctrl->status != GKS_OK) return fail(h, (gks_status)h->hctrl->status, "step produced a non-physical state; state kept");
  return GKS_OK;
}

int gks_launches_per_step(const gks_handle* h) {
  (void)h;
  return kLaunchesPerStep;
}

gks_status gks_debug_recon(gks_handle* h, double* coef) {
  if (!h || !coef) return GKS_EINVAL;
  CK(cudaSetDevice(h->device));
  const Geo& g = h->g;
  const dim3 b2(32, 8);
  if (h->prec == GKS_FP64) {
    launch_ghost<double>(h, 1);
    launch_recon<double, double>(h, 1);
    k_coef_out<double><<<grid2(g.nx, g.ny, b2), b2, 0, h->stream>>>(g, cellbuf<double>(h, 0), cellbuf<double>(h, 1),
                                                                     (const double*)h->rec, h->staging, h->ctrl);
  } else {
    launch_ghost<float>(h, 1);
    launch_recon<float, float>(h, 1);
    k_coef_out<float><<<grid2(g.nx, g.ny, b2), b2, 0, h->stream>>>(g, cellbuf<float>(h, 0), cellbuf<float>(h, 1),
                                                                    (const float*)h->rec, h->staging, h->ctrl);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(coef, h->staging, (size_t)24 * g.nx * g.ny * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return GKS_OK;
}

gks_status gks_debug_flux(gks_handle* h, double dt, double* Fx, double* Fy, double* Wxn, double* Wyn) {
  if (!h || !(dt > 0)) return fail(h, GKS_EINVAL, "gks_debug_flux: dt > 0 required");
  CK(cudaSetDevice(h->device));
  const Geo& g = h->g;
  k_set_dt<<<1, 1, 0, h->stream>>>(h->ctrl, dt);
  gks_status st = h->prec == GKS_FP64 ? launch_step_kernels<double, double>(h, 0, 0, 0, false, false, 1)
                                      : launch_step_kernels<float, float>(h, 0, 0, 0, false, false, 1);
  if (st != GKS_OK) return st;
  st = read_ctrl(h);
  if (st != GKS_OK) return st;
  const int par = (int)(h->hctrl->steps & 1) ^ 1;  // new values were written to the other buffer
  const size_t nfx = (size_t)4 * g.ny * (g.nx + 1), nfy = (size_t)4 * (g.ny + 1) * g.nx;
  struct { void* src; double* dst; size_t n; } parts[4] = {
      {h->Fx, Fx, nfx}, {h->Fy, Fy, nfy}, {h->Wx[par], Wxn, n_wx(g)}, {h->Wy[par], Wyn, n_wy(g)}};
  for (auto& p : parts) {
    if (!p.dst) continue;
    if (h->prec == GKS_FP64)
      k_to_double<double><<<(unsigned)((p.n + 255) / 256), 256, 0, h->stream>>>((const double*)p.src, h->staging, p.n);
    else
      k_to_double<float><<<(unsigned)((p.n + 255) / 256), 256, 0, h->stream>>>((const float*)p.src, h->staging, p.n);
    CK(cudaMemcpyAsync(p.dst, h->staging, p.n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return GKS_OK;
}

// ---- partitioned step (domain decomposition into row slabs) ----

gks_status gks_part_halo_bytes(const gks_handle* h, int what, size_t* bytes) {
  if (!h || !bytes || (what != GKS_PART_STATE && what != GKS_PART_RECORDS)) return GKS_EINVAL;
  const Geo& g = h->g;
  const size_t es = h->prec == GKS_FP64 ? sizeof(double) : sizeof(float);
  // averages: 4 FP64 planes, or the 4 hi and 4 lo FP32 planes, nx + 2 values each
  *bytes = what == GKS_PART_STATE ? (size_t)8 * sizeof(float) * (g.nx + 2) : (size_t)(g.nx + 2) * kRec * es;
  return GKS_OK;
}

gks_status gks_part_bound(gks_handle* h, double* bound) {
  if (!h || !bound) return GKS_EINVAL;
  CK(cudaSetDevice(h->device));
  gks_status st = read_ctrl(h);
  if (st != GKS_OK) return st;
  memcpy(bound, &h->hctrl->bound, sizeof(double));
  if (h->hctrl->status != GKS_OK) return fail(h, (gks_status)h->hctrl->status, "the slab's state is not physical");
  return GKS_OK;
}

gks_status gks_part_recon(gks_handle* h, double dt) {
  if (!h || !(dt > 0)) return fail(h, GKS_EINVAL, "gks_part_recon: dt > 0 required");
  CK(cudaSetDevice(h->device));
  k_part_begin<<<1, 1, 0, h->stream>>>(h->ctrl, dt);
  CK(cudaGetLastError());
  const cudaError_t e = h->prec == GKS_FP64 ? launch_recon<double, double>(h, 0) : launch_recon<float, float>(h, 0);
  CK(e);
  return GKS_OK;
}

gks_status gks_part_finish(gks_handle* h) {
  if (!h) return GKS_EINVAL;
  CK(cudaSetDevice(h->device));
  gks_status st = h->prec == GKS_FP64
                      ? launch_step_kernels<double, double>(h, 0, 0, 0, true, true, 0, nullptr, false)
                      : launch_step_kernels<float, float>(h, 0, 0, 0, true, true, 0, nullptr, false);
  if (st != GKS_OK) return st;
  st = read_ctrl(h);
  if (st != GKS_OK) return st;
  if (h->hctrl->status != GKS_OK) return fail(h, (gks_status)h->hctrl->status, "step produced a non-physical state; state kept");
  return GKS_OK;
}

namespace {
// one edge or halo row: (device address of its first byte, pitch between planes, planes,
// bytes per plane row); row j of the current buffer
gks_status part_row(gks_handle* h, int side, int what, bool halo, char** p, size_t* pitch, int* rows,
                    size_t* width) {
  if (side != 2 && side != 3) return fail(h, GKS_EINVAL, "side must be 2 (y low) or 3 (y high)");
  if (h->g.bc.kind[side] != GKS_BC_EXCHANGE) return fail(h, GKS_EINVAL, "not an exchange side");
  if (what != GKS_PART_STATE && what != GKS_PART_RECORDS) return fail(h, GKS_EINVAL, "what must be state or records");
  gks_status st = read_ctrl(h);
  if (st != GKS_OK) return st;
  const Geo& g = h->g;
  const int j = halo ? (side == 2 ? -1 : g.ny) : (side == 2 ? 0 : g.ny - 1);
  const size_t es = h->prec == GKS_FP64 ? sizeof(double) : sizeof(float);
  if (what == GKS_PART_STATE) {
    const int par = (int)(h->hctrl->steps & 1);
    *p = (char*)h->U[par] + ((size_t)(j + 1) * g.pitch) * es;
    *pitch = g.plane * es;
    *rows = h->prec == GKS_FP64 ? 4 : 8;
    *width = (size_t)(g.nx + 2) * es;
  } else {
    *p = (char*)h->rec + ri(g, -1, j) * es;
    *pitch = 0;
    *rows = 1;
    *width = (size_t)(g.nx + 2) * kRec * es;
  }
  return GKS_OK;
}
}  // namespace

gks_status gks_part_get_edge(gks_handle* h, int side, int what, void* dst) {
  if (!h || !dst) return GKS_EINVAL;
  CK(cudaSetDevice(h->device));
  char* p;
  size_t pitch, width;
  int rows;
  gks_status st = part_row(h, side, what, false, &p, &pitch, &rows, &width);
  if (st != GKS_OK) return st;
  CK(cudaMemcpy2DAsync(dst, width, p, rows > 1 ? pitch : width, width, rows, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return GKS_OK;
}

gks_status gks_part_set_halo(gks_handle* h, int side, int what, const void* src) {
  if (!h || !src) return GKS_EINVAL;
  CK(cudaSetDevice(h->device));
  char* p;
  size_t pitch, width;
  int rows;
  gks_status st = part_row(h, side, what, true, &p, &pitch, &rows, &width);
  if (st != GKS_OK) return st;
  CK(cudaMemcpy2DAsync(p, rows > 1 ? pitch : width, src, width, width, rows, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return GKS_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free single step (gks_step_noalloc).  For callers that must not
// allocate device memory themselves: code running under another runtime's
// memory manager or a hard memory cap, and latency-critical loops where
// cudaMalloc/cudaFree would synchronise the device.  The scratch of one step
// (the padded cell averages before and after, the reconstruction coefficients,
// the face fluxes and the control block) lives in one file-scope device array
// that every GPU loading this library holds until the process exits.
// ===========================================================================
namespace {

// 60 MiB: any grid of up to 65,536 cells.  The padded cell planes and the ghost ring of
// the reconstruction records make the need largest for a single column (nx = 1, rows
// padded to 4 and 3 records wide): 60,885,248 bytes at 1 x 65,536.
constexpr size_t kNoallocBytes = (size_t)60 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// device address of g_noalloc_scratch per device, looked up once with the device current;
// the cache assumes that the device's primary context is never reset (cudaDeviceReset)
void* noalloc_base(int device, std::string& why) {
  static std::atomic<void*> base[64];
  if (device < 0 || device >= 64) { why = "device index out of range"; return nullptr; }
  void* p = base[device].load();
  if (!p) {
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) { why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e); return nullptr; }
    base[device].store(p);
  }
  return p;
}

__global__ void k_noalloc_ctrl(Ctrl* c) {
  c->bound = dbits(INFINITY);
  c->dtb[0] = c->dtb[1] = c->dtb[2] = dbits(INFINITY);
  c->bad_found[0] = c->bad_found[1] = 0;
  c->t = 0.0;
  c->dt = 0.0;
  c->dt_f = 0.0f;
  c->steps = 0;
  c->status = GKS_OK;
  c->skip = 0;
  c->fail_step = -1;
}

}  // namespace

extern "C" gks_status gks_step_noalloc(int nx, int ny, double Lx, double Ly, double gamma, double Pr, double mu,
                                       const gks_bc* bc, const gks_options* opt, const double* dU,
                                       const double* dWx, const double* dWy, double CFL, double dt_max,
                                       double* dU_out, double* dWx_out, double* dWy_out, double* dt_taken,
                                       void* cuda_stream) {
  gks_options o;
  gks_default_options(&o);
  if (opt) o = *opt;
  std::string why;
  if (check_args(nx, ny, Lx, Ly, gamma, Pr, mu, bc, &o, why) != GKS_OK) { g_create_err = why; return GKS_EINVAL; }
  if (o.precision != GKS_FP64) { g_create_err = "gks_step_noalloc: only GKS_FP64"; return GKS_EINVAL; }
  if (!dU || !dWx || !dWy || !dU_out || !dWx_out || !dWy_out || !(CFL > 0) || !(dt_max > 0)) {
    g_create_err = "gks_step_noalloc: all six state pointers, CFL > 0 and dt_max > 0 are required";
    return GKS_EINVAL;
  }
  {
    // outputs must not overlap inputs or each other: the face kernels write new face values
    // that other faces' reconstruction still reads, and the update reads the old averages
    const size_t nu = (size_t)4 * nx * ny, nwx = (size_t)8 * ny * (nx + 1), nwy = (size_t)8 * (ny + 1) * nx;
    const struct { const double* p; size_t n; } in[3] = {{dU, nu}, {dWx, nwx}, {dWy, nwy}},
                                                 out[3] = {{dU_out, nu}, {dWx_out, nwx}, {dWy_out, nwy}};
    auto overlap = [](const double* a, size_t na, const double* b, size_t nb) { return a < b + nb && b < a + na; };
    for (int k = 0; k < 3; ++k)
      for (int m = 0; m < 3; ++m)
        if (overlap(out[k].p, out[k].n, in[m].p, in[m].n) || (m > k && overlap(out[k].p, out[k].n, out[m].p, out[m].n))) {
          g_create_err = "gks_step_noalloc: the output arrays must not overlap the inputs or each other";
          return GKS_EINVAL;
        }
  }
  Geo g;
  make_geo(g, nx, ny, Lx, Ly, gamma, Pr, mu, bc, o);
  // scratch layout: control block | padded U before | padded U after | reconstruction records | Fx | Fy
  const size_t b_ctrl = align256(sizeof(Ctrl));
  const size_t b_u = align256(4 * g.plane * sizeof(double));
  const size_t b_rec = align256(rec_count(g) * sizeof(double));
  const size_t b_fx = align256((size_t)4 * ny * (nx + 1) * sizeof(double));
  const size_t b_fy = align256((size_t)4 * (ny + 1) * nx * sizeof(double));
  const size_t b_bad = align256((size_t)nx * ny);
  const size_t need = b_ctrl + 2 * b_u + b_rec + b_fx + b_fy + b_bad;
  if ((long long)nx * ny > 65536 || need > kNoallocBytes) {
    g_create_err = "gks_step_noalloc: grid too large for the static scratch (at most 65,536 cells; " +
                   std::to_string(kNoallocBytes >> 20) + " MiB); need " + std::to_string(need) + " bytes";
    return GKS_EINVAL;
  }
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) { g_create_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return GKS_ECUDA; }
  unsigned char* base = (unsigned char*)noalloc_base(device, why);
  if (!base) { g_create_err = "gks_step_noalloc: " + why; return GKS_ECUDA; }
  Ctrl* ctrl = (Ctrl*)base;
  double* U0 = (double*)(base + b_ctrl);
  double* U1 = (double*)(base + b_ctrl + b_u);
  double* rec = (double*)(base + b_ctrl + 2 * b_u);
  double* Fx = (double*)(base + b_ctrl + 2 * b_u + b_rec);
  double* Fy = (double*)(base + b_ctrl + 2 * b_u + b_rec + b_fx);
  unsigned char* bad = base + b_ctrl + 2 * b_u + b_rec + b_fx + b_fy;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const dim3 b2(32, 8), bf(32, 4);
  const int per = perimeter(g);
  const Cells<double> C0{U0}, C1{U1};
  // the control block must start from zero state; the rest is fully written before it is read
  k_noalloc_ctrl<<<1, 1, 0, s>>>(ctrl);
  k_scatter_U<double><<<grid2(nx, ny, b2), b2, 0, s>>>(g, dU, C0, C1, ctrl, 1);
  k_ghost<double><<<(per + 127) / 128, 128, 0, s>>>(g, C0, C1, ctrl, 1);
  k_dtbound<double><<<grid2(nx, ny, b2), b2, 0, s>>>(g, C0, C1, ctrl);
  (g.characteristic ? k_recon<double, double, true> : k_recon<double, double, false>)<<<grid2(nx, ny, b2), b2, 0, s>>>(
      g, U0, U1, dWx, dWx_out, dWy, dWy_out, rec, g.dx, g.dy,
                                                            g.weno_eps, g.weno_C, ctrl, 0, 1, CFL,
                                                            dt_max, INFINITY);
  flux_kernel<0, double, double>(g)<<<grid2(nx + 1, ny, bf), bf, 0, s>>>(g, fconst<double>(g, 0), rec,
                                                                  const_cast<double*>(dWx), dWx_out, Fx, ctrl, 0);
  flux_kernel<1, double, double>(g)<<<grid2(nx, ny + 1, bf), bf, 0, s>>>(g, fconst<double>(g, 1), rec,
                                                                  const_cast<double*>(dWy), dWy_out, Fy, ctrl, 0);
  for (int pass = 1; pass <= 3; ++pass)
    k_update<double, double><<<update_grid(g, pass, 0, UpdateBlocks<double>::value), b2, 0, s>>>(g, C0, C1, Fx, Fy, const_cast<double*>(dWx), dWx_out,
                                                              const_cast<double*>(dWy), dWy_out, bad, ctrl, pass);
  k_end<<<1, 1, 0, s>>>(ctrl);
  k_scatter_U<double><<<grid2(nx, ny, b2), b2, 0, s>>>(g, dU_out, C0, C1, ctrl, 0);
  e = cudaGetLastError();
  Ctrl hc;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { g_create_err = std::string("gks_step_noalloc: ") + cudaGetErrorString(e); return GKS_ECUDA; }
  if (dt_taken) *dt_taken = hc.skip ? 0.0 : hc.dt;
  if (hc.status != GKS_OK) {
    g_create_err = "gks_step_noalloc: the step produced a non-physical state; outputs are not valid";
    return (gks_status)hc.status;
  }
  if (hc.skip) { g_create_err = "gks_step_noalloc: dt = 0, no step taken; outputs are not valid"; return GKS_EINVAL; }
  return GKS_OK;
}
