// Batched form: many independent grids of uneven sizes (each with its own gamma,
// mu, Pr, boundary conditions, dt and time) advanced together by ONE persistent
// cooperative kernel per call, captured once in a CUDA graph and replayed.
//
// Inside the kernel every step runs its phases over flat work lists of
// 128-element tiles drawn from all grids (per-grid dt, reconstruction, face
// evolution of x- and y-faces, update + ghost images + CFL minimum, and -- only
// when some cell's update was not physical -- the passes of the positivity
// fallback), separated by a device-wide barrier.  The barrier is a
// counter with a generation word; every wait is bounded in time (globaltimer)
// and gives up with GKS_ETIMEOUT instead of hanging.  The per-element
// arithmetic is that of the single-grid kernels (gks_grid.cuh).
//
// gks_batch_autotune times the tile shape of the face phase and the number of
// resident blocks per SM on the batch itself and keeps the fastest.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/gks.h"
#include "gks_device.cuh"
#include "gks_grid.cuh"

using namespace gks;

namespace {

constexpr int kThreads = 128;  // one work tile = one block: 128 faces, or 2 x 128 cells
constexpr int kCellsPerThread = 2;  // cells per thread in a cell tile (both in flight at once)

struct GridOff {
  size_t u;     // padded cell arrays (4 * plane doubles: Cells<R>)
  size_t wx, wy;
  size_t rec;   // rec_count: reconstruction records with the ghost ring
  size_t fx, fy;
  size_t bad;   // nx * ny flags of the positivity fallback
};

struct Barrier {
  unsigned count;
  unsigned gen;
  int any_bad[2];            // some grid's update pass 1 / 2 left a cell non-physical this step
  int error;
  int skip_block;            // test hook: this block never arrives (-1: none)
  unsigned long long limit;  // wait limit in ns
};

template <class R, class TW>
struct Args {
  int G;
  const Geo* geo;
  const GridOff* off;
  const FaceConst<R>* fc;  // [G][2]
  Ctrl* ctrl;
  double* U[2];
  TW* Wx[2];
  TW* Wy[2];
  R* rec;
  R* Fx;
  R* Fy;
  unsigned char* bad;
  const int4* cell_items;   // (grid, x0, y0, -)
  const int4* face_items;   // (grid, x0, y0, axis)
  int n_cell, n_face;
  int cell_tw;              // cell tile width (height = 2 x 128 / width)
  int face_tw[2];           // face tile widths of x- and y-faces (heights = 128 / width)
  Barrier* bar;
  double cfl;
  unsigned long long* stamps;  // optional: %globaltimer at the end of each phase, kPhases per step (block 0)
};

// phases of one step, each ended by a device-wide barrier: open the step (dt per grid),
// reconstruction, face evolution, update passes 1, 2, 3 (2 and 3 only when needed)
constexpr int kPhases = 6;

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// device-wide barrier with a bounded wait; returns false once any block gave up
__device__ bool grid_barrier(Barrier* b) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    volatile int* verr = &b->error;
    const unsigned my = *vgen;
    __threadfence();
    if ((int)blockIdx.x != b->skip_block) {
      if (atomicAdd(&b->count, 1u) + 1 == gridDim.x) {
        b->count = 0;
        __threadfence();
        atomicAdd(&b->gen, 1u);
      }
    }
    const unsigned long long t0 = now_ns();
    while (*vgen == my && *verr == 0) {
      if (now_ns() - t0 > b->limit) {
        atomicCAS(&b->error, 0, (int)GKS_ETIMEOUT);
        break;
      }
      __nanosleep(200);
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)&b->error == 0;
}

// resident blocks per SM the FP32 batch kernel is compiled for: 3 (168 registers, 12 warps
// per SM; at 4 blocks and 128 registers the Navier-Stokes face routine inside the persistent
// loop spills ~360 bytes; the autotuner may run fewer)
#ifndef GKS_BATCH_MINB_F32
#define GKS_BATCH_MINB_F32 3
#endif
template <class R> struct BatchBlocks;
template <> struct BatchBlocks<double> { static constexpr int value = 1; };
template <> struct BatchBlocks<float> { static constexpr int value = GKS_BATCH_MINB_F32; };

// NSM = 1: every grid has mu > 0 (the Navier-Stokes face routine only); -1: the face
// routine decides per grid.  CHAR: the reconstruction in characteristic variables (an
// option of the whole batch); the kernel without it carries only the conservative one,
// whose registers are far fewer.
template <class R, class TW, int NSM, bool CHAR>
__global__ void __launch_bounds__(kThreads, BatchBlocks<R>::value) k_batch(Args<R, TW> a, int nsteps) {
  const int tid = threadIdx.x;
  auto stamp = [&](int s, int phase) {
    if (a.stamps && blockIdx.x == 0 && tid == 0) a.stamps[(size_t)s * kPhases + phase] = now_ns();
  };
  if (a.stamps && blockIdx.x == 0 && tid == 0) a.stamps[(size_t)nsteps * kPhases] = now_ns();  // start
  for (int s = 0; s < nsteps; ++s) {
    // dt of this step per grid (after ending the previous one)
    for (int g = blockIdx.x * kThreads + tid; g < a.G; g += gridDim.x * kThreads) {
      if (s > 0) ctrl_end(&a.ctrl[g]);
      ctrl_begin(&a.ctrl[g], a.cfl, INFINITY, INFINITY);
    }
    if (!grid_barrier(a.bar)) return;
    stamp(s, 0);
    // every block read the previous step's flags before the barrier above
    if (blockIdx.x == 0 && tid == 0) a.bar->any_bad[0] = a.bar->any_bad[1] = 0;

    // reconstruction (two cells per thread, kThreads / cell_tw rows apart)
    for (int it = blockIdx.x; it < a.n_cell; it += gridDim.x) {
      const int4 w = a.cell_items[it];
      const Ctrl* c = &a.ctrl[w.x];
      if (c->skip) continue;
      const Geo& g = a.geo[w.x];
      const int par = (int)(c->steps & 1);
      const GridOff& o = a.off[w.x];
      const R* U = (const R*)(a.U[par] + o.u);
#pragma unroll
      for (int r = 0; r < kCellsPerThread; ++r) {
        const int i = w.y + tid % a.cell_tw, j = w.z + tid / a.cell_tw + r * (kThreads / a.cell_tw);
        if (i < g.nx && j < g.ny)
          recon_cell<R, TW, CHAR>(g, U, a.Wx[par] + o.wx, a.Wy[par] + o.wy, a.rec + o.rec, i, j, GeoR<R>::dx(g),
                                  GeoR<R>::dy(g), GeoR<R>::weps(g), GeoR<R>::wC(g));
      }
    }
    if (!grid_barrier(a.bar)) return;
    stamp(s, 1);

    // face evolution
    for (int it = blockIdx.x; it < a.n_face; it += gridDim.x) {
      const int4 w = a.face_items[it];
      const Ctrl* c = &a.ctrl[w.x];
      if (c->skip) continue;
      const Geo& g = a.geo[w.x];
      const int tw = a.face_tw[w.w];
      const int i = w.y + tid % tw, j = w.z + tid / tw;
      const int par = (int)(c->steps & 1);
      const GridOff& o = a.off[w.x];
      const R* U = (const R*)(a.U[par] + o.u);
      const R dt = step_dt<R>(c);
      if (w.w == 0) {
        if (i <= g.nx && j < g.ny)
          flux_face<0, R, TW, NSM>(g, a.fc[2 * w.x], a.rec + o.rec, a.Wx[par ^ 1] + o.wx, a.Fx + o.fx, i, j, dt);
      } else {
        if (i < g.nx && j <= g.ny)
          flux_face<1, R, TW, NSM>(g, a.fc[2 * w.x + 1], a.rec + o.rec, a.Wy[par ^ 1] + o.wy, a.Fy + o.fy, i, j,
                                   dt);
      }
    }
    if (!grid_barrier(a.bar)) return;
    stamp(s, 2);

    // update and the CFL minimum of the new state (update_cell): pass 1; pass 2
    // for grids where pass 1 left a cell non-physical; pass 3 for grids where
    // pass 2 still did.  The global flags let every block skip an unneeded pass
    // together.
    for (int pass = 1; pass <= 3; ++pass) {
      if (pass > 1 && *(volatile int*)&a.bar->any_bad[pass - 2] == 0) {
        for (int q = pass; q <= 3; ++q) stamp(s, 2 + q);  // the skipped passes take no time
        break;
      }
      for (int it = blockIdx.x; it < a.n_cell; it += gridDim.x) {
        const int4 w = a.cell_items[it];
        Ctrl* c = &a.ctrl[w.x];
        if (c->skip || (pass == 2 && !c->bad_found[0]) || (pass == 3 && !c->bad_found[1])) continue;  // per block
        const Geo& g = a.geo[w.x];
        const int par = (int)(c->steps & 1);
        const GridOff& o = a.off[w.x];
        R inv = R(0);
#pragma unroll
        for (int r = 0; r < kCellsPerThread; ++r) {
          const int i = w.y + tid % a.cell_tw, j = w.z + tid / a.cell_tw + r * (kThreads / a.cell_tw);
          if (i < g.nx && j < g.ny) {
            bool bad;
            const R iv = update_cell<R, TW>(g, Cells<R>{(R*)(a.U[par] + o.u)}, Cells<R>{(R*)(a.U[par ^ 1] + o.u)},
                                            a.Fx + o.fx, a.Fy + o.fy, a.Wx[par ^ 1] + o.wx, a.Wy[par ^ 1] + o.wy,
                                            a.bad + o.bad, pass, step_dt<R>(c), i, j, bad);
            inv = fmax(inv, iv);
            if (pass == 1) {
              a.bad[o.bad + (size_t)j * g.nx + i] = bad ? 1 : 0;
              if (bad) {
                atomicOr(&c->bad_found[0], 1);
                atomicOr(&a.bar->any_bad[0], 1);
              }
            } else if (pass == 2) {
              if (bad) {
                atomicOr(&c->bad_found[1], 1);
                atomicOr(&a.bar->any_bad[1], 1);
              }
            } else if (bad && atomicCAS(&c->status, GKS_OK, GKS_ENONPHYSICAL) == GKS_OK) {
              c->fail_step = c->steps;
            }
          }
        }
        // per warp: a block barrier per tile would hold every warp of the block until the
        // slowest one's loads return
        warp_bound_to<R>(inv, &c->dtb[pass - 1]);
      }
      if (!grid_barrier(a.bar)) return;
      stamp(s, 2 + pass);
    }
  }
  for (int g = blockIdx.x * kThreads + tid; g < a.G; g += gridDim.x * kThreads)
    if (nsteps > 0) ctrl_end(&a.ctrl[g]);
}

// ---- per-grid state transfer ----
template <class R>
__global__ void kb_scatter(Geo g, const double* src, Cells<R> U, int to_dev) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  for (int v = 0; v < 4; ++v) {
    const size_t o = ((size_t)v * g.ny + j) * g.nx + i;
    if (to_dev) U.set(g, v, i, j, src[o]);
    else const_cast<double*>(src)[o] = U.get(g, v, i, j);
  }
}

template <class R>
__global__ void kb_ghost(Geo g, Cells<R> U) {
  ghost_at<R>(g, U, blockIdx.x * blockDim.x + threadIdx.x);
}

template <class TW>
__global__ void kb_copyW(const double* src, TW* W, size_t n, int to_dev) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (to_dev) W[k] = (TW)src[k];
  else const_cast<double*>(src)[k] = (double)W[k];
}

template <class R>
__global__ void kb_dtbound(Geo g, Cells<R> U, Ctrl* c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
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

dim3 grid2(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

}  // namespace

struct gks_batch {
  int G;
  int prec;
  int device, sms;
  cudaStream_t stream;
  bool own_stream;
  std::vector<Geo> geo;
  std::vector<GridOff> off;
  size_t n_u, n_wx, n_wy, n_coef, n_fx, n_fy;
  long long cells;
  // device
  Geo* d_geo;
  GridOff* d_off;
  void* d_fc;
  Ctrl* d_ctrl;
  double* U[2];  // per grid 4 * plane doubles at off.u (Cells<R>)
  void* Wx[2];
  void* Wy[2];
  void* rec;
  void* Fx;
  void* Fy;
  unsigned char* bad;
  int4* d_cell;
  int4* d_face;
  int n_cell, n_face;
  Barrier* d_bar;
  Ctrl* h_ctrl;  // pinned mirror of all control blocks
  Barrier* h_bar;
  double* staging;
  size_t staging_n;
  // launch configuration
  int face_tw[2], cell_tw, blocks_per_sm, max_blocks_per_sm;
  bool all_ns;  // every grid has mu > 0: the kernel with the Navier-Stokes face routine only
  bool characteristic;  // reconstruction in characteristic variables (batch-wide option)
  double timeout_s;
  int skip_block;
  cudaGraphExec_t graph;
  int graph_steps;
  double graph_cfl;
  bool graph_ok;
  std::string err;
};

namespace {

gks_status bfail(gks_batch* b, gks_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

#define BCK(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return bfail(b, GKS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

size_t wsize(const gks_batch* b) { return b->prec == GKS_FP64 ? 8 : 4; }

gks_status build_items(gks_batch* b) {
  // faces: every grid's x-face tiles first, then the y-face tiles, so that an SM runs one
  // face body at a time (except around the switch)
  std::vector<int4> cell, face;
  const int ch = kCellsPerThread * kThreads / b->cell_tw;
  const int fwx = b->face_tw[0], fhx = kThreads / fwx, fwy = b->face_tw[1], fhy = kThreads / fwy;
  for (int g = 0; g < b->G; ++g) {
    const Geo& G = b->geo[g];
    for (int y = 0; y < G.ny; y += ch)
      for (int x = 0; x < G.nx; x += b->cell_tw) cell.push_back(make_int4(g, x, y, 0));
    for (int y = 0; y < G.ny; y += fhx)
      for (int x = 0; x < G.nx + 1; x += fwx) face.push_back(make_int4(g, x, y, 0));
  }
  for (int g = 0; g < b->G; ++g) {
    const Geo& G = b->geo[g];
    for (int y = 0; y < G.ny + 1; y += fhy)
      for (int x = 0; x < G.nx; x += fwy) face.push_back(make_int4(g, x, y, 1));
  }
  cudaFree(b->d_cell);
  cudaFree(b->d_face);
  b->d_cell = b->d_face = nullptr;
  BCK(cudaMalloc(&b->d_cell, cell.size() * sizeof(int4)));
  BCK(cudaMalloc(&b->d_face, face.size() * sizeof(int4)));
  BCK(cudaMemcpy(b->d_cell, cell.data(), cell.size() * sizeof(int4), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->d_face, face.data(), face.size() * sizeof(int4), cudaMemcpyHostToDevice));
  b->n_cell = (int)cell.size();
  b->n_face = (int)face.size();
  return GKS_OK;
}

template <class R, class TW>
Args<R, TW> make_args(gks_batch* b, double cfl) {
  Args<R, TW> a;
  a.G = b->G;
  a.geo = b->d_geo;
  a.off = b->d_off;
  a.fc = (const FaceConst<R>*)b->d_fc;
  a.ctrl = b->d_ctrl;
  for (int k = 0; k < 2; ++k) {
    a.U[k] = b->U[k];
    a.Wx[k] = (TW*)b->Wx[k];
    a.Wy[k] = (TW*)b->Wy[k];
  }
  a.rec = (R*)b->rec;
  a.Fx = (R*)b->Fx;
  a.Fy = (R*)b->Fy;
  a.bad = b->bad;
  a.cell_items = b->d_cell;
  a.face_items = b->d_face;
  a.n_cell = b->n_cell;
  a.n_face = b->n_face;
  a.cell_tw = b->cell_tw;
  a.face_tw[0] = b->face_tw[0];
  a.face_tw[1] = b->face_tw[1];
  a.bar = b->d_bar;
  a.cfl = cfl;
  a.stamps = nullptr;
  return a;
}

template <class R, class TW>
auto batch_kernel(const gks_batch* b) -> decltype(&k_batch<R, TW, 1, false>) {
  if (b->characteristic) return b->all_ns ? &k_batch<R, TW, 1, true> : &k_batch<R, TW, -1, true>;
  return b->all_ns ? &k_batch<R, TW, 1, false> : &k_batch<R, TW, -1, false>;
}

template <class R, class TW>
gks_status launch(gks_batch* b, int nsteps, double cfl, unsigned long long* stamps = nullptr) {
  Args<R, TW> a = make_args<R, TW>(b, cfl);
  a.stamps = stamps;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(b->sms * b->blocks_per_sm));
  cfg.blockDim = dim3(kThreads);
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BCK(cudaLaunchKernelEx(&cfg, batch_kernel<R, TW>(b), a, nsteps));
  return GKS_OK;
}

gks_status launch_any(gks_batch* b, int nsteps, double cfl, unsigned long long* stamps = nullptr) {
  return b->prec == GKS_FP64 ? launch<double, double>(b, nsteps, cfl, stamps)
                             : launch<float, float>(b, nsteps, cfl, stamps);
}

gks_status reset_barrier(gks_batch* b) {
  b->h_bar->count = 0;
  b->h_bar->gen = 0;
  b->h_bar->any_bad[0] = b->h_bar->any_bad[1] = 0;
  b->h_bar->error = 0;
  b->h_bar->skip_block = b->skip_block;
  b->h_bar->limit = (unsigned long long)(b->timeout_s * 1e9);
  BCK(cudaMemcpyAsync(b->d_bar, b->h_bar, sizeof(Barrier), cudaMemcpyHostToDevice, b->stream));
  return GKS_OK;
}

void drop_graph(gks_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

int occupancy(gks_batch* b) {
  int n = 0;
  if (b->prec == GKS_FP64)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<double, double>(b), kThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<float, float>(b), kThreads, 0);
  return n;
}

}  // namespace

extern "C" {

gks_status gks_batch_create(int n, const gks_grid_desc* grids, const gks_options* opt, void* cuda_stream,
                            gks_batch** out) {
  if (!out || n < 1 || !grids) return GKS_EINVAL;
  *out = nullptr;
  gks_options o;
  gks_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != GKS_FP64 && o.precision != GKS_FP32_BULK) return GKS_EINVAL;
  gks_batch* b = new gks_batch();
  b->G = n;
  b->prec = o.precision;
  b->cell_tw = 32;
  // x-faces: nx + 1 per row, so narrow tall tiles waste least of the extra column;
  // y-faces: ny + 1 rows, wide short tiles (the autotuner may pick others)
  b->face_tw[0] = 8;
  b->face_tw[1] = 32;
  b->timeout_s = 2.0;
  b->skip_block = -1;
  b->all_ns = true;
  b->characteristic = o.characteristic != 0;
  size_t nu = 0, nwx = 0, nwy = 0, nc = 0, nfx = 0, nfy = 0, nbad = 0;
  b->cells = 0;
  for (int g = 0; g < n; ++g) {
    const gks_grid_desc& d = grids[g];
    if (d.nx < 2 || d.ny < 2 || !(d.Lx > 0) || !(d.Ly > 0) || !(d.gamma > 1.0) || !(d.Pr > 0) || !(d.mu >= 0)) {
      delete b;
      return GKS_EINVAL;
    }
    Geo G;
    memset(&G, 0, sizeof(G));
    G.nx = d.nx; G.ny = d.ny;
    G.dx = d.Lx / d.nx; G.dy = d.Ly / d.ny;
    G.gamma = d.gamma; G.mu = d.mu; G.Pr = d.Pr;
    if (!(d.mu > 0)) b->all_ns = false;
    G.weno_eps = o.weno_eps; G.weno_C = o.weno_C; G.tau_eps = o.tau_eps; G.tau_C = o.tau_C;
    G.viscous_dt = o.viscous_dt;
    G.characteristic = o.characteristic;
    for (int k = 0; k < 4; ++k) {
      G.bc.kind[k] = d.bc[k].kind;
      G.bc.uw[k] = d.bc[k].u_wall;
      G.bc.vw[k] = d.bc[k].v_wall;
      G.bc.Tw[k] = d.bc[k].T_wall;
      if (d.bc[k].kind < 0 || d.bc[k].kind > 4) { delete b; return GKS_EINVAL; }
    }
    geo_finish(G);
    if ((G.bc.kind[0] == GKS_BC_PERIODIC) != (G.bc.kind[1] == GKS_BC_PERIODIC) ||
        (G.bc.kind[2] == GKS_BC_PERIODIC) != (G.bc.kind[3] == GKS_BC_PERIODIC)) {
      delete b;
      return GKS_EINVAL;
    }
    GridOff of;
    of.u = nu; nu += 4 * G.plane;
    nu = (nu + 31) & ~(size_t)31;
    of.wx = nwx; nwx += (size_t)8 * d.ny * (d.nx + 1);
    of.wy = nwy; nwy += (size_t)8 * (d.ny + 1) * d.nx;
    of.rec = nc; nc += rec_count(G);
    of.fx = nfx; nfx += (size_t)4 * d.ny * (d.nx + 1);
    of.fy = nfy; nfy += (size_t)4 * (d.ny + 1) * d.nx;
    of.bad = nbad; nbad += (size_t)d.nx * d.ny;
    b->geo.push_back(G);
    b->off.push_back(of);
    b->cells += (long long)d.nx * d.ny;
  }
  b->n_u = nu; b->n_wx = nwx; b->n_wy = nwy; b->n_coef = nc; b->n_fx = nfx; b->n_fy = nfy;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) {
    if (cuda_stream) { b->stream = (cudaStream_t)cuda_stream; b->own_stream = false; }
    else { e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking); b->own_stream = true; }
  }
  const size_t ws = wsize(b);
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  alloc((void**)&b->d_geo, sizeof(Geo) * n);
  alloc((void**)&b->d_off, sizeof(GridOff) * n);
  alloc(&b->d_fc, (b->prec == GKS_FP64 ? sizeof(FaceConst<double>) : sizeof(FaceConst<float>)) * 2 * n);
  alloc((void**)&b->d_ctrl, sizeof(Ctrl) * n);
  for (int k = 0; k < 2; ++k) {
    alloc((void**)&b->U[k], nu * sizeof(double));
    alloc(&b->Wx[k], nwx * ws);
    alloc(&b->Wy[k], nwy * ws);
  }
  alloc(&b->rec, nc * ws);
  alloc(&b->Fx, nfx * ws);
  alloc(&b->Fy, nfy * ws);
  alloc((void**)&b->bad, nbad);
  alloc((void**)&b->d_bar, sizeof(Barrier));
  size_t st = 0;
  for (int g = 0; g < n; ++g) {
    const Geo& G = b->geo[g];
    st = std::max(st, std::max((size_t)4 * G.nx * G.ny, std::max((size_t)8 * G.ny * (G.nx + 1), (size_t)8 * (G.ny + 1) * G.nx)));
  }
  b->staging_n = st;
  alloc((void**)&b->staging, st * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_ctrl, sizeof(Ctrl) * n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_bar, sizeof(Barrier));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_geo, b->geo.data(), sizeof(Geo) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_off, b->off.data(), sizeof(GridOff) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (b->prec == GKS_FP64) {
      std::vector<FaceConst<double>> fc;
      for (int g = 0; g < n; ++g) { fc.push_back(grid_face_const<double>(b->geo[g], 0)); fc.push_back(grid_face_const<double>(b->geo[g], 1)); }
      e = cudaMemcpy(b->d_fc, fc.data(), sizeof(FaceConst<double>) * 2 * n, cudaMemcpyHostToDevice);
    } else {
      std::vector<FaceConst<float>> fc;
      for (int g = 0; g < n; ++g) { fc.push_back(grid_face_const<float>(b->geo[g], 0)); fc.push_back(grid_face_const<float>(b->geo[g], 1)); }
      e = cudaMemcpy(b->d_fc, fc.data(), sizeof(FaceConst<float>) * 2 * n, cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess) {
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaMemset(b->U[k], 0, nu * sizeof(double));
    }
    // control blocks: t = 0, no bound yet
    memset(b->h_ctrl, 0, sizeof(Ctrl) * n);
    const double inf = INFINITY;
    uint64_t bits;
    memcpy(&bits, &inf, 8);
    for (int g = 0; g < n; ++g) b->h_ctrl[g].bound = b->h_ctrl[g].dtb[0] = b->h_ctrl[g].dtb[1] = b->h_ctrl[g].dtb[2] = bits;
    if (e == cudaSuccess) e = cudaMemcpy(b->d_ctrl, b->h_ctrl, sizeof(Ctrl) * n, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    const gks_status s = e == cudaErrorMemoryAllocation ? GKS_ENOMEM : GKS_ECUDA;
    gks_batch_destroy(b);
    return s;
  }
  b->max_blocks_per_sm = occupancy(b);
  b->blocks_per_sm = b->max_blocks_per_sm;
  if (b->max_blocks_per_sm < 1 || build_items(b) != GKS_OK) {
    gks_batch_destroy(b);
    return GKS_ECUDA;
  }
  *out = b;
  return GKS_OK;
}

gks_status gks_batch_set_state(gks_batch* b, int g, const double* U, const double* Wx, const double* Wy, double t) {
  if (!b || g < 0 || g >= b->G || !U || !Wx || !Wy) return bfail(b, GKS_EINVAL, "gks_batch_set_state: bad argument");
  BCK(cudaSetDevice(b->device));
  const Geo& G = b->geo[g];
  const GridOff& o = b->off[g];
  Ctrl& c = b->h_ctrl[g];
  BCK(cudaMemcpyAsync(&c, b->d_ctrl + g, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  const int par = (int)(c.steps & 1);
  const dim3 b2(32, 8);
  BCK(cudaMemcpyAsync(b->staging, U, (size_t)4 * G.nx * G.ny * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  if (b->prec == GKS_FP64) {
    const Cells<double> C{b->U[par] + o.u};
    kb_scatter<double><<<grid2(G.nx, G.ny, b2), b2, 0, b->stream>>>(G, b->staging, C, 1);
    kb_ghost<double><<<(perimeter(G) + 127) / 128, 128, 0, b->stream>>>(G, C);
  } else {
    const Cells<float> C{(float*)(b->U[par] + o.u)};
    kb_scatter<float><<<grid2(G.nx, G.ny, b2), b2, 0, b->stream>>>(G, b->staging, C, 1);
    kb_ghost<float><<<(perimeter(G) + 127) / 128, 128, 0, b->stream>>>(G, C);
  }
  const size_t nx = (size_t)8 * G.ny * (G.nx + 1), ny = (size_t)8 * (G.ny + 1) * G.nx;
  BCK(cudaMemcpyAsync(b->staging, Wx, nx * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  if (b->prec == GKS_FP64) kb_copyW<double><<<(unsigned)((nx + 255) / 256), 256, 0, b->stream>>>(b->staging, (double*)b->Wx[par] + o.wx, nx, 1);
  else kb_copyW<float><<<(unsigned)((nx + 255) / 256), 256, 0, b->stream>>>(b->staging, (float*)b->Wx[par] + o.wx, nx, 1);
  BCK(cudaMemcpyAsync(b->staging, Wy, ny * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  if (b->prec == GKS_FP64) kb_copyW<double><<<(unsigned)((ny + 255) / 256), 256, 0, b->stream>>>(b->staging, (double*)b->Wy[par] + o.wy, ny, 1);
  else kb_copyW<float><<<(unsigned)((ny + 255) / 256), 256, 0, b->stream>>>(b->staging, (float*)b->Wy[par] + o.wy, ny, 1);
  // control block: time t, status cleared, bound of the new state
  c.t = t;
  c.status = GKS_OK;
  c.skip = 0;
  const double inf = INFINITY;
  memcpy(&c.bound, &inf, 8);
  BCK(cudaMemcpyAsync(b->d_ctrl + g, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, b->stream));
  if (b->prec == GKS_FP64)
    kb_dtbound<double><<<grid2(G.nx, G.ny, b2), b2, 0, b->stream>>>(G, Cells<double>{b->U[par] + o.u}, b->d_ctrl + g);
  else
    kb_dtbound<float><<<grid2(G.nx, G.ny, b2), b2, 0, b->stream>>>(G, Cells<float>{(float*)(b->U[par] + o.u)},
                                                                   b->d_ctrl + g);
  BCK(cudaGetLastError());
  BCK(cudaMemcpyAsync(&c, b->d_ctrl + g, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (c.status != GKS_OK) return bfail(b, GKS_ENONPHYSICAL, "gks_batch_set_state: state has rho <= 0 or p <= 0");
  return GKS_OK;
}

gks_status gks_batch_get_state(gks_batch* b, int g, double* U, double* Wx, double* Wy, double* t, long long* steps) {
  if (!b || g < 0 || g >= b->G) return bfail(b, GKS_EINVAL, "gks_batch_get_state: bad argument");
  BCK(cudaSetDevice(b->device));
  const Geo& G = b->geo[g];
  const GridOff& o = b->off[g];
  Ctrl& c = b->h_ctrl[g];
  BCK(cudaMemcpyAsync(&c, b->d_ctrl + g, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  const int par = (int)(c.steps & 1);
  const dim3 b2(32, 8);
  if (U) {
    if (b->prec == GKS_FP64)
      kb_scatter<double><<<grid2(G.nx, G.ny, b2), b2, 0, b->stream>>>(G, b->staging, Cells<double>{b->U[par] + o.u}, 0);
    else
      kb_scatter<float><<<grid2(G.nx, G.ny, b2), b2, 0, b->stream>>>(G, b->staging,
                                                                     Cells<float>{(float*)(b->U[par] + o.u)}, 0);
    BCK(cudaMemcpyAsync(U, b->staging, (size_t)4 * G.nx * G.ny * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  }
  const size_t nx = (size_t)8 * G.ny * (G.nx + 1), ny = (size_t)8 * (G.ny + 1) * G.nx;
  if (Wx) {
    if (b->prec == GKS_FP64) kb_copyW<double><<<(unsigned)((nx + 255) / 256), 256, 0, b->stream>>>(b->staging, (double*)b->Wx[par] + o.wx, nx, 0);
    else kb_copyW<float><<<(unsigned)((nx + 255) / 256), 256, 0, b->stream>>>(b->staging, (float*)b->Wx[par] + o.wx, nx, 0);
    BCK(cudaMemcpyAsync(Wx, b->staging, nx * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  }
  if (Wy) {
    if (b->prec == GKS_FP64) kb_copyW<double><<<(unsigned)((ny + 255) / 256), 256, 0, b->stream>>>(b->staging, (double*)b->Wy[par] + o.wy, ny, 0);
    else kb_copyW<float><<<(unsigned)((ny + 255) / 256), 256, 0, b->stream>>>(b->staging, (float*)b->Wy[par] + o.wy, ny, 0);
    BCK(cudaMemcpyAsync(Wy, b->staging, ny * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  }
  BCK(cudaGetLastError());
  BCK(cudaStreamSynchronize(b->stream));
  if (t) *t = c.t;
  if (steps) *steps = c.steps;
  if (c.status != GKS_OK) return bfail(b, (gks_status)c.status, "grid state is the last good one");
  return GKS_OK;
}

gks_status gks_batch_step(gks_batch* b, int nsteps, double CFL) {
  if (!b || nsteps < 0 || !(CFL > 0)) return bfail(b, GKS_EINVAL, "gks_batch_step: nsteps >= 0 and CFL > 0 required");
  if (nsteps == 0) return GKS_OK;
  BCK(cudaSetDevice(b->device));
  gks_status st = reset_barrier(b);
  if (st != GKS_OK) return st;
  if (!b->graph || b->graph_steps != nsteps || b->graph_cfl != CFL) {
    drop_graph(b);
    // capture the persistent launch once; replay it on later calls
    cudaGraph_t graph = nullptr;
    b->graph_ok = false;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const gks_status ls = launch_any(b, nsteps, CFL);
      const cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
      if (ls == GKS_OK && ee == cudaSuccess && cudaGraphInstantiate(&b->graph, graph, 0) == cudaSuccess)
        b->graph_ok = true;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
    if (!b->graph_ok) {
      drop_graph(b);
      return launch_any(b, nsteps, CFL);  // capture unsupported: plain cooperative launch
    }
    b->graph_steps = nsteps;
    b->graph_cfl = CFL;
  }
  BCK(cudaGraphLaunch(b->graph, b->stream));
  return GKS_OK;
}

gks_status gks_batch_sync(gks_batch* b, long long* steps_min, long long* steps_max) {
  if (!b) return GKS_EINVAL;
  BCK(cudaSetDevice(b->device));
  BCK(cudaMemcpyAsync(b->h_ctrl, b->d_ctrl, sizeof(Ctrl) * b->G, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaMemcpyAsync(b->h_bar, b->d_bar, sizeof(Barrier), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  long long lo = 0, hi = 0;
  int bad = 0;
  for (int g = 0; g < b->G; ++g) {
    const long long s = b->h_ctrl[g].steps;
    if (g == 0 || s < lo) lo = s;
    if (g == 0 || s > hi) hi = s;
    if (b->h_ctrl[g].status != GKS_OK) bad = b->h_ctrl[g].status;
  }
  if (steps_min) *steps_min = lo;
  if (steps_max) *steps_max = hi;
  if (b->h_bar->error) return bfail(b, (gks_status)b->h_bar->error, "a device barrier wait timed out; the step sequence was abandoned");
  if (bad) return bfail(b, (gks_status)bad, "a grid produced a non-physical state; that grid stopped");
  return GKS_OK;
}

gks_status gks_batch_grid_info(gks_batch* b, int g, double* t, long long* steps, int* status) {
  if (!b || g < 0 || g >= b->G) return GKS_EINVAL;
  BCK(cudaMemcpyAsync(&b->h_ctrl[g], b->d_ctrl + g, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (t) *t = b->h_ctrl[g].t;
  if (steps) *steps = b->h_ctrl[g].steps;
  if (status) *status = b->h_ctrl[g].status;
  return GKS_OK;
}

gks_status gks_batch_configure_tiles(gks_batch* b, int width_x, int width_y, int blocks_per_sm) {
  if (!b) return GKS_EINVAL;
  auto ok = [](int w) { return w == 4 || w == 8 || w == 16 || w == 32 || w == 64 || w == 128; };
  if (!ok(width_x) || !ok(width_y)) return bfail(b, GKS_EINVAL, "face tile widths must be 4, 8, 16, 32, 64 or 128");
  if (blocks_per_sm < 1 || blocks_per_sm > b->max_blocks_per_sm)
    return bfail(b, GKS_EINVAL, "blocks_per_sm must lie in [1, " + std::to_string(b->max_blocks_per_sm) + "]");
  BCK(cudaStreamSynchronize(b->stream));
  drop_graph(b);
  b->blocks_per_sm = blocks_per_sm;
  if (width_x != b->face_tw[0] || width_y != b->face_tw[1]) {
    b->face_tw[0] = width_x;
    b->face_tw[1] = width_y;
    return build_items(b);
  }
  return GKS_OK;
}

gks_status gks_batch_configure(gks_batch* b, int face_tile_width, int blocks_per_sm) {
  return gks_batch_configure_tiles(b, face_tile_width, face_tile_width, blocks_per_sm);
}

gks_status gks_batch_autotune(gks_batch* b, double CFL, int trial_steps, int* face_tile_width_x,
                              int* face_tile_width_y, int* blocks_per_sm, float* best_ms) {
  if (!b || !(CFL > 0) || trial_steps < 1) return bfail(b, GKS_EINVAL, "gks_batch_autotune: bad argument");
  BCK(cudaSetDevice(b->device));
  // the trials advance the batch; save and restore the state and control blocks
  const size_t ws = wsize(b);
  void* save[4] = {nullptr};
  const size_t sz[4] = {b->n_u * 8, b->n_wx * ws, b->n_wy * ws, sizeof(Ctrl) * (size_t)b->G};
  BCK(cudaStreamSynchronize(b->stream));
  BCK(cudaMemcpy(b->h_ctrl, b->d_ctrl, sizeof(Ctrl) * b->G, cudaMemcpyDeviceToHost));
  for (int k = 0; k < 4; ++k) BCK(cudaMalloc(&save[k], 2 * sz[k]));
  auto snapshot = [&](bool restore) -> gks_status {
    for (int par = 0; par < 2; ++par) {
      void* live[3] = {b->U[par], b->Wx[par], b->Wy[par]};
      for (int k = 0; k < 3; ++k) {
        if (!save[k]) continue;
        char* s = (char*)save[k] + par * sz[k];
        if (restore) BCK(cudaMemcpyAsync(live[k], s, sz[k], cudaMemcpyDeviceToDevice, b->stream));
        else BCK(cudaMemcpyAsync(s, live[k], sz[k], cudaMemcpyDeviceToDevice, b->stream));
      }
    }
    if (restore) BCK(cudaMemcpyAsync(b->d_ctrl, save[3], sz[3], cudaMemcpyDeviceToDevice, b->stream));
    else BCK(cudaMemcpyAsync(save[3], b->d_ctrl, sz[3], cudaMemcpyDeviceToDevice, b->stream));
    return GKS_OK;
  };
  gks_status st = snapshot(false);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // one timed trial of a configuration (state restored afterwards); +inf if it failed
  auto trial = [&](int wx, int wy, int bps) -> float {
    if (st != GKS_OK) return 1e30f;
    st = gks_batch_configure_tiles(b, wx, wy, bps);
    if (st == GKS_OK) st = reset_barrier(b);
    if (st == GKS_OK) st = launch_any(b, 1, CFL);  // warm-up
    if (st == GKS_OK) st = reset_barrier(b);
    cudaEventRecord(e0, b->stream);
    if (st == GKS_OK) st = launch_any(b, trial_steps, CFL);
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = bfail(b, GKS_ECUDA, "autotune trial failed");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (cudaMemcpy(b->h_bar, b->d_bar, sizeof(Barrier), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = bfail(b, GKS_ECUDA, "autotune trial failed");
    const bool good = st == GKS_OK && b->h_bar->error == 0;
    if (st == GKS_OK) st = snapshot(true);
    return good ? ms : 1e30f;
  };
  // coordinate search: the x-face tile width, then the y-face one, then the resident blocks
  int bx = b->face_tw[0], by = b->face_tw[1], bb = b->max_blocks_per_sm;
  float best = 1e30f;
  for (int w : {4, 8, 16, 32}) {
    const float ms = trial(w, by, bb);
    if (ms < best) { best = ms; bx = w; }
  }
  for (int w : {16, 32, 64, 128}) {
    if (w == by) continue;
    const float ms = trial(bx, w, bb);
    if (ms < best) { best = ms; by = w; }
  }
  for (int bps = 1; bps < b->max_blocks_per_sm; ++bps) {
    const float ms = trial(bx, by, bps);
    if (ms < best) { best = ms; bb = bps; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == GKS_OK) st = gks_batch_configure_tiles(b, bx, by, bb);
  cudaStreamSynchronize(b->stream);
  for (int k = 0; k < 4; ++k) cudaFree(save[k]);
  if (st != GKS_OK) return st;
  if (face_tile_width_x) *face_tile_width_x = bx;
  if (face_tile_width_y) *face_tile_width_y = by;
  if (blocks_per_sm) *blocks_per_sm = bb;
  if (best_ms) *best_ms = best / trial_steps;
  return GKS_OK;
}

gks_status gks_batch_profile(gks_batch* b, int nsteps, double CFL, double* ms) {
  if (!b || nsteps < 1 || !(CFL > 0) || !ms) return bfail(b, GKS_EINVAL, "gks_batch_profile: bad argument");
  BCK(cudaSetDevice(b->device));
  unsigned long long* d = nullptr;
  const size_t n = (size_t)nsteps * kPhases + 1;
  BCK(cudaMalloc(&d, n * sizeof(unsigned long long)));
  gks_status st = reset_barrier(b);
  if (st == GKS_OK) st = launch_any(b, nsteps, CFL, d);
  std::vector<unsigned long long> h(n);
  if (st == GKS_OK && cudaMemcpyAsync(h.data(), d, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                      b->stream) != cudaSuccess)
    st = bfail(b, GKS_ECUDA, "gks_batch_profile: copy");
  if (st == GKS_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) st = bfail(b, GKS_ECUDA, "gks_batch_profile");
  cudaFree(d);
  if (st != GKS_OK) return st;
  for (int p = 0; p < kPhases; ++p) ms[p] = 0.0;
  unsigned long long prev = h[(size_t)nsteps * kPhases];
  for (int s = 0; s < nsteps; ++s)
    for (int p = 0; p < kPhases; ++p) {
      const unsigned long long t = h[(size_t)s * kPhases + p];
      ms[p] += (double)(t - prev) * 1e-6 / nsteps;
      prev = t;
    }
  return GKS_OK;
}

gks_status gks_batch_set_wait_limit(gks_batch* b, double seconds, int test_skip_block) {
  if (!b || !(seconds > 0)) return GKS_EINVAL;
  BCK(cudaStreamSynchronize(b->stream));
  drop_graph(b);
  b->timeout_s = seconds;
  b->skip_block = test_skip_block;
  return GKS_OK;
}

long long gks_batch_cells(const gks_batch* b) { return b ? b->cells : 0; }

int gks_batch_launches_per_call(const gks_batch* b) {
  (void)b;
  return 1;
}

void gks_batch_destroy(gks_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  cudaFree(b->d_geo);
  cudaFree(b->d_off);
  cudaFree(b->d_fc);
  cudaFree(b->d_ctrl);
  for (int k = 0; k < 2; ++k) {
    cudaFree(b->U[k]);
    cudaFree(b->Wx[k]);
    cudaFree(b->Wy[k]);
  }
  cudaFree(b->rec);
  cudaFree(b->Fx);
  cudaFree(b->Fy);
  cudaFree(b->bad);
  cudaFree(b->d_cell);
  cudaFree(b->d_face);
  cudaFree(b->d_bar);
  cudaFree(b->staging);
  if (b->h_ctrl) cudaFreeHost(b->h_ctrl);
  if (b->h_bar) cudaFreeHost(b->h_bar);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* gks_batch_last_error(const gks_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
