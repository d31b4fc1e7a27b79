// Grid-level device work of one time step, per element: the ghost ring, the
// reconstruction of one cell, the evolution at one face and the update of one
// cell.  The single-grid kernels (gks.cu) and the persistent batched kernel
// (gks_batch.cu) both call these, so both compute the same arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/gks.h"
#include "gks_device.cuh"

namespace gks {

// per-grid control block; every step's scalars stay on the device
struct Ctrl {
  unsigned long long bound;   // CFL bound (FP64 bits) of the current state
  unsigned long long dtb[3];  // running minima of the CFL bound of each update pass of the step
  double t;
  double dt;
  float dt_f;                 // dt rounded to FP32, for the FP32 kernels
  long long steps;
  int status;
  int skip;
  long long fail_step;
  int bad_found[2];           // update pass 1 / 2 left a cell non-physical
};

struct BCs {
  int kind[4];
  double uw[4], vw[4], Tw[4];
};

struct Geo {
  int nx, ny, pitch;  // pitch: row length of the padded cell arrays
  size_t plane;       // (ny+2) * pitch
  double dx, dy;
  double idx, idy;                  // 1/dx, 1/dy
  float idx_hi, idx_lo, idy_hi, idy_lo;  // the same as FP32 pairs hi + lo
  double visc;                      // viscous rate bound 2 mu max(4/3, gamma/Pr) / min(dx, dy)^2
  float gamma_f, gm1_f, K_f, visc_f;  // gamma, gamma - 1, K = (4 - 2 gamma) / (gamma - 1), visc in FP32
  float dx_f, dy_f, weno_eps_f, weno_C_f;
  float uwt_f[4], Tw_f[4];          // tangential wall velocity and wall temperature per side
  int visc_on;                      // viscous_dt and mu > 0
  double gamma, mu, Pr;
  double weno_eps, weno_C, tau_eps, tau_C;
  int viscous_dt;
  int characteristic;  // reconstruction in characteristic variables
  BCs bc;
};

__host__ __device__ __forceinline__ size_t ci(const Geo& g, int v, int i, int j) {
  return (size_t)v * g.plane + (size_t)(j + 1) * g.pitch + (i + 1);
}

// ---------------------------------------------------------------------------
// Reconstruction records.  Per cell, ghost ring included, the compute-type cell
// average and the coefficient vectors a2..a6 of Section 3.2, four variables each:
// 24 contiguous values (96 bytes in FP32, 192 in FP64), so that a face reads each
// of its two cells with 16-byte loads from one address instead of gathering 24
// values from separate planes.  Ghost records hold only the average (the images
// of the ghost ring), which the equilibrium polynomial of Section 3.3 reads.
//   [0..3] average, [4 + 4 (k - 2) + v] = a_k of variable v, k = 2..6
// ---------------------------------------------------------------------------
constexpr int kRec = 24;

__host__ __device__ __forceinline__ size_t rec_count(const Geo& g) { return (size_t)(g.nx + 2) * (g.ny + 2) * kRec; }
__host__ __device__ __forceinline__ size_t ri(const Geo& g, int i, int j) {
  return ((size_t)(j + 1) * (g.nx + 2) + (i + 1)) * kRec;
}

template <class R> struct RecIO;
template <> struct RecIO<float> {
  static __device__ __forceinline__ void load(const float* __restrict__ p, float r[kRec]) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < kRec / 4; ++k) {
      const float4 t = q[k];
      r[4 * k] = t.x; r[4 * k + 1] = t.y; r[4 * k + 2] = t.z; r[4 * k + 3] = t.w;
    }
  }
  static __device__ __forceinline__ void load_avg(const float* __restrict__ p, float r[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    r[0] = t.x; r[1] = t.y; r[2] = t.z; r[3] = t.w;
  }
  static __device__ __forceinline__ void store(float* p, const float r[kRec]) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int k = 0; k < kRec / 4; ++k) q[k] = make_float4(r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
  }
  static __device__ __forceinline__ void store_avg(float* p, const float r[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
  }
};
template <> struct RecIO<double> {
  static __device__ __forceinline__ void load(const double* __restrict__ p, double r[kRec]) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int k = 0; k < kRec / 2; ++k) {
      const double2 t = q[k];
      r[2 * k] = t.x; r[2 * k + 1] = t.y;
    }
  }
  static __device__ __forceinline__ void load_avg(const double* __restrict__ p, double r[4]) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = q[0], b = q[1];
    r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
  }
  static __device__ __forceinline__ void store(double* p, const double r[kRec]) {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int k = 0; k < kRec / 2; ++k) q[k] = make_double2(r[2 * k], r[2 * k + 1]);
  }
  static __device__ __forceinline__ void store_avg(double* p, const double r[4]) {
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = make_double2(r[0], r[1]);
    q[1] = make_double2(r[2], r[3]);
  }
};

// derived fields: sizes of the padded arrays, reciprocal cell sizes and FP32
// copies, from nx, ny, dx, dy, gamma, mu and Pr
inline void geo_finish(Geo& g) {
  g.pitch = ((g.nx + 2) + 1) & ~1;
  g.plane = (size_t)(g.ny + 2) * g.pitch;
  g.idx = 1.0 / g.dx;
  g.idy = 1.0 / g.dy;
  g.idx_hi = (float)g.idx;
  g.idx_lo = (float)(g.idx - (double)g.idx_hi);
  g.idy_hi = (float)g.idy;
  g.idy_lo = (float)(g.idy - (double)g.idy_hi);
  const double h = g.dx < g.dy ? g.dx : g.dy;
  const double r = g.gamma / g.Pr > 4.0 / 3.0 ? g.gamma / g.Pr : 4.0 / 3.0;
  g.visc = 2.0 * g.mu * r / (h * h);
  g.gamma_f = (float)g.gamma;
  g.gm1_f = (float)(g.gamma - 1.0);
  g.K_f = (float)((4.0 - 2.0 * g.gamma) / (g.gamma - 1.0));
  g.visc_f = (float)g.visc;
  g.dx_f = (float)g.dx;
  g.dy_f = (float)g.dy;
  g.weno_eps_f = (float)g.weno_eps;
  g.weno_C_f = (float)g.weno_C;
  for (int k = 0; k < 4; ++k) {
    g.uwt_f[k] = (float)(k < 2 ? g.bc.vw[k] : g.bc.uw[k]);
    g.Tw_f[k] = (float)g.bc.Tw[k];
  }
  g.visc_on = g.viscous_dt && g.mu > 0.0;
}

// Geo scalars in the compute type (the FP32 kernels do no FP64 arithmetic)
template <class R> struct GeoR;
template <> struct GeoR<double> {
  static __device__ __forceinline__ double gamma(const Geo& g) { return g.gamma; }
  static __device__ __forceinline__ double gm1(const Geo& g) { return g.gamma - 1.0; }
  static __device__ __forceinline__ double K(const Geo& g) { return (4.0 - 2.0 * g.gamma) / (g.gamma - 1.0); }
  static __device__ __forceinline__ double idx(const Geo& g) { return g.idx; }
  static __device__ __forceinline__ double idy(const Geo& g) { return g.idy; }
  static __device__ __forceinline__ double visc(const Geo& g) { return g.visc; }
  static __device__ __forceinline__ double dx(const Geo& g) { return g.dx; }
  static __device__ __forceinline__ double dy(const Geo& g) { return g.dy; }
  static __device__ __forceinline__ double weps(const Geo& g) { return g.weno_eps; }
  static __device__ __forceinline__ double wC(const Geo& g) { return g.weno_C; }
  // tangential wall velocity in the face frame: y-component on x-sides, x on y-sides
  static __device__ __forceinline__ double uwt(const Geo& g, int side) { return side < 2 ? g.bc.vw[side] : g.bc.uw[side]; }
  static __device__ __forceinline__ double Tw(const Geo& g, int side) { return g.bc.Tw[side]; }
};
template <> struct GeoR<float> {
  static __device__ __forceinline__ float gamma(const Geo& g) { return g.gamma_f; }
  static __device__ __forceinline__ float gm1(const Geo& g) { return g.gm1_f; }
  static __device__ __forceinline__ float K(const Geo& g) { return g.K_f; }
  static __device__ __forceinline__ float idx(const Geo& g) { return g.idx_hi; }
  static __device__ __forceinline__ float idy(const Geo& g) { return g.idy_hi; }
  static __device__ __forceinline__ float visc(const Geo& g) { return g.visc_f; }
  static __device__ __forceinline__ float dx(const Geo& g) { return g.dx_f; }
  static __device__ __forceinline__ float dy(const Geo& g) { return g.dy_f; }
  static __device__ __forceinline__ float weps(const Geo& g) { return g.weno_eps_f; }
  static __device__ __forceinline__ float wC(const Geo& g) { return g.weno_C_f; }
  static __device__ __forceinline__ float uwt(const Geo& g, int side) { return g.uwt_f[side]; }
  static __device__ __forceinline__ float Tw(const Geo& g, int side) { return g.Tw_f[side]; }
};

// dt of the step in the compute type
template <class R> __device__ __forceinline__ R step_dt(const Ctrl* c);
template <> __device__ __forceinline__ double step_dt<double>(const Ctrl* c) { return c->dt; }
template <> __device__ __forceinline__ float step_dt<float>(const Ctrl* c) { return c->dt_f; }

// ---------------------------------------------------------------------------
// Full-precision cell averages, the state the conservative update accumulates
// into (get / set in FP64; put stores a compute-type value).  One allocation of 4 * plane doubles per buffer either way:
//  * FP64 mode: four FP64 planes;
//  * FP32-bulk mode: each average is an unevaluated sum hi + lo of two FP32
//    numbers (a double-float pair), hi planes in the first half and lo planes
//    in the second.  hi is the FP32 rounding of hi + lo, so the hi planes are
//    the FP32 cell averages every FP32 kernel reads.
// view() is the compute-type array of the averages.
// ---------------------------------------------------------------------------
template <class R> struct Cells;
template <> struct Cells<double> {
  double* p;
  __device__ __forceinline__ double get(const Geo& g, int v, int i, int j) const { return p[ci(g, v, i, j)]; }
  __device__ __forceinline__ void set(const Geo& g, int v, int i, int j, double w) const { p[ci(g, v, i, j)] = w; }
  __device__ __forceinline__ void put(const Geo& g, int v, int i, int j, double w) const { p[ci(g, v, i, j)] = w; }
  __host__ __device__ __forceinline__ const double* view() const { return p; }
};
template <> struct Cells<float> {
  float* p;  // hi planes; lo planes at p + 4 * plane
  __device__ __forceinline__ double get(const Geo& g, int v, int i, int j) const {
    const size_t o = ci(g, v, i, j);
    return (double)p[o] + (double)p[o + 4 * g.plane];
  }
  __device__ __forceinline__ void set(const Geo& g, int v, int i, int j, double w) const {
    const size_t o = ci(g, v, i, j);
    const float hi = (float)w;
    p[o] = hi;
    p[o + 4 * g.plane] = (float)(w - (double)hi);
  }
  // a value known only in FP32 (ghost images): lo = 0
  __device__ __forceinline__ void put(const Geo& g, int v, int i, int j, float w) const {
    const size_t o = ci(g, v, i, j);
    p[o] = w;
    p[o + 4 * g.plane] = 0.0f;
  }
  __host__ __device__ __forceinline__ const float* view() const { return p; }
};

// (hi, lo) += f * (sh + sl) for a double-float pair: the product's rounding
// error (from the FMA) and the addition's (Knuth's TwoSum) are carried in lo,
// so the pair loses only the roundings of lo itself, ~2^-48 relative.  The
// _rn intrinsics keep the compiler from fusing the product into the sum.
__device__ __forceinline__ void df_add_product(float& hi, float& lo, float f, float sh, float sl) {
  const float p = __fmul_rn(f, sh);
  const float pe = __fadd_rn(__fmaf_rn(f, sh, -p), __fmul_rn(f, sl));
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

// Programmatic dependent launch: a step kernel launched with programmatic stream
// serialisation first waits for its predecessor grid to complete (and its writes
// to be visible), then lets its own successor be scheduled once every block of
// this grid is resident, so that launch latency overlaps execution.  Without the
// launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

// ---------------------------------------------------------------------------
// control: dt of the coming step from the running minimum, and its end
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ctrl_begin(Ctrl* c, double cfl, double dt_max, double t_end) {
  double dt = fmin(cfl * bitsd(c->bound), dt_max);
  dt = fmin(dt, t_end - c->t);
  c->dt = dt;
  c->dt_f = (float)dt;
  c->skip = (c->status != GKS_OK || !(dt > 0.0)) ? 1 : 0;
  c->dtb[0] = c->dtb[1] = c->dtb[2] = dbits(INFINITY);
  c->bad_found[0] = c->bad_found[1] = 0;
}

// the update pass whose state the step keeps: 1, or 2 / 3 after the fallbacks
__device__ __forceinline__ int last_pass(const Ctrl* c) { return c->bad_found[1] ? 3 : (c->bad_found[0] ? 2 : 1); }

__device__ __forceinline__ void ctrl_end(Ctrl* c) {
  if (c->skip || c->status != GKS_OK) return;
  c->bound = c->dtb[last_pass(c) - 1];
  c->t += c->dt;
  c->steps += 1;
}

// ---------------------------------------------------------------------------
// boundary images of cell averages (ghost ring)
// ---------------------------------------------------------------------------
// in the compute type R: the FP32 kernels read only the FP32 (hi) averages
template <class R>
__device__ __forceinline__ void bc_value(int kind, R gamma, R uwt, R Tw, int axis, const R in[4], R out[4]) {
  if (kind == GKS_BC_PERIODIC || kind == GKS_BC_OUTFLOW) {
    for (int k = 0; k < 4; ++k) out[k] = in[k];
    return;
  }
  R f[4];
  f[0] = in[0];
  f[3] = in[3];
  f[1] = axis == 0 ? in[1] : in[2];
  f[2] = axis == 0 ? in[2] : in[1];
  R o[4];
  if (kind == GKS_BC_SLIPWALL) {
    o[0] = f[0]; o[1] = -f[1]; o[2] = f[2]; o[3] = f[3];
  } else if (kind == GKS_BC_NOSLIP_ADIABATIC) {
    // equal density and temperature: rho E changes by the kinetic energy only
    o[0] = f[0];
    o[1] = -f[1];
    o[2] = R(2) * f[0] * uwt - f[2];
    o[3] = f[3] + R(2) * f[0] * uwt * uwt - R(2) * uwt * f[2];
  } else {
    const R rho = f[0], mn = f[1], mt = f[2];
    o[0] = rho;
    o[1] = -mn;
    o[2] = R(2) * rho * uwt - mt;
    o[3] = R(2) * rho * uwt * uwt - R(2) * uwt * mt + d_div(mn * mn + mt * mt, rho) +
           d_div(R(2) * rho * Tw, gamma - R(1)) - f[3];
  }
  out[0] = o[0];
  out[3] = o[3];
  out[1] = axis == 0 ? o[1] : o[2];
  out[2] = axis == 0 ? o[2] : o[1];
}

// value of a ghost cell from the compute-type averages; y is resolved first, so
// corners are x-images of y-ghosts
template <class R>
__device__ __forceinline__ void ghost_cell(const Geo& g, const R* U, int i, int j, R out[4]) {
  int is = i, js = j;
  int xs = -1, ys = -1;  // boundary side applied
  if (j < 0) { ys = 2; js = g.bc.kind[2] == GKS_BC_PERIODIC ? g.ny - 1 : 0; }
  if (j >= g.ny) { ys = 3; js = g.bc.kind[3] == GKS_BC_PERIODIC ? 0 : g.ny - 1; }
  if (i < 0) { xs = 0; is = g.bc.kind[0] == GKS_BC_PERIODIC ? g.nx - 1 : 0; }
  if (i >= g.nx) { xs = 1; is = g.bc.kind[1] == GKS_BC_PERIODIC ? 0 : g.nx - 1; }
  R w[4], t[4];
  for (int v = 0; v < 4; ++v) w[v] = U[ci(g, v, is, js)];
  if (ys >= 0) {
    bc_value<R>(g.bc.kind[ys], GeoR<R>::gamma(g), GeoR<R>::uwt(g, ys), GeoR<R>::Tw(g, ys), 1, w, t);
    for (int v = 0; v < 4; ++v) w[v] = t[v];
  }
  if (xs >= 0) {
    bc_value<R>(g.bc.kind[xs], GeoR<R>::gamma(g), GeoR<R>::uwt(g, xs), GeoR<R>::Tw(g, xs), 0, w, t);
    for (int v = 0; v < 4; ++v) w[v] = t[v];
  }
  for (int v = 0; v < 4; ++v) out[v] = w[v];
}

__host__ __device__ __forceinline__ int perimeter(const Geo& g) { return 2 * (g.nx + 2) + 2 * g.ny; }

// Every ghost cell is the boundary image of exactly one interior cell (the one
// ghost_cell reads).  ghosts_of_cell refreshes the ghosts whose source is
// interior cell (i, j) from U, so the update that writes (i, j) also writes
// them and a step needs no separate ghost pass.
template <class Fn>
__device__ __forceinline__ void for_each_ghost_of(const Geo& g, int i, int j, Fn fn) {
  const bool px = g.bc.kind[0] == GKS_BC_PERIODIC, py = g.bc.kind[2] == GKS_BC_PERIODIC;
  // candidate x (y) coordinates: the cell's own, the low ghost, the high ghost; across an
  // exchange side the ghost row is the neighbouring slab's, supplied from outside
  const bool xl = i == (px ? g.nx - 1 : 0), xh = i == (px ? 0 : g.nx - 1);
  const bool yl = j == (py ? g.ny - 1 : 0) && g.bc.kind[2] != GKS_BC_EXCHANGE;
  const bool yh = j == (py ? 0 : g.ny - 1) && g.bc.kind[3] != GKS_BC_EXCHANGE;
  if (!(xl || xh || yl || yh)) return;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if ((a == 0 && b == 0) || (a == 1 && !xl) || (a == 2 && !xh) || (b == 1 && !yl) || (b == 2 && !yh)) continue;
      fn(a == 0 ? i : (a == 1 ? -1 : g.nx), b == 0 ? j : (b == 1 ? -1 : g.ny));
    }
}

template <class R>
__device__ __forceinline__ void ghosts_of_cell(const Geo& g, Cells<R> U, int i, int j) {
  for_each_ghost_of(g, i, j, [&](int gi, int gj) {
    R w[4];
    ghost_cell<R>(g, U.view(), gi, gj, w);
#pragma unroll
    for (int v = 0; v < 4; ++v) U.put(g, v, gi, gj, w[v]);
  });
}

// p-th cell of the ghost ring (boundary images are taken in FP64)
template <class R>
__device__ __forceinline__ void ghost_at(const Geo& g, Cells<R> U, int p) {
  const int row = g.nx + 2;
  int i, j;
  if (p < row) { i = p - 1; j = -1; if (g.bc.kind[2] == GKS_BC_EXCHANGE) return; }
  else if (p < 2 * row) { i = p - row - 1; j = g.ny; if (g.bc.kind[3] == GKS_BC_EXCHANGE) return; }
  else if (p < 2 * row + g.ny) { i = -1; j = p - 2 * row; }
  else if (p < 2 * row + 2 * g.ny) { i = g.nx; j = p - 2 * row - g.ny; }
  else return;
  R w[4];
  ghost_cell<R>(g, U.view(), i, j, w);
  for (int v = 0; v < 4; ++v) U.put(g, v, i, j, w[v]);
}

// ---------------------------------------------------------------------------
// reconstruction of cell (i, j); U is the padded cell-average array in the
// compute type, Wx/Wy the face point values; writes the cell's record and the
// averages of the ghost records that are images of the cell
// ---------------------------------------------------------------------------
// Eigenvectors of the Jacobian of the x-flux of the 2D Euler equations at the
// conservative state w: columns of Rv for the eigenvalues u - c, u (entropy), u (shear),
// u + c, and Lv = Rv^-1 (rows).  With b1 = (gamma-1)/c^2, b2 = b1 q^2/2 and the total
// enthalpy H: r1 = (1, u-c, v, H-uc), r2 = (1, u, v, q^2/2), r3 = (0, 0, 1, v),
// r4 = (1, u+c, v, H+uc); l1 = (b2 + u/c, -b1 u - 1/c, -b1 v, b1)/2, l2 = (1-b2, b1 u,
// b1 v, -b1), l3 = (-v, 0, 1, 0), l4 = (b2 - u/c, -b1 u + 1/c, -b1 v, b1)/2.  Returns false
// for a non-physical state.
template <class R>
__device__ __forceinline__ bool char_basis(const R w[4], R gm1, R gam, R Lv[4][4], R Rv[4][4]) {
  const R rho = w[0], ir = d_div(R(1), rho);
  const R u = w[1] * ir, v = w[2] * ir, q2 = u * u + v * v;
  const R p = gm1 * (w[3] - R(0.5) * rho * q2);
  if (!(rho > R(0)) || !(p > R(0))) return false;
  const R c2 = gam * p * ir, c = sqrt(c2), ic = d_div(R(1), c);
  const R H = (w[3] + p) * ir, b1 = d_div(gm1, c2), b2 = R(0.5) * b1 * q2;
  const R rv[4][4] = {{R(1), R(1), R(0), R(1)},
                      {u - c, u, R(0), u + c},
                      {v, v, R(1), v},
                      {H - u * c, R(0.5) * q2, v, H + u * c}};
  const R lv[4][4] = {{R(0.5) * (b2 + u * ic), R(0.5) * (-b1 * u - ic), R(-0.5) * b1 * v, R(0.5) * b1},
                      {R(1) - b2, b1 * u, b1 * v, -b1},
                      {-v, R(0), R(1), R(0)},
                      {R(0.5) * (b2 - u * ic), R(0.5) * (-b1 * u + ic), R(-0.5) * b1 * v, R(0.5) * b1}};
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Rv[r][k] = rv[r][k];
      Lv[r][k] = lv[r][k];
    }
  return true;
}

// Reconstruction of cell (i, j) from its 13 stencil vectors (the cell and its four
// neighbours, the eight face Gauss values), all four variables: in conservative
// variables (CHAR = false), or in characteristic ones: the x-derivative coefficients
// (a2, a4) from a reconstruction of the variables projected on the eigenvectors of the
// x-flux Jacobian of the cell average, the y ones (a3, a5) from the y-flux Jacobian's,
// the cross derivative a6 the mean of both.
template <bool CHAR, class R>
__device__ __forceinline__ void recon_vectors(const R in[13][4], const ReconK<R>& K, R gm1, R gam, R a[4][5]) {
  if constexpr (!CHAR) {
#pragma unroll
    for (int v = 0; v < 4; ++v)
      recon_var<R>(in[0][v], in[1][v], in[2][v], in[3][v], in[4][v], in[5][v], in[6][v], in[7][v], in[8][v],
                   in[9][v], in[10][v], in[11][v], in[12][v], K, a[v]);
  } else {
#pragma unroll
    for (int axis = 0; axis < 2; ++axis) {
      // momenta swapped for the y direction (the x-frame formulas with u <-> v)
      const int m1 = axis == 0 ? 1 : 2, m2 = axis == 0 ? 2 : 1;
      R ref[4] = {in[0][0], in[0][m1], in[0][m2], in[0][3]};
      R Lv[4][4], Rv[4][4];
      if (!char_basis(ref, gm1, gam, Lv, Rv)) {
        recon_vectors<false, R>(in, K, gm1, gam, a);
        return;
      }
      R cc[4][5];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        R pr[13];
#pragma unroll
        for (int k = 0; k < 13; ++k)
          pr[k] = Lv[r][0] * in[k][0] + Lv[r][1] * in[k][m1] + Lv[r][2] * in[k][m2] + Lv[r][3] * in[k][3];
        recon_var<R>(pr[0], pr[1], pr[2], pr[3], pr[4], pr[5], pr[6], pr[7], pr[8], pr[9], pr[10], pr[11], pr[12],
                     K, cc[r]);
      }
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        // a2, a4 (m = 0, 2) from the x pass; a3, a5 (m = 1, 3) from the y pass; a6 from both
        if (m == 4 || (axis == 0) == (m == 0 || m == 2)) {
          R o[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) o[r] = Rv[r][0] * cc[0][m] + Rv[r][1] * cc[1][m] + Rv[r][2] * cc[2][m] + Rv[r][3] * cc[3][m];
          const R s = m == 4 ? R(0.5) : R(1);
          const R w4[4] = {o[0], axis == 0 ? o[1] : o[2], axis == 0 ? o[2] : o[1], o[3]};
#pragma unroll
          for (int v = 0; v < 4; ++v) a[v][m] = (m == 4 && axis == 1) ? a[v][m] + s * w4[v] : s * w4[v];
        }
      }
    }
  }
}

template <class R, class TW, bool CHAR = false>
__device__ __forceinline__ void recon_cell(const Geo& g, const R* __restrict__ U, const TW* __restrict__ Wx,
                                           const TW* __restrict__ Wy, R* __restrict__ rec, int i, int j, R dx,
                                           R dy, R weps, R wC) {
  const int nx = g.nx, ny = g.ny;
  const size_t fxp = (size_t)ny * (nx + 1), fyp = (size_t)(ny + 1) * nx;
  const ReconK<R> K = recon_k(dx, dy, GeoR<R>::idx(g), GeoR<R>::idy(g), weps, wC);
  R a[4][5], cbar[4];
  // stencil vector k of variable v: c, e, w, n, s; east face y-/y+, west y-/y+, north x-/x+,
  // south x-/x+
  auto load = [&](int v, R in[13]) {
    const TW* wx = Wx + (size_t)v * 2 * fxp + (size_t)j * (nx + 1);
    const TW* wy = Wy + (size_t)v * 2 * fyp;
    in[0] = U[ci(g, v, i, j)];
    in[1] = U[ci(g, v, i + 1, j)];
    in[2] = U[ci(g, v, i - 1, j)];
    in[3] = U[ci(g, v, i, j + 1)];
    in[4] = U[ci(g, v, i, j - 1)];
    in[5] = R(wx[i + 1]);
    in[6] = R(wx[fxp + i + 1]);
    in[7] = R(wx[i]);
    in[8] = R(wx[fxp + i]);
    in[9] = R(wy[(size_t)(j + 1) * nx + i]);
    in[10] = R(wy[fyp + (size_t)(j + 1) * nx + i]);
    in[11] = R(wy[(size_t)j * nx + i]);
    in[12] = R(wy[fyp + (size_t)j * nx + i]);
  };
  if constexpr (CHAR) {
    R in[13][4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      R t[13];
      load(v, t);
#pragma unroll
      for (int k = 0; k < 13; ++k) in[k][v] = t[k];
      cbar[v] = t[0];
    }
    recon_vectors<true, R>(in, K, GeoR<R>::gm1(g), GeoR<R>::gamma(g), a);
  } else {
    // one variable at a time: only its 13 stencil values are live
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      R t[13];
      load(v, t);
      cbar[v] = t[0];
      recon_var<R>(t[0], t[1], t[2], t[3], t[4], t[5], t[6], t[7], t[8], t[9], t[10], t[11], t[12], K, a[v]);
    }
  }
  // the polynomial at the four face centres (x = +-dx/2, y = 0 and x = 0, y = +-dy/2):
  // value = e0 +- a2 dx/2 on x-faces, n0 +- a3 dy/2 on y-faces
  R ve[4], vw[4], vn[4], vs[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    // U(x, y) = c + a2 x + a3 y + a4 (x^2 - dx^2/12)/2 + a5 (y^2 - dy^2/12)/2 + a6 x y
    const R cc = cbar[v];
    const R e0 = cc + a[v][2] * K.dx2_12 - a[v][3] * R(0.5) * K.dy2_12;
    const R n0 = cc + a[v][3] * K.dy2_12 - a[v][2] * R(0.5) * K.dx2_12;
    ve[v] = e0 + a[v][0] * (R(0.5) * dx);
    vw[v] = e0 - a[v][0] * (R(0.5) * dx);
    vn[v] = n0 + a[v][1] * (R(0.5) * dy);
    vs[v] = n0 - a[v][1] * (R(0.5) * dy);
  }
  // positivity: rho > 0 and p > 0 (2 rho rho E > |rho u|^2) at the four face centres,
  // else the constant average
  auto ok = [](const R w[4]) { return w[0] > R(0) && R(2) * w[0] * w[3] > w[1] * w[1] + w[2] * w[2]; };
  const bool bad = !(ok(ve) && ok(vw) && ok(vn) && ok(vs));
  R r[kRec];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    r[v] = cbar[v];
#pragma unroll
    for (int k = 0; k < 5; ++k) r[4 + 4 * k + v] = bad ? R(0) : a[v][k];
  }
  RecIO<R>::store(rec + ri(g, i, j), r);
  // the ghost ring's averages (boundary images written by the last update)
  for_each_ghost_of(g, i, j, [&](int gi, int gj) {
    R w[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) w[v] = U[ci(g, v, gi, gj)];
    RecIO<R>::store_avg(rec + ri(g, gi, gj), w);
  });
}

// ---------------------------------------------------------------------------
// face evolution
// ---------------------------------------------------------------------------
// face-frame slot of physical variable v (y-faces swap the momenta)
template <int AX> __device__ __forceinline__ int slot(int v) { return AX == 0 ? v : (v == 1 ? 2 : (v == 2 ? 1 : v)); }

// value and derivatives of cell (i, j)'s polynomial at the centre of its face
// on side s (+1: the face at +h_n/2, -1: at -h_n/2), in the face frame of axis AX
template <int AX, class R>
__device__ __forceinline__ void side_state(const Geo& g, const R* __restrict__ rec, int i, int j, int s, R hn,
                                           R hn2_12, R ht2_24, FaceState<R>& S) {
  R r[kRec];
  RecIO<R>::load(rec + ri(g, i, j), r);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const R c = r[v];
    const R a2 = r[4 + v], a3 = r[8 + v], a4 = r[12 + v], a5 = r[16 + v], a6 = r[20 + v];
    const R an = AX == 0 ? a2 : a3, at = AX == 0 ? a3 : a2;
    const R ann = AX == 0 ? a4 : a5, att = AX == 0 ? a5 : a4;
    const int k = slot<AX>(v);
    const R sh = R(s) * R(0.5) * hn;
    S.w[0][k] = c + an * sh + ann * hn2_12 - att * ht2_24;
    S.w[1][k] = an + ann * sh;
    S.w[2][k] = at + a6 * sh;
    S.w[3][k] = ann;
    S.w[4][k] = a6;
    S.w[5][k] = att;
  }
}

// Inputs of one face, fetched on demand by face_evolution
template <int AX, class R>
struct GridFaceSource {
  const Geo* g;
  const R* U;    // padded compute-type averages (the first-order fallback's constant states)
  const R* rec;  // reconstruction records
  int i, j;            // face index (x-faces: i in [0, nx]; y-faces: j in [0, ny])
  int cl, cr;          // the two cells along the normal, after periodic wrap
  int img_lo, img_hi;  // boundary image on the low / high side: 0 none, else the BC kind
  R hn, ht, hn2_12, ht2_24, gamma, uwt_lo, Tw_lo, uwt_hi, Tw_hi;

  __device__ __forceinline__ int cx(int n) const { return AX == 0 ? n : i; }
  __device__ __forceinline__ int cy(int n) const { return AX == 0 ? j : n; }

  __device__ __forceinline__ void image(int kind, R uwt, R Tw, const FaceState<R>& in, FaceState<R>& out) const {
    if (kind == GKS_BC_OUTFLOW) out = in;
    else wall_image<R>(kind, gamma, uwt, Tw, in, out);
  }

  bool first_order;  // constant states (cell averages) for the positivity fallback

  // the average of cell n (along the normal) as a constant face state
  __device__ __forceinline__ void const_state(int n, FaceState<R>& S) const {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      S.w[0][slot<AX>(v)] = U[ci(*g, v, cx(n), cy(n))];
#pragma unroll
      for (int d = 1; d < 6; ++d) S.w[d][v] = R(0);
    }
  }

  __device__ __forceinline__ void side(int k, FaceState<R>& S) const {
    if (first_order) {
      if (k == 0) {
        if (img_lo) {
          FaceState<R> in;
          const_state(cr, in);
          image(img_lo, uwt_lo, Tw_lo, in, S);
        } else {
          const_state(cl, S);
        }
      } else {
        if (img_hi) {
          FaceState<R> in;
          const_state(cl, in);
          image(img_hi, uwt_hi, Tw_hi, in, S);
        } else {
          const_state(cr, S);
        }
      }
      return;
    }
    if (k == 0) {
      if (img_lo) {
        FaceState<R> in;
        side_state<AX>(*g, rec, cx(cr), cy(cr), -1, hn, hn2_12, ht2_24, in);
        image(img_lo, uwt_lo, Tw_lo, in, S);
      } else {
        side_state<AX>(*g, rec, cx(cl), cy(cl), +1, hn, hn2_12, ht2_24, S);
      }
    } else {
      if (img_hi) {
        FaceState<R> in;
        side_state<AX>(*g, rec, cx(cl), cy(cl), +1, hn, hn2_12, ht2_24, in);
        image(img_hi, uwt_hi, Tw_hi, in, S);
      } else {
        side_state<AX>(*g, rec, cx(cr), cy(cr), -1, hn, hn2_12, ht2_24, S);
      }
    }
  }

  // six cell averages around the face (ghost ring included), face frame
  __device__ __forceinline__ void avg(R a[2][3][4]) const {
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int ii = AX == 0 ? i - 1 + m : i - 1 + k;
        const int jj = AX == 0 ? j - 1 + k : j - 1 + m;
        R w[4];
        RecIO<R>::load_avg(rec + ri(*g, ii, jj), w);
#pragma unroll
        for (int v = 0; v < 4; ++v) a[m][k][slot<AX>(v)] = w[v];
      }
  }
};

// Flux through a wall face (face frame, kind = the boundary kind of the side).  A
// wall lets no mass through, and an adiabatic wall no heat: its energy flux is the
// work u_w F_(m_t) of the shear on the moving wall.  The mirror image behind a
// no-slip wall also reverses the tangential velocity, which the tangential transport
// terms of the evolution do not respect; the wall's definition removes the resulting
// O(dt d(rho u_t)/dt) mass and energy fluxes (a slip wall gives them exactly).
template <class R>
__device__ __forceinline__ void wall_face_flux(int kind, R uwt, R F[4]) {
  if (kind == GKS_BC_SLIPWALL || kind == GKS_BC_NOSLIP_ISOTHERMAL || kind == GKS_BC_NOSLIP_ADIABATIC) F[0] = R(0);
  if (kind == GKS_BC_NOSLIP_ADIABATIC) F[3] = uwt * F[2];
}

// per-launch constants of the face routine for axis AX of grid g
template <class R>
__host__ __device__ inline FaceConst<R> grid_face_const(const Geo& g, int axis) {
  FaceParams P;
  P.gamma = g.gamma; P.mu = g.mu; P.Pr = g.Pr; P.tau_eps = g.tau_eps; P.tau_C = g.tau_C;
  P.dn = axis == 0 ? g.dx : g.dy;
  P.dtan = axis == 0 ? g.dy : g.dx;
  return face_const<R>(P);
}

// the evolution at face (i, j) of axis AX: flux F and new point values Wn
// (NSM: Navier-Stokes 1, Euler 0, decided per grid at run time -1)
template <int AX, class R, class TW, int NSM = -1>
__device__ __forceinline__ void flux_face(const Geo& g, const FaceConst<R>& C, const R* __restrict__ rec,
                                          TW* __restrict__ Wn, R* __restrict__ F, int i, int j, R dt) {
  const int nx = g.nx, ny = g.ny;
  const int fx = AX == 0 ? nx + 1 : nx, fy = AX == 0 ? ny : ny + 1;
  GridFaceSource<AX, R> src;
  src.g = &g;
  src.U = nullptr;
  src.rec = rec;
  src.i = i;
  src.j = j;
  const int f = AX == 0 ? i : j;     // face index along the normal
  const int nf = AX == 0 ? nx : ny;  // faces 0 and nf are on the boundary
  const int lo_side = AX == 0 ? 0 : 2, hi_side = lo_side + 1;
  // the two cells along the normal: across a periodic side the wrapped cell, across an
  // exchange side the neighbouring slab's (its record in the halo row), across any other
  // the image of the inside cell's polynomial
  src.cl = f - 1;
  src.cr = f;
  src.img_lo = src.img_hi = 0;
  if (f == 0) {
    if (g.bc.kind[lo_side] == GKS_BC_PERIODIC) src.cl = nf - 1;
    else if (g.bc.kind[lo_side] != GKS_BC_EXCHANGE) src.img_lo = g.bc.kind[lo_side];
  }
  if (f == nf) {
    if (g.bc.kind[hi_side] == GKS_BC_PERIODIC) src.cr = 0;
    else if (g.bc.kind[hi_side] != GKS_BC_EXCHANGE) src.img_hi = g.bc.kind[hi_side];
  }
  src.hn = C.dn;
  src.ht = C.dtan;
  src.hn2_12 = C.dn2_12;
  src.ht2_24 = C.dt2_24;
  src.gamma = C.gamma;
  src.uwt_lo = GeoR<R>::uwt(g, lo_side);
  src.Tw_lo = GeoR<R>::Tw(g, lo_side);
  src.uwt_hi = GeoR<R>::uwt(g, hi_side);
  src.Tw_hi = GeoR<R>::Tw(g, hi_side);
  src.first_order = false;

  R Fl[4], Wm[4], Wp[4];
  face_evolution<R, NSM>(C, src, dt, Fl, Wm, Wp);
  if (src.img_lo) wall_face_flux<R>(src.img_lo, src.uwt_lo, Fl);
  else if (src.img_hi) wall_face_flux<R>(src.img_hi, src.uwt_hi, Fl);

  const size_t nfaces = (size_t)fx * fy, o = (size_t)j * fx + i;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int k = slot<AX>(v);
    F[(size_t)v * nfaces + o] = Fl[k];
    Wn[(size_t)(v * 2 + 0) * nfaces + o] = TW(Wm[k]);
    Wn[(size_t)(v * 2 + 1) * nfaces + o] = TW(Wp[k]);
  }
}

// ---------------------------------------------------------------------------
// update, CFL bound of the new state, physical check
// ---------------------------------------------------------------------------
// inverse CFL bound max((|U|+c)/dx, (|V|+c)/dy) (and the viscous rate) of a state;
// ok = rho > 0 and p > 0.  The bound itself is 1/inverse.
template <class R>
__device__ __forceinline__ R inv_bound(const Geo& g, const R w[4], bool& ok) {
  const R ir = d_div(R(1), w[0]);
  const R u = w[1] * ir, v = w[2] * ir;
  const R p = GeoR<R>::gm1(g) * (w[3] - R(0.5) * (w[1] * u + w[2] * v));
  ok = w[0] > R(0) && p > R(0);
  const R c = sqrt(GeoR<R>::gamma(g) * p * ir);
  R inv = fmax((fabs(u) + c) * GeoR<R>::idx(g), (fabs(v) + c) * GeoR<R>::idy(g));
  if (g.visc_on) inv = fmax(inv, GeoR<R>::visc(g) * ir);
  return inv;
}

// warp maximum of inv, then the atomic minimum of the bound 1/inv (no block
// barrier: the warps of a block go on independently).  Every lane of the warp must
// call it.
template <class R>
__device__ __forceinline__ void warp_bound_to(R inv, unsigned long long* slot) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) inv = fmax(inv, __shfl_xor_sync(0xffffffffu, inv, o));
  if ((threadIdx.x & 31) == 0 && inv > R(0)) atomicMin(slot, dbits(1.0 / (double)inv));
}

// block maximum of inv, then the atomic minimum of the bound 1/inv.  Every
// thread of the block must call it.
template <class R>
__device__ __forceinline__ void block_bound_to(R inv, unsigned long long* slot) {
  __shared__ R red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) inv = fmax(inv, __shfl_xor_sync(0xffffffffu, inv, o));
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  if (lane == 0) red[warp] = inv;
  __syncthreads();
  if (warp == 0) {
    inv = lane < nw ? red[lane] : R(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) inv = fmax(inv, __shfl_xor_sync(0xffffffffu, inv, o));
    if (lane == 0 && inv > R(0)) atomicMin(slot, dbits(1.0 / (double)inv));
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// positivity fallback: the collisionless (tau -> infinity) evolution of the
// two cell averages at face (i, j) of axis AX -- flux dt (rho_l <u psi>_{u>0} +
// rho_r <u psi>_{u<0}) and point values U0 -- in the physical frame
// ---------------------------------------------------------------------------
template <int AX, class R>
__device__ __forceinline__ void kfvs_face(const Geo& g, const R* U, R gm1, R K, int i, int j, R dt, R F[4],
                                          R W[4]) {
  GridFaceSource<AX, R> src;
  src.g = &g;
  src.U = U;
  src.rec = nullptr;
  src.i = i;
  src.j = j;
  const int f = AX == 0 ? i : j, nf = AX == 0 ? g.nx : g.ny;
  const int lo_side = AX == 0 ? 0 : 2, hi_side = lo_side + 1;
  src.cl = f - 1;
  src.cr = f;
  src.img_lo = src.img_hi = 0;
  if (f == 0) {
    if (g.bc.kind[lo_side] == GKS_BC_PERIODIC) src.cl = nf - 1;
    else if (g.bc.kind[lo_side] != GKS_BC_EXCHANGE) src.img_lo = g.bc.kind[lo_side];
  }
  if (f == nf) {
    if (g.bc.kind[hi_side] == GKS_BC_PERIODIC) src.cr = 0;
    else if (g.bc.kind[hi_side] != GKS_BC_EXCHANGE) src.img_hi = g.bc.kind[hi_side];
  }
  src.gamma = GeoR<R>::gamma(g);
  src.uwt_lo = GeoR<R>::uwt(g, lo_side);
  src.Tw_lo = GeoR<R>::Tw(g, lo_side);
  src.uwt_hi = GeoR<R>::uwt(g, hi_side);
  src.Tw_hi = GeoR<R>::Tw(g, hi_side);
  src.first_order = true;
  R Ff[4] = {R(0), R(0), R(0), R(0)}, Wf[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    FaceState<R> S;
    src.side(k, S);
    R rho, ir, u, v, p;
    prim(S.w[0], gm1, rho, ir, u, v, p);
    Moments<R, 4, 3> m;
    moments(u, v, d_div(R(0.5) * rho, p), p * ir, K, k == 0 ? +1 : -1, m);
    R a[4], b[4];
    psi_mom<0, 0>(m, a);
    psi_mom<1, 0>(m, b);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Wf[q] += rho * a[q];
      Ff[q] += dt * rho * b[q];
    }
  }
  if (src.img_lo) wall_face_flux<R>(src.img_lo, src.uwt_lo, Ff);
  else if (src.img_hi) wall_face_flux<R>(src.img_hi, src.uwt_hi, Ff);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    F[v] = Ff[slot<AX>(v)];
    W[v] = Wf[slot<AX>(v)];
  }
}

// positivity fallback: is face (i, j) of axis AX next to a marked cell?
template <int AX>
__device__ __forceinline__ bool face_needs_fix(const Geo& g, const unsigned char* bad, int i, int j) {
  const int f = AX == 0 ? i : j, nf = AX == 0 ? g.nx : g.ny;
  const int lo_side = AX == 0 ? 0 : 2;
  int a = f - 1, b = f;
  if (f == 0) a = g.bc.kind[lo_side] == GKS_BC_PERIODIC ? nf - 1 : -1;
  if (f == nf) b = g.bc.kind[lo_side + 1] == GKS_BC_PERIODIC ? 0 : -1;
  const int c0 = a < 0 ? -1 : (AX == 0 ? j * g.nx + a : a * g.nx + i);
  const int c1 = b < 0 ? -1 : (AX == 0 ? j * g.nx + b : b * g.nx + i);
  return (c0 >= 0 && bad[c0]) || (c1 >= 0 && bad[c1]);
}

// state of one cell for the update, loaded before any arithmetic: FP64 values or FP32
// (hi, lo) pairs
template <class R> struct CellState;
template <> struct CellState<double> { double w[4]; };
template <> struct CellState<float> { float hi[4], lo[4]; };

__device__ __forceinline__ void load_state(const Geo& g, Cells<double> U, int i, int j, CellState<double>& s) {
#pragma unroll
  for (int v = 0; v < 4; ++v) s.w[v] = U.p[ci(g, v, i, j)];
}
__device__ __forceinline__ void load_state(const Geo& g, Cells<float> U, int i, int j, CellState<float>& s) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const size_t o = ci(g, v, i, j);
    s.hi[v] = U.p[o];
    s.lo[v] = U.p[o + 4 * g.plane];
  }
}

// Eq. finite for one variable: FP64 planes take the FP32 or FP64 fluxes in
// FP64 (differences of FP32 numbers are exact there); the double-float pair
// takes the FP32 fluxes one product at a time with error-free transformations.
// Either way each face flux enters both neighbours with the same rounding, so
// the sum over cells telescopes to roundoff of the accumulation type.
template <class R>
__device__ __forceinline__ R update_var(const Geo& g, const CellState<double>& S, Cells<double> Un, const R f[4][4], int v,
                                        int i, int j, bool& finite) {
  const size_t o = ci(g, v, i, j);
  const double w = S.w[v] + ((double)f[0][v] - (double)f[1][v]) * g.idx + ((double)f[2][v] - (double)f[3][v]) * g.idy;
  Un.p[o] = w;
  finite = isfinite(w);
  return R(w);
}
__device__ __forceinline__ float update_var(const Geo& g, const CellState<float>& S, Cells<float> Un, const float f[4][4],
                                            int v, int i, int j, bool& finite) {
  const size_t o = ci(g, v, i, j), lo_off = 4 * g.plane;
  float hi = S.hi[v], lo = S.lo[v];
  df_add_product(hi, lo, f[0][v], g.idx_hi, g.idx_lo);
  df_add_product(hi, lo, -f[1][v], g.idx_hi, g.idx_lo);
  df_add_product(hi, lo, f[2][v], g.idy_hi, g.idy_lo);
  df_add_product(hi, lo, -f[3][v], g.idy_hi, g.idy_lo);
  // renormalise: hi becomes the FP32 rounding of the pair (Dekker's fast two-sum)
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
  Un.p[o] = hi;
  Un.p[o + lo_off] = lo;
  finite = isfinite(hi) && isfinite(lo);
  return hi;
}

// Eq. finite for cell (i, j) into Un, and the ghost cells that are images of
// (i, j); returns the inverse CFL bound of the new state, 0 with bad = true if
// it is not physical.  pass 1 takes every face
// flux from Fx/Fy; pass 2 replaces the faces next to cells marked in pass 1 by
// the collisionless flux; pass 3 replaces every face.  Replaced faces also get
// their point values in Wxn/Wyn, written by one cell each (its west and south
// faces, and the east / north faces of the last column / row).
template <class R, class TW>
__device__ __forceinline__ R update_cell(const Geo& g, Cells<R> U, Cells<R> Un, const R* __restrict__ Fx,
                                         const R* __restrict__ Fy, TW* __restrict__ Wxn, TW* __restrict__ Wyn,
                                         const unsigned char* __restrict__ marked, int pass, R dt, int i, int j,
                                         bool& bad) {
  const int nx = g.nx, ny = g.ny;
  const size_t nfx = (size_t)ny * (nx + 1), nfy = (size_t)(ny + 1) * nx;
  const R* Ur = U.view();
  // the four face fluxes: west, east, south, north
  R f[4][4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    f[0][v] = Fx[v * nfx + (size_t)j * (nx + 1) + i];
    f[1][v] = Fx[v * nfx + (size_t)j * (nx + 1) + i + 1];
    f[2][v] = Fy[v * nfy + (size_t)j * nx + i];
    f[3][v] = Fy[v * nfy + (size_t)(j + 1) * nx + i];
  }
  CellState<R> S;
  load_state(g, U, i, j, S);
  if (pass > 1) {
    const R gm1 = GeoR<R>::gm1(g), K = GeoR<R>::K(g);
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      const int fi = i + (q == 1), fj = j + (q == 3);
      const bool x = q < 2;
      const bool redo = pass == 3 || (x ? face_needs_fix<0>(g, marked, fi, fj) : face_needs_fix<1>(g, marked, fi, fj));
      if (!redo) continue;
      R W[4], Fq[4];
      if (x) kfvs_face<0, R>(g, Ur, gm1, K, fi, fj, dt, Fq, W);
      else kfvs_face<1, R>(g, Ur, gm1, K, fi, fj, dt, Fq, W);
      // constant indices keep f in registers
#pragma unroll
      for (int qq = 0; qq < 4; ++qq)
        if (qq == q)
#pragma unroll
          for (int v = 0; v < 4; ++v) f[qq][v] = Fq[v];
      const bool owner = q == 0 || q == 2 || (q == 1 && i == nx - 1) || (q == 3 && j == ny - 1);
      if (owner) {
        TW* Wn = x ? Wxn : Wyn;
        const size_t nf = x ? nfx : nfy;
        const size_t o = x ? (size_t)fj * (nx + 1) + fi : (size_t)fj * nx + fi;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          Wn[(size_t)(v * 2 + 0) * nf + o] = TW(W[v]);
          Wn[(size_t)(v * 2 + 1) * nf + o] = TW(W[v]);
        }
      }
    }
  }
  R wr[4];
  bool finite = true;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    bool fv;
    wr[v] = update_var(g, S, Un, f, v, i, j, fv);
    finite = finite && fv;
  }
  ghosts_of_cell<R>(g, Un, i, j);
  bool ok;
  R inv = inv_bound<R>(g, wr, ok);
  bad = !ok || !finite || !(inv < R(INFINITY));
  return bad ? R(0) : inv;
}

}  // namespace gks
