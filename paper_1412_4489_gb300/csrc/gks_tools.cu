// Measurement helpers of the library (include/gks.h):
//  * gks_face_op_count: runs the face routine of gks_device.cuh once on the host
//    with a counting number type, giving the exact arithmetic of one face
//    evaluation (the algorithmic flops of the roofline);
//  * gks_measure_alu_peak: FMA throughput of this GPU in FP32 or FP64 from a
//    kernel of independent FMA chains over every SM.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "../../include/gks.h"

namespace opc {

struct Counts {
  long long add, mul, div, cmp, sqrt, rsqrt, exp, expm1, erfc;
};
static thread_local Counts C;

// a double that counts the arithmetic done with it
template <int PREC>
struct Num {
  double v;
  Num() : v(0) {}
  Num(double x) : v(x) {}
  Num(int x) : v(x) {}
  Num(float x) : v(x) {}
  explicit operator double() const { return v; }
  Num operator-() const { return Num(-v); }
  Num& operator+=(const Num& o) { ++C.add; v += o.v; return *this; }
  Num& operator-=(const Num& o) { ++C.add; v -= o.v; return *this; }
  Num& operator*=(const Num& o) { ++C.mul; v *= o.v; return *this; }
  Num& operator/=(const Num& o) { ++C.div; v /= o.v; return *this; }
};
template <int P> Num<P> operator+(Num<P> a, const Num<P>& b) { ++C.add; return Num<P>(a.v + b.v); }
template <int P> Num<P> operator-(Num<P> a, const Num<P>& b) { ++C.add; return Num<P>(a.v - b.v); }
template <int P> Num<P> operator*(Num<P> a, const Num<P>& b) { ++C.mul; return Num<P>(a.v * b.v); }
template <int P> Num<P> operator/(Num<P> a, const Num<P>& b) { ++C.div; return Num<P>(a.v / b.v); }
template <int P> bool operator<(const Num<P>& a, const Num<P>& b) { ++C.cmp; return a.v < b.v; }
template <int P> bool operator>(const Num<P>& a, const Num<P>& b) { ++C.cmp; return a.v > b.v; }
template <int P> bool operator<(const Num<P>& a, double b) { ++C.cmp; return a.v < b; }
template <int P> bool operator>(const Num<P>& a, double b) { ++C.cmp; return a.v > b; }
template <int P> Num<P> fabs(const Num<P>& a) { return Num<P>(::fabs(a.v)); }
template <int P> Num<P> d_exp(const Num<P>& a) { ++C.exp; return Num<P>(::exp(a.v)); }
template <int P> Num<P> d_expm1(const Num<P>& a) { ++C.expm1; return Num<P>(::expm1(a.v)); }
template <int P> Num<P> d_erfc(const Num<P>& a) { ++C.erfc; return Num<P>(::erfc(a.v)); }
template <int P> Num<P> d_sqrt(const Num<P>& a) { ++C.sqrt; return Num<P>(::sqrt(a.v)); }
template <int P> Num<P> d_rsqrt(const Num<P>& a) { ++C.rsqrt; return Num<P>(1.0 / ::sqrt(a.v)); }
template <int P> Num<P> d_div(const Num<P>& a, const Num<P>& b) { ++C.div; return Num<P>(a.v / b.v); }

}  // namespace opc

#include "gks_device.cuh"

namespace gks {
// the counting types follow the branch thresholds of the precision they stand for
template <> struct Prec<opc::Num<0>> {
  static constexpr double series_below = Prec<double>::series_below;
  static constexpr int series_terms = Prec<double>::series_terms;
  static constexpr double tie = Prec<double>::tie;
};
template <> struct Prec<opc::Num<1>> {
  static constexpr double series_below = Prec<float>::series_below;
  static constexpr int series_terms = Prec<float>::series_terms;
  static constexpr double tie = Prec<float>::tie;
};
}  // namespace gks

namespace {

template <int P>
void count_face(const double* L, const double* R, const double* avg, double dn, double dtan, double dt,
                double gamma, double mu, double Pr, double tau_eps, double tau_C) {
  using N = opc::Num<P>;
  gks::FaceState<N> SL, SR;
  N av[2][3][4];
  for (int d = 0; d < 6; ++d)
    for (int k = 0; k < 4; ++k) {
      SL.w[d][k] = N(L[d * 4 + k]);
      SR.w[d][k] = N(R[d * 4 + k]);
    }
  for (int m = 0; m < 2; ++m)
    for (int n = 0; n < 3; ++n)
      for (int k = 0; k < 4; ++k) av[m][n][k] = N(avg[(m * 3 + n) * 4 + k]);
  gks::FaceParams FP;
  FP.gamma = gamma; FP.mu = mu; FP.Pr = Pr; FP.tau_eps = tau_eps; FP.tau_C = tau_C;
  FP.dn = dn; FP.dtan = dtan;
  N F[4], Wm[4], Wp[4];
  gks::ArrayFaceSource<N> src;
  src.s[0] = &SL;
  src.s[1] = &SR;
  src.a = av;
  const gks::FaceConst<N> C = gks::face_const<N>(FP);
  opc::C = opc::Counts{};  // per-launch constants are not per-face work
  // the routine the face kernels run: Navier-Stokes for mu > 0, Euler otherwise
  if (mu > 0.0) gks::face_evolution<N, 1>(C, src, N(dt), F, Wm, Wp);
  else gks::face_evolution<N, 0>(C, src, N(dt), F, Wm, Wp);
}

template <class R>
__global__ void k_fma_chain(R* out, int iters) {
  // 8 independent chains per thread keep the FMA pipe busy
  R a[8];
  const R m = R(0.999999), c = R(1e-7);
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = R(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  R s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == R(-1.2345)) out[0] = s;  // never true; keeps the chains alive
}

}  // namespace

extern "C" {

gks_status gks_face_op_count(const double* L, const double* R, const double* avg, double dn, double dtan, double dt,
                             double gamma, double mu, double Pr, double tau_eps, double tau_C, int precision,
                             long long* counts) {
  if (!L || !R || !avg || !counts || !(dt > 0) || !(dn > 0) || !(dtan > 0)) return GKS_EINVAL;
  if (precision == GKS_FP64)
    count_face<0>(L, R, avg, dn, dtan, dt, gamma, mu, Pr, tau_eps, tau_C);
  else if (precision == GKS_FP32_BULK)
    count_face<1>(L, R, avg, dn, dtan, dt, gamma, mu, Pr, tau_eps, tau_C);
  else
    return GKS_EINVAL;
  const opc::Counts& c = opc::C;
  const long long v[9] = {c.add, c.mul, c.div, c.cmp, c.sqrt, c.rsqrt, c.exp, c.expm1, c.erfc};
  for (int k = 0; k < 9; ++k) counts[k] = v[k];
  return GKS_OK;
}

gks_status gks_measure_alu_peak(int precision, double* tflops) {
  if (!tflops || (precision != GKS_FP64 && precision != GKS_FP32_BULK)) return GKS_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GKS_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GKS_ECUDA;
  void* out = nullptr;
  if (cudaMalloc(&out, 64) != cudaSuccess) return GKS_ENOMEM;
  const int threads = 512, blocks = sms * 8;
  const int iters = precision == GKS_FP64 ? 1 << 11 : 1 << 14;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    if (precision == GKS_FP64) k_fma_chain<double><<<blocks, threads>>>((double*)out, iters);
    else k_fma_chain<float><<<blocks, threads>>>((float*)out, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return GKS_ECUDA;
  const double flops = 2.0 * 8.0 * (double)iters * threads * blocks;
  *tflops = flops / (best * 1e-3) / 1e12;
  return GKS_OK;
}

}  // extern "C"
