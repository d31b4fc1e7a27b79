// Device arithmetic of the compact third-order gas-kinetic scheme
// (Pan & Xu, arXiv:1412.4489), templated on the compute type R (double or float).
//
//   Section 2.1  Maxwellian moments: full space and the half spaces u > 0, u < 0
//   Section 2.2  closed-form solve of <a> = r, the nine coefficient systems,
//                time weights of Eq. dis1 / Eq. dis2 integrated over [0, dt]
//                and at t = dt, assembly of the flux and of Eq. point
//   Section 3.2  compact reconstruction of one cell
//   Section 3.3  equilibrium polynomial across a face
//   Section 4    collision time
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#ifndef GKS_FN
#define GKS_FN __host__ __device__ __forceinline__
#endif

namespace gks {

template <class R> struct Prec;
// series_below: x = dt/tau below which the time weights are summed from series;
// series_terms: the sums stop before x^series_terms / series_terms!, at which the largest
// relative truncation error over x < series_below is below the type's rounding (FP64: 17
// terms reach it, FP32: 18);
// tie: relative width within which two cross-derivative candidates count as equal.
// FP64: far above its rounding noise, far below any real difference.  FP32: ~16
// ulps, just above the rounding noise of the candidates; a wider band makes FP32
// keep the first stencil where FP64 picks a smaller one of opposite sign, which
// measured worse against the FP64 results on discontinuous data.
template <> struct Prec<double> {
  static constexpr double series_below = 0.5;
  static constexpr int series_terms = 18;
  static constexpr double tie = 1e-8;
};
template <> struct Prec<float> {
  static constexpr float series_below = 2.0f;
  static constexpr int series_terms = 18;
  static constexpr float tie = 1e-6f;
};

__device__ __forceinline__ double d_exp(double x) { return exp(x); }
__device__ __forceinline__ float d_exp(float x) { return __expf(x); }
__device__ __forceinline__ double d_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float d_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double d_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float d_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float d_rsqrt(float x) { return rsqrtf(x); }
// quotient of runtime values: IEEE in FP64; in FP32 the fast division (within
// 2 ulps for divisors below 2^126), far inside the FP32 path's error budget
__device__ __forceinline__ double d_div(double a, double b) { return a / b; }
__device__ __forceinline__ float d_div(float a, float b) { return __fdividef(a, b); }

template <class R> GKS_FN R sq(R a) { return a * a; }

// ---------------------------------------------------------------------------
// Section 2.1: moments of g = rho (lam/pi)^((K+2)/2) exp(-lam((u-U)^2+(v-V)^2+xi^2)),
// normalised by rho.  NU u-moments, NV v-moments.
// ---------------------------------------------------------------------------
template <class R, int NU, int NV>
struct Moments {
  R u[NU];
  R v[NV];
  R xi2, xi4;
  R kap;  // <xi^4> - <xi^2>^2 = 2 K var^2
};

// kind: 0 full space, +1 over u > 0, -1 over u < 0; var = 1/(2 lam) = p/rho, formed
// once per Maxwellian by the caller
template <class R, int NU, int NV>
GKS_FN void moments(R U, R V, R lam, R var, R K, int kind, Moments<R, NU, NV>& m) {
  if (kind == 0) {
    m.u[0] = R(1);
    m.u[1] = U;
  } else {
    const R rs = d_rsqrt(lam);
    const R s = lam * rs;  // sqrt(lam)
    const R h = R(0.5) * d_erfc(-R(kind) * s * U);
    // boundary term of the integration by parts at u = 0
    const R b = d_exp(-lam * U * U) * R(0.28209479177387814) * rs;  // 1/(2 sqrt(pi lam))
    m.u[0] = h;
    m.u[1] = U * h + R(kind) * b;
  }
#pragma unroll
  for (int n = 2; n < NU; ++n) m.u[n] = U * m.u[n - 1] + (n == 2 ? var : R(n - 1) * var) * m.u[n - 2];
  m.v[0] = R(1);
  m.v[1] = V;
  m.v[2] = V * V + var;
#pragma unroll
  for (int n = 3; n < NV; ++n) m.v[n] = V * m.v[n - 1] + R(n - 1) * var * m.v[n - 2];
  m.xi2 = K * var;
  m.xi4 = K * (K + R(2)) * var * var;
  m.kap = R(2) * K * var * var;
}

// The same half-space moments from their first two entries h = <u^0>, g = <u^1>
// (already formed once for the same Maxwellian: no second erfc and exp).
template <class R, int NU, int NV>
GKS_FN void moments_from(R U, R V, R var, R K, R h, R g, Moments<R, NU, NV>& m) {
  m.u[0] = h;
  m.u[1] = g;
#pragma unroll
  for (int n = 2; n < NU; ++n) m.u[n] = U * m.u[n - 1] + (n == 2 ? var : R(n - 1) * var) * m.u[n - 2];
  m.v[0] = R(1);
  m.v[1] = V;
  m.v[2] = V * V + var;
#pragma unroll
  for (int n = 3; n < NV; ++n) m.v[n] = V * m.v[n - 1] + R(n - 1) * var * m.v[n - 2];
  m.xi2 = K * var;
  m.xi4 = K * (K + R(2)) * var * var;
  m.kap = R(2) * K * var * var;
}

// <u^A v^B psi> and <xi^2 u^A v^B psi>, psi = (1, u, v, (u^2+v^2+xi^2)/2)
template <int A, int B, class R, int NU, int NV>
GKS_FN void psi_mom(const Moments<R, NU, NV>& m, R o[4]) {
  static_assert(A + 2 < NU && B + 2 < NV, "moment table too short");
  const R ab = m.u[A] * m.v[B];
  o[0] = ab;
  o[1] = m.u[A + 1] * m.v[B];
  o[2] = m.u[A] * m.v[B + 1];
  o[3] = R(0.5) * (m.u[A + 2] * m.v[B] + m.u[A] * m.v[B + 2] + ab * m.xi2);
}

// ---------------------------------------------------------------------------
// Section 2.2: <a> = rho r for a expanded in psi has a closed-form solution
// (the moment matrix of a Maxwellian is block structured about (U, V)).  The
// factors that depend only on the Maxwellian are formed once per Maxwellian.
// ---------------------------------------------------------------------------
template <class R>
struct SolveK {
  R U, V;
  R l2;  // 2 lam
  R c4;  // 4 lam^2 / N, N = K + 2
  R s0;  // U^2 + V^2 - N / (2 lam)
  R s1;  // (U^2 + V^2) / 2 + N / (4 lam)
  R hq;  // (U^2 + V^2) / 2
  R kc;  // (N + 2) / (4 lam)
};

template <class R>
GKS_FN SolveK<R> solve_k(R U, R V, R lam, R var, R N, R iN) {
  SolveK<R> k;
  const R q2 = U * U + V * V;
  const R nv = N * var;  // N / (2 lam)
  k.U = U;
  k.V = V;
  k.l2 = R(2) * lam;
  k.c4 = R(4) * lam * lam * iN;
  k.s0 = q2 - nv;
  k.s1 = R(0.5) * (q2 + nv);
  k.hq = R(0.5) * q2;
  k.kc = R(0.5) * (nv + R(2) * var);
  return k;
}

// <a> = rho r with r = ir d, ir = 1/rho folded into the factors:
// c4i = c4 ir, l2i = l2 ir
template <class R>
GKS_FN void solve_scaled(const SolveK<R>& k, R c4i, R l2i, R ir, const R d[4], R x[4]) {
  const R x4 = c4i * (R(2) * (d[3] - k.U * d[1] - k.V * d[2]) + k.s0 * d[0]);
  const R x3 = l2i * (d[2] - k.V * d[0]) - k.V * x4;
  const R x2 = l2i * (d[1] - k.U * d[0]) - k.U * x4;
  x[0] = ir * d[0] - k.U * x2 - k.V * x3 - x4 * k.s1;
  x[1] = x2;
  x[2] = x3;
  x[3] = x4;
}

// ---------------------------------------------------------------------------
// Time weights.  With x = dt/tau and e = exp(-x), the flux needs the integrals
// over [0, dt] of C_1..C_8, C_7 t and C_7 t^2; Eq. point needs their values at
// t = dt.  Several are differences of nearly equal terms when x is small; there
// they are summed from their Taylor series in x.
// ---------------------------------------------------------------------------
template <class R>
struct TimeW {
  R I[11];  // integrals, index 1..8 = C_1..C_8, 9 = C_7 t, 10 = C_7 t^2
  R E[11];  // values at t = dt
};

template <class R>
GKS_FN void time_weights(R T, R tau, TimeW<R>& w) {
  const R x = tau > R(0) ? d_div(T, tau) : R(INFINITY);
  const R e = tau > R(0) ? d_exp(-x) : R(0);
  const R om = tau > R(0) ? -d_expm1(-x) : R(1);  // 1 - e
  R f1, f2, f3, f4, f5, f6;  // see below
  if (x < Prec<R>::series_below) {
    // t_n = (-x)^n / n!:  f1 = x-1+e = sum_{n>=2} t_n;  f2 = 1-(1+x)e = sum (n-1) t_n;
    // f3 = 2-2e-x-xe = sum (n-2) t_n;  f4 = x^2/2-x+1-e = -sum_{n>=3} t_n;
    // f5 = 4-(x+2)^2 e = -sum (n-1)(n-4) t_n;  f6 = 2-(x^2+2x+2) e = -sum_{n>=3} (n-1)(n-2) t_n
    R t = R(0.5) * x * x;
    f1 = t; f2 = t; f3 = R(0); f4 = R(0); f5 = R(2) * t; f6 = R(0);
#pragma unroll
    for (int n = 3; n < Prec<R>::series_terms; ++n) {
      t *= -x * R(1.0 / n);
      f1 += t;
      f2 += R(n - 1) * t;
      f3 += R(n - 2) * t;
      f4 -= t;
      f5 -= R((n - 1) * (n - 4)) * t;
      f6 -= R((n - 1) * (n - 2)) * t;
    }
    const R t2 = tau * tau, t3 = t2 * tau;
    w.I[1] = tau * f1;
    w.I[2] = t2 * f3;
    w.I[3] = t2 * f4;
    w.I[4] = -t3 * f5;
    w.I[9] = t2 * f2;
    w.I[10] = t3 * f6;
    w.E[2] = -tau * f2;
    w.E[3] = tau * f1;
  } else {
    const R t2 = tau * tau;
    w.I[1] = T - tau * om;
    w.I[2] = R(2) * t2 * om - tau * T * (R(1) + e);
    w.I[3] = R(0.5) * T * T - tau * T + t2 * om;
    w.I[4] = -R(4) * t2 * tau + tau * sq(T + R(2) * tau) * e;
    w.I[9] = t2 - tau * (tau + T) * e;
    w.I[10] = R(2) * t2 * tau - tau * (T * T + R(2) * T * tau + R(2) * t2) * e;
    w.E[2] = (T + tau) * e - tau;
    w.E[3] = T - tau + tau * e;
  }
  w.I[5] = T * T * T * R(1.0 / 3.0) - tau * T * T;
  w.I[6] = -tau * (R(0.5) * T * T + w.I[9]);
  w.I[7] = tau * om;
  w.I[8] = -w.I[9];
  w.E[1] = om;
  w.E[4] = -(T * T + R(2) * T * tau) * e;
  w.E[5] = T * T - R(2) * T * tau;
  w.E[6] = -T * tau * (R(1) + e);
  w.E[7] = e;
  w.E[8] = -T * e;
  w.E[9] = T * e;
  w.E[10] = T * T * e;
}

// ---------------------------------------------------------------------------
// The nine coefficients of one equilibrium state (system after Eq. dis3).
// The composites (a1^2+d11), (a1 a2+d12), (a2^2+d22), (A a1+b1), (A a2+b2),
// (A^2+B) are single unknowns expanded in psi: Axx, Axy, Ayy, Atx, Aty, Att.
// d[] = (dn, dt, dnn, dnt, dtt) of the conservative variables.
// ---------------------------------------------------------------------------
template <class R>
struct Coefs {
  R a1[4], a2[4], Axx[4], Axy[4], Ayy[4], A[4], Atx[4], Aty[4], Att[4];
};

// A coefficient vector X about the Maxwellian's (U, V) in central coordinates: the
// coefficients of 1, c, d, s = (c^2 + d^2 + xi^2) / 2 with c = u - U, d = v - V
template <class R>
GKS_FN void to_central(const SolveK<R>& k, const R X[4], R Y[4]) {
  Y[0] = X[0] + k.U * X[1] + k.V * X[2] + k.hq * X[3];
  Y[1] = X[1] + k.U * X[3];
  Y[2] = X[2] + k.V * X[3];
  Y[3] = X[3];
}

template <class R>
GKS_FN void from_central(const SolveK<R>& k, const R Y[4], R X[4]) {
  X[3] = Y[3];
  X[1] = Y[1] - k.U * Y[3];
  X[2] = Y[2] - k.V * Y[3];
  X[0] = Y[0] - k.U * X[1] - k.V * X[2] - k.hq * Y[3];
}

// The time coefficient T of <(X u + Y v + T) psi g> = 0 (X, Y, T in central coordinates):
// T = -P(u X + v Y), P the projection on span(psi) in the inner product weighted by the
// Maxwellian.  u X = U X + c X, and the Maxwellian's central moments (<c^2> = 1/(2 lam),
// <c^4> = 3 <c^2>^2, <xi^2> = K <c^2>) give P(c) = c, P(c^2) = (2/N) s, P(c d) = 0 and
// P(c s) = kc c with kc = <c^2 s> / <c^2> = (N + 2) / (4 lam); likewise in d.
template <class R>
GKS_FN void time_coef(const SolveK<R>& k, R i2N, const R X[4], const R Y[4], R T[4]) {
  T[0] = -(k.U * X[0] + k.V * Y[0]);
  T[1] = -(k.U * X[1] + k.V * Y[1] + X[0] + k.kc * X[3]);
  T[2] = -(k.U * X[2] + k.V * Y[2] + Y[0] + k.kc * Y[3]);
  T[3] = -(k.U * X[3] + k.V * Y[3] + i2N * (X[1] + Y[2]));
}

// ir = 1/rho of the Maxwellian, i2N = 2 / N.  The spatial coefficients by the closed-form
// solve; the time coefficients (the compatibility conditions of the system after Eq. dis3)
// by the projection above, in central coordinates, mapped back to the psi basis.
template <class R>
GKS_FN void coef_systems(R ir, const SolveK<R>& sk, R i2N, const R d[5][4], bool time_terms, bool second_time,
                         Coefs<R>& c) {
  const R c4i = sk.c4 * ir, l2i = sk.l2 * ir;
  solve_scaled(sk, c4i, l2i, ir, d[0], c.a1);
  solve_scaled(sk, c4i, l2i, ir, d[1], c.a2);
  solve_scaled(sk, c4i, l2i, ir, d[2], c.Axx);
  solve_scaled(sk, c4i, l2i, ir, d[3], c.Axy);
  solve_scaled(sk, c4i, l2i, ir, d[4], c.Ayy);
  if (!time_terms) return;
  R x[4], y[4], z[4], tx[4], ty[4], t[4];
  to_central(sk, c.a1, x);
  to_central(sk, c.a2, y);
  time_coef(sk, i2N, x, y, t);  // <A + a1 u + a2 v> = 0
  from_central(sk, t, c.A);
  to_central(sk, c.Axx, x);
  to_central(sk, c.Axy, y);
  to_central(sk, c.Ayy, z);
  time_coef(sk, i2N, x, y, tx);  // <Axx u + Axy v + Atx> = 0
  time_coef(sk, i2N, y, z, ty);  // <Axy u + Ayy v + Aty> = 0
  from_central(sk, tx, c.Atx);
  from_central(sk, ty, c.Aty);
  if (!second_time) return;
  time_coef(sk, i2N, tx, ty, t);  // <Atx u + Aty v + Att> = 0
  from_central(sk, t, c.Att);
}

// The interface distribution grouped by velocity monomial: f = sum over
// m in {1, u, v, u^2, u v, v^2} of X_m(psi) m g, plus y X'_m for the part
// linear along the face.  The moments of f are taken by expanding
// P = sum_m m X_m(psi) into monomials u^a v^b (xi^2)^c first (a + b <= 4 for
// c = 0, a + b <= 2 for c = 1) and then pairing each monomial with the moment
// table of g (moments factorise: <u^a v^b xi^2c> = <u^a><v^b><xi^2c>):
//   flux   += rho <u P psi>           (time-integrated weights)
//   point0 += rho <P psi>             (weights at t = dt)
//   point1 += rho <P' psi>            (weights at t = dt, y-linear part)
//   mean   += rho <P psi>             (time-integrated weights; heat flux)
template <class R>
struct Groups {
  R X1[4], Xu[4], Xv[4], Xuu[4], Xuv[4], Xvv[4];
};

// monomial coefficients: c0[(b, a)] for u^a v^b, a + b <= 4, stored by b then a
// (offsets 0, 5, 9, 12, 14); c1[(b, a)] for u^a v^b xi^2, a + b <= 2 (offsets 0, 3, 5)
template <class R>
struct Poly {
  R c0[15], c1[6];
};

GKS_FN constexpr int pidx0(int a, int b) { return (b == 0 ? 0 : b == 1 ? 5 : b == 2 ? 9 : b == 3 ? 12 : 14) + a; }
GKS_FN constexpr int pidx1(int a, int b) { return (b == 0 ? 0 : b == 1 ? 3 : 5) + a; }

// P of the six groups (FULL) or of the first three only (the y-linear part)
template <bool FULL, class R>
GKS_FN void poly_of(const Groups<R>& g, Poly<R>& P) {
  const R h1 = R(0.5) * g.X1[3], hu = R(0.5) * g.Xu[3], hv = R(0.5) * g.Xv[3];
  // X (psi) = X0 + X1 u + X2 v + X3 (u^2 + v^2 + xi^2) / 2, times the group's monomial
  P.c0[pidx0(0, 0)] = g.X1[0];
  P.c0[pidx0(1, 0)] = g.X1[1] + g.Xu[0];
  P.c0[pidx0(0, 1)] = g.X1[2] + g.Xv[0];
  P.c0[pidx0(2, 0)] = h1 + g.Xu[1];
  P.c0[pidx0(1, 1)] = g.Xu[2] + g.Xv[1];
  P.c0[pidx0(0, 2)] = h1 + g.Xv[2];
  P.c0[pidx0(3, 0)] = hu;
  P.c0[pidx0(2, 1)] = hv;
  P.c0[pidx0(1, 2)] = hu;
  P.c0[pidx0(0, 3)] = hv;
  P.c1[pidx1(0, 0)] = h1;
  P.c1[pidx1(1, 0)] = hu;
  P.c1[pidx1(0, 1)] = hv;
  if (FULL) {
    const R huu = R(0.5) * g.Xuu[3], huv = R(0.5) * g.Xuv[3], hvv = R(0.5) * g.Xvv[3];
    P.c0[pidx0(2, 0)] += g.Xuu[0];
    P.c0[pidx0(1, 1)] += g.Xuv[0];
    P.c0[pidx0(0, 2)] += g.Xvv[0];
    P.c0[pidx0(3, 0)] += g.Xuu[1];
    P.c0[pidx0(2, 1)] += g.Xuu[2] + g.Xuv[1];
    P.c0[pidx0(1, 2)] += g.Xuv[2] + g.Xvv[1];
    P.c0[pidx0(0, 3)] += g.Xvv[2];
    P.c0[pidx0(4, 0)] = huu;
    P.c0[pidx0(3, 1)] = huv;
    P.c0[pidx0(2, 2)] = huu + hvv;
    P.c0[pidx0(1, 3)] = huv;
    P.c0[pidx0(0, 4)] = hvv;
    P.c1[pidx1(2, 0)] = huu;
    P.c1[pidx1(1, 1)] = huv;
    P.c1[pidx1(0, 2)] = hvv;
  }
}

// out += rho <u^SU P psi>, psi = (1, u, v, (u^2 + v^2 + xi^2) / 2); D / D1: the
// degree of P in (u, v) for c = 0 / c = 1 (4 / 2, or 3 / 1 for the y-linear part).
// <xi^2> is a number, so the xi^2 monomials fold into the others: with
// q_ab = p0_ab + <xi^2> p1_ab, the first three components are sums of q_ab <u^a><v^b>;
// the fourth's extra xi^2 weight, sum p0 <xi^2> + p1 <xi^4>, is <xi^2> o0 + kap T with
// kap = <xi^4> - <xi^2>^2 and T = sum p1_ab <u^a><v^b> (u-moments shifted by SU).
template <int SU, int D, int D1, class R, int NU, int NV>
GKS_FN void poly_moments(const Poly<R>& P, const Moments<R, NU, NV>& m, R rho, R out[4]) {
  static_assert(D + SU + 2 < NU && D + 2 < NV, "moment table too short");
  R o0 = R(0), o1 = R(0), o2 = R(0), o3 = R(0);
#pragma unroll
  for (int b = 0; b <= D; ++b) {
    // sum_a q u^(a+SU), u^(a+SU+1), u^(a+SU+2) moments (the first term starts each sum)
    R s0 = R(0), s1 = R(0), s2 = R(0);
#pragma unroll
    for (int a = 0; a <= D - b; ++a) {
      const R q = a + b <= D1 ? P.c0[pidx0(a, b)] + m.xi2 * P.c1[pidx1(a, b)] : P.c0[pidx0(a, b)];
      s0 = a == 0 ? q * m.u[SU] : s0 + q * m.u[a + SU];
      s1 = a == 0 ? q * m.u[SU + 1] : s1 + q * m.u[a + SU + 1];
      s2 = a == 0 ? q * m.u[SU + 2] : s2 + q * m.u[a + SU + 2];
    }
    // <v^b>, <v^(b+1)>, <v^(b+2)> (v^0 = 1)
    if (b == 0) {
      o0 = s0;
      o1 = s1;
      o2 = s0 * m.v[1];
      o3 = s2 + s0 * m.v[2];
    } else {
      o0 = o0 + s0 * m.v[b];
      o1 = o1 + s1 * m.v[b];
      o2 = o2 + s0 * m.v[b + 1];
      o3 = o3 + s2 * m.v[b] + s0 * m.v[b + 2];
    }
  }
  R T = R(0);
#pragma unroll
  for (int b = 0; b <= D1; ++b) {
    R t = R(0);
#pragma unroll
    for (int a = 0; a <= D1 - b; ++a) t = a == 0 ? P.c1[pidx1(a, b)] * m.u[SU] : t + P.c1[pidx1(a, b)] * m.u[a + SU];
    T = b == 0 ? t : T + t * m.v[b];
  }
  out[0] += rho * o0;
  out[1] += rho * o1;
  out[2] += rho * o2;
  out[3] += rho * (R(0.5) * (o3 + m.xi2 * o0 + m.kap * T));
}

template <class R, int NU, int NV>
GKS_FN void add_flux(const Groups<R>& g, const Moments<R, NU, NV>& m, R rho, R out[4]) {
  Poly<R> P;
  poly_of<true>(g, P);
  poly_moments<1, 4, 2>(P, m, rho, out);
}

template <class R, int NU, int NV>
GKS_FN void add_point(const Groups<R>& g, const Moments<R, NU, NV>& m, R rho, R out[4]) {
  Poly<R> P;
  poly_of<true>(g, P);
  poly_moments<0, 4, 2>(P, m, rho, out);
}

// the same for groups whose u^2, u v, v^2 parts vanish
template <class R, int NU, int NV>
GKS_FN void add_point_first(const Groups<R>& g, const Moments<R, NU, NV>& m, R rho, R out[4]) {
  Poly<R> P;
  poly_of<false>(g, P);
  poly_moments<0, 3, 1>(P, m, rho, out);
}

template <class R, int NU, int NV>
GKS_FN void add_point_linear(const R Y1[4], const R Yu[4], const R Yv[4], const Moments<R, NU, NV>& m, R rho,
                             R out[4]) {
  Groups<R> g;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    g.X1[k] = Y1[k];
    g.Xu[k] = Yu[k];
    g.Xv[k] = Yv[k];
  }
  Poly<R> P;
  poly_of<false>(g, P);
  poly_moments<0, 3, 1>(P, m, rho, out);
}

// Eq. dis1 grouped: weights W = I (flux, mean) or E (point); y2 = dtan^2/12 is both
// the face mean of y^2 and y^2 at the Gauss points.
// SECOND = false: W[4] = 0, the groups of u^2, u v, v^2 vanish and are not formed.
template <bool SECOND = true, class R>
GKS_FN void hydro_groups(const Coefs<R>& c, const R* W, R y2, Groups<R>& g) {
  const R h5 = R(0.5) * W[5], hy = R(0.5) * y2 * W[1], h4 = R(0.5) * W[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    g.X1[k] = W[3] * c.A[k] + h5 * c.Att[k] + hy * c.Ayy[k];
    g.Xu[k] = W[2] * c.a1[k] + W[6] * c.Atx[k];
    g.Xv[k] = W[2] * c.a2[k] + W[6] * c.Aty[k];
    if (SECOND) {
      g.Xuu[k] = h4 * c.Axx[k];
      g.Xuv[k] = W[4] * c.Axy[k];
      g.Xvv[k] = h4 * c.Ayy[k];
    }
  }
  g.X1[0] += W[1];
}

// Eq. dis2 grouped for one side.  NS: f_G = g_k - tau (a u + A) g_k with the time
// coefficients c.A, c.Atx, c.Aty and tn = tau; Euler: f_G = g_k, and the terms
// with tn are absent (not formed).
template <bool NS, class R>
GKS_FN void kinetic_groups(const Coefs<R>& c, const R* W, R y2, R tn, Groups<R>& g) {
  const R h7 = R(0.5) * y2 * W[7];
  if (NS) {
    const R t7 = tn * W[7], t8 = tn * W[8];
    const R w78 = W[8] - t7, wq = R(0.5) * W[10] - t8, wq2 = W[10] - R(2) * t8;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      g.X1[k] = h7 * c.Ayy[k] - t7 * c.A[k];
      g.Xu[k] = w78 * c.a1[k] - t8 * c.Atx[k];
      g.Xv[k] = w78 * c.a2[k] - t8 * c.Aty[k];
      g.Xuu[k] = wq * c.Axx[k];
      g.Xuv[k] = wq2 * c.Axy[k];
      g.Xvv[k] = wq * c.Ayy[k];
    }
  } else {
    const R wq = R(0.5) * W[10];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      g.X1[k] = h7 * c.Ayy[k];
      g.Xu[k] = W[8] * c.a1[k];
      g.Xv[k] = W[8] * c.a2[k];
      g.Xuu[k] = wq * c.Axx[k];
      g.Xuv[k] = W[10] * c.Axy[k];
      g.Xvv[k] = wq * c.Ayy[k];
    }
  }
  g.X1[0] += W[7];
}

// ---------------------------------------------------------------------------
// Face states in the face frame: value and (dn, dt, dnn, dnt, dtt)
// ---------------------------------------------------------------------------
template <class R>
struct FaceState {
  R w[6][4];
};

template <class R>
GKS_FN void prim(const R w[4], R gm1, R& rho, R& ir, R& U, R& V, R& p) {
  rho = w[0];
  ir = d_div(R(1), rho);
  U = w[1] * ir;
  V = w[2] * ir;
  p = gm1 * (w[3] - R(0.5) * (w[1] * U + w[2] * V));
}

struct FaceParams {
  double gamma, mu, Pr, tau_eps, tau_C;
  double dn, dtan;  // cell size normal to and along the face
};

// Per-launch constants of the face routine in the compute type
template <class R>
struct FaceConst {
  R gamma, gm1, K, N, iN, i2N, dn, dtan, y2, mu, pr_fix, tau_eps, tau_C;
  R dn2_12, dt2_24;             // dn^2 / 12, dtan^2 / 24 (face values of the cell polynomial)
  R i4n, i4t, i8n2, i2nt, i2t2;  // 1/(4 dn), 1/(4 dt), 1/(8 dn^2), 1/(2 dn dt), 1/(2 dt^2)
  bool ns, prandtl;
};

template <class R>
GKS_FN FaceConst<R> face_const(const FaceParams& P) {
  FaceConst<R> c;
  c.gamma = R(P.gamma);
  c.gm1 = R(P.gamma - 1.0);
  c.K = R((4.0 - 2.0 * P.gamma) / (P.gamma - 1.0));  // internal degrees of freedom, Section 2.1
  c.N = R(2.0 / (P.gamma - 1.0));                     // K + 2
  c.iN = R(0.5 * (P.gamma - 1.0));
  c.i2N = R(P.gamma - 1.0);  // 2 / N
  c.dn = R(P.dn);
  c.dtan = R(P.dtan);
  c.y2 = R(P.dtan * P.dtan / 12.0);
  c.dn2_12 = R(P.dn * P.dn / 12.0);
  c.dt2_24 = R(P.dtan * P.dtan / 24.0);
  c.i4n = R(1.0 / (4.0 * P.dn));
  c.i4t = R(1.0 / (4.0 * P.dtan));
  c.i8n2 = R(1.0 / (8.0 * P.dn * P.dn));
  c.i2nt = R(1.0 / (2.0 * P.dn * P.dtan));
  c.i2t2 = R(1.0 / (2.0 * P.dtan * P.dtan));
  c.mu = R(P.mu);
  c.pr_fix = R(1.0 / P.Pr - 1.0);
  c.tau_eps = R(P.tau_eps);
  c.tau_C = R(P.tau_C);
  c.ns = P.mu > 0.0;
  c.prandtl = P.Pr != 1.0;
  return c;
}

// A face source over the two sides and the six averages of one face, for
// callers that hold them in arrays (the host operation count).
template <class R>
struct ArrayFaceSource {
  const FaceState<R>* s[2];
  const R (*a)[3][4];
  GKS_FN void side(int k, FaceState<R>& out) const { out = *s[k]; }
  GKS_FN void avg(R out[2][3][4]) const {
    for (int m = 0; m < 2; ++m)
      for (int n = 0; n < 3; ++n)
        for (int v = 0; v < 4; ++v) out[m][n][v] = a[m][n][v];
  }
};

// Wall images G(n, t) = Phi(P(-n, t)) of the inside face state (face frame).
// kind 2: slip wall (normal momentum negated).  kind 3: isothermal no-slip with
// tangential wall velocity uwt and wall temperature Tw: rho' = rho,
// m' = 2 rho u_w - m, rho E' = 2 rho |u_w|^2 - 2 u_w.m + |m|^2/rho + 2 rho Tw/(gamma-1) - rho E.
// kind 4: adiabatic no-slip: rho' = rho, m' = 2 rho u_w - m, T' = T (a linear map).
template <class R>
GKS_FN void wall_image(int kind, R gamma, R uwt, R Tw, const FaceState<R>& in, FaceState<R>& out) {
  if (kind == 2) {
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const R s = (d == 1 || d == 4) ? R(-1) : R(1);  // odd derivatives in n flip
      out.w[d][0] = s * in.w[d][0];
      out.w[d][1] = -s * in.w[d][1];
      out.w[d][2] = s * in.w[d][2];
      out.w[d][3] = s * in.w[d][3];
    }
    return;
  }
  if (kind == 4) {
    // adiabatic no-slip: the linear map rho' = rho, m_n' = -m_n, m_t' = 2 u_w rho - m_t,
    // rho E' = rho E + 2 u_w^2 rho - 2 u_w m_t applied to the value and every derivative
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const R s = (d == 1 || d == 4) ? R(-1) : R(1);  // odd derivatives in n flip
      const R r = in.w[d][0], mn = in.w[d][1], mt = in.w[d][2], e = in.w[d][3];
      out.w[d][0] = s * r;
      out.w[d][1] = -s * mn;
      out.w[d][2] = s * (R(2) * uwt * r - mt);
      out.w[d][3] = s * (e + R(2) * uwt * uwt * r - R(2) * uwt * mt);
    }
    return;
  }
  const R rho = in.w[0][0], mn = in.w[0][1], mt = in.w[0][2];
  const R ir = d_div(R(1), rho);
  const R m2 = mn * mn + mt * mt;
  const R cT = d_div(R(2) * Tw, gamma - R(1));
  // value
  out.w[0][0] = rho;
  out.w[0][1] = -mn;
  out.w[0][2] = R(2) * rho * uwt - mt;
  out.w[0][3] = R(2) * rho * uwt * uwt - R(2) * uwt * mt + m2 * ir + rho * cT - in.w[0][3];
  // Jacobian rows applied to a derivative vector a
  auto lin = [&](const R a[4], R o[4]) {
    o[0] = a[0];
    o[1] = -a[1];
    o[2] = R(2) * uwt * a[0] - a[2];
    o[3] = (R(2) * uwt * uwt - m2 * ir * ir + cT) * a[0] + R(2) * mn * ir * a[1] +
           (R(2) * mt * ir - R(2) * uwt) * a[2] - a[3];
  };
  // second derivative of |m|^2/rho along a, b
  auto hess = [&](const R a[4], const R b[4]) {
    const R ma = mn * a[1] + mt * a[2], mb = mn * b[1] + mt * b[2];
    return R(2) * m2 * ir * ir * ir * a[0] * b[0] - R(2) * ir * ir * (ma * b[0] + mb * a[0]) +
           R(2) * ir * (a[1] * b[1] + a[2] * b[2]);
  };
  R o[4];
  lin(in.w[1], o);
#pragma unroll
  for (int k = 0; k < 4; ++k) out.w[1][k] = -o[k];
  lin(in.w[2], o);
#pragma unroll
  for (int k = 0; k < 4; ++k) out.w[2][k] = o[k];
  lin(in.w[3], o);
#pragma unroll
  for (int k = 0; k < 4; ++k) out.w[3][k] = o[k];
  out.w[3][3] += hess(in.w[1], in.w[1]);
  lin(in.w[4], o);
#pragma unroll
  for (int k = 0; k < 4; ++k) out.w[4][k] = -o[k];
  out.w[4][3] -= hess(in.w[1], in.w[2]);
  lin(in.w[5], o);
#pragma unroll
  for (int k = 0; k < 4; ++k) out.w[5][k] = o[k];
  out.w[5][3] += hess(in.w[2], in.w[2]);
}

// ---------------------------------------------------------------------------
// Section 2.2 at one face centre.  The two sides (value and derivatives in the
// face frame) and the six cell averages of Section 3.3 (avg[m][k], m = 0 left,
// 1 right; k = tangential -1, 0, 1) come from src.side(k, S) and src.avg(a),
// which are called where they are needed so that they need not stay live in
// registers.  Outputs the time-integrated face-mean flux and the point values
// at the two Gauss points (tangential -/+ sqrt(3)/6 dtan) at t = dt.
// NSM: 1 Navier-Stokes, 0 Euler (mu = 0: the terms of the time derivatives of
// g_k vanish and are not formed), -1 decided at run time by C.ns.
// ---------------------------------------------------------------------------
template <class R, int NSM = -1, class Src>
GKS_FN void face_evolution(const FaceConst<R>& C, const Src& src, R dt, R F[4], R Wm[4], R Wp[4]) {
  const bool ns = NSM < 0 ? C.ns : NSM == 1;
  // per side: rho, 1/rho, U, V, lam = rho / (2 p), 1 / (2 lam) = p / rho, p, and the
  // half-space <u^0>, <u^1>
  R rs[2], irs[2], us[2], vs[2], ls[2], vrs[2], ps[2], h0[2], h1[2];
  R U0[4] = {R(0), R(0), R(0), R(0)};
  // Eq. compatibility2: U0 = rho_l <psi>_{u>0} + rho_r <psi>_{u<0}
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    FaceState<R> S;
    src.side(k, S);
    prim(S.w[0], C.gm1, rs[k], irs[k], us[k], vs[k], ps[k]);
    ls[k] = d_div(R(0.5) * rs[k], ps[k]);
    vrs[k] = ps[k] * irs[k];
    Moments<R, 4, 3> m;
    moments(us[k], vs[k], ls[k], vrs[k], C.K, k == 0 ? +1 : -1, m);
    h0[k] = m.u[0];
    h1[k] = m.u[1];
    R a[4];
    psi_mom<0, 0>(m, a);
#pragma unroll
    for (int v = 0; v < 4; ++v) U0[v] += rs[k] * a[v];
  }
  R r0, ir0, u0, v0, p0;
  prim(U0, C.gm1, r0, ir0, u0, v0, p0);
  const R lam0 = d_div(R(0.5) * r0, p0), var0 = p0 * ir0;

  // Section 4: collision time
  const R jump = fabs(d_div(ps[0] - ps[1], ps[0] + ps[1])) * dt;
  const R tau = ns ? d_div(C.mu, p0) + jump : C.tau_eps * dt + C.tau_C * jump;
  const R tn = ns ? tau : R(0);

  TimeW<R> tw;
  time_weights(dt, tau, tw);
  // e = exp(-dt/tau) >= 0 underflows to exactly 0 once tau is a small enough fraction of dt
  // (smooth Euler flow); the point-value terms whose weights carry it are then not formed
  const bool kin_point = tw.E[7] > R(0);

  R Fl[4] = {0, 0, 0, 0}, P0[4] = {0, 0, 0, 0}, P1[4] = {0, 0, 0, 0}, Mn[4] = {0, 0, 0, 0};

  // ---- equilibrium part, Eq. dis1, with g0 and the polynomial of Section 3.3 ----
  {
    R d[5][4];
    {
      R avg[2][3][4];
      src.avg(avg);
      const R i4n = C.i4n, i4t = C.i4t, i8n2 = C.i8n2, i2nt = C.i2nt, i2t2 = C.i2t2;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const R um = avg[0][0][k], uc = avg[0][1][k], up = avg[0][2][k];
        const R wm = avg[1][0][k], wc = avg[1][1][k], wp = avg[1][2][k];
        d[0][k] = ((wp - up) + R(2) * (wc - uc) + (wm - um)) * i4n;                // b2
        d[1][k] = (wp - wm + up - um) * i4t;                                       // b3
        d[2][k] = (R(26) * (wc + uc) - (wp + up + wm + um) - R(48) * U0[k]) * i8n2;  // b4
        d[3][k] = (wp - up - wm + um) * i2nt;                                      // b6
        d[4][k] = (wp - R(2) * wc + wm + up - R(2) * uc + um) * i2t2;               // b5
      }
    }
    Moments<R, 8, 7> m;
    moments(u0, v0, lam0, var0, C.K, 0, m);
    Coefs<R> c;
    coef_systems(ir0, solve_k(u0, v0, lam0, var0, C.N, C.iN), C.i2N, d, true, true, c);
    Groups<R> g;
    hydro_groups(c, tw.I, C.y2, g);
    add_flux(g, m, r0, Fl);
    if (C.prandtl) add_point(g, m, r0, Mn);
    if (kin_point) {
      hydro_groups(c, tw.E, C.y2, g);
      add_point(g, m, r0, P0);
    } else {
      // e = exp(-dt/tau) = 0: the weight of the second-order groups at t = dt, -(dt^2 + 2 dt tau) e,
      // is exactly 0
      hydro_groups<false>(c, tw.E, C.y2, g);
      add_point_first(g, m, r0, P0);
    }
    R Y1[4], Yu[4], Yv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Y1[k] = tw.E[1] * c.a2[k] + tw.E[3] * c.Aty[k];
      Yu[k] = tw.E[2] * c.Axy[k];
      Yv[k] = tw.E[2] * c.Ayy[k];
    }
    add_point_linear(Y1, Yu, Yv, m, r0, P1);
  }

  // ---- kinetic part, Eq. dis2, for both sides ----
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    // selects, not indexing: a dynamic index would put these arrays in local memory
    const R rho = side ? rs[1] : rs[0], U = side ? us[1] : us[0];
    const R V = side ? vs[1] : vs[0], lam = side ? ls[1] : ls[0];
    const R ir = side ? irs[1] : irs[0], var = side ? vrs[1] : vrs[0];
    Coefs<R> c;
    {
      R d[5][4];
      {
        FaceState<R> S;
        src.side(side, S);
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
          for (int k = 0; k < 4; ++k) d[q][k] = S.w[q + 1][k];
      }
      // the time coefficients of g_k (NS only)
      coef_systems(ir, solve_k(U, V, lam, var, C.N, C.iN), C.i2N, d, ns, false, c);
    }
    Moments<R, 8, 7> mh;
    moments_from(U, V, var, C.K, side ? h0[1] : h0[0], side ? h1[1] : h1[0], mh);
    Groups<R> g;
    if (ns) kinetic_groups<true>(c, tw.I, C.y2, tn, g);
    else kinetic_groups<false>(c, tw.I, C.y2, tn, g);
    add_flux(g, mh, rho, Fl);
    if (C.prandtl) add_point(g, mh, rho, Mn);
    // Every weight of the kinetic part at t = dt carries e = exp(-dt/tau), which underflows to
    // exactly 0 once tau is a small enough fraction of dt (smooth Euler flow): the point
    // values then get exactly nothing from this side
    if (kin_point) {
      R Y1[4], Yu[4], Yv[4];
      if (ns) {
        kinetic_groups<true>(c, tw.E, C.y2, tn, g);
        add_point(g, mh, rho, P0);
        const R wy = -tn * tw.E[7] - tw.E[9];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          Y1[k] = tw.E[7] * (c.a2[k] - tn * c.Aty[k]);
          Yu[k] = wy * c.Axy[k];
          Yv[k] = wy * c.Ayy[k];
        }
      } else {
        kinetic_groups<false>(c, tw.E, C.y2, tn, g);
        add_point(g, mh, rho, P0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          Y1[k] = tw.E[7] * c.a2[k];
          Yu[k] = -tw.E[9] * c.Axy[k];
          Yv[k] = -tw.E[9] * c.Ayy[k];
        }
      }
      add_point_linear(Y1, Yu, Yv, mh, rho, P1);
    }
  }

  // Prandtl-number fix: energy flux += (1/Pr - 1) q, q the time-integrated
  // face-mean heat flux (1/2) int (u-U0)((u-U0)^2+(v-V0)^2+xi^2) f, written with the
  // flux and the time-integrated conservative moments.
  if (C.prandtl) {
    const R q2 = u0 * u0 + v0 * v0;
    const R q = Fl[3] - u0 * Fl[1] - v0 * Fl[2] + (R(0.5) * q2 + u0 * u0) * Fl[0] - u0 * Mn[3] +
                u0 * v0 * Mn[2] - R(0.5) * u0 * q2 * Mn[0];
    Fl[3] += C.pr_fix * q;
  }
  const R yg = R(0.28867513459481287) * C.dtan;  // sqrt(3)/6
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    F[k] = Fl[k];
    Wm[k] = P0[k] - yg * P1[k];
    Wp[k] = P0[k] + yg * P1[k];
  }
}

// ---------------------------------------------------------------------------
// Section 3.2: compact reconstruction of one variable of one cell.
// c: cell average; e, w, n, s: neighbour averages; em/ep: east-face Gauss
// values (y-/y+), wm/wp west face, nm/np north face (x-/x+), sm/sp south face.
// Output a[0..4] = (a2, a3, a4, a5, a6) of
//   U(x,y) = c + a2 x + a3 y + a4 (x^2-dx^2/12)/2 + a5 (y^2-dy^2/12)/2 + a6 x y.
// ---------------------------------------------------------------------------
template <class R>
GKS_FN R minmod(R a, R b) {
  return a * b > R(0) ? (fabs(a) < fabs(b) ? a : b) : R(0);
}

// Cell-size constants of the reconstruction, formed once per cell (not per variable)
template <class R>
struct ReconK {
  R dx, dy, idx, idy;
  R dx6, dy6;          // dx / 6, dy / 6
  R r3;                // sqrt(3) / (dx dy)
  R idx2, idy2;        // 1 / dx^2, 1 / dy^2
  R dx2, dy2;          // smoothness indicator: weights of c2^2, c3^2,
  R kc4, kc5, kc6;     //   c4^2 (13/12 dx^4), c5^2 (13/12 dy^4), c6^2 (7/6 dx^2 dy^2)
  R dx2_12, dy2_12;    // dx^2 / 12, dy^2 / 12 (face values of the polynomial)
  R weps, b1sq;        // eps and (eps + I(U1))^2, I(U1) = C dx dy
};

// idx, idy: 1/dx, 1/dy of the grid (formed once on the host)
template <class R>
GKS_FN ReconK<R> recon_k(R dx, R dy, R idx, R idy, R weps, R wC) {
  ReconK<R> k;
  k.dx = dx;
  k.dy = dy;
  k.idx = idx;
  k.idy = idy;
  k.idx2 = idx * idx;
  k.idy2 = idy * idy;
  k.dx6 = dx * R(1.0 / 6.0);
  k.dy6 = dy * R(1.0 / 6.0);
  k.r3 = R(1.7320508075688772) * idx * idy;  // sqrt(3) / (dx dy)
  k.dx2 = dx * dx;
  k.dy2 = dy * dy;
  k.kc4 = R(13.0 / 12.0) * k.dx2 * k.dx2;
  k.kc5 = R(13.0 / 12.0) * k.dy2 * k.dy2;
  k.kc6 = R(7.0 / 6.0) * k.dx2 * k.dy2;
  k.dx2_12 = k.dx2 * R(1.0 / 12.0);
  k.dy2_12 = k.dy2 * R(1.0 / 12.0);
  k.weps = weps;
  const R b1 = weps + wC * dx * dy;
  k.b1sq = b1 * b1;
  return k;
}

template <class R>
GKS_FN void recon_var(R c, R e, R w, R n, R s, R em, R ep, R wm, R wp, R nm, R np, R sm, R sp,
                      const ReconK<R>& K, R a[5]) {
  // one-sided stencils (Eq. over-sys) from each face's Gauss-point sum (twice its mean) and
  // the neighbour average
  const R se = em + ep, sw = wm + wp, sn = nm + np, ss = sm + sp;
  const R a4 = minmod(R(3) * (c + w - sw) * K.idx2, R(3) * (c + e - se) * K.idx2);
  const R a2 = minmod((R(2) * c - sw) * K.idx + a4 * K.dx6, (se - R(2) * c) * K.idx - a4 * K.dx6);
  const R a5 = minmod(R(3) * (c + s - ss) * K.idy2, R(3) * (c + n - sn) * K.idy2);
  const R a3 = minmod((R(2) * c - ss) * K.idy + a5 * K.dy6, (sn - R(2) * c) * K.idy - a5 * K.dy6);
  // cross derivative of the four one-sided stencils with limited a2, a3:
  // sx (sqrt3 Dx/(dx dy) - a3/dx) + sy (sqrt3 Dy/(dx dy) - a2/dy), smallest magnitude
  const R xe = K.r3 * (ep - em) - a3 * K.idx, xw = K.r3 * (wp - wm) - a3 * K.idx;
  const R yn = K.r3 * (np - nm) - a2 * K.idy, ys = K.r3 * (sp - sm) - a2 * K.idy;
  // magnitudes within a relative Prec<R>::tie of the current choice are ties
  // (piecewise constant data give exact ties of opposite sign); the earlier
  // stencil is kept
  const R keep = R(1) - R(Prec<R>::tie);
  R a6 = xe + yn;        // (+, +)
  R cand = -xw + yn;     // (-, +)
  if (fabs(cand) < fabs(a6) * keep) a6 = cand;
  cand = -xw - ys;       // (-, -)
  if (fabs(cand) < fabs(a6) * keep) a6 = cand;
  cand = xe - ys;        // (+, -)
  if (fabs(cand) < fabs(a6) * keep) a6 = cand;
  // central stencil
  const R c2 = R(0.5) * (e - w) * K.idx, c4 = (e - R(2) * c + w) * K.idx2;
  const R c3 = R(0.5) * (n - s) * K.idy, c5 = (n - R(2) * c + s) * K.idy2;
  const R c6 = R(0.5) * K.r3 * ((ep - em) - (wp - wm) + (np - nm) - (sp - sm));
  // Eq. average: alpha = 1/(eps + I)^2, I(U1) = C dx dy; I(U2), the integral of the
  // squared first and second derivatives of the central polynomial over the cell scaled
  // by |Omega|, collected by coefficient
  const R I2 = c2 * (K.dx2 * c2) + c3 * (K.dy2 * c3) + c4 * (K.kc4 * c4) + c5 * (K.kc5 * c5) + c6 * (K.kc6 * c6);
  const R b2 = K.weps + I2, b2sq = b2 * b2;
  // w1 = (1/b1^2) / (1/b1^2 + 1/b2^2) = b2^2 / (b1^2 + b2^2); a = c + w1 (a_one-sided - c)
  const R w1 = d_div(b2sq, K.b1sq + b2sq);
  a[0] = c2 + w1 * (a2 - c2);
  a[1] = c3 + w1 * (a3 - c3);
  a[2] = c4 + w1 * (a4 - c4);
  a[3] = c5 + w1 * (a5 - c5);
  a[4] = c6 + w1 * (a6 - c6);
}

}  // namespace gks
