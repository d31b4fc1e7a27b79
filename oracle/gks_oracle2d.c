/*
 * Two-dimensional oracle of the compact third-order gas-kinetic scheme
 * (Pan & Xu, arXiv:1412.4489).  TEST INFRASTRUCTURE ONLY: a plain, slow FP64
 * restatement of the paper, loaded only by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark.  No code is shared with the CUDA library.
 *
 * Organisation follows the paper:
 *   Section 2.1  Maxwellian, psi, K and the moments <.> = int g (.) psi dXi
 *   Section 2.2  coefficient systems, C_1..C_8, Eq. dis1 (hydrodynamic part),
 *                Eq. dis2 (kinetic part), Eq. compatibility2 (U_0), Eq. point
 *   Section 3.2  compact 2D reconstruction, Eq. over-sys, limiter, weights
 *   Section 3.3  equilibrium polynomial b_2..b_6
 *   Section 4    collision time tau, CFL time step
 *   Eq. finite   conservative update
 * Velocity moments are taken by expanding every integrand into monomials
 * u^p v^q (xi^2)^r and summing products of one-dimensional Gaussian moments,
 * which is the plain definition of each moment.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "gks_oracle.h"

#define NMOM 10
#define PCAP 320

/* ------------------------------------------------------------------ */
/* Section 2.1: Maxwellian g = rho (lam/pi)^((K+2)/2) exp(-lam((u-U)^2+(v-V)^2+xi^2)) */
/* ------------------------------------------------------------------ */
typedef struct {
  double rho, U, V, lam, K;
  double mu[3][NMOM]; /* <u^n>/rho: [0] full space, [1] u>0, [2] u<0 */
  double mv[NMOM];    /* <v^n>/rho over the full space */
  double mxi[3];      /* <1>, <xi^2>, <xi^4> of the K internal degrees of freedom */
} maxw;

static void maxw_set(maxw* m, double rho, double U, double V, double lam, double K) {
  m->rho = rho; m->U = U; m->V = V; m->lam = lam; m->K = K;
  const double var = 1.0 / (2.0 * lam); /* variance of each velocity component */
  const double root = sqrt(lam);
  const double edge = exp(-lam * U * U) / (2.0 * sqrt(M_PI * lam));
  m->mu[0][0] = 1.0;
  m->mu[0][1] = U;
  m->mu[1][0] = 0.5 * erfc(-root * U);
  m->mu[1][1] = U * m->mu[1][0] + edge;
  m->mu[2][0] = 0.5 * erfc(root * U);
  m->mu[2][1] = U * m->mu[2][0] - edge;
  m->mv[0] = 1.0;
  m->mv[1] = V;
  /* integration by parts of u^(n-1) (u-U) exp(-lam (u-U)^2): the boundary term
   * vanishes at u = 0 for n >= 2, so one recursion serves all three ranges */
  for (int n = 2; n < NMOM; ++n) {
    for (int h = 0; h < 3; ++h) m->mu[h][n] = U * m->mu[h][n - 1] + (n - 1) * var * m->mu[h][n - 2];
    m->mv[n] = V * m->mv[n - 1] + (n - 1) * var * m->mv[n - 2];
  }
  m->mxi[0] = 1.0;
  m->mxi[1] = K * var;
  m->mxi[2] = K * (K + 2.0) * var * var;
}

/* conservative (rho, rho U, rho V, rho E) -> Maxwellian parameters;
 * rho E = rho (U^2+V^2)/2 + (K+2) rho / (4 lam) */
static void maxw_from_cons(maxw* m, const double w[4], double K) {
  const double rho = w[0], U = w[1] / rho, V = w[2] / rho;
  const double lam = (K + 2.0) * rho / (4.0 * (w[3] - 0.5 * rho * (U * U + V * V)));
  maxw_set(m, rho, U, V, lam, K);
}

/* ------------------------------------------------------------------ */
/* Polynomials in (u, v, xi^2): sums of c u^p v^q (xi^2)^r               */
/* ------------------------------------------------------------------ */
typedef struct { double c; int p, q, r; } term;
typedef struct { int n; term t[PCAP]; } poly;

/* terms are appended, not merged: a moment is linear, so repeated monomials
 * simply contribute twice */
static void poly_add(poly* a, double c, int p, int q, int r) {
  if (c == 0.0) return;
  if (a->n >= PCAP) abort();
  a->t[a->n].c = c; a->t[a->n].p = p; a->t[a->n].q = q; a->t[a->n].r = r; a->n++;
}

static void poly_mul(const poly* a, const poly* b, poly* out) {
  out->n = 0;
  for (int i = 0; i < a->n; ++i)
    for (int j = 0; j < b->n; ++j)
      poly_add(out, a->t[i].c * b->t[j].c, a->t[i].p + b->t[j].p, a->t[i].q + b->t[j].q,
               a->t[i].r + b->t[j].r);
}

/* psi = (1, u, v, (u^2+v^2+xi^2)/2) */
static void poly_psi(int beta, poly* out) {
  out->n = 0;
  switch (beta) {
    case 0: poly_add(out, 1.0, 0, 0, 0); break;
    case 1: poly_add(out, 1.0, 1, 0, 0); break;
    case 2: poly_add(out, 1.0, 0, 1, 0); break;
    default:
      poly_add(out, 0.5, 2, 0, 0);
      poly_add(out, 0.5, 0, 2, 0);
      poly_add(out, 0.5, 0, 0, 1);
  }
}

/* a coefficient expanded in psi: X0 + X1 u + X2 v + X3 (u^2+v^2+xi^2)/2 */
static void poly_coef(const double X[4], poly* out) {
  out->n = 0;
  poly_add(out, X[0], 0, 0, 0);
  poly_add(out, X[1], 1, 0, 0);
  poly_add(out, X[2], 0, 1, 0);
  poly_add(out, 0.5 * X[3], 2, 0, 0);
  poly_add(out, 0.5 * X[3], 0, 2, 0);
  poly_add(out, 0.5 * X[3], 0, 0, 1);
}

static void poly_mono(double c, int p, int q, poly* out) {
  out->n = 0;
  poly_add(out, c, p, q, 0);
}

/* normalised moment of a polynomial: int g P dXi / rho over the chosen u-range */
static double maxw_mom(const maxw* m, int half, const poly* a) {
  double s = 0.0;
  for (int k = 0; k < a->n; ++k) {
    const term* t = &a->t[k];
    if (t->p >= NMOM || t->q >= NMOM || t->r > 2) abort();
    s += t->c * m->mu[half][t->p] * m->mv[t->q] * m->mxi[t->r];
  }
  return s;
}

/* normalised 4-vector int g P psi dXi / rho */
static void maxw_mom4(const maxw* m, int half, const poly* a, double out[4]) {
  poly ps, prod;
  for (int b = 0; b < 4; ++b) {
    poly_psi(b, &ps);
    poly_mul(a, &ps, &prod);
    out[b] = maxw_mom(m, half, &prod);
  }
}

/* 4-vector <X u^p v^q psi>/rho over the full space */
static void mom4_coef_mono(const maxw* m, int half, const double X[4], int p, int q, double out[4]) {
  poly px, pm, prod;
  poly_coef(X, &px);
  poly_mono(1.0, p, q, &pm);
  poly_mul(&px, &pm, &prod);
  maxw_mom4(m, half, &prod, out);
}

/* ------------------------------------------------------------------ */
/* Coefficient systems <a> = rhs (Section 2.2, system after Eq. dis3)   */
/* ------------------------------------------------------------------ */
static void solve4(double M[4][5], double x[4]) {
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (piv != c)
      for (int k = 0; k < 5; ++k) { double t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t; }
    for (int r = c + 1; r < 4; ++r) {
      const double f = M[r][c] / M[c][c];
      for (int k = c; k < 5; ++k) M[r][k] -= f * M[c][k];
    }
  }
  for (int r = 3; r >= 0; --r) {
    double s = M[r][4];
    for (int k = r + 1; k < 4; ++k) s -= M[r][k] * x[k];
    x[r] = s / M[r][r];
  }
}

/* solve M a = r with M_{beta alpha} = <psi_alpha psi_beta>/rho (r already / rho) */
static void maxw_solve(const maxw* m, const double r[4], double a[4]) {
  double M[4][5];
  poly pa, pb, prod;
  for (int b = 0; b < 4; ++b) {
    poly_psi(b, &pb);
    for (int al = 0; al < 4; ++al) {
      poly_psi(al, &pa);
      poly_mul(&pa, &pb, &prod);
      M[b][al] = maxw_mom(m, 0, &prod);
    }
    M[b][4] = r[b];
  }
  solve4(M, a);
}

/* The nine coefficients of one equilibrium state.  Composite symbols of the
 * paper ((a1^2+d11), (a1 a2+d12), (a2^2+d22), (A a1+b1), (A a2+b2), (A^2+B))
 * are each one unknown expanded in psi, as they appear in Eq. dis1 / dis2. */
typedef struct {
  double a1[4], a2[4], Axx[4], Axy[4], Ayy[4], A[4], Atx[4], Aty[4], Att[4];
} coefs;

/* d[0..4] = dU/dn, dU/dt, d2U/dn2, d2U/dndt, d2U/dt2 of the conservative variables */
static void coefs_solve(const maxw* m, const double d[5][4], coefs* c) {
  double r[4], t1[4], t2[4];
  const double irho = 1.0 / m->rho;
  for (int k = 0; k < 4; ++k) r[k] = d[0][k] * irho;
  maxw_solve(m, r, c->a1);                             /* <a1> = dU/dx */
  for (int k = 0; k < 4; ++k) r[k] = d[1][k] * irho;
  maxw_solve(m, r, c->a2);                             /* <a2> = dU/dy */
  for (int k = 0; k < 4; ++k) r[k] = d[2][k] * irho;
  maxw_solve(m, r, c->Axx);                            /* <a1^2+d11> = d2U/dx2 */
  for (int k = 0; k < 4; ++k) r[k] = d[4][k] * irho;
  maxw_solve(m, r, c->Ayy);                            /* <a2^2+d22> = d2U/dy2 */
  for (int k = 0; k < 4; ++k) r[k] = d[3][k] * irho;
  maxw_solve(m, r, c->Axy);                            /* <a1 a2+d12> = d2U/dxdy */
  /* <A + a1 u + a2 v> = 0 */
  mom4_coef_mono(m, 0, c->a1, 1, 0, t1);
  mom4_coef_mono(m, 0, c->a2, 0, 1, t2);
  for (int k = 0; k < 4; ++k) r[k] = -(t1[k] + t2[k]);
  maxw_solve(m, r, c->A);
  /* <(a1^2+d11) u + (a1 a2+d12) v + (A a1+b1)> = 0 */
  mom4_coef_mono(m, 0, c->Axx, 1, 0, t1);
  mom4_coef_mono(m, 0, c->Axy, 0, 1, t2);
  for (int k = 0; k < 4; ++k) r[k] = -(t1[k] + t2[k]);
  maxw_solve(m, r, c->Atx);
  /* <(a1 a2+d12) u + (a2^2+d22) v + (A a2+b2)> = 0 */
  mom4_coef_mono(m, 0, c->Axy, 1, 0, t1);
  mom4_coef_mono(m, 0, c->Ayy, 0, 1, t2);
  for (int k = 0; k < 4; ++k) r[k] = -(t1[k] + t2[k]);
  maxw_solve(m, r, c->Aty);
  /* <(A a1+b1) u + (A a2+b2) v + (A^2+B)> = 0 */
  mom4_coef_mono(m, 0, c->Atx, 1, 0, t1);
  mom4_coef_mono(m, 0, c->Aty, 0, 1, t2);
  for (int k = 0; k < 4; ++k) r[k] = -(t1[k] + t2[k]);
  maxw_solve(m, r, c->Att);
}

/* ------------------------------------------------------------------ */
/* Time coefficients C_1..C_8 (Section 2.2) and their integrals          */
/* index 9 = C_7 t, index 10 = C_7 t^2 (from the (-ut), (y-vt) factors   */
/* of the last line of Eq. dis2)                                          */
/* ------------------------------------------------------------------ */
enum { T1 = 1, T2, T3, T4, T5, T6, T7, T8, T7T, T7T2 };

/* exp(-t/tau), with tau = 0 (collision-free limit of the inviscid collision
 * time when epsilon = 0 and the two pressures agree) giving 0 */
static double decay(double t, double tau) { return tau > 0.0 ? exp(-t / tau) : 0.0; }

void orc_time_coefs(double t, double tau, double c[11]) {
  const double e = decay(t, tau);
  c[0] = 0.0;
  c[T1] = 1.0 - e;
  c[T2] = (t + tau) * e - tau;
  c[T3] = t - tau + tau * e;
  c[T4] = -(t * t + 2.0 * t * tau) * e;
  c[T5] = t * t - 2.0 * t * tau;
  c[T6] = -t * tau * (1.0 + e);
  c[T7] = e;
  c[T8] = -t * e;
  c[T7T] = t * e;
  c[T7T2] = t * t * e;
}

/* closed-form integrals over [0, T] of the functions above, written in T and
 * tau so that they stay finite at tau = 0 */
void orc_time_integrals(double T, double tau, double c[11]) {
  const double e = decay(T, tau);
  const double t2 = tau * tau, t3 = t2 * tau;
  c[0] = 0.0;
  c[T1] = T - tau * (1.0 - e);
  c[T2] = 2.0 * t2 * (1.0 - e) - tau * T * (1.0 + e);
  c[T3] = 0.5 * T * T - tau * T + t2 * (1.0 - e);
  c[T4] = -4.0 * t3 + tau * (T + 2.0 * tau) * (T + 2.0 * tau) * e;
  c[T5] = T * T * T / 3.0 - tau * T * T;
  c[T6] = -tau * (0.5 * T * T + t2 - tau * (tau + T) * e);
  c[T7] = tau * (1.0 - e);
  c[T8] = -(t2 - tau * (tau + T) * e);
  c[T7T] = t2 - tau * (tau + T) * e;
  c[T7T2] = 2.0 * t3 - tau * (T * T + 2.0 * T * tau + 2.0 * t2) * e;
}

/* ------------------------------------------------------------------ */
/* The gas distribution function at the interface as a list of terms   */
/* s * C_tid(t) * y^ypow * g_src * X(psi) * u^p v^q                    */
/* src 0: g0 over the full space; 1: g_l over u>0; 2: g_r over u<0      */
/* ------------------------------------------------------------------ */
typedef struct { int src, tid, p, q, ypow; double s; double X[4]; } fterm;
typedef struct { int n; fterm t[64]; } flist;

static const double E0[4] = {1.0, 0.0, 0.0, 0.0}; /* the constant function 1 */

static void fl_add(flist* f, int src, int tid, double s, const double X[4], int p, int q, int ypow) {
  fterm* t = &f->t[f->n++];
  t->src = src; t->tid = tid; t->s = s; t->p = p; t->q = q; t->ypow = ypow;
  memcpy(t->X, X, sizeof(double) * 4);
}

/* Eq. dis1, term by term in the paper's order */
static void fl_hydro(flist* f, const coefs* c) {
  fl_add(f, 0, T1, 1.0, E0, 0, 0, 0);       /* C1 g0 */
  fl_add(f, 0, T2, 1.0, c->a1, 1, 0, 0);    /* C2 g0 a1 u */
  fl_add(f, 0, T2, 1.0, c->a2, 0, 1, 0);    /* C2 g0 a2 v */
  fl_add(f, 0, T1, 1.0, c->a2, 0, 0, 1);    /* C1 g0 a2 y */
  fl_add(f, 0, T3, 1.0, c->A, 0, 0, 0);     /* C3 g0 A */
  fl_add(f, 0, T4, 0.5, c->Axx, 2, 0, 0);   /* 1/2 C4 g0 (a1^2+d11) u^2 */
  fl_add(f, 0, T6, 1.0, c->Atx, 1, 0, 0);   /* C6 g0 (A a1+b1) u */
  fl_add(f, 0, T5, 0.5, c->Att, 0, 0, 0);   /* 1/2 C5 g0 (A^2+B) */
  fl_add(f, 0, T1, 0.5, c->Ayy, 0, 0, 2);   /* 1/2 C1 g0 (a2^2+d22) y^2 */
  fl_add(f, 0, T2, 1.0, c->Ayy, 0, 1, 1);   /* C2 g0 (a2^2+d22) v y */
  fl_add(f, 0, T4, 0.5, c->Ayy, 0, 2, 0);   /* 1/2 C4 g0 (a2^2+d22) v^2 */
  fl_add(f, 0, T2, 1.0, c->Axy, 1, 0, 1);   /* C2 g0 (a1 a2+d12) u y */
  fl_add(f, 0, T4, 1.0, c->Axy, 1, 1, 0);   /* C4 g0 (a1 a2+d12) u v */
  fl_add(f, 0, T3, 1.0, c->Aty, 0, 0, 1);   /* C3 g0 (A a2+b2) y */
  fl_add(f, 0, T6, 1.0, c->Aty, 0, 1, 0);   /* C6 g0 (A a2+b2) v */
}

/* Eq. dis2 for side src (1 = left, 2 = right).  ns = 1: Navier-Stokes initial
 * distribution f_G = g - tau (a1 u + a2 v + A) g; ns = 0: Euler, f_G = g. */
static void fl_kinetic(flist* f, int src, const coefs* c, double tau, int ns) {
  const double mt = ns ? -tau : 0.0;
  /* C7 g [1 - tau (a1 u + a2 v + A)] */
  fl_add(f, src, T7, 1.0, E0, 0, 0, 0);
  if (ns) {
    fl_add(f, src, T7, mt, c->a1, 1, 0, 0);
    fl_add(f, src, T7, mt, c->a2, 0, 1, 0);
    fl_add(f, src, T7, mt, c->A, 0, 0, 0);
  }
  /* C8 g [a1 u - tau ((a1^2+d11) u^2 + (a1 a2+d12) u v + (A a1+b1) u)] */
  fl_add(f, src, T8, 1.0, c->a1, 1, 0, 0);
  if (ns) {
    fl_add(f, src, T8, mt, c->Axx, 2, 0, 0);
    fl_add(f, src, T8, mt, c->Axy, 1, 1, 0);
    fl_add(f, src, T8, mt, c->Atx, 1, 0, 0);
  }
  /* C8 g [a2 v - tau ((a1 a2+d12) u v + (a2^2+d22) v^2 + (A a2+b2) v)] */
  fl_add(f, src, T8, 1.0, c->a2, 0, 1, 0);
  if (ns) {
    fl_add(f, src, T8, mt, c->Axy, 1, 1, 0);
    fl_add(f, src, T8, mt, c->Ayy, 0, 2, 0);
    fl_add(f, src, T8, mt, c->Aty, 0, 1, 0);
  }
  /* C7 g [a2 - tau ((a1 a2+d12) u + (a2^2+d22) v + (A a2+b2))] y */
  fl_add(f, src, T7, 1.0, c->a2, 0, 0, 1);
  if (ns) {
    fl_add(f, src, T7, mt, c->Axy, 1, 0, 1);
    fl_add(f, src, T7, mt, c->Ayy, 0, 1, 1);
    fl_add(f, src, T7, mt, c->Aty, 0, 0, 1);
  }
  /* 1/2 C7 g [(a1^2+d11)(-ut)^2 + 2 (a1 a2+d12)(-ut)(y-vt) + (a2^2+d22)(y-vt)^2] */
  fl_add(f, src, T7T2, 0.5, c->Axx, 2, 0, 0);   /* u^2 t^2 */
  fl_add(f, src, T7T, -1.0, c->Axy, 1, 0, 1);   /* -u t y */
  fl_add(f, src, T7T2, 1.0, c->Axy, 1, 1, 0);   /* u v t^2 */
  fl_add(f, src, T7, 0.5, c->Ayy, 0, 0, 2);     /* y^2 */
  fl_add(f, src, T7T, -1.0, c->Ayy, 0, 1, 1);   /* -2 y v t / 2 */
  fl_add(f, src, T7T2, 0.5, c->Ayy, 0, 2, 0);   /* v^2 t^2 */
}

static void cons_prim(const double w[4], double gamma, double* rho, double* u, double* v, double* p) {
  *rho = w[0];
  *u = w[1] / w[0];
  *v = w[2] / w[0];
  *p = (gamma - 1.0) * (w[3] - 0.5 * w[0] * (*u * *u + *v * *v));
}

/* first_order = 1: the first-order evolution used by the positivity fallback of
 * the update -- both sides are constant (their derivatives are ignored) and the
 * equilibrium state has no slopes (b2..b6 = 0) */
static void face_impl(const orc_params* P, const double L[6][4], const double R[6][4],
                      const double avg[2][3][4], double dn, double dtan, double dt,
                      double Fhat[4], double Wg[2][4], double* dbg, int first_order) {
  const double gam = P->gamma;
  const double K = (4.0 - 2.0 * gam) / (gam - 1.0); /* Section 2.1 */
  maxw gl, gr, g0;
  maxw_from_cons(&gl, L[0], K);
  maxw_from_cons(&gr, R[0], K);

  /* Eq. compatibility2: U0 = int_{u>0} psi g_l + int_{u<0} psi g_r */
  double U0[4], hl[4], hr[4];
  {
    poly one;
    poly_mono(1.0, 0, 0, &one);
    maxw_mom4(&gl, 1, &one, hl);
    maxw_mom4(&gr, 2, &one, hr);
    for (int k = 0; k < 4; ++k) U0[k] = gl.rho * hl[k] + gr.rho * hr[k];
  }
  maxw_from_cons(&g0, U0, K);

  /* Section 3.3: equilibrium polynomial U0 + b2 x + b3 y + b4 x^2/2 + b5 y^2/2 + b6 x y
   * from the six cell averages avg[m][n+1], m = 0,1 (normal), n = -1,0,1 */
  double b[7][4];
  for (int k = 0; k < 4; ++k) {
    const double um1 = avg[0][0][k], u0 = avg[0][1][k], up1 = avg[0][2][k];
    const double vm1 = avg[1][0][k], v0 = avg[1][1][k], vp1 = avg[1][2][k];
    b[2][k] = ((vp1 - up1) + 2.0 * (v0 - u0) + (vm1 - um1)) / (4.0 * dn);
    b[3][k] = (vp1 - vm1 + up1 - um1) / (4.0 * dtan);
    b[4][k] = (26.0 * (v0 + u0) - (vp1 + up1 + vm1 + um1) - 48.0 * U0[k]) / (8.0 * dn * dn);
    b[5][k] = (vp1 - 2.0 * v0 + vm1 + up1 - 2.0 * u0 + um1) / (2.0 * dtan * dtan);
    b[6][k] = (vp1 - up1 - vm1 + um1) / (2.0 * dn * dtan);
    if (first_order) b[2][k] = b[3][k] = b[4][k] = b[5][k] = b[6][k] = 0.0;
  }

  /* Section 4: collision time */
  double rl, ul, vl, pl, rr, ur, vr, pr, r0, u0, v0, p0;
  cons_prim(L[0], gam, &rl, &ul, &vl, &pl);
  cons_prim(R[0], gam, &rr, &ur, &vr, &pr);
  cons_prim(U0, gam, &r0, &u0, &v0, &p0);
  const double jump = fabs((pl - pr) / (pl + pr)) * dt;
  const int ns = P->mu > 0.0;
  const double tau = ns ? P->mu / p0 + jump : P->tau_eps * dt + P->tau_C * jump;

  /* coefficient systems for g0 (derivatives of the equilibrium polynomial)
   * and for both sides (derivatives of the reconstructed polynomials) */
  coefs c0, cl, cr;
  {
    double d0[5][4], dl[5][4], dr[5][4];
    for (int k = 0; k < 4; ++k) {
      d0[0][k] = b[2][k]; d0[1][k] = b[3][k]; d0[2][k] = b[4][k]; d0[3][k] = b[6][k]; d0[4][k] = b[5][k];
      for (int s = 0; s < 5; ++s) {
        dl[s][k] = first_order ? 0.0 : L[s + 1][k];
        dr[s][k] = first_order ? 0.0 : R[s + 1][k];
      }
    }
    coefs_solve(&g0, d0, &c0);
    coefs_solve(&gl, dl, &cl);
    coefs_solve(&gr, dr, &cr);
  }

  /* the distribution function at the interface: Eq. integral = Eq. dis1 + Eq. dis2 */
  flist f;
  f.n = 0;
  fl_hydro(&f, &c0);
  fl_kinetic(&f, 1, &cl, tau, ns);
  fl_kinetic(&f, 2, &cr, tau, ns);

  double Cint[11], Cend[11];
  orc_time_integrals(dt, tau, Cint);
  orc_time_coefs(dt, tau, Cend);
  const maxw* src[3] = {&g0, &gl, &gr};
  const int half[3] = {0, 1, 2};
  const double yavg[3] = {1.0, 0.0, dtan * dtan / 12.0}; /* face means of 1, y, y^2 */
  const double yg = sqrt(3.0) / 6.0 * dtan;

  /* heat flux weight (u-U0) ((u-U0)^2 + (v-V0)^2 + xi^2) / 2 for the Prandtl fix */
  poly qw;
  {
    poly cu, cv, e2, t;
    cu.n = 0; poly_add(&cu, 1.0, 1, 0, 0); poly_add(&cu, -u0, 0, 0, 0);
    cv.n = 0; poly_add(&cv, 1.0, 0, 1, 0); poly_add(&cv, -v0, 0, 0, 0);
    poly cu2, cv2;
    poly_mul(&cu, &cu, &cu2);
    poly_mul(&cv, &cv, &cv2);
    e2.n = 0;
    for (int k = 0; k < cu2.n; ++k) poly_add(&e2, 0.5 * cu2.t[k].c, cu2.t[k].p, cu2.t[k].q, cu2.t[k].r);
    for (int k = 0; k < cv2.n; ++k) poly_add(&e2, 0.5 * cv2.t[k].c, cv2.t[k].p, cv2.t[k].q, cv2.t[k].r);
    poly_add(&e2, 0.5, 0, 0, 1);
    poly_mul(&cu, &e2, &t);
    qw = t;
  }

  double F[4] = {0, 0, 0, 0}, Wm[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}}, q = 0.0;
  for (int k = 0; k < f.n; ++k) {
    const fterm* t = &f.t[k];
    const maxw* g = src[t->src];
    poly px, pm, base, wu, tmp;
    poly_coef(t->X, &px);
    poly_mono(1.0, t->p, t->q, &pm);
    poly_mul(&px, &pm, &base);
    /* flux: int_0^dt (1/dtan) int_face int u psi f */
    const double wflux = t->s * Cint[t->tid] * yavg[t->ypow] * g->rho;
    if (wflux != 0.0) {
      double m4[4];
      poly_mono(1.0, 1, 0, &pm);
      poly_mul(&base, &pm, &wu);
      maxw_mom4(g, half[t->src], &wu, m4);
      for (int b2 = 0; b2 < 4; ++b2) F[b2] += wflux * m4[b2];
      if (P->Pr != 1.0) {
        poly_mul(&base, &qw, &tmp);
        q += wflux * maxw_mom(g, half[t->src], &tmp);
      }
    }
    /* Eq. point at t = dt, y = -/+ yg */
    {
      double m4[4];
      maxw_mom4(g, half[t->src], &base, m4);
      for (int gp = 0; gp < 2; ++gp) {
        const double y = gp == 0 ? -yg : yg;
        const double w = t->s * Cend[t->tid] * pow(y, t->ypow) * g->rho;
        for (int b2 = 0; b2 < 4; ++b2) Wm[gp][b2] += w * m4[b2];
      }
    }
  }
  /* Prandtl-number fix of the energy flux: add (1/Pr - 1) times the heat flux */
  if (P->Pr != 1.0) F[3] += (1.0 / P->Pr - 1.0) * q;

  for (int k = 0; k < 4; ++k) {
    Fhat[k] = F[k];
    Wg[0][k] = Wm[0][k];
    Wg[1][k] = Wm[1][k];
  }
  if (dbg) {
    for (int k = 0; k < 4; ++k) dbg[k] = U0[k];
    dbg[4] = tau;
    for (int s = 2; s <= 6; ++s)
      for (int k = 0; k < 4; ++k) dbg[5 + (s - 2) * 4 + k] = b[s][k];
    dbg[25] = q;
  }
}

void orc_face(const orc_params* P, const double L[6][4], const double R[6][4],
              const double avg[2][3][4], double dn, double dtan, double dt,
              double Fhat[4], double Wg[2][4], double* dbg) {
  face_impl(P, L, R, avg, dn, dtan, dt, Fhat, Wg, dbg, 0);
}

/* The fallback evolution: the collisionless (tau -> infinity) limit of Eq.
 * integral for constant states, f = f0: the flux over [0, dt] is
 * dt (rho_l <u psi>_{u>0,l} + rho_r <u psi>_{u<0,r}) and the point values are
 * U0 of Eq. compatibility2 at every point of the face. */
void orc_face_first_order(const orc_params* P, const double L[6][4], const double R[6][4],
                          double dn, double dtan, double dt, double Fhat[4], double Wg[2][4],
                          double* dbg) {
  (void)dn;
  (void)dtan;
  const double gam = P->gamma;
  const double K = (4.0 - 2.0 * gam) / (gam - 1.0);
  maxw gl, gr;
  maxw_from_cons(&gl, L[0], K);
  maxw_from_cons(&gr, R[0], K);
  poly one, u;
  poly_mono(1.0, 0, 0, &one);
  poly_mono(1.0, 1, 0, &u);
  double hl[4], hr[4], fl[4], fr[4];
  maxw_mom4(&gl, 1, &one, hl);
  maxw_mom4(&gr, 2, &one, hr);
  maxw_mom4(&gl, 1, &u, fl);
  maxw_mom4(&gr, 2, &u, fr);
  for (int k = 0; k < 4; ++k) {
    Fhat[k] = dt * (gl.rho * fl[k] + gr.rho * fr[k]);
    Wg[0][k] = Wg[1][k] = gl.rho * hl[k] + gr.rho * hr[k];
  }
  if (dbg)
    for (int k = 0; k < 4; ++k) dbg[k] = Wg[0][k];
}

/* ------------------------------------------------------------------ */
/* Boundary images (the paper names its boundary conditions but does   */
/* not define them; this is the reading used throughout)               */
/* ------------------------------------------------------------------ */

/* pointwise map of a face-frame state to its image behind the wall */
static void wall_map(int kind, double gam, double uwt, double Tw, const double w[4], double o[4]) {
  if (kind == ORC_BC_SLIPWALL) {
    o[0] = w[0]; o[1] = -w[1]; o[2] = w[2]; o[3] = w[3];
    return;
  }
  if (kind == ORC_BC_NOSLIP_ADIABATIC) {
    /* rho' = rho, u' = 2 u_w - u, T' = T: the internal energy is kept, the kinetic energy
     * changes by (|m'|^2 - |m|^2) / (2 rho) = 2 rho u_w^2 - 2 u_w m_t (linear in the state) */
    o[0] = w[0];
    o[1] = -w[1];
    o[2] = 2.0 * w[0] * uwt - w[2];
    o[3] = w[3] + 2.0 * w[0] * uwt * uwt - 2.0 * uwt * w[2];
    return;
  }
  /* no-slip isothermal: rho' = rho, u' = 2 u_w - u, T' = 2 T_w - T */
  const double rho = w[0], mn = w[1], mt = w[2], e = w[3];
  o[0] = rho;
  o[1] = -mn;
  o[2] = 2.0 * rho * uwt - mt;
  o[3] = 2.0 * rho * uwt * uwt - 2.0 * uwt * mt + (mn * mn + mt * mt) / rho +
         2.0 * rho * Tw / (gam - 1.0) - e;
}

/* Jacobian and the Hessian of the energy component of wall_map */
static void wall_jac(int kind, double gam, double uwt, double Tw, const double w[4], double J[4][4]) {
  memset(J, 0, sizeof(double) * 16);
  if (kind == ORC_BC_SLIPWALL) {
    J[0][0] = 1; J[1][1] = -1; J[2][2] = 1; J[3][3] = 1;
    return;
  }
  if (kind == ORC_BC_NOSLIP_ADIABATIC) {
    J[0][0] = 1; J[1][1] = -1;
    J[2][0] = 2.0 * uwt; J[2][2] = -1;
    J[3][0] = 2.0 * uwt * uwt; J[3][2] = -2.0 * uwt; J[3][3] = 1;
    return;
  }
  const double rho = w[0], mn = w[1], mt = w[2];
  J[0][0] = 1.0;
  J[1][1] = -1.0;
  J[2][0] = 2.0 * uwt; J[2][2] = -1.0;
  J[3][0] = 2.0 * uwt * uwt - (mn * mn + mt * mt) / (rho * rho) + 2.0 * Tw / (gam - 1.0);
  J[3][1] = 2.0 * mn / rho;
  J[3][2] = -2.0 * uwt + 2.0 * mt / rho;
  J[3][3] = -1.0;
}

static double wall_hess_e(int kind, const double w[4], const double a[4], const double bb[4]) {
  if (kind == ORC_BC_SLIPWALL || kind == ORC_BC_NOSLIP_ADIABATIC) return 0.0;  /* linear maps */
  /* second derivative of |m|^2 / rho along a and b */
  const double rho = w[0], mn = w[1], mt = w[2];
  const double m2 = mn * mn + mt * mt;
  const double ma = mn * a[1] + mt * a[2], mb = mn * bb[1] + mt * bb[2];
  return 2.0 * m2 / (rho * rho * rho) * a[0] * bb[0] - 2.0 * ma * bb[0] / (rho * rho) -
         2.0 * mb * a[0] / (rho * rho) + 2.0 * (a[1] * bb[1] + a[2] * bb[2]) / rho;
}

void orc_bc_image(const orc_params* P, int kind, double uwt, double Tw, const double in[6][4],
                  double out[6][4]) {
  if (kind == ORC_BC_OUTFLOW || kind == ORC_BC_PERIODIC) {
    /* outflow: the inside polynomial continued across the face */
    memcpy(out, in, sizeof(double) * 24);
    return;
  }
  /* image G(n, t) = Phi(P(-n, t)) of the inside polynomial P */
  double J[4][4];
  wall_map(kind, P->gamma, uwt, Tw, in[0], out[0]);
  wall_jac(kind, P->gamma, uwt, Tw, in[0], J);
  for (int r = 0; r < 4; ++r) {
    double s[5] = {0, 0, 0, 0, 0};
    for (int c = 0; c < 4; ++c)
      for (int d = 0; d < 5; ++d) s[d] += J[r][c] * in[d + 1][c];
    out[1][r] = -s[0]; /* d/dn */
    out[2][r] = s[1];  /* d/dt */
    out[3][r] = s[2];  /* d2/dn2 */
    out[4][r] = -s[3]; /* d2/dndt */
    out[5][r] = s[4];  /* d2/dt2 */
  }
  out[3][3] += wall_hess_e(kind, in[0], in[1], in[1]);
  out[4][3] -= wall_hess_e(kind, in[0], in[1], in[2]);
  out[5][3] += wall_hess_e(kind, in[0], in[2], in[2]);
}

/* ------------------------------------------------------------------ */
/* Section 3.2: compact reconstruction                                 */
/* ------------------------------------------------------------------ */
static double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return a > 0.0 ? fmin(a, b) : fmax(a, b);
}

/* smoothness indicator sum_{|alpha|=1,2} |cell|^(|alpha|-1) int (D^alpha P)^2 / |cell|
 * for P = Ubar + a2 x + a3 y + a4 wx + a5 wy + a6 x y */
static double indicator(const double a[6], double dx, double dy) {
  const double ux2 = a[1] * a[1] + a[3] * a[3] * dx * dx / 12.0 + a[5] * a[5] * dy * dy / 12.0;
  const double uy2 = a[2] * a[2] + a[4] * a[4] * dy * dy / 12.0 + a[5] * a[5] * dx * dx / 12.0;
  return dx * dx * ux2 + dy * dy * uy2 + dx * dx * dx * dx * a[3] * a[3] +
         dx * dx * dy * dy * a[5] * a[5] + dy * dy * dy * dy * a[4] * a[4];
}

static void recon_var(const orc_params* P, double Uc, double Ue, double Uw, double Un, double Us,
                      double em, double ep, double wm, double wp, double nm, double np, double sm,
                      double sp, double dx, double dy, double out[6]) {
  /* one-sided stencils (Eq. over-sys): face Gauss mean and the neighbour average */
  const double Se = 0.5 * (em + ep), Sw = 0.5 * (wm + wp);
  const double Sn = 0.5 * (nm + np), Ss = 0.5 * (sm + sp);
  const double a4e = 3.0 * (Uc + Ue - 2.0 * Se) / (dx * dx), t2e = 2.0 * (Se - Uc) / dx;
  const double a4w = 3.0 * (Uc + Uw - 2.0 * Sw) / (dx * dx), t2w = 2.0 * (Sw - Uc) / dx;
  const double a5n = 3.0 * (Uc + Un - 2.0 * Sn) / (dy * dy), t3n = 2.0 * (Sn - Uc) / dy;
  const double a5s = 3.0 * (Uc + Us - 2.0 * Ss) / (dy * dy), t3s = 2.0 * (Ss - Uc) / dy;
  /* Eq. limiter, normal (a2, a4) and tangential (a3, a5) pairs separately */
  const double a4 = minmod(a4w, a4e);
  const double a2 = minmod(-t2w + a4 * dx / 6.0, t2e - a4 * dx / 6.0);
  const double a5 = minmod(a5s, a5n);
  const double a3 = minmod(-t3s + a5 * dy / 6.0, t3n - a5 * dy / 6.0);
  /* cross derivative of the four one-sided stencils with the limited a2, a3;
   * keep the smallest in magnitude.  The paper gives no tie rule, and piecewise
   * constant data produce exact ties of opposite sign: magnitudes within a
   * relative 1e-8 of the current choice count as ties, and the first stencil in
   * the order (+,+), (-,+), (-,-), (+,-) is kept */
  const double dxe = ep - em, dxw = wp - wm, dyn = np - nm, dys = sp - sm;
  const double r3 = sqrt(3.0);
  const int sx[4] = {1, -1, -1, 1}, sy[4] = {1, 1, -1, -1};
  double a6 = 0.0;
  for (int k = 0; k < 4; ++k) {
    const double Dx = sx[k] > 0 ? dxe : dxw, Dy = sy[k] > 0 ? dyn : dys;
    const double c = sx[k] * (r3 * Dx / (dx * dy) - a3 / dx) + sy[k] * (r3 * Dy / (dx * dy) - a2 / dy);
    if (k == 0 || fabs(c) < fabs(a6) * (1.0 - 1e-8)) a6 = c;
  }
  const double U1[6] = {Uc, a2, a3, a4, a5, a6};
  /* central stencil */
  const double U2[6] = {Uc,
                        (Ue - Uw) / (2.0 * dx),
                        (Un - Us) / (2.0 * dy),
                        (Ue - 2.0 * Uc + Uw) / (dx * dx),
                        (Un - 2.0 * Uc + Us) / (dy * dy),
                        r3 * ((dxe - dxw) + (dyn - dys)) / (2.0 * dx * dy)};
  /* Eq. average: nonlinear weights, I(U1) = C dx dy */
  const double I1 = P->weno_C * dx * dy, I2 = indicator(U2, dx, dy);
  const double al1 = 1.0 / ((P->weno_eps + I1) * (P->weno_eps + I1));
  const double al2 = 1.0 / ((P->weno_eps + I2) * (P->weno_eps + I2));
  const double w1 = al1 / (al1 + al2), w2 = al2 / (al1 + al2);
  out[0] = Uc;
  for (int k = 1; k < 6; ++k) out[k] = w1 * U1[k] + w2 * U2[k];
}

/* value and derivatives of P at (x, y): P, Px, Py, Pxx, Pxy, Pyy */
static void poly_eval(const double a[6], double dx, double dy, double x, double y, double o[6]) {
  o[0] = a[0] + a[1] * x + a[2] * y + a[3] * 0.5 * (x * x - dx * dx / 12.0) +
         a[4] * 0.5 * (y * y - dy * dy / 12.0) + a[5] * x * y;
  o[1] = a[1] + a[3] * x + a[5] * y;
  o[2] = a[2] + a[4] * y + a[5] * x;
  o[3] = a[3];
  o[4] = a[5];
  o[5] = a[4];
}

/* Eigenvectors of the Jacobian dF/dU of the x-flux of the 2D Euler equations at the
 * conservative state w: columns of R for the eigenvalues u - c, u (entropy), u (shear),
 * u + c, and L = R^-1 (rows).  With b1 = (gamma-1)/c^2, b2 = b1 (u^2+v^2)/2 and the total
 * enthalpy H:  r1 = (1, u-c, v, H-uc), r2 = (1, u, v, q^2/2), r3 = (0, 0, 1, v),
 * r4 = (1, u+c, v, H+uc);  l1 = (b2 + u/c, -b1 u - 1/c, -b1 v, b1)/2,
 * l2 = (1-b2, b1 u, b1 v, -b1), l3 = (-v, 0, 1, 0), l4 = (b2 - u/c, -b1 u + 1/c, -b1 v, b1)/2. */
void orc_char_basis(const double w[4], double gam, double L[4][4], double R[4][4]) {
  const double rho = w[0], u = w[1] / rho, v = w[2] / rho;
  const double q2 = u * u + v * v;
  const double p = (gam - 1.0) * (w[3] - 0.5 * rho * q2);
  const double c = sqrt(gam * p / rho), H = (w[3] + p) / rho;
  const double b1 = (gam - 1.0) / (c * c), b2 = 0.5 * b1 * q2;
  const double Rm[4][4] = {{1.0, 1.0, 0.0, 1.0},
                           {u - c, u, 0.0, u + c},
                           {v, v, 1.0, v},
                           {H - u * c, 0.5 * q2, v, H + u * c}};
  const double Lm[4][4] = {{0.5 * (b2 + u / c), 0.5 * (-b1 * u - 1.0 / c), -0.5 * b1 * v, 0.5 * b1},
                           {1.0 - b2, b1 * u, b1 * v, -b1},
                           {-v, 0.0, 1.0, 0.0},
                           {0.5 * (b2 - u / c), 0.5 * (-b1 * u + 1.0 / c), -0.5 * b1 * v, 0.5 * b1}};
  memcpy(R, Rm, sizeof(Rm));
  memcpy(L, Lm, sizeof(Lm));
}

/* momenta swapped: the y-direction quantities in the x-frame formulas */
static void swap_uv(const double a[4], double o[4]) {
  o[0] = a[0]; o[1] = a[2]; o[2] = a[1]; o[3] = a[3];
}

/* Reconstruction in the characteristic variables of one direction (axis 0: x, 1: y) of the
 * cell average: every stencil value is projected with L, each characteristic variable is
 * reconstructed as a scalar, and the coefficients are projected back with R. */
static void recon_char_axis(const orc_params* P, int axis, const double nb[5][4], const double fx[4][4],
                            const double fy[4][4], double dx, double dy, double co[4][6]) {
  double L[4][4], R[4][4], ref[4];
  if (axis == 0) memcpy(ref, nb[0], sizeof(ref)); else swap_uv(nb[0], ref);
  orc_char_basis(ref, P->gamma, L, R);
  /* the 13 stencil vectors, projected */
  double in[13][4], pr[13][4];
  for (int k = 0; k < 5; ++k) memcpy(in[k], nb[k], sizeof(in[k]));
  for (int k = 0; k < 4; ++k) memcpy(in[5 + k], fx[k], sizeof(in[k]));
  for (int k = 0; k < 4; ++k) memcpy(in[9 + k], fy[k], sizeof(in[k]));
  for (int k = 0; k < 13; ++k) {
    double a[4];
    if (axis == 0) memcpy(a, in[k], sizeof(a)); else swap_uv(in[k], a);
    for (int r = 0; r < 4; ++r) {
      pr[k][r] = 0.0;
      for (int c = 0; c < 4; ++c) pr[k][r] += L[r][c] * a[c];
    }
  }
  double cc[4][6];
  for (int r = 0; r < 4; ++r)
    recon_var(P, pr[0][r], pr[1][r], pr[2][r], pr[3][r], pr[4][r], pr[5][r], pr[6][r], pr[7][r],
              pr[8][r], pr[9][r], pr[10][r], pr[11][r], pr[12][r], dx, dy, cc[r]);
  for (int m = 0; m < 6; ++m) {
    double a[4], o[4];
    for (int r = 0; r < 4; ++r) {
      a[r] = 0.0;
      for (int c = 0; c < 4; ++c) a[r] += R[r][c] * cc[c][m];
    }
    if (axis == 0) memcpy(o, a, sizeof(o)); else swap_uv(a, o);
    for (int v = 0; v < 4; ++v) co[v][m] = o[v];
  }
}

void orc_recon_cell(const orc_params* P, const double nb[5][4], const double fx[4][4],
                    const double fy[4][4], double dx, double dy, double co[4][6]) {
  if (P->characteristic) {
    /* x-derivative coefficients (a2, a4) from the x-characteristic reconstruction, y ones
     * (a3, a5) from the y-characteristic one, the cross derivative a6 their mean */
    double cx[4][6], cy[4][6];
    recon_char_axis(P, 0, nb, fx, fy, dx, dy, cx);
    recon_char_axis(P, 1, nb, fx, fy, dx, dy, cy);
    for (int v = 0; v < 4; ++v) {
      co[v][0] = nb[0][v];
      co[v][1] = cx[v][1];
      co[v][2] = cy[v][2];
      co[v][3] = cx[v][3];
      co[v][4] = cy[v][4];
      co[v][5] = 0.5 * (cx[v][5] + cy[v][5]);
    }
  } else {
    for (int v = 0; v < 4; ++v)
      recon_var(P, nb[0][v], nb[1][v], nb[2][v], nb[3][v], nb[4][v], fx[0][v], fx[1][v], fx[2][v],
                fx[3][v], fy[0][v], fy[1][v], fy[2][v], fy[3][v], dx, dy, co[v]);
  }
  /* positivity: a cell whose polynomial gives rho <= 0 or p <= 0 at a face
   * centre falls back to its constant average */
  const double pts[4][2] = {{0.5 * dx, 0}, {-0.5 * dx, 0}, {0, 0.5 * dy}, {0, -0.5 * dy}};
  int bad = 0;
  for (int k = 0; k < 4 && !bad; ++k) {
    double w[4], o[6];
    for (int v = 0; v < 4; ++v) {
      poly_eval(co[v], dx, dy, pts[k][0], pts[k][1], o);
      w[v] = o[0];
    }
    double r, u, vv, p;
    cons_prim(w, P->gamma, &r, &u, &vv, &p);
    if (!(r > 0.0) || !(p > 0.0)) bad = 1;
  }
  if (bad)
    for (int v = 0; v < 4; ++v)
      for (int k = 1; k < 6; ++k) co[v][k] = 0.0;
}

/* ------------------------------------------------------------------ */
/* Grid level                                                          */
/* ------------------------------------------------------------------ */
#define UI(v, j, i) ((size_t)(v) * ny * nx + (size_t)(j) * nx + (i))
#define WXI(v, g, j, i) ((((size_t)(v) * 2 + (g)) * ny + (j)) * (nx + 1) + (i))
#define WYI(v, g, j, i) ((((size_t)(v) * 2 + (g)) * (ny + 1) + (j)) * nx + (i))
#define CI(v, k, j, i) ((((size_t)(v) * 6 + (k)) * ny + (j)) * nx + (i))

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n);
#else
  (void)n;
#endif
}

double orc_dt2d(const orc_params* P, int nx, int ny, double Lx, double Ly, const double* U,
                double CFL, double dt_max, int viscous_dt) {
  const double dx = Lx / nx, dy = Ly / ny;
  double m = INFINITY;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double w[4] = {U[UI(0, j, i)], U[UI(1, j, i)], U[UI(2, j, i)], U[UI(3, j, i)]};
      double r, u, v, p;
      cons_prim(w, P->gamma, &r, &u, &v, &p);
      const double c = sqrt(P->gamma * p / r);
      double d = fmin(dx / (fabs(u) + c), dy / (fabs(v) + c));
      if (viscous_dt && P->mu > 0.0) {
        const double h = fmin(dx, dy);
        d = fmin(d, r * h * h / (2.0 * P->mu * fmax(4.0 / 3.0, P->gamma / P->Pr)));
      }
      m = fmin(m, d);
    }
  return fmin(CFL * m, dt_max);
}

/* cell average at (i, j) including the one-cell ghost ring */
typedef struct {
  int nx, ny;
  double* g; /* [4][ny+2][nx+2] */
} ghosts;

#define GI(G, v, j, i) ((size_t)(v) * ((G)->ny + 2) * ((G)->nx + 2) + (size_t)((j) + 1) * ((G)->nx + 2) + ((i) + 1))

/* physical <-> face frame: y-faces swap the two momentum components */
static void to_frame(int axis, const double w[4], double o[4]) {
  o[0] = w[0]; o[3] = w[3];
  if (axis == 0) { o[1] = w[1]; o[2] = w[2]; } else { o[1] = w[2]; o[2] = w[1]; }
}

static double wall_tangent_velocity(const orc_bc* b, int axis) {
  return axis == 0 ? b->v_wall : b->u_wall;
}

static void ghost_value(const orc_params* P, const orc_bc* b, int axis, const double in[4], double out[4]) {
  if (b->kind == ORC_BC_OUTFLOW || b->kind == ORC_BC_PERIODIC) {
    memcpy(out, in, sizeof(double) * 4);
    return;
  }
  double f[4], o[4];
  to_frame(axis, in, f);
  wall_map(b->kind, P->gamma, wall_tangent_velocity(b, axis), b->T_wall, f, o);
  to_frame(axis, o, out);
}

/* Flux through a wall face (face frame).  A wall lets no mass through, and an
 * adiabatic wall no heat: its energy flux is the work u_w F_(m_t) of the shear on the
 * moving wall.  The mirror images give these exactly for a slip wall; behind a no-slip
 * wall the image also reverses the tangential velocity, which the tangential
 * transport terms of the evolution do not respect, so the evaluated mass and energy
 * fluxes carry an O(dt d(rho u_t)/dt) error that the wall's definition removes. */
static void wall_face_flux(const orc_bc* b, int axis, double F[4]) {
  if (b->kind == ORC_BC_SLIPWALL || b->kind == ORC_BC_NOSLIP_ISOTHERMAL || b->kind == ORC_BC_NOSLIP_ADIABATIC)
    F[0] = 0.0;
  if (b->kind == ORC_BC_NOSLIP_ADIABATIC) F[3] = wall_tangent_velocity(b, axis) * F[2];
}

/* ghost ring: first the y-ghost rows of interior columns, then the x-ghost
 * columns of all rows (corners are x-images of y-ghosts) */
static void fill_ghosts(const orc_params* P, int nx, int ny, const orc_bc bc[4], const double* U, ghosts* G) {
  G->nx = nx; G->ny = ny;
  for (int v = 0; v < 4; ++v)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) G->g[GI(G, v, j, i)] = U[UI(v, j, i)];
  for (int i = 0; i < nx; ++i) {
    double in[4], out[4];
    for (int side = 0; side < 2; ++side) {
      const int jg = side == 0 ? -1 : ny;
      const int js = bc[2 + side].kind == ORC_BC_PERIODIC ? (side == 0 ? ny - 1 : 0) : (side == 0 ? 0 : ny - 1);
      for (int v = 0; v < 4; ++v) in[v] = G->g[GI(G, v, js, i)];
      ghost_value(P, &bc[2 + side], 1, in, out);
      for (int v = 0; v < 4; ++v) G->g[GI(G, v, jg, i)] = out[v];
    }
  }
  for (int j = -1; j <= ny; ++j) {
    double in[4], out[4];
    for (int side = 0; side < 2; ++side) {
      const int ig = side == 0 ? -1 : nx;
      const int is = bc[side].kind == ORC_BC_PERIODIC ? (side == 0 ? nx - 1 : 0) : (side == 0 ? 0 : nx - 1);
      for (int v = 0; v < 4; ++v) in[v] = G->g[GI(G, v, j, is)];
      ghost_value(P, &bc[side], 0, in, out);
      for (int v = 0; v < 4; ++v) G->g[GI(G, v, j, ig)] = out[v];
    }
  }
}

void orc_recon2d(const orc_params* P, int nx, int ny, double Lx, double Ly, const orc_bc bc[4],
                 const double* U, const double* Wx, const double* Wy, double* coef) {
  const double dx = Lx / nx, dy = Ly / ny;
  ghosts G;
  G.g = (double*)malloc(sizeof(double) * 4 * (nx + 2) * (ny + 2));
  fill_ghosts(P, nx, ny, bc, U, &G);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double nb[5][4], fx[4][4], fy[4][4], co[4][6];
      for (int v = 0; v < 4; ++v) {
        nb[0][v] = G.g[GI(&G, v, j, i)];
        nb[1][v] = G.g[GI(&G, v, j, i + 1)];
        nb[2][v] = G.g[GI(&G, v, j, i - 1)];
        nb[3][v] = G.g[GI(&G, v, j + 1, i)];
        nb[4][v] = G.g[GI(&G, v, j - 1, i)];
        fx[0][v] = Wx[WXI(v, 0, j, i + 1)]; fx[1][v] = Wx[WXI(v, 1, j, i + 1)];
        fx[2][v] = Wx[WXI(v, 0, j, i)];     fx[3][v] = Wx[WXI(v, 1, j, i)];
        fy[0][v] = Wy[WYI(v, 0, j + 1, i)]; fy[1][v] = Wy[WYI(v, 1, j + 1, i)];
        fy[2][v] = Wy[WYI(v, 0, j, i)];     fy[3][v] = Wy[WYI(v, 1, j, i)];
      }
      orc_recon_cell(P, nb, fx, fy, dx, dy, co);
      for (int v = 0; v < 4; ++v)
        for (int k = 0; k < 6; ++k) coef[CI(v, k, j, i)] = co[v][k];
    }
  free(G.g);
}

/* face-frame value and derivatives (n, t, nn, nt, tt) of cell (i, j)'s
 * polynomial at the point (x, y) of its local coordinates */
static void side_state(const double* coef, int nx, int ny, int i, int j, int axis, double dx,
                       double dy, double x, double y, double S[6][4]) {
  double w[6][4];
  for (int v = 0; v < 4; ++v) {
    double a[6], o[6];
    for (int k = 0; k < 6; ++k) a[k] = coef[CI(v, k, j, i)];
    poly_eval(a, dx, dy, x, y, o);
    for (int d = 0; d < 6; ++d) w[d][v] = o[d];
  }
  /* o = (P, Px, Py, Pxx, Pxy, Pyy); face frame order (P, Pn, Pt, Pnn, Pnt, Ptt) */
  const int ord_x[6] = {0, 1, 2, 3, 4, 5};
  const int ord_y[6] = {0, 2, 1, 5, 4, 3};
  for (int d = 0; d < 6; ++d) to_frame(axis, w[axis == 0 ? ord_x[d] : ord_y[d]], S[d]);
}

void orc_flux2d(const orc_params* P, int nx, int ny, double Lx, double Ly, const orc_bc bc[4],
                const double* U, const double* Wx, const double* Wy, double dt, double* Fx,
                double* Fy, double* Wxn, double* Wyn) {
  const double dx = Lx / nx, dy = Ly / ny;
  double* coef = (double*)malloc(sizeof(double) * 24 * nx * ny);
  orc_recon2d(P, nx, ny, Lx, Ly, bc, U, Wx, Wy, coef);
  ghosts G;
  G.g = (double*)malloc(sizeof(double) * 4 * (nx + 2) * (ny + 2));
  fill_ghosts(P, nx, ny, bc, U, &G);

  /* x-faces: face i lies between cells i-1 and i */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      double L[6][4], R[6][4], avg[2][3][4], F[4], Wg[2][4];
      int il = i - 1, ir = i;
      const int lo = (i == 0), hi = (i == nx);
      if (lo && bc[0].kind == ORC_BC_PERIODIC) il = nx - 1;
      if (hi && bc[1].kind == ORC_BC_PERIODIC) ir = 0;
      if (lo && bc[0].kind != ORC_BC_PERIODIC) {
        side_state(coef, nx, ny, ir, j, 0, dx, dy, -0.5 * dx, 0.0, R);
        orc_bc_image(P, bc[0].kind, bc[0].v_wall, bc[0].T_wall, R, L);
      } else if (hi && bc[1].kind != ORC_BC_PERIODIC) {
        side_state(coef, nx, ny, il, j, 0, dx, dy, 0.5 * dx, 0.0, L);
        orc_bc_image(P, bc[1].kind, bc[1].v_wall, bc[1].T_wall, L, R);
      } else {
        side_state(coef, nx, ny, il, j, 0, dx, dy, 0.5 * dx, 0.0, L);
        side_state(coef, nx, ny, ir, j, 0, dx, dy, -0.5 * dx, 0.0, R);
      }
      for (int m = 0; m < 2; ++m)
        for (int n = -1; n <= 1; ++n) {
          double w[4];
          for (int v = 0; v < 4; ++v) w[v] = G.g[GI(&G, v, j + n, i - 1 + m)];
          to_frame(0, w, avg[m][n + 1]);
        }
      orc_face(P, L, R, avg, dx, dy, dt, F, Wg, NULL);
      if (lo && bc[0].kind != ORC_BC_PERIODIC) wall_face_flux(&bc[0], 0, F);
      else if (hi && bc[1].kind != ORC_BC_PERIODIC) wall_face_flux(&bc[1], 0, F);
      for (int v = 0; v < 4; ++v) {
        Fx[((size_t)v * ny + j) * (nx + 1) + i] = F[v];
        Wxn[WXI(v, 0, j, i)] = Wg[0][v];
        Wxn[WXI(v, 1, j, i)] = Wg[1][v];
      }
    }

  /* y-faces: face j lies between cells j-1 and j; face frame n = y, t = x */
#pragma omp parallel for schedule(static)
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double L[6][4], R[6][4], avg[2][3][4], F[4], Wg[2][4], Ff[4], Wf[2][4];
      int jl = j - 1, jr = j;
      const int lo = (j == 0), hi = (j == ny);
      if (lo && bc[2].kind == ORC_BC_PERIODIC) jl = ny - 1;
      if (hi && bc[3].kind == ORC_BC_PERIODIC) jr = 0;
      if (lo && bc[2].kind != ORC_BC_PERIODIC) {
        side_state(coef, nx, ny, i, jr, 1, dx, dy, 0.0, -0.5 * dy, R);
        orc_bc_image(P, bc[2].kind, bc[2].u_wall, bc[2].T_wall, R, L);
      } else if (hi && bc[3].kind != ORC_BC_PERIODIC) {
        side_state(coef, nx, ny, i, jl, 1, dx, dy, 0.0, 0.5 * dy, L);
        orc_bc_image(P, bc[3].kind, bc[3].u_wall, bc[3].T_wall, L, R);
      } else {
        side_state(coef, nx, ny, i, jl, 1, dx, dy, 0.0, 0.5 * dy, L);
        side_state(coef, nx, ny, i, jr, 1, dx, dy, 0.0, -0.5 * dy, R);
      }
      for (int m = 0; m < 2; ++m)
        for (int n = -1; n <= 1; ++n) {
          double w[4];
          for (int v = 0; v < 4; ++v) w[v] = G.g[GI(&G, v, j - 1 + m, i + n)];
          to_frame(1, w, avg[m][n + 1]);
        }
      orc_face(P, L, R, avg, dy, dx, dt, Ff, Wf, NULL);
      if (lo && bc[2].kind != ORC_BC_PERIODIC) wall_face_flux(&bc[2], 1, Ff);
      else if (hi && bc[3].kind != ORC_BC_PERIODIC) wall_face_flux(&bc[3], 1, Ff);
      to_frame(1, Ff, F);
      to_frame(1, Wf[0], Wg[0]);
      to_frame(1, Wf[1], Wg[1]);
      for (int v = 0; v < 4; ++v) {
        Fy[((size_t)v * (ny + 1) + j) * nx + i] = F[v];
        Wyn[WYI(v, 0, j, i)] = Wg[0][v];
        Wyn[WYI(v, 1, j, i)] = Wg[1][v];
      }
    }
  free(G.g);
  free(coef);
}

/* state of cell (i, j) as a constant face state (value only), face frame */
static void const_state(const double* U, int nx, int ny, int i, int j, int axis, double S[6][4]) {
  double w[4];
  memset(S, 0, sizeof(double) * 24);
  for (int v = 0; v < 4; ++v) w[v] = U[UI(v, j, i)];
  to_frame(axis, w, S[0]);
}

/* first-order evolution at x-face (i, j) (axis 0) or y-face (i, j) (axis 1) */
static void face_first_order(const orc_params* P, int nx, int ny, double dx, double dy, const orc_bc bc[4],
                             const double* U, int axis, int i, int j, double dt, double F[4], double Wg[2][4]) {
  double L[6][4], R[6][4], Ff[4], Wf[2][4];
  const int f = axis == 0 ? i : j, nf = axis == 0 ? nx : ny;
  const orc_bc* blo = &bc[axis == 0 ? 0 : 2];
  const orc_bc* bhi = &bc[axis == 0 ? 1 : 3];
  int cl = f - 1, cr = f;
  if (f == 0 && blo->kind == ORC_BC_PERIODIC) cl = nf - 1;
  if (f == nf && bhi->kind == ORC_BC_PERIODIC) cr = 0;
#define CELL_I(n) (axis == 0 ? (n) : i)
#define CELL_J(n) (axis == 0 ? j : (n))
  if (f == 0 && blo->kind != ORC_BC_PERIODIC) {
    const_state(U, nx, ny, CELL_I(cr), CELL_J(cr), axis, R);
    orc_bc_image(P, blo->kind, wall_tangent_velocity(blo, axis), blo->T_wall, R, L);
  } else if (f == nf && bhi->kind != ORC_BC_PERIODIC) {
    const_state(U, nx, ny, CELL_I(cl), CELL_J(cl), axis, L);
    orc_bc_image(P, bhi->kind, wall_tangent_velocity(bhi, axis), bhi->T_wall, L, R);
  } else {
    const_state(U, nx, ny, CELL_I(cl), CELL_J(cl), axis, L);
    const_state(U, nx, ny, CELL_I(cr), CELL_J(cr), axis, R);
  }
#undef CELL_I
#undef CELL_J
  orc_face_first_order(P, L, R, axis == 0 ? dx : dy, axis == 0 ? dy : dx, dt, Ff, Wf, NULL);
  if (f == 0 && blo->kind != ORC_BC_PERIODIC) wall_face_flux(blo, axis, Ff);
  else if (f == nf && bhi->kind != ORC_BC_PERIODIC) wall_face_flux(bhi, axis, Ff);
  to_frame(axis, Ff, F);
  to_frame(axis, Wf[0], Wg[0]);
  to_frame(axis, Wf[1], Wg[1]);
}

/* Eq. finite into Un; returns the number of non-physical cells and marks them */
static int update_cells(const orc_params* P, int nx, int ny, double dx, double dy, const double* U,
                        const double* Fx, const double* Fy, double* Un, unsigned char* bad) {
  int nbad = 0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double w[4];
      for (int v = 0; v < 4; ++v) {
        const double fw = Fx[((size_t)v * ny + j) * (nx + 1) + i];
        const double fe = Fx[((size_t)v * ny + j) * (nx + 1) + i + 1];
        const double gs = Fy[((size_t)v * (ny + 1) + j) * nx + i];
        const double gn = Fy[((size_t)v * (ny + 1) + j + 1) * nx + i];
        w[v] = U[UI(v, j, i)] + (fw - fe) / dx + (gs - gn) / dy;
        Un[UI(v, j, i)] = w[v];
      }
      double r, u, vv, p;
      cons_prim(w, P->gamma, &r, &u, &vv, &p);
      const int b = !(r > 0.0) || !(p > 0.0) || !isfinite(w[0]) || !isfinite(w[1]) || !isfinite(w[2]) ||
                    !isfinite(w[3]);
      bad[(size_t)j * nx + i] = (unsigned char)b;
      nbad += b;
    }
  return nbad;
}

void orc_flux2d_faces(const orc_params* P, int nx, int ny, double Lx, double Ly, const orc_bc bc[4],
                      const double* U, const double* Wx, const double* Wy, double dt, int n, const int* faces,
                      double* F, double* Wg) {
  const double dx = Lx / nx, dy = Ly / ny;
  double* coef = (double*)malloc(sizeof(double) * 24 * nx * ny);
  orc_recon2d(P, nx, ny, Lx, Ly, bc, U, Wx, Wy, coef);
  ghosts G;
  G.g = (double*)malloc(sizeof(double) * 4 * (nx + 2) * (ny + 2));
  fill_ghosts(P, nx, ny, bc, U, &G);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < n; ++k) {
    const int axis = faces[3 * k], i = faces[3 * k + 1], j = faces[3 * k + 2];
    double L[6][4], R[6][4], avg[2][3][4], Ff[4], Wf[2][4];
    const int f = axis == 0 ? i : j, nf = axis == 0 ? nx : ny;
    const orc_bc* blo = &bc[axis == 0 ? 0 : 2];
    const orc_bc* bhi = &bc[axis == 0 ? 1 : 3];
    int cl = f - 1, cr = f;
    if (f == 0 && blo->kind == ORC_BC_PERIODIC) cl = nf - 1;
    if (f == nf && bhi->kind == ORC_BC_PERIODIC) cr = 0;
    const double hn = axis == 0 ? 0.5 * dx : 0.5 * dy;
    const int ci0 = axis == 0 ? cl : i, cj0 = axis == 0 ? j : cl;
    const int ci1 = axis == 0 ? cr : i, cj1 = axis == 0 ? j : cr;
    const double px = axis == 0 ? hn : 0.0, py = axis == 0 ? 0.0 : hn;
    if (f == 0 && blo->kind != ORC_BC_PERIODIC) {
      side_state(coef, nx, ny, ci1, cj1, axis, dx, dy, -px, -py, R);
      orc_bc_image(P, blo->kind, wall_tangent_velocity(blo, axis), blo->T_wall, R, L);
    } else if (f == nf && bhi->kind != ORC_BC_PERIODIC) {
      side_state(coef, nx, ny, ci0, cj0, axis, dx, dy, px, py, L);
      orc_bc_image(P, bhi->kind, wall_tangent_velocity(bhi, axis), bhi->T_wall, L, R);
    } else {
      side_state(coef, nx, ny, ci0, cj0, axis, dx, dy, px, py, L);
      side_state(coef, nx, ny, ci1, cj1, axis, dx, dy, -px, -py, R);
    }
    for (int m = 0; m < 2; ++m)
      for (int t = -1; t <= 1; ++t) {
        double w[4];
        for (int v = 0; v < 4; ++v)
          w[v] = axis == 0 ? G.g[GI(&G, v, j + t, i - 1 + m)] : G.g[GI(&G, v, j - 1 + m, i + t)];
        to_frame(axis, w, avg[m][t + 1]);
      }
    orc_face(P, L, R, avg, axis == 0 ? dx : dy, axis == 0 ? dy : dx, dt, Ff, Wf, NULL);
    if (f == 0 && blo->kind != ORC_BC_PERIODIC) wall_face_flux(blo, axis, Ff);
    else if (f == nf && bhi->kind != ORC_BC_PERIODIC) wall_face_flux(bhi, axis, Ff);
    double Fp[4], W0[4], W1[4];
    to_frame(axis, Ff, Fp);
    to_frame(axis, Wf[0], W0);
    to_frame(axis, Wf[1], W1);
    for (int v = 0; v < 4; ++v) {
      F[4 * k + v] = Fp[v];
      Wg[8 * k + v] = W0[v];
      Wg[8 * k + 4 + v] = W1[v];
    }
  }
  free(G.g);
  free(coef);
}

int orc_step2d(const orc_params* P, int nx, int ny, double Lx, double Ly, const orc_bc bc[4],
               double CFL, double dt_max, int viscous_dt, double* U, double* Wx, double* Wy,
               double* dt_out) {
  const double dx = Lx / nx, dy = Ly / ny;
  const double dt = orc_dt2d(P, nx, ny, Lx, Ly, U, CFL, dt_max, viscous_dt);
  const size_t nU = (size_t)4 * nx * ny, nWx = (size_t)8 * ny * (nx + 1), nWy = (size_t)8 * (ny + 1) * nx;
  double* Fx = (double*)malloc(sizeof(double) * 4 * ny * (nx + 1));
  double* Fy = (double*)malloc(sizeof(double) * 4 * (ny + 1) * nx);
  double* Wxn = (double*)malloc(sizeof(double) * nWx);
  double* Wyn = (double*)malloc(sizeof(double) * nWy);
  double* Un = (double*)malloc(sizeof(double) * nU);
  unsigned char* bad = (unsigned char*)malloc((size_t)nx * ny);
  orc_flux2d(P, nx, ny, Lx, Ly, bc, U, Wx, Wy, dt, Fx, Fy, Wxn, Wyn);
  /* Eq. finite with the analytically time-integrated, face-averaged fluxes */
  int nbad = update_cells(P, nx, ny, dx, dy, U, Fx, Fy, Un, bad);
  /* positivity fallback (the paper is silent on positivity): if the update makes
   * some cell non-physical, every face of such a cell is evolved again with the
   * collisionless first-order flux and the update is redone; if some cell is
   * still non-physical, every face of the grid gets that flux for this step */
  for (int level = 1; nbad && level <= 2; ++level) {
    unsigned char* marked = (unsigned char*)malloc((size_t)nx * ny);
    for (size_t c = 0; c < (size_t)nx * ny; ++c) marked[c] = level == 2 ? 1 : bad[c];
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        const int il = i == 0 ? (bc[0].kind == ORC_BC_PERIODIC ? nx - 1 : -1) : i - 1;
        const int ir = i == nx ? (bc[1].kind == ORC_BC_PERIODIC ? 0 : -1) : i;
        if (!((il >= 0 && marked[(size_t)j * nx + il]) || (ir >= 0 && marked[(size_t)j * nx + ir]))) continue;
        double F[4], Wg[2][4];
        face_first_order(P, nx, ny, dx, dy, bc, U, 0, i, j, dt, F, Wg);
        for (int v = 0; v < 4; ++v) {
          Fx[((size_t)v * ny + j) * (nx + 1) + i] = F[v];
          Wxn[WXI(v, 0, j, i)] = Wg[0][v];
          Wxn[WXI(v, 1, j, i)] = Wg[1][v];
        }
      }
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int jl = j == 0 ? (bc[2].kind == ORC_BC_PERIODIC ? ny - 1 : -1) : j - 1;
        const int jr = j == ny ? (bc[3].kind == ORC_BC_PERIODIC ? 0 : -1) : j;
        if (!((jl >= 0 && marked[(size_t)jl * nx + i]) || (jr >= 0 && marked[(size_t)jr * nx + i]))) continue;
        double F[4], Wg[2][4];
        face_first_order(P, nx, ny, dx, dy, bc, U, 1, i, j, dt, F, Wg);
        for (int v = 0; v < 4; ++v) {
          Fy[((size_t)v * (ny + 1) + j) * nx + i] = F[v];
          Wyn[WYI(v, 0, j, i)] = Wg[0][v];
          Wyn[WYI(v, 1, j, i)] = Wg[1][v];
        }
      }
    free(marked);
    nbad = update_cells(P, nx, ny, dx, dy, U, Fx, Fy, Un, bad);
  }
  if (!nbad) {
    memcpy(U, Un, sizeof(double) * nU);
    memcpy(Wx, Wxn, sizeof(double) * nWx);
    memcpy(Wy, Wyn, sizeof(double) * nWy);
  }
  free(Fx); free(Fy); free(Wxn); free(Wyn); free(Un); free(bad);
  if (dt_out) *dt_out = dt;
  return nbad ? ORC_ENONPHYSICAL : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* unit-level exports                                                  */
/* ------------------------------------------------------------------ */
void orc_moments(double U, double V, double lam, double K, int half, double mu_out[10],
                 double mv_out[10], double mxi_out[3]) {
  maxw m;
  maxw_set(&m, 1.0, U, V, lam, K);
  for (int n = 0; n < NMOM; ++n) { mu_out[n] = m.mu[half][n]; mv_out[n] = m.mv[n]; }
  for (int n = 0; n < 3; ++n) mxi_out[n] = m.mxi[n];
}

void orc_solve_coef(double rho, double U, double V, double lam, double K, const double rhs[4],
                    double a_out[4]) {
  maxw m;
  maxw_set(&m, rho, U, V, lam, K);
  double r[4];
  for (int k = 0; k < 4; ++k) r[k] = rhs[k] / rho;
  maxw_solve(&m, r, a_out);
}
