/*
 * One-dimensional oracle of the compact third-order gas-kinetic scheme
 * (Pan & Xu, arXiv:1412.4489).  TEST INFRASTRUCTURE ONLY (see gks_oracle.h).
 *
 * An independent restatement of Section 3.1 (compact 1D reconstruction) and
 * of the 1D form of Section 2.2 (all tangential terms of Eq. dis1 / dis2
 * dropped), with psi = (1, u, (u^2+xi^2)/2) and K1 = (3-gamma)/(gamma-1)
 * internal degrees of freedom.  It shares no routine with the 2D oracle, so
 * 2D runs on data that do not depend on y can be checked against it.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "gks_oracle.h"

#define M1 10
#define Q1CAP 96

typedef struct {
  double rho, U, lam, K;
  double mu[3][M1]; /* <u^n>/rho over all u, u>0, u<0 */
  double mxi[3];
} g1;

static void g1_set(g1* g, double rho, double U, double lam, double K) {
  g->rho = rho; g->U = U; g->lam = lam; g->K = K;
  const double s2 = 0.5 / lam;
  const double b = exp(-lam * U * U) * 0.5 / sqrt(M_PI * lam);
  g->mu[0][0] = 1.0;                      g->mu[0][1] = U;
  g->mu[1][0] = 0.5 * erfc(-sqrt(lam) * U); g->mu[1][1] = U * g->mu[1][0] + b;
  g->mu[2][0] = 0.5 * erfc(sqrt(lam) * U);  g->mu[2][1] = U * g->mu[2][0] - b;
  for (int n = 2; n < M1; ++n)
    for (int h = 0; h < 3; ++h) g->mu[h][n] = U * g->mu[h][n - 1] + (n - 1) * s2 * g->mu[h][n - 2];
  g->mxi[0] = 1.0;
  g->mxi[1] = K * s2;
  g->mxi[2] = K * (K + 2.0) * s2 * s2;
}

/* (rho, rho U, rho E) with rho E = rho U^2/2 + (K+1) rho/(4 lam) */
static void g1_from_cons(g1* g, const double w[3], double K) {
  const double U = w[1] / w[0];
  const double lam = (K + 1.0) * w[0] / (4.0 * (w[2] - 0.5 * w[0] * U * U));
  g1_set(g, w[0], U, lam, K);
}

/* polynomials c u^p (xi^2)^r */
typedef struct { int n; double c[Q1CAP]; int p[Q1CAP], r[Q1CAP]; } q1;

static void q1_add(q1* a, double c, int p, int r) {
  if (c == 0.0) return;
  if (a->n >= Q1CAP) abort();
  a->c[a->n] = c; a->p[a->n] = p; a->r[a->n] = r; a->n++;
}

static void q1_mul(const q1* a, const q1* b, q1* o) {
  o->n = 0;
  for (int i = 0; i < a->n; ++i)
    for (int j = 0; j < b->n; ++j) q1_add(o, a->c[i] * b->c[j], a->p[i] + b->p[j], a->r[i] + b->r[j]);
}

static void q1_psi(int k, q1* o) {
  o->n = 0;
  if (k == 0) q1_add(o, 1.0, 0, 0);
  else if (k == 1) q1_add(o, 1.0, 1, 0);
  else { q1_add(o, 0.5, 2, 0); q1_add(o, 0.5, 0, 1); }
}

static void q1_coef(const double X[3], q1* o) {
  o->n = 0;
  q1_add(o, X[0], 0, 0);
  q1_add(o, X[1], 1, 0);
  q1_add(o, 0.5 * X[2], 2, 0);
  q1_add(o, 0.5 * X[2], 0, 1);
}

static double g1_mom(const g1* g, int h, const q1* a) {
  double s = 0.0;
  for (int k = 0; k < a->n; ++k) {
    if (a->p[k] >= M1 || a->r[k] > 2) abort();
    s += a->c[k] * g->mu[h][a->p[k]] * g->mxi[a->r[k]];
  }
  return s;
}

static void g1_mom3(const g1* g, int h, const q1* a, double o[3]) {
  q1 ps, pr;
  for (int b = 0; b < 3; ++b) {
    q1_psi(b, &ps);
    q1_mul(a, &ps, &pr);
    o[b] = g1_mom(g, h, &pr);
  }
}

static void g1_solve(const g1* g, const double r[3], double x[3]) {
  double M[3][4];
  q1 pa, pb, pr;
  for (int b = 0; b < 3; ++b) {
    q1_psi(b, &pb);
    for (int a = 0; a < 3; ++a) {
      q1_psi(a, &pa);
      q1_mul(&pa, &pb, &pr);
      M[b][a] = g1_mom(g, 0, &pr);
    }
    M[b][3] = r[b];
  }
  for (int c = 0; c < 3; ++c) {
    int piv = c;
    for (int k = c + 1; k < 3; ++k)
      if (fabs(M[k][c]) > fabs(M[piv][c])) piv = k;
    for (int k = 0; k < 4; ++k) { double t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t; }
    for (int k = c + 1; k < 3; ++k) {
      const double f = M[k][c] / M[c][c];
      for (int l = c; l < 4; ++l) M[k][l] -= f * M[c][l];
    }
  }
  for (int k = 2; k >= 0; --k) {
    double s = M[k][3];
    for (int l = k + 1; l < 3; ++l) s -= M[k][l] * x[l];
    x[k] = s / M[k][k];
  }
}

/* <X u psi>/rho over the full space */
static void g1_mom_u(const g1* g, const double X[3], double o[3]) {
  q1 px, pu, pr;
  q1_coef(X, &px);
  pu.n = 0;
  q1_add(&pu, 1.0, 1, 0);
  q1_mul(&px, &pu, &pr);
  g1_mom3(g, 0, &pr, o);
}

typedef struct { double a1[3], Axx[3], A[3], Atx[3], Att[3]; } c1d;

/* <a1> = U_x, <a1^2+d11> = U_xx, <A + a1 u> = 0, <(a1^2+d11) u + (A a1+b1)> = 0,
 * <(A a1+b1) u + (A^2+B)> = 0 */
static void c1d_solve(const g1* g, const double ux[3], const double uxx[3], c1d* c) {
  double r[3], t[3];
  for (int k = 0; k < 3; ++k) r[k] = ux[k] / g->rho;
  g1_solve(g, r, c->a1);
  for (int k = 0; k < 3; ++k) r[k] = uxx[k] / g->rho;
  g1_solve(g, r, c->Axx);
  g1_mom_u(g, c->a1, t);
  for (int k = 0; k < 3; ++k) r[k] = -t[k];
  g1_solve(g, r, c->A);
  g1_mom_u(g, c->Axx, t);
  for (int k = 0; k < 3; ++k) r[k] = -t[k];
  g1_solve(g, r, c->Atx);
  g1_mom_u(g, c->Atx, t);
  for (int k = 0; k < 3; ++k) r[k] = -t[k];
  g1_solve(g, r, c->Att);
}

/* time functions, same numbering as the 2D file: 1..8 = C_1..C_8,
 * 9 = C_7 t, 10 = C_7 t^2 */
static double t1d_decay(double t, double tau) { return tau > 0.0 ? exp(-t / tau) : 0.0; }

static void t1d_at(double t, double tau, double c[11]) {
  const double e = t1d_decay(t, tau);
  c[1] = 1.0 - e; c[2] = (t + tau) * e - tau; c[3] = t - tau + tau * e;
  c[4] = -(t * t + 2.0 * t * tau) * e; c[5] = t * t - 2.0 * t * tau; c[6] = -t * tau * (1.0 + e);
  c[7] = e; c[8] = -t * e; c[9] = t * e; c[10] = t * t * e;
}

/* integrals of the above over [0, T] */
static void t1d_int(double T, double tau, double c[11]) {
  const double e = t1d_decay(T, tau), t2 = tau * tau;
  const double q = t2 - tau * (tau + T) * e; /* int_0^T t exp(-t/tau) dt */
  c[1] = T - tau * (1.0 - e);
  c[2] = q + tau * tau * (1.0 - e) - tau * T;
  c[3] = 0.5 * T * T - tau * T + t2 * (1.0 - e);
  c[4] = -(2.0 * t2 * tau - tau * (T * T + 2.0 * T * tau + 2.0 * t2) * e) - 2.0 * tau * q;
  c[5] = T * T * T / 3.0 - tau * T * T;
  c[6] = -tau * (0.5 * T * T + q);
  c[7] = tau * (1.0 - e);
  c[8] = -q;
  c[9] = q;
  c[10] = 2.0 * t2 * tau - tau * (T * T + 2.0 * T * tau + 2.0 * t2) * e;
}

typedef struct { int src, tid, p; double s, X[3]; } t1term;

void orc1d_face(const orc_params* P, const double L[3][3], const double R[3][3],
                const double avg[2][3], double dx, double dt, double Fhat[3], double W[3],
                double* dbg) {
  const double gam = P->gamma;
  const double K = (3.0 - gam) / (gam - 1.0);
  g1 gl, gr, g0;
  g1_from_cons(&gl, L[0], K);
  g1_from_cons(&gr, R[0], K);
  double U0[3], hl[3], hr[3];
  q1 one;
  one.n = 0;
  q1_add(&one, 1.0, 0, 0);
  g1_mom3(&gl, 1, &one, hl);
  g1_mom3(&gr, 2, &one, hr);
  for (int k = 0; k < 3; ++k) U0[k] = gl.rho * hl[k] + gr.rho * hr[k];
  g1_from_cons(&g0, U0, K);

  /* 1D equilibrium polynomial U0 + b2 x + b4 x^2/2 matching the two averages */
  double b2[3], b4[3];
  for (int k = 0; k < 3; ++k) {
    b2[k] = (avg[1][k] - avg[0][k]) / dx;
    b4[k] = 3.0 * (avg[0][k] + avg[1][k] - 2.0 * U0[k]) / (dx * dx);
  }
  const double pl = (gam - 1.0) * (L[0][2] - 0.5 * L[0][1] * L[0][1] / L[0][0]);
  const double pr = (gam - 1.0) * (R[0][2] - 0.5 * R[0][1] * R[0][1] / R[0][0]);
  const double p0 = (gam - 1.0) * (U0[2] - 0.5 * U0[1] * U0[1] / U0[0]);
  const double jump = fabs((pl - pr) / (pl + pr)) * dt;
  const int ns = P->mu > 0.0;
  const double tau = ns ? P->mu / p0 + jump : P->tau_eps * dt + P->tau_C * jump;

  c1d c0, cl, cr;
  c1d_solve(&g0, b2, b4, &c0);
  {
    double lx[3], lxx[3], rx[3], rxx[3];
    for (int k = 0; k < 3; ++k) { lx[k] = L[1][k]; lxx[k] = L[2][k]; rx[k] = R[1][k]; rxx[k] = R[2][k]; }
    c1d_solve(&gl, lx, lxx, &cl);
    c1d_solve(&gr, rx, rxx, &cr);
  }

  t1term T[40];
  int n = 0;
  const double e0[3] = {1, 0, 0};
#define ADD(S, TID, SC, XX, PP) do { T[n].src = S; T[n].tid = TID; T[n].s = SC; T[n].p = PP; \
    memcpy(T[n].X, XX, sizeof(double) * 3); ++n; } while (0)
  /* hydrodynamic part (1D Eq. dis1) */
  ADD(0, 1, 1.0, e0, 0);
  ADD(0, 2, 1.0, c0.a1, 1);
  ADD(0, 3, 1.0, c0.A, 0);
  ADD(0, 4, 0.5, c0.Axx, 2);
  ADD(0, 6, 1.0, c0.Atx, 1);
  ADD(0, 5, 0.5, c0.Att, 0);
  /* kinetic part (1D Eq. dis2) for both sides */
  for (int s = 1; s <= 2; ++s) {
    const c1d* c = s == 1 ? &cl : &cr;
    ADD(s, 7, 1.0, e0, 0);
    ADD(s, 8, 1.0, c->a1, 1);
    ADD(s, 10, 0.5, c->Axx, 2);
    if (ns) {
      ADD(s, 7, -tau, c->a1, 1);
      ADD(s, 7, -tau, c->A, 0);
      ADD(s, 8, -tau, c->Axx, 2);
      ADD(s, 8, -tau, c->Atx, 1);
    }
  }
#undef ADD
  double Ci[11], Ce[11];
  t1d_int(dt, tau, Ci);
  t1d_at(dt, tau, Ce);
  const g1* gs[3] = {&g0, &gl, &gr};
  double F[3] = {0, 0, 0}, Wv[3] = {0, 0, 0}, q = 0.0;
  q1 qw;
  {
    /* (u-U0) ((u-U0)^2 + xi^2)/2 */
    const double u0 = U0[1] / U0[0];
    q1 cu, cu2, e, tmp;
    cu.n = 0; q1_add(&cu, 1.0, 1, 0); q1_add(&cu, -u0, 0, 0);
    q1_mul(&cu, &cu, &cu2);
    e.n = 0;
    for (int k = 0; k < cu2.n; ++k) q1_add(&e, 0.5 * cu2.c[k], cu2.p[k], cu2.r[k]);
    q1_add(&e, 0.5, 0, 1);
    q1_mul(&cu, &e, &tmp);
    qw = tmp;
  }
  for (int k = 0; k < n; ++k) {
    const g1* g = gs[T[k].src];
    q1 px, pm, base, bu, bq;
    q1_coef(T[k].X, &px);
    pm.n = 0;
    q1_add(&pm, 1.0, T[k].p, 0);
    q1_mul(&px, &pm, &base);
    double m3[3];
    g1_mom3(g, T[k].src, &base, m3);
    for (int b = 0; b < 3; ++b) Wv[b] += T[k].s * Ce[T[k].tid] * g->rho * m3[b];
    pm.n = 0;
    q1_add(&pm, 1.0, 1, 0);
    q1_mul(&base, &pm, &bu);
    g1_mom3(g, T[k].src, &bu, m3);
    for (int b = 0; b < 3; ++b) F[b] += T[k].s * Ci[T[k].tid] * g->rho * m3[b];
    if (P->Pr != 1.0) {
      q1_mul(&base, &qw, &bq);
      q += T[k].s * Ci[T[k].tid] * g->rho * g1_mom(g, T[k].src, &bq);
    }
  }
  if (P->Pr != 1.0) F[2] += (1.0 / P->Pr - 1.0) * q;
  for (int k = 0; k < 3; ++k) { Fhat[k] = F[k]; W[k] = Wv[k]; }
  if (dbg) {
    for (int k = 0; k < 3; ++k) dbg[k] = U0[k];
    dbg[3] = tau;
    dbg[4] = q;
  }
}

static double mm(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

/* nb = (U_i, U_{i-1}, U_{i+1}), fw = (U_{i-1/2}, U_{i+1/2}); coef = (Ubar, a2, a3) */
void orc1d_recon_cell(const orc_params* P, const double nb[3][3], const double fw[2][3],
                      double dx, double coef[3][3]) {
  for (int v = 0; v < 3; ++v) {
    const double Ui = nb[0][v], Um = nb[1][v], Up = nb[2][v];
    /* one-sided stencils S1 = {U_{i-1}, U_{i-1/2}, U_i}, S2 = {U_i, U_{i+1/2}, U_{i+1}} */
    const double a31 = 3.0 * (Ui + Um - 2.0 * fw[0][v]) / (dx * dx);
    const double a32 = 3.0 * (Ui + Up - 2.0 * fw[1][v]) / (dx * dx);
    const double t21 = 2.0 * (fw[0][v] - Ui) / dx;
    const double t22 = 2.0 * (fw[1][v] - Ui) / dx;
    const double a3 = mm(a31, a32);                                      /* Eq. limiter */
    const double a2 = mm(-t21 + a3 * dx / 6.0, t22 - a3 * dx / 6.0);
    /* central stencil S3 */
    const double c2 = (Up - Um) / (2.0 * dx);
    const double c3 = (Up - 2.0 * Ui + Um) / (dx * dx);
    /* Eq. average with I(U) = sum_l int h^(2l-1) (U^(l))^2, I(U1) = C h^2 */
    const double I1 = P->weno_C * dx * dx;
    const double I2 = dx * dx * c2 * c2 + 13.0 / 12.0 * dx * dx * dx * dx * c3 * c3;
    const double al1 = 1.0 / ((P->weno_eps + I1) * (P->weno_eps + I1));
    const double al2 = 1.0 / ((P->weno_eps + I2) * (P->weno_eps + I2));
    const double w1 = al1 / (al1 + al2), w2 = 1.0 - w1;
    coef[v][0] = Ui;
    coef[v][1] = w1 * a2 + w2 * c2;
    coef[v][2] = w1 * a3 + w2 * c3;
    (void)w2;
  }
  /* fall back to the constant when a face value is not physical */
  for (int s = -1; s <= 1; s += 2) {
    double w[3];
    for (int v = 0; v < 3; ++v) w[v] = coef[v][0] + coef[v][1] * s * 0.5 * dx + coef[v][2] * dx * dx / 12.0;
    const double p = (P->gamma - 1.0) * (w[2] - 0.5 * w[1] * w[1] / w[0]);
    if (!(w[0] > 0.0) || !(p > 0.0)) {
      for (int v = 0; v < 3; ++v) coef[v][1] = coef[v][2] = 0.0;
      break;
    }
  }
}

double orc1d_dt(const orc_params* P, int nx, double Lx, const double* U, double CFL, double dt_max) {
  const double dx = Lx / nx;
  double m = INFINITY;
  for (int i = 0; i < nx; ++i) {
    const double r = U[i], u = U[nx + i] / r;
    const double p = (P->gamma - 1.0) * (U[2 * nx + i] - 0.5 * r * u * u);
    m = fmin(m, dx / (fabs(u) + sqrt(P->gamma * p / r)));
  }
  return fmin(CFL * m, dt_max);
}

int orc1d_step(const orc_params* P, int nx, double Lx, int periodic, double CFL, double dt_max,
               double* U, double* W, double* dt_out) {
  const double dx = Lx / nx;
  const double dt = orc1d_dt(P, nx, Lx, U, CFL, dt_max);
  double* co = (double*)malloc(sizeof(double) * 9 * nx);
  double* F = (double*)malloc(sizeof(double) * 3 * (nx + 1));
  double* Wn = (double*)malloc(sizeof(double) * 3 * (nx + 1));
#define CELL(v, i) U[(size_t)(v) * nx + (periodic ? (((i) % nx) + nx) % nx : ((i) < 0 ? 0 : ((i) >= nx ? nx - 1 : (i))))]
  for (int i = 0; i < nx; ++i) {
    double nb[3][3], fw[2][3], c[3][3];
    for (int v = 0; v < 3; ++v) {
      nb[0][v] = CELL(v, i); nb[1][v] = CELL(v, i - 1); nb[2][v] = CELL(v, i + 1);
      fw[0][v] = W[(size_t)v * (nx + 1) + i];
      fw[1][v] = W[(size_t)v * (nx + 1) + i + 1];
    }
    orc1d_recon_cell(P, nb, fw, dx, c);
    for (int v = 0; v < 3; ++v)
      for (int k = 0; k < 3; ++k) co[((size_t)v * 3 + k) * nx + i] = c[v][k];
  }
  for (int f = 0; f <= nx; ++f) {
    int il = f - 1, ir = f;
    if (periodic) { il = (il + nx) % nx; ir = ir % nx; }
    double L[3][3], R[3][3], avg[2][3], Fh[3], Wf[3];
    for (int v = 0; v < 3; ++v) {
      if (il >= 0) {
        const double a = co[((size_t)v * 3 + 0) * nx + il], b = co[((size_t)v * 3 + 1) * nx + il],
                     c = co[((size_t)v * 3 + 2) * nx + il];
        L[0][v] = a + b * 0.5 * dx + c * dx * dx / 12.0; L[1][v] = b + c * 0.5 * dx; L[2][v] = c;
      }
      if (ir < nx) {
        const double a = co[((size_t)v * 3 + 0) * nx + ir], b = co[((size_t)v * 3 + 1) * nx + ir],
                     c = co[((size_t)v * 3 + 2) * nx + ir];
        R[0][v] = a - b * 0.5 * dx + c * dx * dx / 12.0; R[1][v] = b - c * 0.5 * dx; R[2][v] = c;
      }
    }
    if (il < 0) memcpy(L, R, sizeof(L));     /* outflow: continue the inside polynomial */
    if (ir >= nx) memcpy(R, L, sizeof(R));
    for (int v = 0; v < 3; ++v) { avg[0][v] = CELL(v, f - 1); avg[1][v] = CELL(v, f); }
    orc1d_face(P, L, R, avg, dx, dt, Fh, Wf, NULL);
    for (int v = 0; v < 3; ++v) { F[(size_t)v * (nx + 1) + f] = Fh[v]; Wn[(size_t)v * (nx + 1) + f] = Wf[v]; }
  }
#undef CELL
  int bad = 0;
  double* Un = (double*)malloc(sizeof(double) * 3 * nx);
  for (int i = 0; i < nx; ++i) {
    for (int v = 0; v < 3; ++v)
      Un[(size_t)v * nx + i] = U[(size_t)v * nx + i] + (F[(size_t)v * (nx + 1) + i] - F[(size_t)v * (nx + 1) + i + 1]) / dx;
    const double r = Un[i], u = Un[nx + i] / r, p = (P->gamma - 1.0) * (Un[2 * nx + i] - 0.5 * r * u * u);
    if (!(r > 0.0) || !(p > 0.0)) bad = 1;
  }
  if (!bad) {
    memcpy(U, Un, sizeof(double) * 3 * nx);
    memcpy(W, Wn, sizeof(double) * 3 * (nx + 1));
  }
  free(Un); free(co); free(F); free(Wn);
  if (dt_out) *dt_out = dt;
  return bad ? ORC_ENONPHYSICAL : ORC_OK;
}
