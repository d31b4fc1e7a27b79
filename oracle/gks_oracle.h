/*
 * Oracle of the compact third-order gas-kinetic scheme (Pan & Xu, "A compact
 * third-order gas-kinetic scheme for compressible Euler and Navier-Stokes
 * equations", arXiv:1412.4489).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow FP64 CPU restatement of the
 * scheme, written from the paper to check the CUDA library against.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Layout of the 2D state (structure of arrays, row-major, x fastest):
 *   U [4][ny][nx]          cell averages (rho, rho*U, rho*V, rho*E)      (Eq. finite)
 *   Wx[4][2][ny][nx+1]     point values on x-faces at the two Gauss points
 *                          y_j -/+ (sqrt(3)/6) dy   (g = 0, 1)          (Eq. point)
 *   Wy[4][2][ny+1][nx]     point values on y-faces at x_i -/+ (sqrt(3)/6) dx
 * 1D state: U[3][nx] (rho, rho*U, rho*E), W[3][nx+1] (one point per face).
 */
#ifndef GKS_ORACLE_H
#define GKS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Physical and scheme constants.  weno_eps / weno_C are the epsilon and C of
 * the nonlinear weights (Section 3.1, Eq. average; the paper gives neither
 * value); tau_eps / tau_C the constants of the inviscid collision time
 * (Section 4: 0.05 and 1). */
typedef struct {
  double gamma, mu, Pr;
  double weno_eps, weno_C;
  double tau_eps, tau_C;
  int characteristic;  /* 1: reconstruct in characteristic variables (Section 4's choice for
                          flows with discontinuities), 0: conservative variables */
} orc_params;

enum { ORC_BC_PERIODIC = 0, ORC_BC_OUTFLOW = 1, ORC_BC_SLIPWALL = 2, ORC_BC_NOSLIP_ISOTHERMAL = 3,
       ORC_BC_NOSLIP_ADIABATIC = 4 };

/* One side of the domain.  T_wall is the wall temperature p/rho. */
typedef struct {
  int kind;
  double u_wall, v_wall, T_wall;
} orc_bc;

enum { ORC_OK = 0, ORC_ENONPHYSICAL = 4 };

/* ---- unit-level entry points (used by the pins) ---- */

/* Normalised Maxwellian moments <u^n> (n = 0..9) over the full space (half=0),
 * u>0 (half=1) or u<0 (half=2); <v^n> over the full space; <xi^0,2,4>. */
void orc_moments(double U, double V, double lam, double K, int half,
                 double mu_out[10], double mv_out[10], double mxi_out[3]);

/* Solves <a> = rhs for a coefficient a = a1 + a2 u + a3 v + a4 (u^2+v^2+xi^2)/2,
 * where <.> = int g (.) psi dXi and g is the Maxwellian (rho, U, V, lam). */
void orc_solve_coef(double rho, double U, double V, double lam, double K,
                    const double rhs[4], double a_out[4]);

/* C_1..C_8, C_7 t and C_7 t^2 at time t (out[1..10]); and their integrals over
 * [0, T] (out_int[1..10]).  out[0] is unused. */
void orc_time_coefs(double t, double tau, double out[11]);
void orc_time_integrals(double T, double tau, double out_int[11]);

/* Gas evolution at one cell-interface centre (Section 2.2), in the face frame:
 * n = normal, t = tangential, conservative variables (rho, rho*u_n, rho*u_t, rho*E).
 * L, R: value and derivatives (d/dn, d/dt, d2/dn2, d2/dndt, d2/dt2) of the left
 * (n<0) and right (n>0) reconstructed polynomials at the face centre.
 * avg[m][k]: cell averages U_{m, k-1} (m = 0 left / 1 right cell column,
 * k-1 = -1,0,1 tangential offset) for the equilibrium polynomial (Section 3.3).
 * dn, dtan: cell size normal / along the face.  dt: time step.
 * Outputs: Fhat = time-integrated, face-averaged flux per unit face length;
 * Wg[g] = point values at t = dt at the Gauss points t = -/+ (sqrt(3)/6) dtan.
 * dbg (may be NULL, 64 doubles): U0[4], tau, b2..b6 (20), then unused. */
void orc_face(const orc_params* P, const double L[6][4], const double R[6][4],
              const double avg[2][3][4], double dn, double dtan, double dt,
              double Fhat[4], double Wg[2][4], double* dbg);

/* The evolution of the positivity fallback: the collisionless first-order
 * limit for constant states L[0], R[0] (derivatives ignored).  Outputs as
 * orc_face; dbg[0..3] = U0. */
void orc_face_first_order(const orc_params* P, const double L[6][4], const double R[6][4],
                          double dn, double dtan, double dt, double Fhat[4], double Wg[2][4],
                          double* dbg);

/* Same for a face whose outside state is the boundary image of the inside one
 * (outflow continuation or a wall mirror).  inside_right = 1 when the inside
 * cell lies at n>0.  The face frame's tangential wall velocity is u_wall_t. */
void orc_bc_image(const orc_params* P, int kind, double u_wall_t, double T_wall,
                  const double in[6][4], double out[6][4]);

/* Compact reconstruction of one cell (Section 3.2), all four variables.
 * nb[0..4] = U of the cell, east, west, north, south neighbours ([k][var]);
 * fx[0..3][var] = east face y-/y+, west face y-/y+ Gauss values;
 * fy[0..3][var] = north face x-/x+, south face x-/x+ Gauss values.
 * coef_out[var][6] = (Ubar, a2, a3, a4, a5, a6). */
void orc_recon_cell(const orc_params* P, const double nb[5][4], const double fx[4][4],
                    const double fy[4][4], double dx, double dy, double coef_out[4][6]);

/* Eigenvectors of the x-direction flux Jacobian of the 2D Euler equations at the
 * conservative state w (columns of R, rows of L = R^-1), for the characteristic
 * reconstruction. */
void orc_char_basis(const double w[4], double gamma, double L[4][4], double R[4][4]);

/* ---- grid-level entry points ---- */

/* CFL time step of the state U: CFL * min over cells of min(dx/(|U|+c), dy/(|V|+c)),
 * optionally also bounded by the viscous limit, clipped to dt_max. */
double orc_dt2d(const orc_params* P, int nx, int ny, double Lx, double Ly, const double* U,
                double CFL, double dt_max, int viscous_dt);

/* Reconstructed coefficients of every cell: coef[4][6][ny][nx]. */
void orc_recon2d(const orc_params* P, int nx, int ny, double Lx, double Ly, const orc_bc bc[4],
                 const double* U, const double* Wx, const double* Wy, double* coef);

/* Face fluxes and new point values for a given dt: Fx[4][ny][nx+1], Fy[4][ny+1][nx],
 * Wx_new, Wy_new as in the state layout. */
void orc_flux2d(const orc_params* P, int nx, int ny, double Lx, double Ly, const orc_bc bc[4],
                const double* U, const double* Wx, const double* Wy, double dt,
                double* Fx, double* Fy, double* Wx_new, double* Wy_new);

/* The evolution at n listed faces only (faces[3k..3k+2] = axis, i, j; axis 0 =
 * x-face i between cells i-1 and i of row j, axis 1 = y-face j of column i),
 * for sampled checks of large grids: F[4k..] the flux, Wg[8k..] the two point
 * values (state layout order).  The reconstruction is done for the whole grid. */
void orc_flux2d_faces(const orc_params* P, int nx, int ny, double Lx, double Ly, const orc_bc bc[4],
                      const double* U, const double* Wx, const double* Wy, double dt, int n, const int* faces,
                      double* F, double* Wg);

/* One full step in place.  bc order: x-low, x-high, y-low, y-high.  If the
 * update makes cells non-physical, their faces are evolved again with the
 * collisionless first-order flux and the update is redone; if cells are still
 * non-physical, every face of the grid gets that flux.  Returns ORC_OK or
 * ORC_ENONPHYSICAL (still not physical; state left unchanged). */
int orc_step2d(const orc_params* P, int nx, int ny, double Lx, double Ly, const orc_bc bc[4],
               double CFL, double dt_max, int viscous_dt, double* U, double* Wx, double* Wy,
               double* dt_out);

/* Number of OpenMP threads the grid-level calls use (1 if built without OpenMP). */
int orc_num_threads(void);
void orc_set_num_threads(int n);

/* ---- independent 1D scheme (Section 3.1, 1D solver of Section 2.2) ---- */
void orc1d_face(const orc_params* P, const double L[3][3], const double R[3][3],
                const double avg[2][3], double dx, double dt, double Fhat[3], double W[3],
                double* dbg);
void orc1d_recon_cell(const orc_params* P, const double nb[3][3], const double fw[2][3],
                      double dx, double coef_out[3][3]);
double orc1d_dt(const orc_params* P, int nx, double Lx, const double* U, double CFL, double dt_max);
int orc1d_step(const orc_params* P, int nx, double Lx, int periodic, double CFL, double dt_max,
               double* U, double* W, double* dt_out);

#ifdef __cplusplus
}
#endif
#endif
