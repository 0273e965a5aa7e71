/*
 * UGKS oracle: a plain, slow FP64 CPU implementation of one explicit step of the
 * 2D Unified Gas-Kinetic Scheme (Liu, Hu & Li, arXiv:1810.08137, Sec. 2, Eqs. 1-4,
 * with the flux construction steps S1-S8 of the Sec. 2.B table).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this code: only the tests, the smoke check and the CPU-baseline leg of the bench do.
 * It shares no code, header or constant table with the CUDA library.
 *
 * Layouts (the same public layout the CUDA library uses, restated independently):
 *   cell index   c = j*nx + i            (x fastest)
 *   velocity     q = m*nu + k            (u fastest); u_k, v_m
 *   f[c][q][2]   component 0 = h = int f dxi, component 1 = b = int xi^2 f dxi
 *   W[4][c]      (rho, rho U, rho V, rho E)
 */
#ifndef UGKS_ORACLE_H
#define UGKS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_PERIODIC = 0, ORC_BC_WALL = 1, ORC_BC_PRESSURE = 2 };
enum { ORC_W = 0, ORC_E = 1, ORC_S = 2, ORC_N = 3 };

typedef struct {
  int nx, ny;
  double lx, ly;
  int nu, nv;
  double umin, umax, vmin, vmax;
  int K;                       /* internal degrees of freedom (1 = monatomic in 2D) */
  double kn, omega, alpha;     /* tau from Kn through the VHS/VSS viscosity law */
  double cfl, dt;              /* dt <= 0: dt from the CFL number */
  int bc_kind[4];              /* W, E, S, N */
  double bc_rho[4], bc_T[4], bc_U[4];
  double pr;                   /* Prandtl number: 1 = BGK (Eq. 1); otherwise the Shakhov model */
} orc_cfg;

void   orc_set_threads(int n);
int    orc_get_threads(void);
void   orc_vgrid(const orc_cfg* c, double* u, double* v, double* w);
double orc_dt(const orc_cfg* c);
double orc_tau(const orc_cfg* c, double rho, double lam);
void   orc_mt(double dt, double tau, double Mt[5]);
void   orc_gauss_moments(double U, double lam, int nmax, double* full, double* pos, double* neg);
void   orc_slope_solve(const double prim[4], int K, const double s[4], double a[4]);
void   orc_init_maxwellian(const orc_cfg* c, const double* rho, const double* U, const double* V,
                           const double* T, double* f, double* W);
/* All face fluxes of one step from state (f, W):
 *   Fx[(nx+1)*ny][4], Fy[nx*(ny+1)][4]   time-integrated macroscopic fluxes (x frame)
 *   fx[(nx+1)*ny][nq][2], fy[nx*(ny+1)][nq][2]  time-integrated micro fluxes
 * x-face (i+1/2, j), i = -1..nx-1, is stored at  j*(nx+1) + (i+1);
 * y-face (i, j+1/2), j = -1..ny-1, is stored at (j+1)*nx + i.  Any output may be NULL. */
void   orc_fluxes(const orc_cfg* c, const double* f, const double* W,
                  double* Fx, double* Fy, double* fx, double* fy);
/* nsteps explicit UGKS steps in place (Eq. 3 for f, Eq. 4 for W). */
void   orc_step(const orc_cfg* c, double* f, double* W, int nsteps);
/* Shakhov equilibrium of prim = (rho, U, V, lam) with heat flux q = (qx, qy) at the n
 * velocities (u[i], v[i]): out[i][0] = h, out[i][1] = b (reduced over the internal variable). */
void   orc_shakhov_eq(const double prim[4], int K, double pr, const double q[2], int n,
                      const double* u, const double* v, double* out);
/* Heat flux q = 1/2 sum w c (|c|^2 h + b) of one cell's f[nq][2] about the velocity of W. */
void   orc_heat_flux(const orc_cfg* c, const double* f, const double W[4], double q[2]);
/* One step for the listed cells only: f_out[n][nq][2], W_out[n][4] for cell ids[n]. */
void   orc_step_cells(const orc_cfg* c, const double* f, const double* W, int ncell,
                      const int* ids, double* f_out, double* W_out);

#ifdef __cplusplus
}
#endif
#endif
