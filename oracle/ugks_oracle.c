/*
 * UGKS oracle -- plain, slow, FP64 CPU implementation of the explicit 2D Unified
 * Gas-Kinetic Scheme step of Liu, Hu & Li (arXiv:1810.08137).
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the CPU-baseline
 * leg of the bench, never by the product path.  It shares no code with the CUDA library.
 *
 * What it follows, in order:
 *   Eq. 1   BGK model, Maxwellian g = rho (lam/pi) exp(-lam((u-U)^2+(v-V)^2)) (reduced form)
 *   Eq. 2   integral solution at a cell interface; its time integral gives Mt1..Mt5
 *   Sec. 2.B table, steps S1-S8, done face by face in that order
 *   Eq. 4   conservative update of W;  Eq. 3  implicit (trapezoidal) update of f
 * The paper does not print the flux construction (it defers to its refs [1,2]); where it is
 * silent this file takes these readings (the same ones the CUDA library takes):
 *   - K internal degrees of freedom carried by reduced distributions h = int f dxi and
 *     b = int xi^2 f dxi; psi = (1, u, v, (u^2+v^2+xi^2)/2).
 *   - velocities in units of sqrt(2kT0/m): lam = 1/T, p = rho/(2 lam).
 *   - tau = mu/p with mu = mu_ref T^omega, mu_ref = 5(a+1)(a+2)sqrt(pi)/(4a(5-2w)(7-2w)) Kn.
 *   - dt = CFL / (max|u|/dx + max|v|/dy) unless given.
 *   - uniform velocity grid including the end points, trapezoid weights; the grid is laid out
 *     symmetrically about the centre of the interval.
 *   - van Leer limited slopes per velocity and component; upwind choice H(un) with H(0)=1/2.
 *   - W0 = sum w psi f_up; normal slopes of W from (W0-W_L)/(dx/2), (W_R-W0)/(dx/2); the
 *     tangential slope of W from sum w psi sigma_t,up; the time slope A from compatibility.
 *   - equilibrium part of the macroscopic flux from analytic (half-range) moments, the
 *     free-transport part from discrete sums.
 *   - boundaries: periodic; diffuse isothermal wall (zero net mass flux, first order in
 *     time); pressure ghost = Maxwellian(rho_bc, U and V of the adjacent cell, T_bc) with
 *     zero slopes.
 *   - Prandtl number pr != 1 (not in the paper, which uses the BGK model of Eq. 1): the
 *     Shakhov model.  Its equilibrium g+ = g [1 + (1 - Pr) (c.q) (c_t^2/RT - (D+2)) /
 *     ((D+2) p RT)] (D = 2 + K degrees of freedom, c the peculiar velocity, c_t^2 = |c|^2 +
 *     xi^2, q the heat flux, RT = 1/(2 lam)) replaces g in the collision term.  At an
 *     interface the heat flux is that of the upwind interface values f_up about the
 *     interface velocity, and the Shakhov part enters the integral solution through the
 *     zeroth-order equilibrium term only (its Mt1 weight); the slopes a_L, a_R, b, A are
 *     those of the Maxwellian.  In Eq. 3 both g+^n and g+^{n+1} carry the heat flux of f^n
 *     about the cell's velocity (the heat flux of f^{n+1} is not known before f^{n+1}).
 */
#include "ugks_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;
void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------------------ */
/* Velocity grid (Sec. 2: K x M discrete velocities per cell).                          */
/* ------------------------------------------------------------------------------------ */
static void axis_grid(int n, double lo, double hi, double* x, double* wt) {
  if (n == 1) { x[0] = 0.5 * (lo + hi); wt[0] = 1.0; return; }
  double h = (hi - lo) / (n - 1), mid = 0.5 * (lo + hi);
  for (int k = 0; k < n; k++) {
    x[k] = mid + (k - 0.5 * (n - 1)) * h;
    wt[k] = (k == 0 || k == n - 1) ? 0.5 * h : h;
  }
}

void orc_vgrid(const orc_cfg* c, double* u, double* v, double* w) {
  double* wu = malloc(sizeof(double) * c->nu);
  double* wv = malloc(sizeof(double) * c->nv);
  axis_grid(c->nu, c->umin, c->umax, u, wu);
  axis_grid(c->nv, c->vmin, c->vmax, v, wv);
  for (int m = 0; m < c->nv; m++)
    for (int k = 0; k < c->nu; k++) w[m * c->nu + k] = wu[k] * wv[m];
  free(wu);
  free(wv);
}

double orc_dt(const orc_cfg* c) {
  if (c->dt > 0) return c->dt;
  double* u = malloc(sizeof(double) * c->nu);
  double* v = malloc(sizeof(double) * c->nv);
  double* w = malloc(sizeof(double) * c->nu * c->nv);
  orc_vgrid(c, u, v, w);
  double um = 0, vm = 0;
  for (int k = 0; k < c->nu; k++) um = fmax(um, fabs(u[k]));
  for (int m = 0; m < c->nv; m++) vm = fmax(vm, fabs(v[m]));
  free(u); free(v); free(w);
  double dx = c->lx / c->nx, dy = c->ly / c->ny;
  return c->cfl / (um / dx + vm / dy);
}

/* Collision time tau = mu / p, mu = mu_ref T^omega, p = rho/(2 lam), T = 1/lam. */
double orc_tau(const orc_cfg* c, double rho, double lam) {
  double a = c->alpha, om = c->omega;
  double mu_ref = 5.0 * (a + 1.0) * (a + 2.0) * sqrt(M_PI) /
                  (4.0 * a * (5.0 - 2.0 * om) * (7.0 - 2.0 * om)) * c->kn;
  double T = 1.0 / lam;
  double mu = mu_ref * pow(T, om);
  double p = rho / (2.0 * lam);
  return mu / p;
}

/* ------------------------------------------------------------------------------------ */
/* S3: time integrals of the Eq. 2 weights over one step, with x = dt/tau:              */
/*   Mt1 = int (1 - e^{-t/tau})             Mt4 = int e^{-t/tau}                         */
/*   Mt2 = int (tau(e^{-t/tau}-1) + t e^{-t/tau})   Mt5 = int t e^{-t/tau}                  */
/*   Mt3 = int (t - tau + tau e^{-t/tau})                                                */
/* written as dt*c1, dt^2*c2, dt^2*c3, dt*c4, dt^2*c5; power series below x = 0.1.      */
/* ------------------------------------------------------------------------------------ */
void orc_mt(double dt, double tau, double Mt[5]) {
  double x = dt / tau;
  double c1, c2, c3, c4, c5;
  if (x < 0.1) {
    /* c4 = sum (-x)^n/(n+1)!, c1 = 1-c4, c5 = sum (-1)^n (n+1) x^n/(n+2)!,
       c3 = sum_{n>=1} (-1)^{n+1} x^n/(n+2)!, c2 = sum_{n>=1} (-1)^n n x^n/(n+2)! */
    c1 = c2 = c3 = c4 = c5 = 0.0;
    double xn = 1.0;            /* x^n */
    double f1 = 1.0, f2 = 2.0;  /* (n+1)!, (n+2)! */
    for (int n = 0; n < 16; n++) {
      double sg = (n % 2 == 0) ? 1.0 : -1.0;
      c4 += sg * xn / f1;
      if (n >= 1) c1 += -sg * xn / f1;
      c5 += sg * (n + 1) * xn / f2;
      if (n >= 1) c3 += -sg * xn / f2;
      if (n >= 1) c2 += sg * n * xn / f2;
      xn *= x;
      f1 *= (n + 2);
      f2 *= (n + 3);
    }
  } else {
    double e = exp(-x);
    double em = -expm1(-x); /* 1 - e^{-x} */
    c4 = em / x;
    c1 = 1.0 - c4;
    c5 = (c4 - e) / x;
    c3 = 0.5 - c1 / x;
    c2 = c5 - c1 / x;
  }
  Mt[0] = dt * c1;
  Mt[1] = dt * dt * c2;
  Mt[2] = dt * dt * c3;
  Mt[3] = dt * c4;
  Mt[4] = dt * dt * c5;
}

/* ------------------------------------------------------------------------------------ */
/* S2: moments <x^n> of the 1D normalised Gaussian sqrt(lam/pi) exp(-lam (x-U)^2),       */
/* full range and the half ranges x>0 and x<0 (integration by parts gives the recursion  */
/* <x^{n+2}> = U <x^{n+1}> + (n+1)/(2 lam) <x^n>).                                        */
/* ------------------------------------------------------------------------------------ */
void orc_gauss_moments(double U, double lam, int nmax, double* full, double* pos, double* neg) {
  double e = exp(-lam * U * U) / (2.0 * sqrt(M_PI * lam));
  full[0] = 1.0;
  pos[0] = 0.5 * erfc(-sqrt(lam) * U);
  neg[0] = 0.5 * erfc(sqrt(lam) * U);
  if (nmax >= 1) {
    full[1] = U;
    pos[1] = U * pos[0] + e;
    neg[1] = U * neg[0] - e;
  }
  for (int n = 0; n + 2 <= nmax; n++) {
    full[n + 2] = U * full[n + 1] + (n + 1) / (2.0 * lam) * full[n];
    pos[n + 2] = U * pos[n + 1] + (n + 1) / (2.0 * lam) * pos[n];
    neg[n + 2] = U * neg[n + 1] + (n + 1) / (2.0 * lam) * neg[n];
  }
}

/* Polynomials in (un, ut, xi): sum of c * un^pu * ut^pv * |xi|^px. */
typedef struct { double c; int pu, pv, px; } term_t;
typedef struct { int n; term_t t[8]; } poly_t;

/* psi_i for i = 0..3: 1, un, ut, (un^2 + ut^2 + xi^2)/2 */
static poly_t psi_poly(int i) {
  poly_t p; memset(&p, 0, sizeof p);
  switch (i) {
    case 0: p.n = 1; p.t[0] = (term_t){1.0, 0, 0, 0}; break;
    case 1: p.n = 1; p.t[0] = (term_t){1.0, 1, 0, 0}; break;
    case 2: p.n = 1; p.t[0] = (term_t){1.0, 0, 1, 0}; break;
    default:
      p.n = 3;
      p.t[0] = (term_t){0.5, 2, 0, 0};
      p.t[1] = (term_t){0.5, 0, 2, 0};
      p.t[2] = (term_t){0.5, 0, 0, 2};
  }
  return p;
}

/* a . psi */
static poly_t apsi_poly(const double a[4]) {
  poly_t p; memset(&p, 0, sizeof p);
  p.n = 6;
  p.t[0] = (term_t){a[0], 0, 0, 0};
  p.t[1] = (term_t){a[1], 1, 0, 0};
  p.t[2] = (term_t){a[2], 0, 1, 0};
  p.t[3] = (term_t){0.5 * a[3], 2, 0, 0};
  p.t[4] = (term_t){0.5 * a[3], 0, 2, 0};
  p.t[5] = (term_t){0.5 * a[3], 0, 0, 2};
  return p;
}

/* Moments of the normalised Maxwellian with K internal degrees of freedom. */
typedef struct {
  double un[3][12]; /* 0: full, 1: un > 0, 2: un < 0 */
  double ut[12];
  double xi[7];     /* <|xi|^n>, n even */
} gmom_t;

static void gmom_init(double Un, double Ut, double lam, int K, gmom_t* g) {
  double dummy_p[12], dummy_n[12];
  orc_gauss_moments(Un, lam, 11, g->un[0], g->un[1], g->un[2]);
  orc_gauss_moments(Ut, lam, 11, g->ut, dummy_p, dummy_n);
  memset(g->xi, 0, sizeof g->xi);
  g->xi[0] = 1.0;
  g->xi[2] = K / (2.0 * lam);
  g->xi[4] = (K * K + 2.0 * K) / (4.0 * lam * lam);
}

/* < un^m ut^n P Q > over the un-range r. */
static double mom_pq(const gmom_t* g, int r, int m, int n, const poly_t* P, const poly_t* Q) {
  double s = 0.0;
  for (int a = 0; a < P->n; a++)
    for (int b = 0; b < Q->n; b++) {
      const term_t* x = &P->t[a];
      const term_t* y = &Q->t[b];
      s += x->c * y->c * g->un[r][x->pu + y->pu + m] * g->ut[x->pv + y->pv + n] *
           g->xi[x->px + y->px];
    }
  return s;
}

static double mom_p(const gmom_t* g, int r, int m, int n, const poly_t* P) {
  poly_t one; memset(&one, 0, sizeof one);
  one.n = 1; one.t[0] = (term_t){1.0, 0, 0, 0};
  return mom_pq(g, r, m, n, P, &one);
}

/* Larger polynomial in (un, ut, xi) for the Shakhov term, and its product moments. */
typedef struct { int n; term_t t[40]; } bpoly_t;

/* S(un, ut, xi) / alpha = (qn cn + qt ct) (2 lam (cn^2 + ct^2 + xi^2) - (K + 4)),
   cn = un - Un, ct = ut - Ut, expanded into monomials: a product of 4 and 8 terms. */
static bpoly_t shakhov_poly(double Un, double Ut, double lam, int K, const double q[2],
                            double alpha) {
  term_t a[4] = {{q[0], 1, 0, 0}, {-q[0] * Un, 0, 0, 0}, {q[1], 0, 1, 0}, {-q[1] * Ut, 0, 0, 0}};
  term_t b[8] = {{2.0 * lam, 2, 0, 0}, {-4.0 * lam * Un, 1, 0, 0}, {2.0 * lam * Un * Un, 0, 0, 0},
                 {2.0 * lam, 0, 2, 0}, {-4.0 * lam * Ut, 0, 1, 0}, {2.0 * lam * Ut * Ut, 0, 0, 0},
                 {2.0 * lam, 0, 0, 2}, {-(K + 4.0), 0, 0, 0}};
  bpoly_t p;
  p.n = 0;
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 8; j++)
      p.t[p.n++] = (term_t){alpha * a[i].c * b[j].c, a[i].pu + b[j].pu, a[i].pv + b[j].pv,
                            a[i].px + b[j].px};
  return p;
}

/* < un^m ut^n P B > over the un-range r (B a bpoly_t). */
static double mom_pb(const gmom_t* g, int r, int m, int n, const poly_t* P, const bpoly_t* B) {
  double s = 0.0;
  for (int a = 0; a < P->n; a++)
    for (int b = 0; b < B->n; b++) {
      const term_t* x = &P->t[a];
      const term_t* y = &B->t[b];
      s += x->c * y->c * g->un[r][x->pu + y->pu + m] * g->ut[x->pv + y->pv + n] *
           g->xi[x->px + y->px];
    }
  return s;
}

/* S4: solve <psi (a.psi)> = s for a, with the 4x4 moment matrix of the normalised
   Maxwellian (prim = rho, U, V, lam) and Gaussian elimination with partial pivoting. */
void orc_slope_solve(const double prim[4], int K, const double s[4], double a[4]) {
  gmom_t g;
  gmom_init(prim[1], prim[2], prim[3], K, &g);
  double M[4][5];
  for (int i = 0; i < 4; i++) {
    poly_t pi = psi_poly(i);
    for (int j = 0; j < 4; j++) {
      poly_t pj = psi_poly(j);
      M[i][j] = mom_pq(&g, 0, 0, 0, &pi, &pj);
    }
    M[i][4] = s[i];
  }
  for (int col = 0; col < 4; col++) {
    int piv = col;
    for (int r = col + 1; r < 4; r++)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    if (piv != col)
      for (int k = 0; k < 5; k++) { double t = M[col][k]; M[col][k] = M[piv][k]; M[piv][k] = t; }
    for (int r = col + 1; r < 4; r++) {
      double fct = M[r][col] / M[col][col];
      for (int k = col; k < 5; k++) M[r][k] -= fct * M[col][k];
    }
  }
  for (int r = 3; r >= 0; r--) {
    double t = M[r][4];
    for (int k = r + 1; k < 4; k++) t -= M[r][k] * a[k];
    a[r] = t / M[r][r];
  }
}

/* Primitive variables (rho, U, V, lam) from W, K internal degrees of freedom. */
static void prim_of(const double W[4], int K, double prim[4]) {
  double rho = W[0], U = W[1] / rho, V = W[2] / rho;
  double eint = W[3] - 0.5 * rho * (U * U + V * V);
  prim[0] = rho;
  prim[1] = U;
  prim[2] = V;
  prim[3] = (K + 2) * rho / (4.0 * eint);
}

/* Shakhov model: the factors sh, sb with which g_h = rho (lam/pi) exp(-lam |c|^2) gives the
   Shakhov part of the reduced equilibrium, g+_h = g_h (1 + sh), g+_b = g_h (<xi^2> + sb).
   S = alpha (c.q) (c_t^2/RT - (D+2)), alpha = (1 - Pr) / ((D+2) p RT) = (1 - Pr) 4 lam^2 /
   ((K+4) rho); sh = <S> and sb = <xi^2 S> over the internal variable, with <xi^2> = K/(2 lam)
   and <xi^4> = K (K+2) / (4 lam^2) the moments of its normalised Gaussian. */
static void shakhov_factor(const double prim[4], int K, double pr, const double q[2], double u,
                           double v, double* sh, double* sb) {
  double rho = prim[0], lam = prim[3];
  double d2 = K + 4.0;
  double alpha = (1.0 - pr) * 4.0 * lam * lam / (d2 * rho);
  double cu = u - prim[1], cv = v - prim[2];
  double cq = cu * q[0] + cv * q[1];
  double c2 = 2.0 * lam * (cu * cu + cv * cv);
  double xi2 = K / (2.0 * lam), xi4 = K * (K + 2.0) / (4.0 * lam * lam);
  *sh = alpha * cq * (c2 + 2.0 * lam * xi2 - d2);
  *sb = alpha * cq * ((c2 - d2) * xi2 + 2.0 * lam * xi4);
}

void orc_shakhov_eq(const double prim[4], int K, double pr, const double q[2], int n,
                    const double* u, const double* v, double* out) {
  for (int i = 0; i < n; i++) {
    double du = u[i] - prim[1], dv = v[i] - prim[2];
    double gh = prim[0] * (prim[3] / M_PI) * exp(-prim[3] * (du * du + dv * dv));
    double sh, sb;
    shakhov_factor(prim, K, pr, q, u[i], v[i], &sh, &sb);
    out[2 * i] = gh * (1.0 + sh);
    out[2 * i + 1] = gh * (K / (2.0 * prim[3]) + sb);
  }
}

/* Heat flux q = 1/2 sum w c (|c|^2 h + b), c = (u - U, v - V), of a reduced f[nq][2]. */
static void heat_flux(int nq, const double* w, const double* uq, const double* vq,
                      const double* f, double U, double V, double q[2]) {
  q[0] = q[1] = 0.0;
  for (int k = 0; k < nq; k++) {
    double cu = uq[k] - U, cv = vq[k] - V;
    double e = (cu * cu + cv * cv) * f[2 * k] + f[2 * k + 1];
    q[0] += 0.5 * w[k] * cu * e;
    q[1] += 0.5 * w[k] * cv * e;
  }
}

void orc_heat_flux(const orc_cfg* c, const double* f, const double W[4], double q[2]) {
  int nq = c->nu * c->nv;
  double* u = malloc(sizeof(double) * c->nu);
  double* v = malloc(sizeof(double) * c->nv);
  double* w = malloc(sizeof(double) * nq);
  double* uq = malloc(sizeof(double) * nq);
  double* vq = malloc(sizeof(double) * nq);
  orc_vgrid(c, u, v, w);
  for (int m = 0; m < c->nv; m++)
    for (int k = 0; k < c->nu; k++) { uq[m * c->nu + k] = u[k]; vq[m * c->nu + k] = v[m]; }
  heat_flux(nq, w, uq, vq, f, W[1] / W[0], W[2] / W[0], q);
  free(u); free(v); free(w); free(uq); free(vq);
}

void orc_init_maxwellian(const orc_cfg* c, const double* rho, const double* U, const double* V,
                         const double* T, double* f, double* W) {
  int nq = c->nu * c->nv, nc = c->nx * c->ny;
  double* u = malloc(sizeof(double) * c->nu);
  double* v = malloc(sizeof(double) * c->nv);
  double* w = malloc(sizeof(double) * nq);
  orc_vgrid(c, u, v, w);
  for (int cell = 0; cell < nc; cell++) {
    double lam = 1.0 / T[cell];
    for (int m = 0; m < c->nv; m++)
      for (int k = 0; k < c->nu; k++) {
        double du = u[k] - U[cell], dv = v[m] - V[cell];
        double gh = rho[cell] * (lam / M_PI) * exp(-lam * (du * du + dv * dv));
        size_t o = ((size_t)cell * nq + (size_t)m * c->nu + k) * 2;
        f[o] = gh;
        f[o + 1] = c->K / (2.0 * lam) * gh;
      }
    W[0 * nc + cell] = rho[cell];
    W[1 * nc + cell] = rho[cell] * U[cell];
    W[2 * nc + cell] = rho[cell] * V[cell];
    W[3 * nc + cell] = rho[cell] * (0.5 * (U[cell] * U[cell] + V[cell] * V[cell]) +
                                    (c->K + 2) / (4.0 * lam));
  }
  free(u); free(v); free(w);
}

/* ------------------------------------------------------------------------------------ */
/* Step context: velocity arrays and a ring of two ghost layers.                       */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  const orc_cfg* c;
  int nx, ny, nq, K;
  double dx, dy, dt;
  double *w, *uq, *vq;    /* per velocity q */
  const double* f;
  const double* W;
  int* slot;              /* extended cell -> ghost slot, -1 for interior */
  double* gf;             /* ghost f */
  double* gW;             /* ghost W, 4 per slot */
} ctx_t;

static int ext_index(const ctx_t* x, int i, int j) { return (j + 2) * (x->nx + 4) + (i + 2); }
static int is_interior(const ctx_t* x, int i, int j) {
  return i >= 0 && i < x->nx && j >= 0 && j < x->ny;
}

static const double* cell_f(const ctx_t* x, int i, int j) {
  if (is_interior(x, i, j)) return x->f + ((size_t)j * x->nx + i) * x->nq * 2;
  return x->gf + (size_t)x->slot[ext_index(x, i, j)] * x->nq * 2;
}

static void cell_W(const ctx_t* x, int i, int j, double out[4]) {
  if (is_interior(x, i, j)) {
    int nc = x->nx * x->ny, cell = j * x->nx + i;
    for (int k = 0; k < 4; k++) out[k] = x->W[k * nc + cell];
  } else {
    const double* g = x->gW + 4 * (size_t)x->slot[ext_index(x, i, j)];
    for (int k = 0; k < 4; k++) out[k] = g[k];
  }
}

/* Pressure ghost cell: Maxwellian with the boundary density and temperature and the
   velocity of the adjacent cell; W analytic. */
static void pressure_ghost(const ctx_t* x, int side, const double Wadj[4], double* gf, double* gW) {
  const orc_cfg* c = x->c;
  double rho = c->bc_rho[side], lam = 1.0 / c->bc_T[side];
  double U = Wadj[1] / Wadj[0], V = Wadj[2] / Wadj[0];
  for (int q = 0; q < x->nq; q++) {
    double du = x->uq[q] - U, dv = x->vq[q] - V;
    double gh = rho * (lam / M_PI) * exp(-lam * (du * du + dv * dv));
    gf[2 * q] = gh;
    gf[2 * q + 1] = x->K / (2.0 * lam) * gh;
  }
  gW[0] = rho;
  gW[1] = rho * U;
  gW[2] = rho * V;
  gW[3] = rho * (0.5 * (U * U + V * V) + (x->K + 2) / (4.0 * lam));
}

static void fill_ghost(ctx_t* x, int i, int j, int side, int src_i, int src_j) {
  int s = x->slot[ext_index(x, i, j)];
  double* gf = x->gf + (size_t)s * x->nq * 2;
  double* gW = x->gW + 4 * (size_t)s;
  double Wsrc[4];
  cell_W(x, src_i, src_j, Wsrc);
  if (x->c->bc_kind[side] == ORC_BC_PRESSURE) {
    pressure_ghost(x, side, Wsrc, gf, gW);
  } else { /* periodic image or zero-gradient copy for a wall */
    memcpy(gf, cell_f(x, src_i, src_j), sizeof(double) * x->nq * 2);
    memcpy(gW, Wsrc, sizeof(double) * 4);
  }
}

static void ctx_init(ctx_t* x, const orc_cfg* c, const double* f, const double* W) {
  memset(x, 0, sizeof *x);
  x->c = c; x->nx = c->nx; x->ny = c->ny; x->nq = c->nu * c->nv; x->K = c->K;
  x->dx = c->lx / c->nx; x->dy = c->ly / c->ny; x->dt = orc_dt(c);
  x->f = f; x->W = W;
  double* u = malloc(sizeof(double) * c->nu);
  double* v = malloc(sizeof(double) * c->nv);
  x->w = malloc(sizeof(double) * x->nq);
  x->uq = malloc(sizeof(double) * x->nq);
  x->vq = malloc(sizeof(double) * x->nq);
  orc_vgrid(c, u, v, x->w);
  for (int m = 0; m < c->nv; m++)
    for (int k = 0; k < c->nu; k++) { x->uq[m * c->nu + k] = u[k]; x->vq[m * c->nu + k] = v[m]; }
  free(u); free(v);

  int ne = (x->nx + 4) * (x->ny + 4), ng = 0;
  x->slot = malloc(sizeof(int) * ne);
  for (int j = -2; j < x->ny + 2; j++)
    for (int i = -2; i < x->nx + 2; i++)
      x->slot[ext_index(x, i, j)] = is_interior(x, i, j) ? -1 : ng++;
  x->gf = malloc(sizeof(double) * (size_t)ng * x->nq * 2);
  x->gW = malloc(sizeof(double) * (size_t)ng * 4);

  int nx = x->nx, ny = x->ny;
  /* x-sides first, rows 0..ny-1 */
  for (int j = 0; j < ny; j++)
    for (int l = 1; l <= 2; l++) {
      int kW = c->bc_kind[ORC_W], kE = c->bc_kind[ORC_E];
      fill_ghost(x, -l, j, ORC_W, kW == ORC_BC_PERIODIC ? nx - l : 0, j);
      fill_ghost(x, nx - 1 + l, j, ORC_E, kE == ORC_BC_PERIODIC ? l - 1 : nx - 1, j);
    }
  /* then y-sides over every column, x-ghost columns included (corners) */
  for (int i = -2; i < nx + 2; i++)
    for (int l = 1; l <= 2; l++) {
      int kS = c->bc_kind[ORC_S], kN = c->bc_kind[ORC_N];
      fill_ghost(x, i, -l, ORC_S, i, kS == ORC_BC_PERIODIC ? ny - l : 0);
      fill_ghost(x, i, ny - 1 + l, ORC_N, i, kN == ORC_BC_PERIODIC ? l - 1 : ny - 1);
    }
}

static void ctx_free(ctx_t* x) {
  free(x->w); free(x->uq); free(x->vq); free(x->slot); free(x->gf); free(x->gW);
}

static int is_pressure_ghost(const ctx_t* x, int i, int j) {
  const int* k = x->c->bc_kind;
  return (i < 0 && k[ORC_W] == ORC_BC_PRESSURE) || (i >= x->nx && k[ORC_E] == ORC_BC_PRESSURE) ||
         (j < 0 && k[ORC_S] == ORC_BC_PRESSURE) || (j >= x->ny && k[ORC_N] == ORC_BC_PRESSURE);
}

/* van Leer limited slope of cell (i,j) in direction dir (0: x, 1: y), per q and component. */
static void slope(const ctx_t* x, int i, int j, int dir, double* out) {
  if (is_pressure_ghost(x, i, j)) { memset(out, 0, sizeof(double) * x->nq * 2); return; }
  int di = dir == 0 ? 1 : 0, dj = dir == 0 ? 0 : 1;
  double h = dir == 0 ? x->dx : x->dy;
  const double* a = cell_f(x, i - di, j - dj);
  const double* b = cell_f(x, i, j);
  const double* cc = cell_f(x, i + di, j + dj);
  for (int n = 0; n < x->nq * 2; n++) {
    double s1 = (b[n] - a[n]) / h, s2 = (cc[n] - b[n]) / h;
    out[n] = (s1 * s2 > 0.0) ? 2.0 * s1 * s2 / (s1 + s2) : 0.0;
  }
}

/* Reduced polynomial weights of (a.psi) g for h and for b, divided by g_h. */
static double P_h(const double a[4], double un, double ut, double xi2) {
  return a[0] + a[1] * un + a[2] * ut + a[3] * (0.5 * (un * un + ut * ut) + 0.5 * xi2);
}
static double P_b(const double a[4], double un, double ut, double xi2, double xi4) {
  return (a[0] + a[1] * un + a[2] * ut + 0.5 * a[3] * (un * un + ut * ut)) * xi2 + 0.5 * a[3] * xi4;
}

typedef struct { double *fup, *snup, *stup, *H; } face_scratch;

/* One UGKS interface in the face frame (un normal, ut tangential), steps S1-S8. */
static void ugks_face(const ctx_t* x, const double* un, const double* ut,
                      const double* fL, const double* snL, const double* stL, const double WL[4],
                      const double* fR, const double* snR, const double* stR, const double WR[4],
                      double delta, face_scratch* sc, double F[4], double* ft) {
  int nq = x->nq, K = x->K;
  const double* w = x->w;
  double dt = x->dt;

  /* S1: upwind interface values; W0 and the tangential slope of W (8 reductions) */
  double W0[4] = {0, 0, 0, 0}, St[4] = {0, 0, 0, 0};
  for (int q = 0; q < nq; q++) {
    double H = un[q] > 0.0 ? 1.0 : (un[q] < 0.0 ? 0.0 : 0.5);
    sc->H[q] = H;
    for (int cp = 0; cp < 2; cp++) {
      int n = 2 * q + cp;
      double fLf = fL[n] + snL[n] * delta / 2.0;
      double fRf = fR[n] - snR[n] * delta / 2.0;
      sc->fup[n] = H * fLf + (1.0 - H) * fRf;
      sc->snup[n] = H * snL[n] + (1.0 - H) * snR[n];
      sc->stup[n] = H * stL[n] + (1.0 - H) * stR[n];
    }
    double e2 = 0.5 * (un[q] * un[q] + ut[q] * ut[q]);
    double fh = sc->fup[2 * q], fb = sc->fup[2 * q + 1];
    W0[0] += w[q] * fh;
    W0[1] += w[q] * un[q] * fh;
    W0[2] += w[q] * ut[q] * fh;
    W0[3] += w[q] * (e2 * fh + 0.5 * fb);
    double sh = sc->stup[2 * q], sb = sc->stup[2 * q + 1];
    St[0] += w[q] * sh;
    St[1] += w[q] * un[q] * sh;
    St[2] += w[q] * ut[q] * sh;
    St[3] += w[q] * (e2 * sh + 0.5 * sb);
  }

  /* S2: interface primitive variables and Maxwellian moments */
  double prim0[4];
  prim_of(W0, K, prim0);
  double rho0 = prim0[0], lam0 = prim0[3];
  gmom_t g;
  gmom_init(prim0[1], prim0[2], lam0, K, &g);

  /* S3: collision time and time-integration weights */
  double tau0 = orc_tau(x->c, rho0, lam0);
  double Mt[5];
  orc_mt(dt, tau0, Mt);

  /* S4: micro slopes a_L, a_R (normal), b (tangential), A (time) */
  double sL[4], sR[4], sT[4], aL[4], aR[4], bT[4], A[4], sA[4];
  for (int k = 0; k < 4; k++) {
    sL[k] = (W0[k] - WL[k]) / (rho0 * delta / 2.0);
    sR[k] = (WR[k] - W0[k]) / (rho0 * delta / 2.0);
    sT[k] = St[k] / rho0;
  }
  orc_slope_solve(prim0, K, sL, aL);
  orc_slope_solve(prim0, K, sR, aR);
  orc_slope_solve(prim0, K, sT, bT);
  poly_t pL = apsi_poly(aL), pR = apsi_poly(aR), pB = apsi_poly(bT);
  for (int i = 0; i < 4; i++) {
    poly_t psi = psi_poly(i);
    sA[i] = -(mom_pq(&g, 1, 1, 0, &psi, &pL) + mom_pq(&g, 2, 1, 0, &psi, &pR) +
              mom_pq(&g, 0, 0, 1, &psi, &pB));
  }
  orc_slope_solve(prim0, K, sA, A);
  poly_t pA = apsi_poly(A);

  /* S5: equilibrium part of the macroscopic flux (analytic moments) */
  double Feq[4];
  for (int i = 0; i < 4; i++) {
    poly_t psi = psi_poly(i);
    Feq[i] = rho0 * (Mt[0] * mom_p(&g, 0, 1, 0, &psi) +
                     Mt[1] * (mom_pq(&g, 1, 2, 0, &psi, &pL) + mom_pq(&g, 2, 2, 0, &psi, &pR) +
                              mom_pq(&g, 0, 1, 1, &psi, &pB)) +
                     Mt[2] * mom_pq(&g, 0, 1, 0, &psi, &pA));
  }

  /* Shakhov model (pr != 1): heat flux of the interface values about (U0, V0), and the
     Shakhov part of the zeroth-order equilibrium term in the macroscopic flux */
  double pr = x->c->pr, q0[2] = {0.0, 0.0};
  int shk = pr != 1.0;
  if (shk) {
    heat_flux(nq, w, un, ut, sc->fup, prim0[1], prim0[2], q0);
    double alpha = (1.0 - pr) * 4.0 * lam0 * lam0 / ((K + 4.0) * rho0);
    bpoly_t S0 = shakhov_poly(prim0[1], prim0[2], lam0, K, q0, alpha);
    for (int i = 0; i < 4; i++) {
      poly_t psi = psi_poly(i);
      Feq[i] += rho0 * Mt[0] * mom_pb(&g, 0, 1, 0, &psi, &S0);
    }
  }

  /* S7: free-transport part of the macroscopic flux (4 reductions) */
  double Sf[4] = {0, 0, 0, 0}, Ss[4] = {0, 0, 0, 0};
  for (int q = 0; q < nq; q++) {
    double e2 = 0.5 * (un[q] * un[q] + ut[q] * ut[q]);
    double fh = sc->fup[2 * q], fb = sc->fup[2 * q + 1];
    double dh = un[q] * sc->snup[2 * q] + ut[q] * sc->stup[2 * q];
    double db = un[q] * sc->snup[2 * q + 1] + ut[q] * sc->stup[2 * q + 1];
    double wu = w[q] * un[q];
    Sf[0] += wu * fh;            Ss[0] += wu * dh;
    Sf[1] += wu * un[q] * fh;    Ss[1] += wu * un[q] * dh;
    Sf[2] += wu * ut[q] * fh;    Ss[2] += wu * ut[q] * dh;
    Sf[3] += wu * (e2 * fh + 0.5 * fb);
    Ss[3] += wu * (e2 * dh + 0.5 * db);
  }
  for (int i = 0; i < 4; i++) F[i] = Feq[i] + Mt[3] * Sf[i] - Mt[4] * Ss[i];

  /* S6 + S8: interface Maxwellian and the micro flux of h and b per velocity */
  if (ft) {
    double xi2 = g.xi[2], xi4 = g.xi[4];
    for (int q = 0; q < nq; q++) {
      double du = un[q] - prim0[1], dv = ut[q] - prim0[2];
      double gh = rho0 * (lam0 / M_PI) * exp(-lam0 * (du * du + dv * dv));
      double gb = K / (2.0 * lam0) * gh;
      double H = sc->H[q];
      double Pha = H * P_h(aL, un[q], ut[q], xi2) + (1.0 - H) * P_h(aR, un[q], ut[q], xi2);
      double Pba = H * P_b(aL, un[q], ut[q], xi2, xi4) + (1.0 - H) * P_b(aR, un[q], ut[q], xi2, xi4);
      double Phb = P_h(bT, un[q], ut[q], xi2), Pbb = P_b(bT, un[q], ut[q], xi2, xi4);
      double PhA = P_h(A, un[q], ut[q], xi2), PbA = P_b(A, un[q], ut[q], xi2, xi4);
      double dh = un[q] * sc->snup[2 * q] + ut[q] * sc->stup[2 * q];
      double db = un[q] * sc->snup[2 * q + 1] + ut[q] * sc->stup[2 * q + 1];
      double sh = 0.0, sb = 0.0;
      if (shk) shakhov_factor(prim0, K, pr, q0, un[q], ut[q], &sh, &sb);
      ft[2 * q] = un[q] * (Mt[0] * (gh + gh * sh) + (Mt[1] * (un[q] * Pha + ut[q] * Phb) + Mt[2] * PhA) * gh +
                           Mt[3] * sc->fup[2 * q] - Mt[4] * dh);
      ft[2 * q + 1] = un[q] * (Mt[0] * (gb + gh * sb) + (Mt[1] * (un[q] * Pba + ut[q] * Pbb) + Mt[2] * PbA) * gh +
                               Mt[3] * sc->fup[2 * q + 1] - Mt[4] * db);
    }
  }
}

/* Diffuse isothermal wall in the face frame.  interior_high: the gas is on the high-index
   side of the face.  Incoming molecules carry the reconstructed interior f at the face,
   outgoing ones a wall Maxwellian whose density makes the net mass flux zero. */
static void wall_face(const ctx_t* x, const double* un, const double* ut, const double* fint,
                      const double* snint, int interior_high, int side, double delta,
                      double F[4], double* ft) {
  const orc_cfg* c = x->c;
  int nq = x->nq, K = x->K;
  double lamw = 1.0 / c->bc_T[side], Uw = c->bc_U[side];
  double num = 0.0, den = 0.0;
  for (int q = 0; q < nq; q++) {
    int incoming = interior_high ? (un[q] < 0.0) : (un[q] > 0.0);
    int outgoing = interior_high ? (un[q] > 0.0) : (un[q] < 0.0);
    if (incoming) {
      double ff = interior_high ? fint[2 * q] - snint[2 * q] * delta / 2.0
                                : fint[2 * q] + snint[2 * q] * delta / 2.0;
      num += x->w[q] * un[q] * ff;
    } else if (outgoing) {
      double du = ut[q] - Uw, dn = un[q];
      den += x->w[q] * un[q] * (lamw / M_PI) * exp(-lamw * (du * du + dn * dn));
    }
  }
  double rhow = -num / den;
  for (int k = 0; k < 4; k++) F[k] = 0.0;
  for (int q = 0; q < nq; q++) {
    int incoming = interior_high ? (un[q] < 0.0) : (un[q] > 0.0);
    int outgoing = interior_high ? (un[q] > 0.0) : (un[q] < 0.0);
    double fh = 0.0, fb = 0.0;
    if (incoming) {
      for (int cp = 0; cp < 2; cp++) {
        int n = 2 * q + cp;
        double ff = interior_high ? fint[n] - snint[n] * delta / 2.0 : fint[n] + snint[n] * delta / 2.0;
        if (cp == 0) fh = ff; else fb = ff;
      }
    } else if (outgoing) {
      double du = ut[q] - Uw, dn = un[q];
      fh = rhow * (lamw / M_PI) * exp(-lamw * (du * du + dn * dn));
      fb = K / (2.0 * lamw) * fh;
    }
    double th = x->dt * un[q] * fh, tb = x->dt * un[q] * fb;
    if (ft) { ft[2 * q] = th; ft[2 * q + 1] = tb; }
    double e2 = 0.5 * (un[q] * un[q] + ut[q] * ut[q]);
    F[0] += x->w[q] * th;
    F[1] += x->w[q] * un[q] * th;
    F[2] += x->w[q] * ut[q] * th;
    F[3] += x->w[q] * (e2 * th + 0.5 * tb);
  }
}

typedef struct { double *snL, *stL, *snR, *stR; face_scratch sc; } work_t;

static void work_alloc(work_t* wk, int nq) {
  size_t n = (size_t)nq * 2;
  wk->snL = malloc(sizeof(double) * n); wk->stL = malloc(sizeof(double) * n);
  wk->snR = malloc(sizeof(double) * n); wk->stR = malloc(sizeof(double) * n);
  wk->sc.fup = malloc(sizeof(double) * n); wk->sc.snup = malloc(sizeof(double) * n);
  wk->sc.stup = malloc(sizeof(double) * n); wk->sc.H = malloc(sizeof(double) * nq);
}
static void work_free(work_t* wk) {
  free(wk->snL); free(wk->stL); free(wk->snR); free(wk->stR);
  free(wk->sc.fup); free(wk->sc.snup); free(wk->sc.stup); free(wk->sc.H);
}

/* x-face (i+1/2, j), i = -1..nx-1; flux in the x frame. */
static void face_x(const ctx_t* x, work_t* wk, int i, int j, double F[4], double* ft) {
  const int* kind = x->c->bc_kind;
  if (i == -1 && kind[ORC_W] == ORC_BC_WALL) {
    slope(x, 0, j, 0, wk->snR);
    wall_face(x, x->uq, x->vq, cell_f(x, 0, j), wk->snR, 1, ORC_W, x->dx, F, ft);
    return;
  }
  if (i == x->nx - 1 && kind[ORC_E] == ORC_BC_WALL) {
    slope(x, i, j, 0, wk->snL);
    wall_face(x, x->uq, x->vq, cell_f(x, i, j), wk->snL, 0, ORC_E, x->dx, F, ft);
    return;
  }
  double WL[4], WR[4];
  cell_W(x, i, j, WL);
  cell_W(x, i + 1, j, WR);
  slope(x, i, j, 0, wk->snL);     slope(x, i, j, 1, wk->stL);
  slope(x, i + 1, j, 0, wk->snR); slope(x, i + 1, j, 1, wk->stR);
  ugks_face(x, x->uq, x->vq, cell_f(x, i, j), wk->snL, wk->stL, WL, cell_f(x, i + 1, j), wk->snR,
            wk->stR, WR, x->dx, &wk->sc, F, ft);
}

/* y-face (i, j+1/2), j = -1..ny-1; computed in the frame (un, ut) = (v, u), returned in
   the x frame. */
static void face_y(const ctx_t* x, work_t* wk, int i, int j, double F[4], double* ft) {
  const int* kind = x->c->bc_kind;
  double Fr[4];
  if (j == -1 && kind[ORC_S] == ORC_BC_WALL) {
    slope(x, i, 0, 1, wk->snR);
    wall_face(x, x->vq, x->uq, cell_f(x, i, 0), wk->snR, 1, ORC_S, x->dy, Fr, ft);
  } else if (j == x->ny - 1 && kind[ORC_N] == ORC_BC_WALL) {
    slope(x, i, j, 1, wk->snL);
    wall_face(x, x->vq, x->uq, cell_f(x, i, j), wk->snL, 0, ORC_N, x->dy, Fr, ft);
  } else {
    double WL[4], WR[4], a[4], b[4];
    cell_W(x, i, j, a);
    cell_W(x, i, j + 1, b);
    WL[0] = a[0]; WL[1] = a[2]; WL[2] = a[1]; WL[3] = a[3];
    WR[0] = b[0]; WR[1] = b[2]; WR[2] = b[1]; WR[3] = b[3];
    slope(x, i, j, 1, wk->snL);     slope(x, i, j, 0, wk->stL);
    slope(x, i, j + 1, 1, wk->snR); slope(x, i, j + 1, 0, wk->stR);
    ugks_face(x, x->vq, x->uq, cell_f(x, i, j), wk->snL, wk->stL, WL, cell_f(x, i, j + 1),
              wk->snR, wk->stR, WR, x->dy, &wk->sc, Fr, ft);
  }
  F[0] = Fr[0]; F[1] = Fr[2]; F[2] = Fr[1]; F[3] = Fr[3];
}

void orc_fluxes(const orc_cfg* c, const double* f, const double* W, double* Fx, double* Fy,
                double* fx, double* fy) {
  ctx_t x;
  ctx_init(&x, c, f, W);
  int nx = x.nx, ny = x.ny, nq = x.nq;
  int nfx = (nx + 1) * ny, nfy = nx * (ny + 1);
#pragma omp parallel num_threads(g_threads)
  {
    work_t wk;
    work_alloc(&wk, nq);
    double* tmp = malloc(sizeof(double) * nq * 2);
    double Fl[4];
#pragma omp for schedule(dynamic, 8)
    for (int n = 0; n < nfx + nfy; n++) {
      if (n < nfx) {
        int j = n / (nx + 1), i = n % (nx + 1) - 1;
        face_x(&x, &wk, i, j, Fl, fx ? fx + (size_t)n * nq * 2 : tmp);
        if (Fx) memcpy(Fx + 4 * (size_t)n, Fl, sizeof Fl);
      } else {
        int m = n - nfx;
        int j = m / nx - 1, i = m % nx;
        face_y(&x, &wk, i, j, Fl, fy ? fy + (size_t)m * nq * 2 : tmp);
        if (Fy) memcpy(Fy + 4 * (size_t)m, Fl, sizeof Fl);
      }
    }
    free(tmp);
    work_free(&wk);
  }
  ctx_free(&x);
}

/* Cell update: Eq. 4 for W and Eq. 3 (trapezoidal in the collision term, solved for
   f^{n+1}) for f.  The flux terms are the time-integrated fluxes per unit face length. */
static void update_cell(const orc_cfg* c, const double* uq, const double* vq, const double* wq,
                        double dt, const double Wn[4], const double FxW[4], const double FxE[4],
                        const double FyS[4], const double FyN[4], const double* fxW,
                        const double* fxE, const double* fyS, const double* fyN,
                        const double* fn, double* fnew, double Wnew[4]) {
  int nq = c->nu * c->nv, K = c->K;
  double dx = c->lx / c->nx, dy = c->ly / c->ny;
  for (int k = 0; k < 4; k++)
    Wnew[k] = Wn[k] + (FxW[k] - FxE[k]) / dx + (FyS[k] - FyN[k]) / dy;
  double pn[4], pn1[4];
  prim_of(Wn, K, pn);
  prim_of(Wnew, K, pn1);
  double tn = orc_tau(c, pn[0], pn[3]), tn1 = orc_tau(c, pn1[0], pn1[3]);
  /* Shakhov model: the heat flux of f^n about the cell's velocity, in g+^n and g+^{n+1} */
  int shk = c->pr != 1.0;
  double qn[2] = {0.0, 0.0};
  if (shk) heat_flux(nq, wq, uq, vq, fn, pn[1], pn[2], qn);
  for (int q = 0; q < nq; q++) {
    double du = uq[q] - pn[1], dv = vq[q] - pn[2];
    double gnh = pn[0] * (pn[3] / M_PI) * exp(-pn[3] * (du * du + dv * dv));
    double gnb = K / (2.0 * pn[3]) * gnh;
    du = uq[q] - pn1[1]; dv = vq[q] - pn1[2];
    double g1h = pn1[0] * (pn1[3] / M_PI) * exp(-pn1[3] * (du * du + dv * dv));
    double g1b = K / (2.0 * pn1[3]) * g1h;
    if (shk) {
      double sh, sb;
      shakhov_factor(pn, K, c->pr, qn, uq[q], vq[q], &sh, &sb);
      gnb = gnb + gnh * sb;
      gnh = gnh + gnh * sh;
      shakhov_factor(pn1, K, c->pr, qn, uq[q], vq[q], &sh, &sb);
      g1b = g1b + g1h * sb;
      g1h = g1h + g1h * sh;
    }
    for (int cp = 0; cp < 2; cp++) {
      int n = 2 * q + cp;
      double gn = cp == 0 ? gnh : gnb, g1 = cp == 0 ? g1h : g1b;
      double rhs = fn[n] + (fxW[n] - fxE[n]) / dx + (fyS[n] - fyN[n]) / dy +
                   dt / 2.0 * (g1 / tn1 + (gn - fn[n]) / tn);
      fnew[n] = rhs / (1.0 + dt / (2.0 * tn1));
    }
  }
}

void orc_step(const orc_cfg* c, double* f, double* W, int nsteps) {
  int nx = c->nx, ny = c->ny, nq = c->nu * c->nv, nc = nx * ny;
  int nfx = (nx + 1) * ny, nfy = nx * (ny + 1);
  double* Fx = malloc(sizeof(double) * 4 * nfx);
  double* Fy = malloc(sizeof(double) * 4 * nfy);
  double* fx = malloc(sizeof(double) * (size_t)nfx * nq * 2);
  double* fy = malloc(sizeof(double) * (size_t)nfy * nq * 2);
  double* uq = malloc(sizeof(double) * nq);
  double* vq = malloc(sizeof(double) * nq);
  double* wq = malloc(sizeof(double) * nq);
  {
    double* u = malloc(sizeof(double) * c->nu);
    double* v = malloc(sizeof(double) * c->nv);
    orc_vgrid(c, u, v, wq);
    for (int m = 0; m < c->nv; m++)
      for (int k = 0; k < c->nu; k++) { uq[m * c->nu + k] = u[k]; vq[m * c->nu + k] = v[m]; }
    free(u); free(v);
  }
  double dt = orc_dt(c);
  for (int s = 0; s < nsteps; s++) {
    orc_fluxes(c, f, W, Fx, Fy, fx, fy);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int cell = 0; cell < nc; cell++) {
      int i = cell % nx, j = cell / nx;
      size_t xw = (size_t)j * (nx + 1) + i, xe = xw + 1;
      size_t ys = (size_t)j * nx + i, yn = (size_t)(j + 1) * nx + i;
      double Wn[4], Wnew[4];
      for (int k = 0; k < 4; k++) Wn[k] = W[k * nc + cell];
      double* fc = f + (size_t)cell * nq * 2;
      update_cell(c, uq, vq, wq, dt, Wn, Fx + 4 * xw, Fx + 4 * xe, Fy + 4 * ys, Fy + 4 * yn,
                  fx + xw * nq * 2, fx + xe * nq * 2, fy + ys * nq * 2, fy + yn * nq * 2, fc, fc,
                  Wnew);
      for (int k = 0; k < 4; k++) W[k * nc + cell] = Wnew[k];
    }
  }
  free(Fx); free(Fy); free(fx); free(fy); free(uq); free(vq); free(wq);
}

/* One step for a list of cells only (the rest of the state is read, not written):
   f_out[n][nq][2], W_out[n][4] for cells ids[n].  Used to check large cases by sampling. */
void orc_step_cells(const orc_cfg* c, const double* f, const double* W, int ncell,
                    const int* ids, double* f_out, double* W_out) {
  ctx_t x;
  ctx_init(&x, c, f, W);
  int nx = x.nx, nq = x.nq, nc = x.nx * x.ny;
#pragma omp parallel num_threads(g_threads)
  {
    work_t wk;
    work_alloc(&wk, nq);
    double* fxw = malloc(sizeof(double) * nq * 2);
    double* fxe = malloc(sizeof(double) * nq * 2);
    double* fys = malloc(sizeof(double) * nq * 2);
    double* fyn = malloc(sizeof(double) * nq * 2);
#pragma omp for schedule(dynamic, 1)
    for (int n = 0; n < ncell; n++) {
      int cell = ids[n], i = cell % nx, j = cell / nx;
      double FW[4], FE[4], FS[4], FN[4], Wn[4];
      face_x(&x, &wk, i - 1, j, FW, fxw);
      face_x(&x, &wk, i, j, FE, fxe);
      face_y(&x, &wk, i, j - 1, FS, fys);
      face_y(&x, &wk, i, j, FN, fyn);
      for (int k = 0; k < 4; k++) Wn[k] = W[k * nc + cell];
      update_cell(c, x.uq, x.vq, x.w, x.dt, Wn, FW, FE, FS, FN, fxw, fxe, fys, fyn,
                  f + (size_t)cell * nq * 2, f_out + (size_t)n * nq * 2, W_out + 4 * (size_t)n);
    }
    free(fxw); free(fxe); free(fys); free(fyn);
    work_free(&wk);
  }
  ctx_free(&x);
}
