/*
 * ns3d_oracle.c -- plain, slow, FP64 CPU oracle for the right-hand side of the
 * 3D compressible Navier-Stokes equations of arXiv 2211.16718 (Kim, Ghosh,
 * Constantinescu, Balakrishnan), Sec. 2.1-2.2, and for the Runge-Kutta update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared [-fopenmp]
 *   (-ffp-contract=off keeps the same rounding on x86-64 and aarch64).
 *
 * Layout of every state array: u[v*N + (k*ny + j)*nx + i], v = 0..4 for
 * (rho, rho*u, rho*v, rho*w, e), x fastest, N = nx*ny*nz, grid point
 * x_i = i*dx with dx = lx/nx (triply periodic box).
 *
 * Readings of the paper taken here where it is silent or garbled:
 *  - viscous stress uses the symmetric strain rate (du_i/dx_j + du_j/dx_i); the
 *    printed minus sign in Sec. 2.1 would make tau antisymmetric;
 *  - e is the total energy per unit volume (the formula of Sec. 2.1);
 *  - exponent p of the WENO weights is 2 (Jiang-Shu), eps = 1e-6 added to beta;
 *  - each of the 5 components of u and of f is reconstructed separately in
 *    conservative variables, left- and right-biased (Sec. 2.2);
 *  - the Roe average uses the grid-point states i and i+1 on either side of the
 *    interface (roe_state = 0) or the reconstructed states (roe_state = 1);
 *  - Harten's entropy fix acts on the two acoustic eigenvalues only:
 *    |lambda| < delta -> (lambda^2 + delta^2)/(2 delta), delta = harten_delta*c~;
 *  - viscous terms: 4th-order central first derivatives of u, v, w, T at the
 *    grid points, then the same operator applied to the viscous fluxes;
 *  - mu is constant, so mu_eff = mu*M_inf/Re_inf is the only viscous parameter;
 *    heat flux coefficient mu_eff/((gamma-1) Pr).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int nx, ny, nz;
  int weno_p;       /* exponent p in alpha_k = c_k/(eps+beta_k)^p */
  int weno_linear;  /* 1: use the optimal weights c_k (debug/pin mode) */
  int roe_state;    /* 0: Roe average of grid points i, i+1; 1: of uL, uR */
  double lx, ly, lz;
  double gamma;
  double mu_eff;    /* mu*M_inf/Re_inf; 0 disables the viscous terms */
  double prandtl;
  double weno_eps;
  double harten_delta; /* entropy-fix width as a fraction of c~; 0 = off */
} orc_params;

static int g_threads = 1;

void orc_set_threads(int n) {
  if (n < 1) n = 1;
  g_threads = n;
#ifdef _OPENMP
  omp_set_num_threads(n);
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return g_threads;
#else
  return 1;
#endif
}

int orc_has_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

static long wrap(long i, long n) {
  long r = i % n;
  return r < 0 ? r + n : r;
}

static double sq(double a) { return a * a; }

static void dims(const orc_params *P, long n[3], long stride[3], double h[3]) {
  n[0] = P->nx; n[1] = P->ny; n[2] = P->nz;
  stride[0] = 1; stride[1] = P->nx; stride[2] = (long)P->nx * P->ny;
  h[0] = P->lx / P->nx; h[1] = P->ly / P->ny; h[2] = P->lz / P->nz;
}

/* ---------------------------------------------------------------------------
 * Equation of state and convective flux, Sec. 2.1:
 *   e = p/(gamma-1) + rho (u^2+v^2+w^2)/2, T = gamma p / rho.
 * ------------------------------------------------------------------------ */
typedef struct { double rho, u, v, w, p, T, H; } prim_t;

static prim_t orc_prim(const double U[5], double gamma) {
  prim_t q;
  q.rho = U[0];
  q.u = U[1] / U[0];
  q.v = U[2] / U[0];
  q.w = U[3] / U[0];
  q.p = (gamma - 1.0) * (U[4] - 0.5 * q.rho * (q.u * q.u + q.v * q.v + q.w * q.w));
  q.T = gamma * q.p / q.rho;
  q.H = (U[4] + q.p) / q.rho;
  return q;
}

/* Convective flux along direction d (f, g, h of Sec. 2.1). */
void orc_flux(const double U[5], int d, double gamma, double F[5]) {
  prim_t q = orc_prim(U, gamma);
  double vel[3] = {q.u, q.v, q.w};
  double un = vel[d];
  F[0] = U[1 + d];                 /* rho*u_d (the momentum component itself) */
  F[1] = U[1] * un;                /* rho u u_d */
  F[2] = U[2] * un;                /* rho v u_d */
  F[3] = U[3] * un;                /* rho w u_d */
  F[1 + d] += q.p;                 /* + p on the diagonal */
  F[4] = (U[4] + q.p) * un;        /* (e + p) u_d */
}

/* ---------------------------------------------------------------------------
 * WENO5 (Sec. 2.2): q[0..4] = f_{j-2}, ..., f_{j+2}; value at j+1/2.
 * ------------------------------------------------------------------------ */
/* The three third-order candidates and their optimal weights c = (1,6,3)/10. */
void orc_weno5_candidates(const double *q, double *cand) {
  cand[0] = (1.0 / 3.0) * q[0] - (7.0 / 6.0) * q[1] + (11.0 / 6.0) * q[2];
  cand[1] = -(1.0 / 6.0) * q[1] + (5.0 / 6.0) * q[2] + (1.0 / 3.0) * q[3];
  cand[2] = (1.0 / 3.0) * q[2] + (5.0 / 6.0) * q[3] - (1.0 / 6.0) * q[4];
}

/* Smoothness indicators beta_1..beta_3. */
void orc_weno5_beta(const double *q, double *beta) {
  beta[0] = (13.0 / 12.0) * sq(q[0] - 2.0 * q[1] + q[2]) + 0.25 * sq(q[0] - 4.0 * q[1] + 3.0 * q[2]);
  beta[1] = (13.0 / 12.0) * sq(q[1] - 2.0 * q[2] + q[3]) + 0.25 * sq(q[1] - q[3]);
  beta[2] = (13.0 / 12.0) * sq(q[2] - 2.0 * q[3] + q[4]) + 0.25 * sq(3.0 * q[2] - 4.0 * q[3] + q[4]);
}

/* Nonlinear weights omega_k = alpha_k / sum(alpha), alpha_k = c_k/(eps+beta_k)^p. */
void orc_weno5_weights(const double *q, double eps, int p, int linear, double *w) {
  const double c[3] = {0.1, 0.6, 0.3};
  if (linear) {
    w[0] = c[0]; w[1] = c[1]; w[2] = c[2];
    return;
  }
  double beta[3], alpha[3], sum = 0.0;
  orc_weno5_beta(q, beta);
  for (int k = 0; k < 3; ++k) {
    double den = 1.0;
    for (int m = 0; m < p; ++m) den *= (eps + beta[k]);
    alpha[k] = c[k] / den;
    sum += alpha[k];
  }
  for (int k = 0; k < 3; ++k) w[k] = alpha[k] / sum;
}

/* Weighted interpolation sum_k omega_k * candidate_k. */
double orc_weno5(const double *q, double eps, int p, int linear) {
  double cand[3], w[3];
  orc_weno5_candidates(q, cand);
  orc_weno5_weights(q, eps, p, linear, w);
  return w[0] * cand[0] + w[1] * cand[1] + w[2] * cand[2];
}

/* Left- and right-biased interface values of a periodic scalar line of length
 * n: qL[i], qR[i] at interface i+1/2.  The right-biased value is the left
 * formula applied to the stencil mirrored about i+1/2 (q_{i+3}, ..., q_{i-1}). */
void orc_weno5_line(const double *q, int n, double eps, int p, int linear, double *qL, double *qR) {
  for (int i = 0; i < n; ++i) {
    double a[5], b[5];
    for (int t = 0; t < 5; ++t) {
      a[t] = q[wrap(i - 2 + t, n)];
      b[t] = q[wrap(i + 3 - t, n)];
    }
    qL[i] = orc_weno5(a, eps, p, linear);
    qR[i] = orc_weno5(b, eps, p, linear);
  }
}

/* ---------------------------------------------------------------------------
 * Roe upwinding (Sec. 2.2, Eq. Roe): Roe-averaged state, eigenvalues, right
 * eigenvectors X (columns) and left eigenvectors X^{-1} (rows) of the 3D Euler
 * flux Jacobian along direction d.  Textbook closed forms for the basis
 *   r1 = (1, V - c n, H - c u_n), r2 = (1, V, |V|^2/2),
 *   r3 = (0, t1, t1.V), r4 = (0, t2, t2.V), r5 = (1, V + c n, H + c u_n),
 * where n = e_d and t1, t2 are the two other unit axes in increasing order.
 * ------------------------------------------------------------------------ */
typedef struct { double u, v, w, H, c; } roe_t;

static roe_t roe_average(const double UL[5], const double UR[5], double gamma) {
  prim_t a = orc_prim(UL, gamma), b = orc_prim(UR, gamma);
  double sa = sqrt(a.rho), sb = sqrt(b.rho);
  roe_t r;
  r.u = (sa * a.u + sb * b.u) / (sa + sb);
  r.v = (sa * a.v + sb * b.v) / (sa + sb);
  r.w = (sa * a.w + sb * b.w) / (sa + sb);
  r.H = (sa * a.H + sb * b.H) / (sa + sb);
  r.c = sqrt((gamma - 1.0) * (r.H - 0.5 * (r.u * r.u + r.v * r.v + r.w * r.w)));
  return r;
}

static void eigensystem(roe_t r, int d, double gamma, double X[5][5], double Xi[5][5], double lam[5]) {
  double V[3] = {r.u, r.v, r.w};
  double nv[3] = {0, 0, 0};
  nv[d] = 1.0;
  int t1 = (d == 0) ? 1 : 0;
  int t2 = (d == 2) ? 1 : 2;
  double tv1[3] = {0, 0, 0}, tv2[3] = {0, 0, 0};
  tv1[t1] = 1.0;
  tv2[t2] = 1.0;
  double un = V[d], c = r.c, q2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
  double b1 = (gamma - 1.0) / (c * c), b2 = 0.5 * q2 * b1;

  /* right eigenvectors as columns */
  X[0][0] = 1.0; X[0][1] = 1.0; X[0][2] = 0.0; X[0][3] = 0.0; X[0][4] = 1.0;
  for (int m = 0; m < 3; ++m) {
    X[1 + m][0] = V[m] - c * nv[m];
    X[1 + m][1] = V[m];
    X[1 + m][2] = tv1[m];
    X[1 + m][3] = tv2[m];
    X[1 + m][4] = V[m] + c * nv[m];
  }
  X[4][0] = r.H - c * un;
  X[4][1] = 0.5 * q2;
  X[4][2] = V[t1];
  X[4][3] = V[t2];
  X[4][4] = r.H + c * un;

  /* left eigenvectors as rows */
  Xi[0][0] = 0.5 * (b2 + un / c);
  Xi[1][0] = 1.0 - b2;
  Xi[2][0] = -V[t1];
  Xi[3][0] = -V[t2];
  Xi[4][0] = 0.5 * (b2 - un / c);
  for (int m = 0; m < 3; ++m) {
    Xi[0][1 + m] = 0.5 * (-b1 * V[m] - nv[m] / c);
    Xi[1][1 + m] = b1 * V[m];
    Xi[2][1 + m] = tv1[m];
    Xi[3][1 + m] = tv2[m];
    Xi[4][1 + m] = 0.5 * (-b1 * V[m] + nv[m] / c);
  }
  Xi[0][4] = 0.5 * b1;
  Xi[1][4] = -b1;
  Xi[2][4] = 0.0;
  Xi[3][4] = 0.0;
  Xi[4][4] = 0.5 * b1;

  lam[0] = un - c;
  lam[1] = un;
  lam[2] = un;
  lam[3] = un;
  lam[4] = un + c;
}

/* |lambda| with Harten's entropy fix on the acoustic eigenvalues (k = 0, 4). */
static void abs_eigenvalues(const double lam[5], double c, double harten_delta, double out[5]) {
  double delta = harten_delta * c;
  for (int k = 0; k < 5; ++k) {
    double a = fabs(lam[k]);
    if ((k == 0 || k == 4) && delta > 0.0 && a < delta) a = (lam[k] * lam[k] + delta * delta) / (2.0 * delta);
    out[k] = a;
  }
}

/* A = X g(Lambda) X^{-1} at the Roe average of (UL, UR) along d; absval = 0
 * gives the Roe matrix itself, absval = 1 the dissipation matrix |A|. */
void orc_roe_matrix(const double UL[5], const double UR[5], int d, double gamma, int absval,
                    double harten_delta, double *A) {
  double X[5][5], Xi[5][5], lam[5], g[5];
  roe_t r = roe_average(UL, UR, gamma);
  eigensystem(r, d, gamma, X, Xi, lam);
  if (absval) abs_eigenvalues(lam, r.c, harten_delta, g);
  else for (int k = 0; k < 5; ++k) g[k] = lam[k];
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) {
      double s = 0.0;
      for (int k = 0; k < 5; ++k) s += X[a][k] * g[k] * Xi[k][b];
      A[a * 5 + b] = s;
    }
}

/* X and X^{-1} as flat row-major 5x5 arrays plus the eigenvalues (for pins). */
void orc_roe_eigensystem(const double UL[5], const double UR[5], int d, double gamma,
                         double *X, double *Xi, double *lam) {
  double x[5][5], xi[5][5];
  roe_t r = roe_average(UL, UR, gamma);
  eigensystem(r, d, gamma, x, xi, lam);
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) {
      X[a * 5 + b] = x[a][b];
      Xi[a * 5 + b] = xi[a][b];
    }
}

/* Numerical flux at interface i+1/2 of one grid line along d.
 * Us[m], Fs[m] = state and convective flux at grid points i-2+m, m = 0..5. */
static void interface_flux(const orc_params *P, int d, const double Us[6][5], const double Fs[6][5],
                           double Fh[5]) {
  double uL[5], uR[5], fL[5], fR[5];
  for (int m = 0; m < 5; ++m) {
    double a[5], b[5], fa[5], fb[5];
    for (int t = 0; t < 5; ++t) {
      a[t] = Us[t][m];       /* left-biased: i-2 .. i+2 */
      b[t] = Us[5 - t][m];   /* right-biased: i+3 .. i-1 */
      fa[t] = Fs[t][m];
      fb[t] = Fs[5 - t][m];
    }
    uL[m] = orc_weno5(a, P->weno_eps, P->weno_p, P->weno_linear);
    uR[m] = orc_weno5(b, P->weno_eps, P->weno_p, P->weno_linear);
    fL[m] = orc_weno5(fa, P->weno_eps, P->weno_p, P->weno_linear);
    fR[m] = orc_weno5(fb, P->weno_eps, P->weno_p, P->weno_linear);
  }
  double X[5][5], Xi[5][5], lam[5], g[5];
  roe_t r = P->roe_state ? roe_average(uL, uR, P->gamma) : roe_average(Us[2], Us[3], P->gamma);
  eigensystem(r, d, P->gamma, X, Xi, lam);
  abs_eigenvalues(lam, r.c, P->harten_delta, g);
  double du[5], wv[5];
  for (int m = 0; m < 5; ++m) du[m] = uR[m] - uL[m];
  for (int k = 0; k < 5; ++k) {
    double s = 0.0;
    for (int m = 0; m < 5; ++m) s += Xi[k][m] * du[m];
    wv[k] = g[k] * s;
  }
  for (int m = 0; m < 5; ++m) {
    double diss = 0.0;
    for (int k = 0; k < 5; ++k) diss += X[m][k] * wv[k];
    Fh[m] = 0.5 * (fL[m] + fR[m]) - 0.5 * diss;
  }
}

/* Single-interface Roe flux from 6 point states (for pins). us: 6x5 row-major. */
void orc_interface_flux(const orc_params *P, int d, const double *us, double *Fh) {
  double Us[6][5], Fs[6][5];
  for (int m = 0; m < 6; ++m) {
    for (int v = 0; v < 5; ++v) Us[m][v] = us[m * 5 + v];
    orc_flux(Us[m], d, P->gamma, Fs[m]);
  }
  interface_flux(P, d, Us, Fs, Fh);
}

/* Gather the state of point (line base + idx*stride) into s[5]. */
static void gather(const double *u, long N, long pt, double s[5]) {
  for (int v = 0; v < 5; ++v) s[v] = u[v * N + pt];
}

/* ---------------------------------------------------------------------------
 * Hyperbolic part: rhs -= (Fhat_{i+1/2} - Fhat_{i-1/2}) / dx_d, d = x, y, z
 * (conservative finite difference, Sec. 2.2).  rhs is accumulated into.
 * ------------------------------------------------------------------------ */
void orc_rhs_hyp_accum(const orc_params *P, const double *u, double *rhs) {
  long n[3], st[3];
  double h[3];
  dims(P, n, st, h);
  long N = n[0] * n[1] * n[2];
  for (int d = 0; d < 3; ++d) {
    int a = (d == 0) ? 1 : 0, b = (d == 2) ? 1 : 2; /* the two other axes */
    long nlines = n[a] * n[b];
    long nd = n[d];
#pragma omp parallel for schedule(static)
    for (long line = 0; line < nlines; ++line) {
      long ia = line % n[a], ib = line / n[a];
      long base = ia * st[a] + ib * st[b];
      double (*Ul)[5] = malloc(sizeof(double[5]) * nd);
      double (*Fl)[5] = malloc(sizeof(double[5]) * nd);
      double (*Fh)[5] = malloc(sizeof(double[5]) * nd);
      for (long i = 0; i < nd; ++i) {
        gather(u, N, base + i * st[d], Ul[i]);
        orc_flux(Ul[i], d, P->gamma, Fl[i]);
      }
      for (long i = 0; i < nd; ++i) {
        double Us[6][5], Fs[6][5];
        for (int m = 0; m < 6; ++m) {
          long j = wrap(i - 2 + m, nd);
          memcpy(Us[m], Ul[j], sizeof(double[5]));
          memcpy(Fs[m], Fl[j], sizeof(double[5]));
        }
        interface_flux(P, d, Us, Fs, Fh[i]);
      }
      for (long i = 0; i < nd; ++i) {
        long im = wrap(i - 1, nd);
        for (int v = 0; v < 5; ++v) rhs[v * N + base + i * st[d]] -= (Fh[i][v] - Fh[im][v]) / h[d];
      }
      free(Ul); free(Fl); free(Fh);
    }
  }
}

/* ---------------------------------------------------------------------------
 * Viscous part (Sec. 2.1 stresses and heat flux; 4th-order central
 * differences): first derivatives of (u, v, w, T) at grid points, viscous flux
 * vectors f^v, g^v, h^v at grid points, then their 4th-order central
 * derivative.  rhs is accumulated into.
 * ------------------------------------------------------------------------ */
/* 4th-order central first derivative (q_{j-2} - 8 q_{j-1} + 8 q_{j+1} - q_{j+2})/(12 h),
 * evaluated in difference form so that a constant gives exactly zero. */
static double d4(double qm2, double qm1, double qp1, double qp2, double hh) {
  return (8.0 * (qp1 - qm1) - (qp2 - qm2)) / (12.0 * hh);
}

/* Viscous flux along d at one point: G[q][e] = d(q)/dx_e for q = u, v, w, T. */
static void visc_flux(const orc_params *P, const double vel[3], const double G[4][3], int d, double Fv[4]) {
  double mu = P->mu_eff;
  double kappa = P->mu_eff / ((P->gamma - 1.0) * P->prandtl);
  double div = G[0][0] + G[1][1] + G[2][2];
  double tau[3]; /* tau_{m d}, m = x, y, z */
  for (int m = 0; m < 3; ++m) {
    tau[m] = mu * (G[m][d] + G[d][m]);
    if (m == d) tau[m] -= mu * (2.0 / 3.0) * div;
  }
  double qd = -kappa * G[3][d];
  Fv[0] = tau[0];
  Fv[1] = tau[1];
  Fv[2] = tau[2];
  Fv[3] = vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] - qd;
}

void orc_rhs_visc_accum(const orc_params *P, const double *u, double *rhs) {
  if (P->mu_eff == 0.0) return;
  long n[3], st[3];
  double h[3];
  dims(P, n, st, h);
  long N = n[0] * n[1] * n[2];
  double *W = malloc(sizeof(double) * 4 * N);   /* u, v, w, T */
  double *G = malloc(sizeof(double) * 12 * N);  /* G[(q*3+e)*N + pt] */
  double *Fv = malloc(sizeof(double) * 4 * N);
#pragma omp parallel for schedule(static)
  for (long pt = 0; pt < N; ++pt) {
    double s[5];
    gather(u, N, pt, s);
    prim_t q = orc_prim(s, P->gamma);
    W[0 * N + pt] = q.u;
    W[1 * N + pt] = q.v;
    W[2 * N + pt] = q.w;
    W[3 * N + pt] = q.T;
  }
#pragma omp parallel for schedule(static)
  for (long pt = 0; pt < N; ++pt) {
    long idx[3] = {pt % n[0], (pt / n[0]) % n[1], pt / (n[0] * n[1])};
    for (int e = 0; e < 3; ++e) {
      long nb[5];
      for (int o = -2; o <= 2; ++o) {
        long id2[3] = {idx[0], idx[1], idx[2]};
        id2[e] = wrap(idx[e] + o, n[e]);
        nb[o + 2] = id2[0] + id2[1] * st[1] + id2[2] * st[2];
      }
      for (int qv = 0; qv < 4; ++qv) {
        const double *A = W + qv * N;
        G[(qv * 3 + e) * N + pt] = d4(A[nb[0]], A[nb[1]], A[nb[3]], A[nb[4]], h[e]);
      }
    }
  }
  for (int d = 0; d < 3; ++d) {
#pragma omp parallel for schedule(static)
    for (long pt = 0; pt < N; ++pt) {
      double vel[3] = {W[pt], W[N + pt], W[2 * N + pt]};
      double Gp[4][3], f[4];
      for (int qv = 0; qv < 4; ++qv)
        for (int e = 0; e < 3; ++e) Gp[qv][e] = G[(qv * 3 + e) * N + pt];
      visc_flux(P, vel, Gp, d, f);
      for (int c = 0; c < 4; ++c) Fv[c * N + pt] = f[c];
    }
#pragma omp parallel for schedule(static)
    for (long pt = 0; pt < N; ++pt) {
      long idx[3] = {pt % n[0], (pt / n[0]) % n[1], pt / (n[0] * n[1])};
      long nb[5];
      for (int o = -2; o <= 2; ++o) {
        long id2[3] = {idx[0], idx[1], idx[2]};
        id2[d] = wrap(idx[d] + o, n[d]);
        nb[o + 2] = id2[0] + id2[1] * st[1] + id2[2] * st[2];
      }
      for (int c = 0; c < 4; ++c) {
        const double *A = Fv + c * N;
        rhs[(1 + c) * N + pt] += d4(A[nb[0]], A[nb[1]], A[nb[3]], A[nb[4]], h[d]);
      }
    }
  }
  free(W); free(G); free(Fv);
}

/* Full right-hand side: rhs = -sum_d D_d(fhat_d) + sum_d D_d(f^v_d), Eq. (NS). */
void orc_rhs(const orc_params *P, const double *u, double *rhs) {
  long N = (long)P->nx * P->ny * P->nz;
  memset(rhs, 0, sizeof(double) * 5 * N);
  orc_rhs_hyp_accum(P, u, rhs);
  orc_rhs_visc_accum(P, u, rhs);
}

void orc_rhs_hyp(const orc_params *P, const double *u, double *rhs) {
  long N = (long)P->nx * P->ny * P->nz;
  memset(rhs, 0, sizeof(double) * 5 * N);
  orc_rhs_hyp_accum(P, u, rhs);
}

void orc_rhs_visc(const orc_params *P, const double *u, double *rhs) {
  long N = (long)P->nx * P->ny * P->nz;
  memset(rhs, 0, sizeof(double) * 5 * N);
  orc_rhs_visc_accum(P, u, rhs);
}

/* ---------------------------------------------------------------------------
 * The same right-hand side evaluated at selected points only, from the local
 * stencil: every quantity is computed by the same functions and in the same
 * order as in orc_rhs, so the values equal orc_rhs at those points.
 * idx[m] is a flat point index; out[m*5 + v].
 * ------------------------------------------------------------------------ */
static long flat_of(const long n[3], long i, long j, long k) { return i + n[0] * (j + n[1] * k); }

static void point_W(const orc_params *P, const double *u, long N, long pt, double Wv[4]) {
  double s[5];
  gather(u, N, pt, s);
  prim_t q = orc_prim(s, P->gamma);
  Wv[0] = q.u; Wv[1] = q.v; Wv[2] = q.w; Wv[3] = q.T;
}

static void point_G(const orc_params *P, const double *u, long N, const long n[3], const double h[3],
                    const long idx[3], double Gp[4][3]) {
  for (int e = 0; e < 3; ++e) {
    double Wn[5][4];
    for (int o = -2; o <= 2; ++o) {
      if (o == 0) continue;
      long id2[3] = {idx[0], idx[1], idx[2]};
      id2[e] = wrap(idx[e] + o, n[e]);
      point_W(P, u, N, flat_of(n, id2[0], id2[1], id2[2]), Wn[o + 2]);
    }
    for (int qv = 0; qv < 4; ++qv) Gp[qv][e] = d4(Wn[0][qv], Wn[1][qv], Wn[3][qv], Wn[4][qv], h[e]);
  }
}

void orc_rhs_points(const orc_params *P, const double *u, long npts, const long *pidx, double *out) {
  long n[3], st[3];
  double h[3];
  dims(P, n, st, h);
  long N = n[0] * n[1] * n[2];
#pragma omp parallel for schedule(dynamic, 1)
  for (long m = 0; m < npts; ++m) {
    long pt = pidx[m];
    long idx[3] = {pt % n[0], (pt / n[0]) % n[1], pt / (n[0] * n[1])};
    double r[5] = {0, 0, 0, 0, 0};
    for (int d = 0; d < 3; ++d) {
      double Fh[2][5];
      for (int side = 0; side < 2; ++side) { /* interfaces i-1/2 (side 0), i+1/2 (side 1) */
        long i0 = idx[d] - 1 + side;
        double Us[6][5], Fs[6][5];
        for (int mm = 0; mm < 6; ++mm) {
          long id2[3] = {idx[0], idx[1], idx[2]};
          id2[d] = wrap(i0 - 2 + mm, n[d]);
          gather(u, N, flat_of(n, id2[0], id2[1], id2[2]), Us[mm]);
          orc_flux(Us[mm], d, P->gamma, Fs[mm]);
        }
        interface_flux(P, d, Us, Fs, Fh[side]);
      }
      for (int v = 0; v < 5; ++v) r[v] -= (Fh[1][v] - Fh[0][v]) / h[d];
    }
    if (P->mu_eff != 0.0) {
      for (int d = 0; d < 3; ++d) {
        double fv[5][4];
        for (int o = -2; o <= 2; ++o) {
          if (o == 0) continue;
          long id2[3] = {idx[0], idx[1], idx[2]};
          id2[d] = wrap(idx[d] + o, n[d]);
          double Wv[4], Gp[4][3];
          point_W(P, u, N, flat_of(n, id2[0], id2[1], id2[2]), Wv);
          point_G(P, u, N, n, h, id2, Gp);
          visc_flux(P, Wv, Gp, d, fv[o + 2]);
        }
        for (int c = 0; c < 4; ++c) r[1 + c] += d4(fv[0][c], fv[1][c], fv[3][c], fv[4][c], h[d]);
      }
    }
    for (int v = 0; v < 5; ++v) out[m * 5 + v] = r[v];
  }
}

/* ---------------------------------------------------------------------------
 * Runge-Kutta time integration (Sec. 2.2): classical RK4 (scheme 0) and the
 * three-stage TVD (SSP) RK3 in Shu-Osher form (scheme 1).
 * ------------------------------------------------------------------------ */
typedef void (*orc_rhs_fn)(void *ctx, const double *u, double *r);

void orc_rk_generic(long n, double *u, double dt, int scheme, orc_rhs_fn f, void *ctx) {
  double *un = malloc(sizeof(double) * n);
  double *us = malloc(sizeof(double) * n);
  double *k = malloc(sizeof(double) * n);
  memcpy(un, u, sizeof(double) * n);
  if (scheme == 0) {
    double *k1 = malloc(sizeof(double) * n), *k2 = malloc(sizeof(double) * n);
    double *k3 = malloc(sizeof(double) * n);
    f(ctx, un, k1);
    for (long m = 0; m < n; ++m) us[m] = un[m] + 0.5 * dt * k1[m];
    f(ctx, us, k2);
    for (long m = 0; m < n; ++m) us[m] = un[m] + 0.5 * dt * k2[m];
    f(ctx, us, k3);
    for (long m = 0; m < n; ++m) us[m] = un[m] + dt * k3[m];
    f(ctx, us, k);
    for (long m = 0; m < n; ++m)
      u[m] = un[m] + (dt / 6.0) * (k1[m] + 2.0 * k2[m] + 2.0 * k3[m] + k[m]);
    free(k1); free(k2); free(k3);
  } else {
    f(ctx, un, k);
    for (long m = 0; m < n; ++m) us[m] = un[m] + dt * k[m];
    f(ctx, us, k);
    for (long m = 0; m < n; ++m) us[m] = 0.75 * un[m] + 0.25 * (us[m] + dt * k[m]);
    f(ctx, us, k);
    for (long m = 0; m < n; ++m) u[m] = (1.0 / 3.0) * un[m] + (2.0 / 3.0) * (us[m] + dt * k[m]);
  }
  free(un); free(us); free(k);
}

static void rhs_cb(void *ctx, const double *u, double *r) { orc_rhs((const orc_params *)ctx, u, r); }

void orc_rk_step(const orc_params *P, double *u, double dt, int nsteps, int scheme) {
  long n = 5L * P->nx * P->ny * P->nz;
  for (int s = 0; s < nsteps; ++s) orc_rk_generic(n, u, dt, scheme, rhs_cb, (void *)P);
}

/* ---------------------------------------------------------------------------
 * Statistics: out[0..4] = sums of rho, rho u, rho v, rho w, e times the cell
 * volume; out[5] = mean of rho|v|^2/2; out[6] = mean of rho|omega|^2/2 with
 * omega from the 4th-order central derivative; out[7] = min rho;
 * out[8] = min p; out[9] = max over points and directions of (|u_d| + c)/dx_d.
 * ------------------------------------------------------------------------ */
void orc_stats(const orc_params *P, const double *u, double *out) {
  long n[3], st[3];
  double h[3];
  dims(P, n, st, h);
  long N = n[0] * n[1] * n[2];
  double vol = h[0] * h[1] * h[2];
  double s[5] = {0, 0, 0, 0, 0}, ke = 0.0, ens = 0.0;
  double rmin = INFINITY, pmin = INFINITY, wmax = 0.0;
  for (long pt = 0; pt < N; ++pt) {
    double U[5];
    gather(u, N, pt, U);
    prim_t q = orc_prim(U, P->gamma);
    for (int v = 0; v < 5; ++v) s[v] += U[v];
    ke += 0.5 * q.rho * (q.u * q.u + q.v * q.v + q.w * q.w);
    long idx[3] = {pt % n[0], (pt / n[0]) % n[1], pt / (n[0] * n[1])};
    double Gp[4][3];
    point_G(P, u, N, n, h, idx, Gp);
    double wx = Gp[2][1] - Gp[1][2], wy = Gp[0][2] - Gp[2][0], wz = Gp[1][0] - Gp[0][1];
    ens += 0.5 * q.rho * (wx * wx + wy * wy + wz * wz);
    if (q.rho < rmin) rmin = q.rho;
    if (q.p < pmin) pmin = q.p;
    double c = sqrt(P->gamma * q.p / q.rho);
    double vel[3] = {q.u, q.v, q.w};
    for (int d = 0; d < 3; ++d) {
      double ws = (fabs(vel[d]) + c) / h[d];
      if (ws > wmax) wmax = ws;
    }
  }
  for (int v = 0; v < 5; ++v) out[v] = s[v] * vol;
  out[5] = ke / N;
  out[6] = ens / N;
  out[7] = rmin;
  out[8] = pmin;
  out[9] = wmax;
}
