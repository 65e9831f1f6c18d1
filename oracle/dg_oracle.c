/*
 * dg_oracle.c -- plain FP64 CPU oracle of the DG method of arXiv:1805.01443.
 *
 * TEST INFRASTRUCTURE ONLY (see dg_oracle.h): used by tests/, smoke() and
 * bench.py's CPU baseline; never by the product library.  Shares no code
 * with the CUDA path.
 *
 * Conventions (readings of the paper are marked READING):
 *   reference element [-1,1]^2, xi = 2(x - x_c)/dx, eta = 2(y - y_c)/dy;
 *   basis phi_ab(xi,eta) = sqrt(2a+1) P_a(xi) sqrt(2b+1) P_b(eta), a,b = 0..p,
 *   mode index k = a*m + b (a: x degree, b: y degree), m = p + 1.
 *   READING (Sec. 2.2): the basis is orthonormal under the MEAN inner product
 *   (1/4) int int phi_i phi_j = delta_ij, so the mass matrix is the identity and
 *   mode 0 is the element average (Sec. 3.1 uses mode 0 as the average).
 *   Operator quadrature: m Gauss-Legendre points per direction on faces and in
 *   the volume (READING of L and M in Eq. 2); IC projection: m+1 points.
 *   Canonical state layout: u[var][k][j][i].
 */
#include "dg_oracle.h"

#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846264338327950288
#endif
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXM 6            /* operator uses m <= 5; IC projection m + 1 <= 6 */
#define MAXN 25           /* modes / nodes per element, m^2 <= 25 */
#define MAXV 4
#define TWO_PI 6.283185307179586476925286766559

struct ref_state {
  ref_mesh mesh;
  ref_eos eos;
  ref_planet pl;
  ref_disc d;
  int p, m, M, nv;
  double dx, dy;
  double xg[MAXM], wg[MAXM];                 /* m-point Gauss-Legendre on [-1,1] */
  double Phi[MAXN][MAXN];                    /* phi_k at node n = q*m + r */
  double DXm[MAXN][MAXN];                    /* d phi_k / d xi at node n */
  double DYm[MAXN][MAXN];                    /* d phi_k / d eta at node n */
  double W[MAXN];                            /* w_q w_r / 4: weights normalised to sum 1 */
  double FxP[MAXN][MAXM], FxM[MAXN][MAXM];   /* phi_k(+-1, eta_r) */
  double FyP[MAXN][MAXM], FyM[MAXN][MAXM];   /* phi_k(xi_q, +-1) */
  size_t ncoef;
  double *u;
  double *ghost[4];                          /* 0: i=-1, 1: i=nx, 2: j=-1, 3: j=ny; [v][k][idx] */
  int glen[4];
  double *kbuf[6];
  double *tmp;
  double t, dt;
  long step;
  double torque, torque_abs;
};

/* ------------------------------------------------------------------------ */
/* Legendre polynomials and Gauss-Legendre quadrature (textbook definitions) */

int ref_legendre(int n, double x, double *P, double *dP) {
  /* Bonnet recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};
     derivative from P'_{k+1} = P'_{k-1} + (2k+1) P_k. */
  if (n < 0) return -1;
  P[0] = 1.0;
  dP[0] = 0.0;
  if (n == 0) return 0;
  P[1] = x;
  dP[1] = 1.0;
  for (int k = 1; k < n; k++) {
    P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
    dP[k + 1] = dP[k - 1] + (2.0 * k + 1.0) * P[k];
  }
  return 0;
}

int ref_gauss_legendre(int m, double *x, double *w) {
  /* Newton iteration on P_m from the usual cosine initial guesses;
     w = 2 / ((1 - x^2) P'_m(x)^2).  Nodes returned in ascending order. */
  if (m < 1 || m > 16) return -1;
  double P[18], dP[18];
  for (int i = 0; i < m; i++) {
    double z = cos(M_PI * (i + 0.75) / (m + 0.5));
    for (int it = 0; it < 100; it++) {
      ref_legendre(m, z, P, dP);
      double dz = P[m] / dP[m];
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    ref_legendre(m, z, P, dP);
    z -= P[m] / dP[m];
    ref_legendre(m, z, P, dP);
    x[m - 1 - i] = z;
    w[m - 1 - i] = 2.0 / ((1.0 - z * z) * dP[m] * dP[m]);
  }
  if (m % 2 == 1) x[m / 2] = 0.0;
  return 0;
}

/* normalised 1D basis sqrt(2a+1) P_a and its derivative */
static void basis1d(int p, double x, double *phi, double *dphi) {
  double P[MAXM + 1], dP[MAXM + 1];
  ref_legendre(p, x, P, dP);
  for (int a = 0; a <= p; a++) {
    double s = sqrt(2.0 * a + 1.0);
    phi[a] = s * P[a];
    dphi[a] = s * dP[a];
  }
}

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a counter-based
   generator: value(counter) = mix64(seed + (counter + 1) * golden gamma). */
static unsigned long long splitmix64(unsigned long long seed, unsigned long long counter) {
  unsigned long long z = seed + (counter + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

int ref_splitmix64_uniform(unsigned long long seed, unsigned long long counter, double *u) {
  *u = (double)(splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Runge-Kutta tableaux (Appendix A), with the readings listed below.        */

typedef struct {
  int s;
  double c[6];
  double a[6][6];
  double b[6];
} tableau;

static int get_tableau(int rk, tableau *T) {
  memset(T, 0, sizeof(*T));
  if (rk == 2) {
    /* READING (Table A4 is printed with c2 = a21 = 1/2, b = (1/2, 1/2), which fails
       the second-order condition sum b_i c_i = 1/2): use Heun's SSP(2,2), c2 = a21 = 1. */
    T->s = 2;
    T->c[1] = 1.0;
    T->a[1][0] = 1.0;
    T->b[0] = 0.5;
    T->b[1] = 0.5;
  } else if (rk == 3) {
    /* READING (Table A5 prints c3 = 3/4 while its row sums to a31 + a32 = 1/2):
       use the Shu-Osher SSP(3,3) stage times c = (0, 1, 1/2). */
    T->s = 3;
    T->c[1] = 1.0;
    T->c[2] = 0.5;
    T->a[1][0] = 1.0;
    T->a[2][0] = 0.25;
    T->a[2][1] = 0.25;
    T->b[0] = 1.0 / 6.0;
    T->b[1] = 1.0 / 6.0;
    T->b[2] = 2.0 / 3.0;
  } else if (rk == 4) {
    /* Table A1, SSP-RK(4,5).  READING: the printed b sums to 1 - 8.8e-11, so the
       weights are divided by their sum (first-order condition restored). */
    static const double c[5] = {0.0, 0.39175222700392, 0.58607968896779, 0.47454236302687,
                                0.93501063100924};
    static const double a[5][4] = {{0, 0, 0, 0},
                                   {0.39175222700392, 0, 0, 0},
                                   {0.21766909633821, 0.36841059262959, 0, 0},
                                   {0.08269208670950, 0.13995850206999, 0.25189177424738, 0},
                                   {0.06796628370320, 0.11503469844438, 0.20703489864929,
                                    0.54497475021237}};
    static const double b[5] = {0.14681187618661, 0.24848290924556, 0.10425883036650,
                                0.27443890091960, 0.22600748319395};
    double sb = 0.0;
    for (int i = 0; i < 5; i++) sb += b[i];
    T->s = 5;
    for (int i = 0; i < 5; i++) {
      T->c[i] = c[i];
      T->b[i] = b[i] / sb;
      for (int j = 0; j < 4; j++) T->a[i][j] = a[i][j];
    }
  } else if (rk == 5) {
    /* Table A2, 6-stage Cash-Karp, fifth-order weights. */
    T->s = 6;
    double c[6] = {0.0, 1.0 / 5, 3.0 / 10, 3.0 / 5, 1.0, 7.0 / 8};
    double a[6][5] = {{0, 0, 0, 0, 0},
                      {1.0 / 5, 0, 0, 0, 0},
                      {3.0 / 40, 9.0 / 40, 0, 0, 0},
                      {3.0 / 10, -9.0 / 10, 6.0 / 5, 0, 0},
                      {-11.0 / 54, 5.0 / 2, -70.0 / 27, 35.0 / 27, 0},
                      {1631.0 / 55296, 175.0 / 512, 575.0 / 13824, 44275.0 / 110592, 253.0 / 4096}};
    double b[6] = {37.0 / 378, 0.0, 250.0 / 621, 125.0 / 594, 0.0, 512.0 / 1771};
    for (int i = 0; i < 6; i++) {
      T->c[i] = c[i];
      T->b[i] = b[i];
      for (int j = 0; j < 5; j++) T->a[i][j] = a[i][j];
    }
  } else {
    return -2;
  }
  return 0;
}

typedef void (*rhs_fn)(void *ctx, double t, const double *u, double *out);

/* One explicit RK step in Butcher form (Appendix A):
   k_i = L(t + c_i h, u + h sum_{j<i} a_ij k_j);  u <- u + h sum_i b_i k_i. */
static void rk_butcher(const tableau *T, size_t N, rhs_fn f, void *ctx, double *u, double t, double h,
                       double **k, double *tmp) {
  for (int i = 0; i < T->s; i++) {
    long NN = (long)N;
#pragma omp parallel for schedule(static)
    for (long e = 0; e < NN; e++) {
      double acc = 0.0;
      for (int j = 0; j < i; j++) acc += T->a[i][j] * k[j][e];
      tmp[e] = u[e] + h * acc;
    }
    f(ctx, t + T->c[i] * h, tmp, k[i]);
  }
  long NN = (long)N;
#pragma omp parallel for schedule(static)
  for (long e = 0; e < NN; e++) {
    double acc = 0.0;
    for (int i = 0; i < T->s; i++) acc += T->b[i] * k[i][e];
    u[e] += h * acc;
  }
}

typedef struct {
  double a, b;
} lin_ctx;

static void lin_rhs(void *ctx, double t, const double *u, double *out) {
  (void)t;
  lin_ctx *c = (lin_ctx *)ctx;
  out[0] = c->a * u[0] - c->b * u[1];
  out[1] = c->b * u[0] + c->a * u[1];
}

int ref_rk_linear(int rk, double a, double b, double dt, double *re, double *im) {
  tableau T;
  if (get_tableau(rk, &T)) return -2;
  double u[2] = {1.0, 0.0}, tmp[2], kb[6][2];
  double *k[6];
  for (int i = 0; i < 6; i++) k[i] = kb[i];
  lin_ctx c = {a, b};
  rk_butcher(&T, 2, lin_rhs, &c, u, 0.0, dt, k, tmp);
  *re = u[0];
  *im = u[1];
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Physics: EOS, fluxes, potentials (Sec. 2.1, Sec. 5.1)                     */

static inline size_t cidx(const ref_state *s, int v, int k, int i, int j) {
  return (((size_t)v * s->M + k) * s->mesh.ny + j) * s->mesh.nx + i;
}

/* Keplerian speed squared of the softened star potential (READING of the
   solid-body core of Sec. 5.1 with core radius r_s): r dPhi_s/dr. */
static double vk2_at(const ref_state *s, double r) {
  double rs = s->d.r_soft;
  if (r >= rs) return 1.0 / r;
  return r * r / (rs * rs * rs);
}

/* isothermal sound speed squared at a point (EOS kinds 0 and 2) */
static double cs2_at(const ref_state *s, double x, double y) {
  double h = s->eos.h;
  if (s->eos.kind == 2) return h * h;
  if (s->eos.kind == 0) return h * h * vk2_at(s, sqrt(x * x + y * y));
  return 0.0;
}

/* directional physical flux f_dir(u) and wave speed |v_dir| + c (Eq. 1) */
static void phys_flux(const ref_state *s, const double *u, double cs2, int dir, double *f,
                      double *speed) {
  double rho = u[0], mx = u[1], my = u[2];
  double vx = mx / rho, vy = my / rho;
  double p, c;
  if (s->eos.kind == 1) {
    double g = s->eos.gamma;
    p = (g - 1.0) * (u[3] - 0.5 * (mx * vx + my * vy));
    c = sqrt(g * p / rho);
  } else {
    p = cs2 * rho;
    c = sqrt(cs2);
  }
  double vn = (dir == 0) ? vx : vy;
  f[0] = rho * vn;
  f[1] = mx * vn + ((dir == 0) ? p : 0.0);
  f[2] = my * vn + ((dir == 1) ? p : 0.0);
  if (s->eos.kind == 1) f[3] = (u[3] + p) * vn;
  *speed = fabs(vn) + c;
}

/* READING (Eq. 2: flux type unstated): local Lax-Friedrichs (Rusanov) flux
   h = (f(uL) + f(uR))/2 . n - alpha (uR - uL)/2, alpha = max over both sides of |v.n| + c,
   with uL on the lower-coordinate side and n the +dir unit vector. */
static void llf(const ref_state *s, const double *uL, const double *uR, int dir, double x,
                double y, double *h) {
  double cs2 = cs2_at(s, x, y);
  double fL[MAXV], fR[MAXV], aL, aR;
  phys_flux(s, uL, cs2, dir, fL, &aL);
  phys_flux(s, uR, cs2, dir, fR, &aR);
  double a = aL > aR ? aL : aR;
  for (int v = 0; v < s->nv; v++) h[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * a * (uR[v] - uL[v]);
}

static void planet_pos(const ref_state *s, double t, double *xp, double *yp) {
  double ph = s->pl.omega_p * t + s->pl.phi0;
  *xp = s->pl.r_p * cos(ph);
  *yp = s->pl.r_p * sin(ph);
}

/* grad Phi at (x,y): softened star (READING: C^1 solid-body core of radius r_s,
   Sec. 5.1) plus Plummer-softened planet (smoothing eps, as in the torque equation). */
static void grad_phi(const ref_state *s, double x, double y, double xp, double yp, double *gx,
                     double *gy) {
  double ax = 0.0, ay = 0.0;
  if (s->d.star) {
    double r2 = x * x + y * y, r = sqrt(r2), rs = s->d.r_soft, inv;
    if (r >= rs)
      inv = 1.0 / (r2 * r);
    else
      inv = 1.0 / (rs * rs * rs);
    ax += x * inv;
    ay += y * inv;
  }
  if (s->pl.enabled) {
    double ddx = x - xp, ddy = y - yp;
    double d2 = ddx * ddx + ddy * ddy + s->pl.eps * s->pl.eps;
    double inv = s->pl.q / (d2 * sqrt(d2));
    ax += ddx * inv;
    ay += ddy * inv;
  }
  *gx = ax;
  *gy = ay;
}

/* background primitive state (rho, vx, vy, p) of the chosen initial condition,
   without noise: the damping target Q0 and the fixed ghost state */
static void background_prim(const ref_state *s, double x, double y, double *w) {
  if (s->d.ic == 0 || s->d.ic == 3) {
    /* READING (configs): Sigma = max(r^slope, floor); rotational equilibrium
       v_phi^2 = r dPhi_s/dr + (r/Sigma) d(c_s^2 Sigma)/dr (Sec. 5.1) with c_s = h v_K,
       which for Sigma ~ r^s gives (1 + (s-1) h^2)/r outside r_s and
       (1 + (s+2) h^2) r^2 / r_s^3 inside. */
    double r = sqrt(x * x + y * y);
    if (r < 1e-12) r = 1e-12;
    double sl = s->d.sigma_slope, h = s->eos.h, rs = s->d.r_soft;
    double sig = pow(r, sl);
    if (sig < s->d.sigma_floor) sig = s->d.sigma_floor;
    double vphi2;
    if (r >= rs)
      vphi2 = (1.0 + (sl - 1.0) * h * h) / r;
    else
      vphi2 = (1.0 + (sl + 2.0) * h * h) * r * r / (rs * rs * rs);
    double vphi = sqrt(vphi2 > 0.0 ? vphi2 : 0.0);
    w[0] = sig;
    w[1] = -vphi * y / r;
    w[2] = vphi * x / r;
    w[3] = h * h * vk2_at(s, r) * sig; /* p = c_s,iso^2 Sigma (adiabatic disc) */
    /* READING (config 5): the imposed shock ring is a pressure step, p x ring_p
       inside r < ring_r, on the same disc (sharp at the nodes, then projected) */
    if (s->d.ic == 3 && r < s->d.ring_r) w[3] *= s->d.ring_p;
  } else if (s->d.ic == 6) {
    /* Sec. 5.1, the paper's own disc: Sigma = Sigma_0 / (1 + f), p = p_0 / (1 + f),
       f = exp((r - r_ex) / (r_p h)), in rotational equilibrium
       v_phi^2 = r^2 Omega^2 + (r / Sigma) d(c_s,iso^2 Sigma)/dr with Omega solid-body
       inside r_in and Keplerian outside.  READINGS: the printed first term
       "Omega^2" is r^2 Omega^2 (the first equality and the units say so);
       Sigma_0 = r_p = 1 and c_s,iso = h (p_0 = h^2 Sigma_0, the printed
       2.5e-3 for h = 0.05); r_in is the star's solid-body core r_s, so that
       r^2 Omega^2 = v_K^2; r_ex is the outer damping radius times 1.15^(3/2)
       (the paper places r_d = r_ex 1.15^(-3/2)).  p / Sigma = h^2 everywhere,
       so d(c_s,iso^2 Sigma)/dr = h^2 dSigma/dr = -h f Sigma / (1 + f).
       READING: Sigma is floored at sigma_floor (1e-4 in the configurations,
       as for the other discs), beyond r ~ r_ex + h ln(1/floor); unfloored the
       box corners hold Sigma ~ 4e-13 and p ~ 1e-15, below the positivity
       limiter's absolute floor.  Where the floor holds there is no pressure
       gradient and v_phi is the star's alone. */
    double r = sqrt(x * x + y * y);
    if (r < 1e-12) r = 1e-12;
    const double h = s->eos.h, rex = s->d.rdamp_out * pow(1.15, 1.5);
    const double f = exp((r - rex) / h);
    double sig = 1.0 / (1.0 + f), g = f / (1.0 + f);
    if (sig < s->d.sigma_floor) {
      sig = s->d.sigma_floor;
      g = 0.0;
    }
    const double vphi2 = vk2_at(s, r) - r * h * g;
    const double vphi = sqrt(vphi2 > 0.0 ? vphi2 : 0.0);
    w[0] = sig;
    w[1] = -vphi * y / r;
    w[2] = vphi * x / r;
    w[3] = h * h * sig;
  } else if (s->d.ic == 4) {
    /* Sec. 4.1 isentropic vortex (Yee et al.) about (x0 + x1, y0 + y1)/2 in
       the free stream rho = p = 1, v = (vx0, vy0); READING: the vortex
       strength beta is not printed, beta = amp (5 in the workloads) */
    const double g = s->eos.gamma, beta = s->d.amp;
    const double xc = 0.5 * (s->mesh.x0 + s->mesh.x1), yc = 0.5 * (s->mesh.y0 + s->mesh.y1);
    const double dx = x - xc, dy = y - yc, r2 = dx * dx + dy * dy;
    const double T = 1.0 - (g - 1.0) * beta * beta / (8.0 * g * M_PI * M_PI) * exp(1.0 - r2);
    const double du = beta / (2.0 * M_PI) * exp(0.5 * (1.0 - r2));
    w[0] = pow(T, 1.0 / (g - 1.0));
    w[1] = s->d.vx0 - du * dy;
    w[2] = s->d.vy0 + du * dx;
    w[3] = pow(w[0], g);
  } else if (s->d.ic == 5) {
    /* Sec. 4.2 Gresho vortex about the box centre: rho = 1, v_phi and p(r) piecewise */
    const double xc = 0.5 * (s->mesh.x0 + s->mesh.x1), yc = 0.5 * (s->mesh.y0 + s->mesh.y1);
    const double dx = x - xc, dy = y - yc, r = sqrt(dx * dx + dy * dy);
    double vphi, p;
    if (r < 0.2) {
      vphi = 5.0 * r;
      p = 5.0 + 12.5 * r * r;
    } else if (r < 0.4) {
      vphi = 2.0 - 5.0 * r;
      p = 9.0 - 4.0 * log(0.2) + 12.5 * r * r - 20.0 * r + 4.0 * log(r);
    } else {
      vphi = 0.0;
      p = 3.0 + 4.0 * log(2.0);
    }
    w[0] = 1.0;
    w[1] = r > 0.0 ? -vphi * dy / r : 0.0;
    w[2] = r > 0.0 ? vphi * dx / r : 0.0;
    w[3] = p;
  } else if (s->d.ic == 1) {
    double lx = s->mesh.x1 - s->mesh.x0, ly = s->mesh.y1 - s->mesh.y0;
    double ph = TWO_PI * ((x - s->mesh.x0) / lx + (y - s->mesh.y0) / ly);
    w[0] = 1.0 + s->d.amp * sin(ph);
    w[1] = s->d.vx0;
    w[2] = s->d.vy0;
    w[3] = 1.0;
  } else {
    w[0] = 1.0;
    w[1] = s->d.vx0;
    w[2] = s->d.vy0;
    w[3] = 1.0;
  }
}

static void prim_to_cons(const ref_state *s, const double *w, double *u) {
  u[0] = w[0];
  u[1] = w[0] * w[1];
  u[2] = w[0] * w[2];
  if (s->eos.kind == 1)
    u[3] = w[3] / (s->eos.gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2]);
}

/* ------------------------------------------------------------------------ */
/* Initial data: L2 projection with m+1 GL points (Eq. 2, first line)        */

static void project_element(const ref_state *s, int i, int j, int noise, double c[MAXV][MAXN]) {
  int m = s->m, mq = m + 1;
  double xq[MAXM + 1], wq[MAXM + 1], ph[MAXM + 1][MAXM], dph[MAXM];
  ref_gauss_legendre(mq, xq, wq);
  for (int q = 0; q < mq; q++) basis1d(s->p, xq[q], ph[q], dph);
  double xc = s->mesh.x0 + (i + 0.5) * s->dx, yc = s->mesh.y0 + (j + 0.5) * s->dy;
  for (int v = 0; v < s->nv; v++)
    for (int k = 0; k < s->M; k++) c[v][k] = 0.0;
  for (int q = 0; q < mq; q++)
    for (int r = 0; r < mq; r++) {
      double x = xc + 0.5 * s->dx * xq[q], y = yc + 0.5 * s->dy * xq[r];
      double w[4], u[4];
      background_prim(s, x, y, w);
      if (noise && (s->d.ic == 0 || s->d.ic == 3) && s->d.noise_amp > 0.0) {
        /* READING (configs): additive U(-amp, amp) on Sigma at each projection node,
           keyed by (seed, element, node). */
        double U;
        unsigned long long ctr =
            ((unsigned long long)j * s->mesh.nx + i) * (unsigned long long)(mq * mq) + q * mq + r;
        ref_splitmix64_uniform(s->d.seed, ctr, &U);
        w[0] += s->d.noise_amp * (2.0 * U - 1.0);
      }
      prim_to_cons(s, w, u);
      double wt = 0.25 * wq[q] * wq[r];
      for (int a = 0; a < m; a++)
        for (int b = 0; b < m; b++)
          for (int v = 0; v < s->nv; v++) c[v][a * m + b] += wt * u[v] * ph[q][a] * ph[r][b];
    }
}

static void init_ic(ref_state *s) {
  int nx = s->mesh.nx, ny = s->mesh.ny;
#pragma omp parallel for schedule(static)
  for (long e = 0; e < (long)nx * ny; e++) {
    int i = (int)(e % nx), j = (int)(e / nx);
    double c[MAXV][MAXN];
    project_element(s, i, j, 1, c);
    for (int v = 0; v < s->nv; v++)
      for (int k = 0; k < s->M; k++) s->u[cidx(s, v, k, i, j)] = c[v][k];
  }
  /* READING (outer boundary, unstated in the paper): ghost elements hold the
     projected background state, consistent with the damping target. */
  for (int side = 0; side < 4; side++) {
    int len = s->glen[side];
    for (int idx = 0; idx < len; idx++) {
      int i, j;
      if (side == 0) { i = -1; j = idx; }
      else if (side == 1) { i = nx; j = idx; }
      else if (side == 2) { i = idx; j = -1; }
      else { i = idx; j = ny; }
      double c[MAXV][MAXN];
      project_element(s, i, j, 0, c);
      for (int v = 0; v < s->nv; v++)
        for (int k = 0; k < s->M; k++) s->ghost[side][((size_t)v * s->M + k) * len + idx] = c[v][k];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Spatial operator L(u, t): right-hand side of Eq. 2 divided by |K|          */

/* coefficients of element (i,j), which may lie outside the mesh; returns 0
   for a transmissive boundary (the caller then mirrors its own trace).
   READING (Sec. 4.2 "gradient free" boundaries): bc 3 is a zero-gradient
   ghost layer, the ghost element a copy of the adjacent interior element */
static int gather(const ref_state *s, const double *u, int i, int j, double c[MAXV][MAXN]) {
  int nx = s->mesh.nx, ny = s->mesh.ny;
  int inside = (i >= 0 && i < nx && j >= 0 && j < ny);
  if (!inside) {
    if (s->mesh.bc == 0) {
      i = (i + nx) % nx;
      j = (j + ny) % ny;
      inside = 1;
    } else if (s->mesh.bc == 3) {
      i = i < 0 ? 0 : (i >= nx ? nx - 1 : i);
      j = j < 0 ? 0 : (j >= ny ? ny - 1 : j);
      inside = 1;
    } else if (s->mesh.bc == 1) {
      int side = (i < 0) ? 0 : (i >= nx) ? 1 : (j < 0) ? 2 : 3;
      int idx = (side < 2) ? j : i;
      int len = s->glen[side];
      for (int v = 0; v < s->nv; v++)
        for (int k = 0; k < s->M; k++) c[v][k] = s->ghost[side][((size_t)v * s->M + k) * len + idx];
      return 1;
    } else {
      return 0;
    }
  }
  for (int v = 0; v < s->nv; v++)
    for (int k = 0; k < s->M; k++) c[v][k] = u[cidx(s, v, k, i, j)];
  return 1;
}

/* trace of an element polynomial at face node r: sum_k c_k F[k][r] */
static void trace(const ref_state *s, double c[MAXV][MAXN], double F[MAXN][MAXM], int r, double *out) {
  for (int v = 0; v < s->nv; v++) {
    double acc = 0.0;
    for (int k = 0; k < s->M; k++) acc += c[v][k] * F[k][r];
    out[v] = acc;
  }
}

typedef struct {
  ref_state *s;
} op_ctx;

static void rhs_eval(void *vctx, double t, const double *u, double *out) {
  ref_state *s = ((op_ctx *)vctx)->s;
  const int nx = s->mesh.nx, ny = s->mesh.ny, m = s->m, M = s->M, nv = s->nv;
  const double dx = s->dx, dy = s->dy;
  double xp, yp;
  planet_pos(s, t, &xp, &yp);
#pragma omp parallel for schedule(static)
  for (long e = 0; e < (long)nx * ny; e++) {
    int i = (int)(e % nx), j = (int)(e / nx);
    double c[MAXV][MAXN], cn[MAXV][MAXN], un[MAXV][MAXN], R[MAXV][MAXN];
    gather(s, u, i, j, c);
    double xc = s->mesh.x0 + (i + 0.5) * dx, yc = s->mesh.y0 + (j + 0.5) * dy;
    /* modal -> nodal at the m x m GL nodes */
    for (int v = 0; v < nv; v++)
      for (int n = 0; n < M; n++) {
        double acc = 0.0;
        for (int k = 0; k < M; k++) acc += c[v][k] * s->Phi[k][n];
        un[v][n] = acc;
      }
    for (int v = 0; v < nv; v++)
      for (int k = 0; k < M; k++) R[v][k] = 0.0;
    /* volume flux and source terms of Eq. 2 */
    for (int n = 0; n < M; n++) {
      int q = n / m, r = n % m;
      double x = xc + 0.5 * dx * s->xg[q], y = yc + 0.5 * dy * s->xg[r];
      double uu[MAXV], fx[MAXV], fy[MAXV], S[MAXV], sp, gx, gy;
      for (int v = 0; v < nv; v++) uu[v] = un[v][n];
      double cs2 = cs2_at(s, x, y);
      phys_flux(s, uu, cs2, 0, fx, &sp);
      phys_flux(s, uu, cs2, 1, fy, &sp);
      grad_phi(s, x, y, xp, yp, &gx, &gy);
      S[0] = 0.0;
      S[1] = -uu[0] * gx;
      S[2] = -uu[0] * gy;
      if (nv == 4) S[3] = -(uu[1] * gx + uu[2] * gy);
      for (int v = 0; v < nv; v++)
        for (int k = 0; k < M; k++)
          R[v][k] += s->W[n] * ((2.0 / dx) * fx[v] * s->DXm[k][n] + (2.0 / dy) * fy[v] * s->DYm[k][n] +
                                S[v] * s->Phi[k][n]);
    }
    /* surface terms: numerical flux times test function on each of the four faces */
    double uL[MAXV], uR[MAXV], h[MAXV];
    /* left face (i-1 | i), x = x0 + i dx */
    int has = gather(s, u, i - 1, j, cn);
    for (int r = 0; r < m; r++) {
      trace(s, c, s->FxM, r, uR);
      if (has) trace(s, cn, s->FxP, r, uL);
      else memcpy(uL, uR, sizeof(uL));
      llf(s, uL, uR, 0, s->mesh.x0 + i * dx, yc + 0.5 * dy * s->xg[r], h);
      double wf = 0.5 * s->wg[r] / dx;
      for (int v = 0; v < nv; v++)
        for (int k = 0; k < M; k++) R[v][k] += wf * h[v] * s->FxM[k][r];
    }
    /* right face (i | i+1), x = x0 + (i+1) dx */
    has = gather(s, u, i + 1, j, cn);
    for (int r = 0; r < m; r++) {
      trace(s, c, s->FxP, r, uL);
      if (has) trace(s, cn, s->FxM, r, uR);
      else memcpy(uR, uL, sizeof(uR));
      llf(s, uL, uR, 0, s->mesh.x0 + (i + 1) * dx, yc + 0.5 * dy * s->xg[r], h);
      double wf = 0.5 * s->wg[r] / dx;
      for (int v = 0; v < nv; v++)
        for (int k = 0; k < M; k++) R[v][k] -= wf * h[v] * s->FxP[k][r];
    }
    /* bottom face (j-1 | j), y = y0 + j dy */
    has = gather(s, u, i, j - 1, cn);
    for (int q = 0; q < m; q++) {
      trace(s, c, s->FyM, q, uR);
      if (has) trace(s, cn, s->FyP, q, uL);
      else memcpy(uL, uR, sizeof(uL));
      llf(s, uL, uR, 1, xc + 0.5 * dx * s->xg[q], s->mesh.y0 + j * dy, h);
      double wf = 0.5 * s->wg[q] / dy;
      for (int v = 0; v < nv; v++)
        for (int k = 0; k < M; k++) R[v][k] += wf * h[v] * s->FyM[k][q];
    }
    /* top face (j | j+1), y = y0 + (j+1) dy */
    has = gather(s, u, i, j + 1, cn);
    for (int q = 0; q < m; q++) {
      trace(s, c, s->FyP, q, uL);
      if (has) trace(s, cn, s->FyM, q, uR);
      else memcpy(uR, uL, sizeof(uR));
      llf(s, uL, uR, 1, xc + 0.5 * dx * s->xg[q], s->mesh.y0 + (j + 1) * dy, h);
      double wf = 0.5 * s->wg[q] / dy;
      for (int v = 0; v < nv; v++)
        for (int k = 0; k < M; k++) R[v][k] -= wf * h[v] * s->FyP[k][q];
    }
    for (int v = 0; v < nv; v++)
      for (int k = 0; k < M; k++) out[cidx(s, v, k, i, j)] = R[v][k];
  }
}

/* ------------------------------------------------------------------------ */
/* Time step, damping, torque                                                */

/* Sec. 2.3: dt_K = C/(2p+1) * (sum_i (|v_i| + c_s)/dx_i)^-1 from the element
   averages (mode 0), global minimum.  READING: for the isothermal EOS c_s is
   taken at the element centre. */
/* the factor of C in the CFL step (Sec. 2.3): 1/(2p+1), and with the
   positivity limiter (Sec. 2.4) min(1/(2p+1), w_1/2) where w_1 is the first weight of the
   N-point Gauss-Lobatto rule normalised to sum 1.  READING: N is the smallest
   count with 2N - 3 >= p (the rule Zhang & Shu use for degree p), and the
   endpoint weight of that rule is 2/(N(N-1)) on [-1,1], i.e. 1/(N(N-1)). */
static double cfl_factor(const ref_state *s) {
  double f = 1.0 / (2.0 * s->p + 1.0);
  if (s->d.positivity) {
    int N = 2;
    while (2 * N - 3 < s->p) N++;
    double w1 = 1.0 / (N * (N - 1.0));
    if (0.5 * w1 < f) f = 0.5 * w1;
  }
  return f;
}

static double cfl_dt(const ref_state *s, const double *u) {
  const int nx = s->mesh.nx, ny = s->mesh.ny;
  double best = INFINITY;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      double rho = u[cidx(s, 0, 0, i, j)], mx = u[cidx(s, 1, 0, i, j)], my = u[cidx(s, 2, 0, i, j)];
      double vx = mx / rho, vy = my / rho, c;
      if (s->eos.kind == 1) {
        double g = s->eos.gamma, E = u[cidx(s, 3, 0, i, j)];
        double p = (g - 1.0) * (E - 0.5 * (mx * vx + my * vy));
        c = sqrt(g * p / rho);
      } else {
        double xc = s->mesh.x0 + (i + 0.5) * s->dx, yc = s->mesh.y0 + (j + 0.5) * s->dy;
        c = sqrt(cs2_at(s, xc, yc));
      }
      double dtk = s->d.cfl * cfl_factor(s) / ((fabs(vx) + c) / s->dx + (fabs(vy) + c) / s->dy);
      if (!(dtk >= best)) best = dtk; /* NaN propagates */
    }
  return best;
}

/* damping ramp R(r) of Sec. 5.1 for one zone; READING: the configured radius is
   the paper's damping radius r_d and the boundary radius sits at the paper's
   ratio 1.15^(3/2) beyond it; R is clamped to [0, 1]. */
static double ramp(double r, double rd, int inner) {
  double f = pow(1.15, 1.5);
  double rb = inner ? rd / f : rd * f;
  if (inner ? !(r < rd) : !(r > rd)) return 0.0;
  double x = (r - rd) / (rb - rd);
  double R = x * x;
  return R > 1.0 ? 1.0 : R;
}

static void damp_apply(ref_state *s, double *u, double dt) {
  const int nx = s->mesh.nx, ny = s->mesh.ny, m = s->m, M = s->M, nv = s->nv;
  double rin = s->d.rdamp_in, rout = s->d.rdamp_out;
  if (!(rin > 0.0) && !(rout > 0.0)) return;
#pragma omp parallel for schedule(static)
  for (long e = 0; e < (long)nx * ny; e++) {
    int i = (int)(e % nx), j = (int)(e / nx);
    double xc = s->mesh.x0 + (i + 0.5) * s->dx, yc = s->mesh.y0 + (j + 0.5) * s->dy;
    double tau_fac[MAXN];
    int any = 0;
    for (int n = 0; n < M; n++) {
      int q = n / m, r = n % m;
      double x = xc + 0.5 * s->dx * s->xg[q], y = yc + 0.5 * s->dy * s->xg[r];
      double rr = sqrt(x * x + y * y), R = 0.0, rd = 0.0;
      if (rin > 0.0 && rr < rin) { R = ramp(rr, rin, 1); rd = rin; }
      else if (rout > 0.0 && rr > rout) { R = ramp(rr, rout, 0); rd = rout; }
      /* tau = 2 pi sqrt(r_d^3 / (G M_*)) / R(r); zero R means no damping */
      tau_fac[n] = (R > 0.0) ? TWO_PI * sqrt(rd * rd * rd) / R : -1.0;
      if (R > 0.0) any = 1;
    }
    if (!any) continue;
    double c[MAXV][MAXN], un[MAXV][MAXN];
    for (int v = 0; v < nv; v++)
      for (int k = 0; k < M; k++) c[v][k] = u[cidx(s, v, k, i, j)];
    for (int v = 0; v < nv; v++)
      for (int n = 0; n < M; n++) {
        double acc = 0.0;
        for (int k = 0; k < M; k++) acc += c[v][k] * s->Phi[k][n];
        un[v][n] = acc;
      }
    for (int n = 0; n < M; n++) {
      double tau = tau_fac[n];
      if (tau < 0.0) continue;
      int q = n / m, r = n % m;
      double x = xc + 0.5 * s->dx * s->xg[q], y = yc + 0.5 * s->dy * s->xg[r];
      double w0[4];
      background_prim(s, x, y, w0);
      /* damped fields: density, velocities (and temperature p/rho, adiabatic) */
      double Q[4], Q0[4];
      Q[0] = un[0][n];
      Q[1] = un[1][n] / un[0][n];
      Q[2] = un[2][n] / un[0][n];
      Q0[0] = w0[0];
      Q0[1] = w0[1];
      Q0[2] = w0[2];
      if (nv == 4) {
        double g = s->eos.gamma;
        double p = (g - 1.0) * (un[3][n] - 0.5 * (un[1][n] * Q[1] + un[2][n] * Q[2]));
        Q[3] = p / un[0][n];
        Q0[3] = w0[3] / w0[0];
      }
      for (int v = 0; v < nv; v++) Q[v] = (dt * Q0[v] + tau * Q[v]) / (tau + dt);
      double w[4] = {Q[0], Q[1], Q[2], (nv == 4) ? Q[3] * Q[0] : 0.0}, uu[4];
      prim_to_cons(s, w, uu);
      for (int v = 0; v < nv; v++) un[v][n] = uu[v];
    }
    /* back to modes by the m-point quadrature projection */
    for (int v = 0; v < nv; v++)
      for (int k = 0; k < M; k++) {
        double acc = 0.0;
        for (int n = 0; n < M; n++) acc += s->W[n] * un[v][n] * s->Phi[k][n];
        u[cidx(s, v, k, i, j)] = acc;
      }
  }
}

/* Sec. 5.2: Gamma = r_p x sum_n G M_n (r_n - r_p) / [(r_n - r_p)^2 + eps^2]^(3/2).
   READING: the "cells" are the quadrature nodes, M_n = Sigma(x_n) w_q w_r |K| / 4.
   Serial sum in fixed (element, node) order; also returns sum_n |Gamma_n|. */
static void torque_eval(const ref_state *s, const double *u, double t, double *gz, double *gabs) {
  const int nx = s->mesh.nx, ny = s->mesh.ny, m = s->m, M = s->M;
  double xp, yp;
  planet_pos(s, t, &xp, &yp);
  double gx = 0.0, gy = 0.0, ab = 0.0, area = s->dx * s->dy, e2 = s->pl.eps * s->pl.eps;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      double xc = s->mesh.x0 + (i + 0.5) * s->dx, yc = s->mesh.y0 + (j + 0.5) * s->dy;
      for (int n = 0; n < M; n++) {
        int q = n / m, r = n % m;
        double sig = 0.0;
        for (int k = 0; k < M; k++) sig += u[cidx(s, 0, k, i, j)] * s->Phi[k][n];
        double x = xc + 0.5 * s->dx * s->xg[q], y = yc + 0.5 * s->dy * s->xg[r];
        double mass = sig * s->W[n] * area;
        double ddx = x - xp, ddy = y - yp, d2 = ddx * ddx + ddy * ddy + e2;
        double f = mass / (d2 * sqrt(d2));
        double gxn = f * ddx, gyn = f * ddy;
        gx += gxn;
        gy += gyn;
        ab += fabs(xp * gyn - yp * gxn);
      }
    }
  *gz = xp * gy - yp * gx;
  *gabs = ab;
}

/* ------------------------------------------------------------------------ */
/* Public entry points                                                       */

/* ------------------------------------------------------------------------ */
/* Troubled-cell indicator and limiters                                       */

static int all_finite(const ref_state *s);

#define SQRT3 1.7320508075688772935274463415059 /* phi_1(+1) / phi_0: the linear mode's face increment */

/* minmod of three numbers */
static double minmod3(double a, double b, double c) {
  if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
  if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
  return 0.0;
}

/* Cockburn & Shu's TVB-modified minmod: a1 itself when |a1| <= M h^2 */
static double tvb_minmod(double a1, double a2, double a3, double mh2) {
  if (fabs(a1) <= mh2) return a1;
  return minmod3(a1, a2, a3);
}

/* element mean (mode 0) of each variable of element (i, j) of u, outside
   elements by the boundary rule (transmissive: the element's own mean) */
static void mean_at(const ref_state *s, const double *u, int i, int j, int ii, int jj, double *out) {
  double c[MAXV][MAXN];
  if (!gather(s, u, ii, jj, c)) gather(s, u, i, j, c);
  for (int v = 0; v < s->nv; v++) out[v] = c[v][0];
}

/* TVB test of element (i, j): per variable and direction, the face increment
   of the linear mode, sqrt(3) u_(1,0) in x and sqrt(3) u_(0,1) in y, against
   the forward and backward differences of the element means.  Returns 1 when
   any of them would be changed (the element is troubled) and gives the
   limited increments. */
static int tvb_element(const ref_state *s, const double *u, int i, int j, double M, double *sx,
                       double *sy) {
  const int m = s->m, nv = s->nv;
  double mL[MAXV], mR[MAXV], mB[MAXV], mT[MAXV];
  mean_at(s, u, i, j, i - 1, j, mL);
  mean_at(s, u, i, j, i + 1, j, mR);
  mean_at(s, u, i, j, i, j - 1, mB);
  mean_at(s, u, i, j, i, j + 1, mT);
  const double mhx = M * s->dx * s->dx, mhy = M * s->dy * s->dy;
  int troubled = 0;
  for (int v = 0; v < nv; v++) {
    const double mean = u[cidx(s, v, 0, i, j)];
    const double ax = SQRT3 * u[cidx(s, v, m, i, j)];   /* mode (a, b) = (1, 0) */
    const double ay = SQRT3 * u[cidx(s, v, 1, i, j)];   /* mode (0, 1) */
    sx[v] = tvb_minmod(ax, mR[v] - mean, mean - mL[v], mhx);
    sy[v] = tvb_minmod(ay, mT[v] - mean, mean - mB[v], mhy);
    if (sx[v] != ax || sy[v] != ay) troubled = 1;
  }
  return troubled;
}

static void tvb_flags(const ref_state *s, const double *u, double M, unsigned char *flags) {
  const int nx = s->mesh.nx, ny = s->mesh.ny;
#pragma omp parallel for schedule(static)
  for (long e = 0; e < (long)nx * ny; e++) {
    double sx[MAXV], sy[MAXV];
    flags[e] = (unsigned char)tvb_element(s, u, (int)(e % nx), (int)(e / nx), M, sx, sy);
  }
}

/* A troubled element becomes its mean plus the limited linear modes in x and
   y, every other mode zero (all variables).  Means are kept, so limiting in
   place does not change what the neighbours see. */
static void limit_p1(const ref_state *s, double *u, const unsigned char *flags) {
  const int nx = s->mesh.nx, ny = s->mesh.ny, m = s->m, M = s->M, nv = s->nv;
  double *lim = s->tmp; /* limited increments, [e][2 * nv] */
#pragma omp parallel for schedule(static)
  for (long e = 0; e < (long)nx * ny; e++) {
    if (!flags[e]) continue;
    double sx[MAXV], sy[MAXV];
    tvb_element(s, u, (int)(e % nx), (int)(e / nx), s->d.tvb_m, sx, sy);
    for (int v = 0; v < nv; v++) {
      lim[e * 2 * MAXV + v] = sx[v];
      lim[e * 2 * MAXV + MAXV + v] = sy[v];
    }
  }
#pragma omp parallel for schedule(static)
  for (long e = 0; e < (long)nx * ny; e++) {
    if (!flags[e]) continue;
    const int i = (int)(e % nx), j = (int)(e / nx);
    for (int v = 0; v < nv; v++) {
      for (int k = 1; k < M; k++) u[cidx(s, v, k, i, j)] = 0.0;
      u[cidx(s, v, m, i, j)] = lim[e * 2 * MAXV + v] / SQRT3;
      u[cidx(s, v, 1, i, j)] = lim[e * 2 * MAXV + MAXV + v] / SQRT3;
    }
  }
}

static double pressure_of(const ref_state *s, const double *U) {
  return (s->eos.gamma - 1.0) * (U[3] - 0.5 * (U[1] * U[1] + U[2] * U[2]) / U[0]);
}

/* point values of element coefficients c at check point n: the m x m volume
   nodes (n < M), then the m points of the faces x = +1, x = -1, y = +1, y = -1 */
static void eval_point(const ref_state *s, double c[MAXV][MAXN], int n, double *U) {
  const int M = s->M, m = s->m;
  for (int v = 0; v < s->nv; v++) {
    double acc = 0.0;
    for (int k = 0; k < M; k++) {
      double phi;
      if (n < M) phi = s->Phi[k][n];
      else {
        int f = (n - M) / m, r = (n - M) % m;
        phi = f == 0 ? s->FxP[k][r] : f == 1 ? s->FxM[k][r] : f == 2 ? s->FyP[k][r] : s->FyM[k][r];
      }
      acc += c[v][k] * phi;
    }
    U[v] = acc;
  }
}

/* Zhang & Shu's positivity limiter (Sec. 2.4) on one element.  READING: the
   check points are the points where the operator evaluates the solution (the
   m x m volume nodes and the 4m face points), eps = 1e-13; density first
   (theta = (mean - eps)/(mean - min)), then pressure with
   theta = min over points with p < eps of (p(mean) - eps)/(p(mean) - p(point)),
   which keeps p >= eps because p is concave in the conserved variables. */
static void positivity_element(const ref_state *s, double c[MAXV][MAXN]) {
  const double eps = 1e-13;
  const int M = s->M, np = s->M + 4 * s->m, nv = s->nv;
  double U[MAXV];
  double rmin = INFINITY;
  for (int n = 0; n < np; n++) {
    eval_point(s, c, n, U);
    if (U[0] < rmin) rmin = U[0];
  }
  const double rbar = c[0][0];
  if (rmin < eps && rbar > eps) {
    double th = (rbar - eps) / (rbar - rmin);
    if (th < 0.0) th = 0.0;
    for (int k = 1; k < M; k++) c[0][k] *= th;
  }
  if (nv < 4) return;
  double Ub[MAXV];
  for (int v = 0; v < nv; v++) Ub[v] = c[v][0];
  const double pbar = pressure_of(s, Ub);
  if (!(pbar > eps)) return;
  double th = 1.0;
  for (int n = 0; n < np; n++) {
    eval_point(s, c, n, U);
    const double p = pressure_of(s, U);
    if (p < eps) {
      const double t = (pbar - eps) / (pbar - p);
      if (t < th) th = t;
    }
  }
  if (th < 1.0) {
    if (th < 0.0) th = 0.0;
    for (int v = 0; v < nv; v++)
      for (int k = 1; k < M; k++) c[v][k] *= th;
  }
}

static void positivity_all(const ref_state *s, double *u) {
  const int nx = s->mesh.nx, ny = s->mesh.ny;
#pragma omp parallel for schedule(static)
  for (long e = 0; e < (long)nx * ny; e++) {
    const int i = (int)(e % nx), j = (int)(e / nx);
    double c[MAXV][MAXN];
    gather(s, u, i, j, c);
    positivity_element(s, c);
    for (int v = 0; v < s->nv; v++)
      for (int k = 0; k < s->M; k++) u[cidx(s, v, k, i, j)] = c[v][k];
  }
}

/* the limiter of a stage value: troubled cells by the TVB test (limiter 1) or
   by the given flags, then positivity */
static void limit_apply(ref_state *s, double *u, const unsigned char *given) {
  const size_t ne = (size_t)s->mesh.nx * s->mesh.ny;
  if (given || s->d.limiter == 1) {
    unsigned char *fl = (unsigned char *)malloc(ne);
    if (given) memcpy(fl, given, ne);
    else tvb_flags(s, u, s->d.tvb_m, fl);
    limit_p1(s, u, fl);
    free(fl);
  }
  if (s->d.positivity) positivity_all(s, u);
}

/* One SSP(3,3) step in Shu-Osher form (Sec. 3.1, Table A5 with c = (0, 1, 1/2)),
   each stage value limited.  READING: after the last stage the damping, the
   torque and the CFL data are taken first (limiting keeps the element means
   the CFL step uses) and the limiter closes the step. */
static int do_step_so(ref_state *s, int fixed, double dtf) {
  double dt = fixed ? dtf : cfl_dt(s, s->u);
  if (!(dt > 0.0) || !isfinite(dt)) return -4;
  const long N = (long)s->ncoef;
  double *k = s->kbuf[0], *u1 = s->kbuf[1], *u2 = s->kbuf[2], *u = s->u;
  op_ctx ctx = {s};
  const double t = s->t;
  rhs_eval(&ctx, t, u, k);
#pragma omp parallel for schedule(static)
  for (long e = 0; e < N; e++) u1[e] = u[e] + dt * k[e];
  limit_apply(s, u1, NULL);
  rhs_eval(&ctx, t + dt, u1, k);
#pragma omp parallel for schedule(static)
  for (long e = 0; e < N; e++) u2[e] = 0.75 * u[e] + 0.25 * (u1[e] + dt * k[e]);
  limit_apply(s, u2, NULL);
  rhs_eval(&ctx, t + 0.5 * dt, u2, k);
#pragma omp parallel for schedule(static)
  for (long e = 0; e < N; e++) u[e] = u[e] / 3.0 + 2.0 / 3.0 * (u2[e] + dt * k[e]);
  damp_apply(s, u, dt);
  torque_eval(s, u, t + dt, &s->torque, &s->torque_abs);
  limit_apply(s, u, NULL);
  s->t += dt;
  s->dt = dt;
  s->step += 1;
  if (!all_finite(s)) return -4;
  return 0;
}

int ref_indicator(ref_state *s, double M, unsigned char *flags) {
  if (!s || !flags || !(M >= 0.0)) return -1;
  tvb_flags(s, s->u, M, flags);
  return 0;
}

int ref_limit(ref_state *s) {
  if (!s) return -1;
  limit_apply(s, s->u, NULL);
  return 0;
}

int ref_limit_flags(ref_state *s, const unsigned char *flags) {
  if (!s || !flags) return -1;
  limit_apply(s, s->u, flags);
  return 0;
}

int ref_step_so(ref_state *s, int n) {
  if (!s || n < 0 || s->d.rk != 3) return -1;
  for (int i = 0; i < n; i++) {
    int rc = do_step_so(s, 0, 0.0);
    if (rc) return rc;
  }
  return 0;
}

int ref_nthreads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* threads of the element loops (results do not depend on it: every element
   writes only itself and the reductions are serial) */
void ref_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int ref_init(ref_state **out, const ref_mesh *mesh, int order, const ref_eos *eos,
             const ref_planet *pl, const ref_disc *disc) {
  if (!out || !mesh || !eos || !pl || !disc) return -1;
  *out = NULL;
  if (order < 1 || order > 4) return -2;
  if (mesh->nx < 1 || mesh->ny < 1 || !(mesh->x1 > mesh->x0) || !(mesh->y1 > mesh->y0)) return -1;
  if (mesh->bc < 0 || mesh->bc > 3) return -1;
  if (eos->kind < 0 || eos->kind > 2) return -2;
  if (eos->kind == 1 && !(eos->gamma > 1.0)) return -1;
  if ((eos->kind == 0 || disc->star || disc->ic == 0 || disc->ic == 3) && !(disc->r_soft > 0.0)) return -1;
  if (disc->ic < 0 || disc->ic > 6) return -2;
  if ((disc->ic == 4 || disc->ic == 5 || disc->ic == 6) && eos->kind != 1) return -1;
  if (disc->ic == 6 && (!disc->star || !(disc->r_soft > 0.0) || !(disc->rdamp_out > 0.0) || !(eos->h > 0.0)))
    return -1;
  if (disc->ic == 3 && (eos->kind != 1 || !(disc->ring_p > 0.0))) return -1;
  if (disc->limiter < 0 || disc->limiter > 1 || disc->positivity < 0 || disc->positivity > 1) return -1;
  if ((disc->limiter || disc->positivity) && disc->rk != 3) return -2;
  if (disc->limiter && !(disc->tvb_m >= 0.0)) return -1;
  tableau T;
  if (get_tableau(disc->rk, &T)) return -2;
  ref_state *s = (ref_state *)calloc(1, sizeof(ref_state));
  if (!s) return -1;
  s->mesh = *mesh;
  s->eos = *eos;
  s->pl = *pl;
  s->d = *disc;
  s->p = order;
  s->m = order + 1;
  s->M = s->m * s->m;
  s->nv = (eos->kind == 1) ? 4 : 3;
  s->dx = (mesh->x1 - mesh->x0) / mesh->nx;
  s->dy = (mesh->y1 - mesh->y0) / mesh->ny;
  ref_gauss_legendre(s->m, s->xg, s->wg);
  double ph[MAXM][MAXM], dph[MAXM][MAXM], pp[MAXM], dpp[MAXM], pm[MAXM], dpm[MAXM];
  for (int q = 0; q < s->m; q++) basis1d(s->p, s->xg[q], ph[q], dph[q]);
  basis1d(s->p, 1.0, pp, dpp);
  basis1d(s->p, -1.0, pm, dpm);
  for (int a = 0; a < s->m; a++)
    for (int b = 0; b < s->m; b++) {
      int k = a * s->m + b;
      for (int q = 0; q < s->m; q++)
        for (int r = 0; r < s->m; r++) {
          int n = q * s->m + r;
          s->Phi[k][n] = ph[q][a] * ph[r][b];
          s->DXm[k][n] = dph[q][a] * ph[r][b];
          s->DYm[k][n] = ph[q][a] * dph[r][b];
        }
      for (int r = 0; r < s->m; r++) {
        s->FxP[k][r] = pp[a] * ph[r][b];
        s->FxM[k][r] = pm[a] * ph[r][b];
        s->FyP[k][r] = ph[r][a] * pp[b];
        s->FyM[k][r] = ph[r][a] * pm[b];
      }
    }
  for (int q = 0; q < s->m; q++)
    for (int r = 0; r < s->m; r++) s->W[q * s->m + r] = 0.25 * s->wg[q] * s->wg[r];
  s->ncoef = (size_t)s->nv * s->M * mesh->nx * mesh->ny;
  s->u = (double *)calloc(s->ncoef, sizeof(double));
  s->tmp = (double *)calloc(s->ncoef, sizeof(double));
  int ok = s->u && s->tmp;
  for (int i = 0; i < T.s; i++) {
    s->kbuf[i] = (double *)calloc(s->ncoef, sizeof(double));
    ok = ok && s->kbuf[i];
  }
  s->glen[0] = s->glen[1] = mesh->ny;
  s->glen[2] = s->glen[3] = mesh->nx;
  for (int side = 0; side < 4; side++) {
    s->ghost[side] = (double *)calloc((size_t)s->nv * s->M * s->glen[side], sizeof(double));
    ok = ok && s->ghost[side];
  }
  if (!ok) {
    ref_destroy(s);
    return -1;
  }
  init_ic(s);
  /* READING: with the limiters on they also act on the projected initial
     data (the adiabatic disc's pressure vanishes at the centre, so its
     projection dips below zero at some nodes) */
  if (s->d.limiter || s->d.positivity) limit_apply(s, s->u, NULL);
  s->t = 0.0;
  s->dt = 0.0;
  s->step = 0;
  *out = s;
  return 0;
}

int ref_destroy(ref_state *s) {
  if (!s) return 0;
  free(s->u);
  free(s->tmp);
  for (int i = 0; i < 6; i++) free(s->kbuf[i]);
  for (int i = 0; i < 4; i++) free(s->ghost[i]);
  free(s);
  return 0;
}

static int all_finite(const ref_state *s) {
  for (size_t e = 0; e < s->ncoef; e++)
    if (!isfinite(s->u[e])) return 0;
  return 1;
}

/* One step of the algorithm of Sec. 3.1: CFL time step from u^n, the RK
   stages (planet at t^n + c_i dt), damping with that dt (Sec. 5.1), then the
   torque on u^{n+1} at t^{n+1} (READING: torque after damping). */
static int do_step(ref_state *s, int fixed, double dtf) {
  double dt = fixed ? dtf : cfl_dt(s, s->u);
  if (!(dt > 0.0) || !isfinite(dt)) return -4;
  tableau T;
  get_tableau(s->d.rk, &T);
  op_ctx ctx = {s};
  rk_butcher(&T, s->ncoef, rhs_eval, &ctx, s->u, s->t, dt, s->kbuf, s->tmp);
  damp_apply(s, s->u, dt);
  torque_eval(s, s->u, s->t + dt, &s->torque, &s->torque_abs);
  s->t += dt;
  s->dt = dt;
  s->step += 1;
  if (!all_finite(s)) return -4;
  return 0;
}

int ref_step(ref_state *s, int n) {
  if (!s || n < 0) return -1;
  const int lim = s->d.limiter || s->d.positivity;
  for (int i = 0; i < n; i++) {
    int rc = lim ? do_step_so(s, 0, 0.0) : do_step(s, 0, 0.0);
    if (rc) return rc;
  }
  return 0;
}

int ref_step_dt(ref_state *s, int n, double dt) {
  if (!s || n < 0 || !(dt > 0.0)) return -1;
  const int lim = s->d.limiter || s->d.positivity;
  for (int i = 0; i < n; i++) {
    int rc = lim ? do_step_so(s, 1, dt) : do_step(s, 1, dt);
    if (rc) return rc;
  }
  return 0;
}

int ref_rhs(ref_state *s, double *out) {
  if (!s || !out) return -1;
  op_ctx ctx = {s};
  rhs_eval(&ctx, s->t, s->u, out);
  return 0;
}

int ref_cfl_dt(ref_state *s, double *dt) {
  if (!s || !dt) return -1;
  *dt = cfl_dt(s, s->u);
  return 0;
}

int ref_damp(ref_state *s, double dt) {
  if (!s || !(dt > 0.0)) return -1;
  damp_apply(s, s->u, dt);
  return 0;
}

int ref_torque(ref_state *s, double *gz, double *abs_sum) {
  if (!s || !gz) return -1;
  *gz = s->torque;
  if (abs_sum) *abs_sum = s->torque_abs;
  return 0;
}

int ref_torque_now(ref_state *s, double t, double *gz, double *abs_sum) {
  if (!s || !gz) return -1;
  double a;
  torque_eval(s, s->u, t, gz, &a);
  if (abs_sum) *abs_sum = a;
  return 0;
}

int ref_fetch(ref_state *s, double *coeffs) {
  if (!s || !coeffs) return -1;
  memcpy(coeffs, s->u, s->ncoef * sizeof(double));
  return 0;
}

int ref_set_state(ref_state *s, const double *coeffs, double t, long step) {
  if (!s || !coeffs) return -1;
  memcpy(s->u, coeffs, s->ncoef * sizeof(double));
  s->t = t;
  s->step = step;
  return 0;
}

int ref_get_time(ref_state *s, double *t, double *dt, long *step) {
  if (!s) return -1;
  if (t) *t = s->t;
  if (dt) *dt = s->dt;
  if (step) *step = s->step;
  return 0;
}

int ref_nodal(ref_state *s, double *out) {
  if (!s || !out) return -1;
  const int nx = s->mesh.nx, ny = s->mesh.ny, M = s->M;
  for (int v = 0; v < s->nv; v++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++)
        for (int n = 0; n < M; n++) {
          double acc = 0.0;
          for (int k = 0; k < M; k++) acc += s->u[cidx(s, v, k, i, j)] * s->Phi[k][n];
          out[(((size_t)v * M + n) * ny + j) * nx + i] = acc;
        }
  return 0;
}

int ref_ghosts(ref_state *s, double *out) {
  if (!s || !out) return -1;
  size_t off = 0;
  for (int side = 0; side < 4; side++) {
    size_t n = (size_t)s->nv * s->M * s->glen[side];
    memcpy(out + off, s->ghost[side], n * sizeof(double));
    off += n;
  }
  return 0;
}

/* Sec. 4.1: L1 = sum_K (1/4) sum_ij |u_h(x_i,y_j) - u(x_i,y_j)| w_i w_j dx dy over the
   (N_p+1)^2 GL nodes, against the exact translated density wave (ic 1). */
int ref_l1_wave(ref_state *s, double t, int var, double *err) {
  if (!s || !err || var < 0 || var >= s->nv) return -1;
  const int nx = s->mesh.nx, ny = s->mesh.ny, m = s->m, M = s->M;
  double lx = s->mesh.x1 - s->mesh.x0, ly = s->mesh.y1 - s->mesh.y0, acc = 0.0;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      double xc = s->mesh.x0 + (i + 0.5) * s->dx, yc = s->mesh.y0 + (j + 0.5) * s->dy;
      for (int n = 0; n < M; n++) {
        int q = n / m, r = n % m;
        double uh = 0.0;
        for (int k = 0; k < M; k++) uh += s->u[cidx(s, var, k, i, j)] * s->Phi[k][n];
        double x = xc + 0.5 * s->dx * s->xg[q], y = yc + 0.5 * s->dy * s->xg[r];
        double ph = TWO_PI * ((x - s->d.vx0 * t - s->mesh.x0) / lx + (y - s->d.vy0 * t - s->mesh.y0) / ly);
        double w[4] = {1.0 + s->d.amp * sin(ph), s->d.vx0, s->d.vy0, 1.0}, ue[4];
        prim_to_cons(s, w, ue);
        acc += 0.25 * fabs(uh - ue[var]) * s->wg[q] * s->wg[r] * s->dx * s->dy;
      }
    }
  *err = acc;
  return 0;
}
