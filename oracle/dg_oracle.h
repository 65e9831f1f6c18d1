/*
 * dg_oracle.h -- plain FP64 CPU oracle for the DG spatial operator of
 * Velasco Romero et al. (arXiv:1805.01443), "Planet-disc interactions with
 * Discontinuous Galerkin Methods using GPUs".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file.  It is used by tests/, by __graft_entry__.smoke() and by
 * bench.py's cpu_baseline / reference arm, and it shares no code, header,
 * table or helper with the CUDA path (its structs mirror the product ABI
 * field for field but are declared here independently).
 *
 * What it computes (paper section / equation in brackets):
 *   - Euler equations with gravity source             [Sec. 2.1, Eq. 1]
 *   - tensor-product Legendre modal basis            [Sec. 2.2]
 *   - L2 projection of initial data                   [Sec. 2.2, Eq. 2 first line]
 *   - semi-discrete weak form with GL quadrature      [Sec. 2.2, Eq. 2]
 *   - local Lax-Friedrichs numerical flux             [Sec. 2.2 after Eq. 2; flux type is a reading]
 *   - explicit Runge-Kutta in Butcher form            [Algorithm 1, Appendix A, Tables A1-A5]
 *   - CFL time step from element averages             [Sec. 2.3]
 *   - wave-killing damping zones                      [Sec. 5.1]
 *   - specific torque on the planet                   [Sec. 5.2, torque equation]
 *   - L1 error norm by quadrature                     [Sec. 4.1]
 *
 * Every element-level operation is written as dense per-element matrix
 * products in plain loops (no sum factorisation), in FP64, with reductions
 * in fixed element order.  Compile with -ffp-contract=off so that x86 and
 * Arm hosts give identical arithmetic.
 *
 * Return codes mirror the product's: 0 ok, -1 bad argument, -2 unsupported,
 * -4 numeric failure (non-finite or non-positive time step).
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny;                 /* elements per direction */
  double x0, x1, y0, y1;      /* box */
  int bc;                     /* 0 periodic, 1 fixed background ghosts, 2 transmissive,
                                 3 zero-gradient ghosts (copies of the adjacent element) */
} ref_mesh;

typedef struct {
  int kind;                   /* 0 locally isothermal c_s = h v_K(r); 1 adiabatic; 2 isothermal c_s = h */
  double gamma;               /* adiabatic index (kind 1) */
  double h;                   /* aspect ratio (kind 0) or constant sound speed (kind 2) */
} ref_eos;

typedef struct {
  double q;                   /* planet-to-star mass ratio (G = M_* = 1) */
  double r_p;                 /* orbital radius */
  double eps;                 /* potential smoothing length */
  double omega_p;             /* orbital frequency */
  double phi0;                /* orbital phase at t = 0 */
  int enabled;                /* planet potential in the source term */
} ref_planet;

typedef struct {
  int ic;                     /* 0 Keplerian disc, 1 density wave, 2 uniform state, 3 disc with a pressure ring,
                                 4 isentropic vortex (strength amp), 5 Gresho vortex (adiabatic),
                                 6 the paper's disc of Sec. 5.1 (adiabatic; r_ex from rdamp_out) */
  int star;                   /* 1: softened point-mass star potential in the source */
  double r_soft;              /* star softening radius r_s */
  double sigma_slope;         /* Sigma ~ r^slope */
  double sigma_floor;
  double noise_amp;           /* additive uniform noise amplitude on Sigma at IC nodes */
  unsigned long long seed;
  double rdamp_in, rdamp_out; /* damping radii r_d (<= 0 disables that zone) */
  double cfl;                 /* Courant number C */
  int rk;                     /* 2 SSP(2,2), 3 SSP(3,3), 4 SSP-RK(4,5), 5 Cash-Karp */
  int prec;                   /* ignored by the oracle (always FP64) */
  double amp, vx0, vy0;       /* wave amplitude and uniform velocity (ic 1, 2) */
  int limiter;                /* 0 none; 1 TVB-minmod troubled cells reduced to limited P1 after each stage */
  double tvb_m;               /* TVB constant M of the modified minmod (0: plain minmod) */
  int positivity;             /* 1: Zhang-Shu positivity limiter after each stage (Sec. 2.4) */
  double ring_r, ring_p;      /* ic 3: the disc of ic 0 with pressure x ring_p inside r < ring_r */
} ref_disc;

typedef struct ref_state ref_state;

int  ref_init(ref_state **s, const ref_mesh *mesh, int order, const ref_eos *eos,
              const ref_planet *pl, const ref_disc *disc);
int  ref_destroy(ref_state *s);
int  ref_step(ref_state *s, int n);                      /* n full steps, CFL dt each */
int  ref_step_dt(ref_state *s, int n, double dt);        /* n full steps with a fixed dt */
int  ref_rhs(ref_state *s, double *out);                 /* L(u^n, t^n), canonical layout */
int  ref_cfl_dt(ref_state *s, double *dt);               /* CFL dt of the current state */
int  ref_damp(ref_state *s, double dt);                  /* one damping application */
int  ref_torque(ref_state *s, double *gz, double *abs_sum); /* torque of the last step */
int  ref_torque_now(ref_state *s, double t, double *gz, double *abs_sum);
int  ref_fetch(ref_state *s, double *coeffs);            /* [var][a*m+b][j][i] */
int  ref_set_state(ref_state *s, const double *coeffs, double t, long step);
int  ref_get_time(ref_state *s, double *t, double *dt, long *step);
int  ref_nodal(ref_state *s, double *out);               /* [var][q*m+r][j][i] at GL nodes */
int  ref_l1_wave(ref_state *s, double t, int var, double *err); /* Sec. 4.1 L1 norm vs exact wave */
int  ref_ghosts(ref_state *s, double *out);              /* bc 1 ghost coefficients: [side][var][k][n] */
int  ref_nthreads(void);
void ref_set_threads(int n);
/* troubled-cell flags (1 byte per element, [j][i]) of the current state by the
   TVB-modified minmod test with constant M */
int  ref_indicator(ref_state *s, double M, unsigned char *flags);
/* the limiter of the step (TVB limiting of troubled cells if limiter = 1, then
   positivity if set) applied once to the current state */
int  ref_limit(ref_state *s);
/* limited-P1 reconstruction of the elements flagged in `flags` (then
   positivity if set), for flags from another indicator */
int  ref_limit_flags(ref_state *s, const unsigned char *flags);
/* n SSP(3,3) steps in Shu-Osher form (limiters applied if configured) */
int  ref_step_so(ref_state *s, int n);

/* tables and building blocks exposed for pinning */
int  ref_gauss_legendre(int m, double *x, double *w);
int  ref_legendre(int n, double x, double *P, double *dP);
int  ref_splitmix64_uniform(unsigned long long seed, unsigned long long counter, double *u);
/* one step of tableau `rk` on the 2x2 linear system u' = [[a, -b], [b, a]] u (i.e. u' = lambda u,
   lambda = a + i b) with step dt: returns the amplification factor R(z) applied to (1, 0). */
int  ref_rk_linear(int rk, double a, double b, double dt, double *re, double *im);

#ifdef __cplusplus
}
#endif
#endif
