/*
 * dg.h -- C ABI of the GB300 (sm_103a) discontinuous-Galerkin operator for the
 * 2D Euler equations with star + planet gravity on a Cartesian mesh of
 * rectangular elements, tensor-product Legendre modal basis of degree p <= 4
 * (Velasco Romero et al., arXiv:1805.01443).
 *
 * The calls follow the paper's statement of the problem:
 *   dg_init   -- mesh, order, EOS and planet of Sec. 5.1; initial nodes of the
 *                primitive variables -> conserved -> modes (Sec. 3.1 step i,
 *                Eq. 2 first line: L2 projection of the initial data)
 *   dg_step   -- CFL step (Sec. 2.3) + SSP Runge-Kutta stages (Algorithm 1,
 *                Appendix A) of the semi-discrete operator of Eq. 2, damping
 *                zones (Sec. 5.1) and the torque on the planet (Sec. 5.2)
 *   dg_torque -- specific torque Gamma_z on the planet (Sec. 5.2 torque equation)
 *   dg_fetch  -- copy of the modes to the host (Sec. 3.1 step iv)
 *
 * Conventions.
 *   Mode (a, b) of variable v in element (i, j) -- a the degree in x, b in y,
 *   m = p + 1 -- is element [v][a*m + b][j][i] of every canonical coefficient
 *   array (FP64, C order, nv*m*m*ny*nx doubles; nv = 3 for the isothermal
 *   kinds (Sigma, Sigma vx, Sigma vy), 4 for the adiabatic kind (+ E)).
 *   The basis sqrt(2a+1) P_a(xi) sqrt(2b+1) P_b(eta) is orthonormal under the
 *   mean inner product over the element, so mode 0 is the element average
 *   (Sec. 3.1 computes the time step from mode 0 as the average).
 *   Units: G = M_* = 1 (Sec. 5.1).
 *
 * Ownership.  The library owns all device memory of a handle (allocated by
 * dg_init, or carved from a caller-provided workspace by dg_init_ex).  Host
 * buffers passed in are owned by the caller and only read or written during
 * the call.  A handle is not thread safe; distinct handles are independent.
 *
 * Asynchrony.  dg_step/dg_step_dt only enqueue work on the handle's stream and
 * return; errors found on the device (non-finite or non-positive state or time
 * step) are reported by the next synchronising call (dg_torque,
 * dg_torque_series, dg_fetch, dg_get_time, dg_conserved, dg_rhs, dg_sync), and
 * after such an error every later step is a no-op so that the state stays at
 * the last good step.
 *
 * Errors.  Every call returns DG_OK (0) or a negative DG_ERR_* code; a
 * description of the last error of a handle is returned by dg_last_error(h)
 * (or of the last failed call without a handle -- dg_init, dg_batch_*,
 * dg_conserved_static -- of this thread by dg_last_error(NULL)).
 */
#ifndef DG_H
#define DG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DG_OK 0
#define DG_ERR_ARG (-1)         /* invalid argument (null pointer, bad size, bad enum) */
#define DG_ERR_UNSUPPORTED (-2) /* order, EOS, RK scheme or precision not built */
#define DG_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define DG_ERR_NUMERIC (-4)     /* non-finite or non-positive state or time step on the device */
#define DG_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */
#define DG_ERR_NOMEM (-6)       /* device allocation failed or workspace too small */

typedef struct dg_handle dg_handle;

/* Mesh of nx x ny rectangular elements on [x0,x1] x [y0,y1] (Sec. 2.2). */
typedef struct {
  int nx, ny;
  double x0, x1, y0, y1;
  int bc; /* 0 periodic; 1 ghost elements holding the projected background
             state of the initial condition (fixed); 2 transmissive (exterior
             trace = interior trace); 3 zero-gradient ghost elements, each a
             copy of the adjacent boundary element (the "gradient free"
             boundary of Sec. 4.2) */
} dg_mesh;

/* Equation of state (Sec. 2.1). */
typedef struct {
  int kind;     /* 0 locally isothermal, c_s = h v_K(r), 3 variables;
                   1 adiabatic ideal gas p = (gamma - 1) e, 4 variables;
                   2 isothermal with constant c_s = h, 3 variables */
  double gamma; /* adiabatic index (kind 1) */
  double h;     /* disc aspect ratio (kind 0) or sound speed (kind 2) */
} dg_eos;

/* Planet on a fixed circular orbit (Sec. 5.1) with Plummer-softened potential
   Phi_p = -q / sqrt(d^2 + eps^2) (the smoothing of the torque equation, Sec. 5.2). */
typedef struct {
  double q;       /* planet / star mass ratio */
  double r_p;     /* orbital radius */
  double eps;     /* smoothing length (0.6 H in the planet-disc workloads) */
  double omega_p; /* orbital frequency: position r_p (cos, sin)(omega_p t + phi0) */
  double phi0;
  int enabled;    /* 1: planet potential in the gravity source */
} dg_planet;

/* Initial condition, star potential, damping zones and numerics. */
typedef struct {
  int ic;             /* 0 rotational-equilibrium disc Sigma = max(r^slope, floor)
                         (Sec. 5.1 equilibrium with c_s = h v_K); 1 density wave
                         rho = 1 + amp sin(2 pi (x~ + y~)), v = (vx0, vy0), p = 1;
                         2 uniform rho = 1, v = (vx0, vy0), p = 1; 3 the disc of
                         ic 0 (adiabatic only) with pressure x ring_p inside
                         r < ring_r (an imposed shock ring); 4 the isentropic
                         vortex of Sec. 4.1 (strength amp, free stream rho = p = 1,
                         v = (vx0, vy0), centred in the box); 5 the Gresho vortex
                         of Sec. 4.2 (centred in the box); 6 the paper's own
                         disc of Sec. 5.1: Sigma = max(1/(1+f), sigma_floor),
                         p = h^2 Sigma, f = exp((r - r_ex)/h), r_ex =
                         rdamp_out * 1.15^(3/2), rotational equilibrium with
                         solid-body rotation inside r_soft (needs the star and
                         rdamp_out > 0); 4, 5 and 6 adiabatic.  Other values
                         give DG_ERR_UNSUPPORTED. */
  int star;           /* 1: softened point-mass star at the origin in the source;
                         Phi_* = -1/r for r >= r_soft, solid-body core inside */
  double r_soft;      /* star softening radius (> 0 for kind 0, star or ic 0) */
  double sigma_slope; /* disc Sigma ~ r^slope */
  double sigma_floor;
  double noise_amp;   /* additive U(-a, a) noise on Sigma at the projection nodes
                         (SplitMix64 keyed by seed, element and node) */
  unsigned long long seed;
  double rdamp_in;    /* inner damping radius r_d (Sec. 5.1), <= 0 disables */
  double rdamp_out;   /* outer damping radius r_d, <= 0 disables */
  double cfl;         /* Courant number C of Sec. 2.3 */
  int rk;             /* Appendix A: 3 SSP(3,3); 2 SSP(2,2); 4 SSP-RK(4,5) (weights
                         divided by their sum); 5 6-stage Cash-Karp; 4 and 5 in the
                         FP64 form only */
  int prec;           /* 0: FP64 operator.  1: precision form (locally isothermal
                         disc only): FP32 operator on delta = u - u_b about the
                         projected equilibrium u_b, with R_b = L(u_b) evaluated
                         in FP64 once, FP64 torque reduction and sums; delta is
                         held as its values at the Gauss-Legendre nodes and the
                         state is exchanged as FP64 modes u = u_b + delta.
                         2 (3xTF32) and 3 (split-BF16 tensor-core contractions)
                         are not built: DG_ERR_UNSUPPORTED (the nodal form's
                         contractions are ~8 % of a stage's instructions) */
  double amp, vx0, vy0;
  int limiter;        /* troubled-cell limiting after every RK stage (FP64 form,
                         SSP(3,3)): 0 none; 1 the TVB-modified minmod test
                         (Cockburn-Shu) per variable and direction on the linear
                         modes against the differences of the neighbours' means,
                         troubled elements reduced to their mean plus the limited
                         linear modes; 2 the same reduction on the flags of the
                         learned indicator (dg_set_indicator), the TVB test while
                         no network is set */
  double tvb_m;       /* TVB constant M (|slope| <= M h^2 is never limited); 0: minmod */
  int positivity;     /* 1: Zhang-Shu positivity limiter after every stage
                         (Sec. 2.4; density, and pressure for the adiabatic
                         EOS, >= 1e-13 at the volume and face quadrature points),
                         with the time-step factor min(1/(2p+1), w_1/2) */
  double ring_r, ring_p; /* ic 3 ring radius and pressure factor */
} dg_disc;

/* Create a handle: validates the arguments, allocates device memory with
   cudaMalloc on the current device, evaluates the initial condition on the
   device and computes the first CFL step.  Synchronises before returning. */
int dg_init(dg_handle **h, const dg_mesh *mesh, int order, const dg_eos *eos,
            const dg_planet *planet, const dg_disc *disc);

/* Bytes of device workspace that dg_init_ex needs for these arguments. */
int dg_workspace_bytes(const dg_mesh *mesh, int order, const dg_eos *eos, const dg_disc *disc,
                       size_t *bytes);

/* As dg_init, but all device memory of the handle is carved out of the
   caller's device buffer `workspace` (>= dg_workspace_bytes, 256-byte aligned,
   owned by the caller and valid until dg_destroy), and work is issued on
   `stream` (a cudaStream_t, NULL for the legacy default stream).  A workspace
   that is not device memory of the current device is refused with
   DG_ERR_ARG; a smaller one with DG_ERR_NOMEM. */
int dg_init_ex(dg_handle **h, const dg_mesh *mesh, int order, const dg_eos *eos,
               const dg_planet *planet, const dg_disc *disc, void *workspace,
               size_t workspace_bytes, void *stream);

/* Advance n >= 0 full time steps, each with the CFL step of the current state
   (Sec. 2.3), the RK stages with the planet at t^n + c_i dt, damping (Sec. 5.1)
   and the torque on the new state at t^{n+1}.  Asynchronous. */
int dg_step(dg_handle *h, int n);

/* As dg_step with a fixed time step dt > 0 instead of the CFL step. */
int dg_step_dt(dg_handle *h, int n, double dt);

/* Wait for the handle's stream; returns the device status. */
int dg_sync(dg_handle *h);

/* Evaluate the operator L(u^n, t^n) of Eq. 2 (right-hand side divided by |K|)
   into the caller's canonical host array.  Synchronises. */
int dg_rhs(dg_handle *h, double *out);

/* Specific torque Gamma_z (Sec. 5.2) of the last completed step; 0 before the
   first step.  Synchronises. */
int dg_torque(dg_handle *h, double *gamma_z);

/* Per-step torque series since the previous call (at most cap values, oldest
   first; the device keeps the last 65536).  *n receives the count.  Synchronises. */
int dg_torque_series(dg_handle *h, double *out, int cap, int *n);

/* Copy the current modes to the caller's canonical host array.  Synchronises. */
int dg_fetch(dg_handle *h, double *coeffs);

/* Replace the modes (canonical host array), the time and the step counter,
   clear the device status and recompute the CFL step.  Synchronises.
   Page-locked host memory that is mapped into the device's address space
   (cudaHostAlloc, pinned tensors) is read in place by the conversion kernel;
   any other host memory is first copied to a device staging buffer. */
int dg_set_state(dg_handle *h, const double *coeffs, double t, long step);

/* dg_set_state without waiting: queue the replacement of the modes (a
   canonical array in page-locked host memory), the time and the step counter,
   and return.  The copy runs on the handle's own copy stream into one of two
   staging buffers (device memory of the handle, allocated at the first call),
   so it overlaps the work already queued on the handle's stream (the step
   before); the conversion, the status reset and the CFL step follow on the
   handle's stream once the copy has landed.  The host array must stay
   unchanged until the next synchronising call on the handle.  Errors of the
   queued work are reported by the next synchronising call.  DG_ERR_ARG for
   host memory that is not page-locked. */
int dg_set_state_async(dg_handle *h, const double *coeffs, double t, long step);

/* Precision form only (DG_ERR_UNSUPPORTED otherwise): its state is the FP32
   perturbation delta = u - u_b about the projected background u_b, so a caller
   that holds delta can exchange it directly, at half the bytes of the FP64
   state.  Values: delta at the m x m Gauss-Legendre nodes of each element
   (the form's own state; the node (xi_q, eta_r) of the m-point rule at index
   q*m+r), not Legendre modes.  Layout: canonical, FP32, [var][q*m+r][j][i].
   dg_set_delta_async: as dg_set_state_async with u = u_b + delta (the same
   copy stream and staging buffers; page-locked host memory only, unchanged
   until the next synchronising call), except that the conversion and its
   CFL step also overlap the work queued before the call: they run on a
   third stream of the handle into a spare state buffer, which becomes the
   state once that work is done (the first call allocates the stream, the
   spare buffer -- one FP32 state, 78.6 MB at P4 512^2 -- and two small CFL
   slots, released by dg_destroy).  The result is the same, bit for bit.  A
   handle held by a batch converts in place on its own stream instead (the
   batch keeps the addresses of its state buffers).
   dg_fetch_delta: copy the current delta to the caller's host array;
   synchronises. */
int dg_set_delta_async(dg_handle *h, const float *delta, double t, long step);
int dg_fetch_delta(dg_handle *h, float *delta);

/* dg_torque without waiting: queue the copy of the torque of the last step
   queued before it into *gz (page-locked host memory), valid after the next
   synchronising call.  DG_ERR_ARG for memory that is not page-locked. */
int dg_torque_async(dg_handle *h, double *gz);

/* Current time, the time step of the next step, and the step counter. */
int dg_get_time(dg_handle *h, double *t, double *dt, long *step);

/* FP64 sums over the elements of (element average x |K|) for each variable:
   total mass, momentum (and energy).  out has nv doubles.  Synchronises. */
int dg_conserved(dg_handle *h, double *out);

/* Issue later work on `stream` (cudaStream_t; NULL = legacy default stream). */
int dg_set_stream(dg_handle *h, void *stream);

/* Number of variables (3 or 4) and of modes per variable (m*m) of a handle. */
int dg_shape(dg_handle *h, int *nv, int *nmodes, int *nx, int *ny);

/* Static data of the precision form's stage kernel, for its traffic figures:
   the number of 32-element tiles, of tiles that keep the background residual
   R_b (the others hold no coefficient above 1e-10 of max |R_b| and read none),
   and of tiles whose box touches a damping zone (they read the damping
   offsets in the last stage).  DG_ERR_UNSUPPORTED for the FP64 form. */
int dg_prec_tiles(dg_handle *h, long long *ntiles, long long *rb_tiles, long long *zone_tiles);

/* Kernel timing for benchmarks: while enabled, the RK-stage kernel launches of
   the handle are bracketed by pairs of CUDA events recorded on the handle's
   stream (no extra synchronisation): each launch of the FP64 form, the
   back-to-back stage launches of one step of the precision form.  Enabling
   or disabling synchronises and discards earlier records. */
int dg_set_timing(dg_handle *h, int enable);

/* Sum of the recorded stage-kernel durations in milliseconds and the number of
   stage launches they cover since the previous call; synchronises and clears
   the records. */
int dg_timing(dg_handle *h, double *stage_ms, long long *nstage);

/* Largest input of dg_conserved_static, in elements (nx * ny). */
#define DG_STATIC_MAX_ELEMENTS 1048576

/* dg_conserved_static -- the totals of dg_conserved (per variable, the sum over
   the elements of the element average times |K|, in FP64) for a canonical
   coefficient array that the caller already holds in device memory, computed
   without allocating any device memory.  The paper has no counterpart to this
   call: it serves callers that cannot call cudaMalloc when they need the sums,
   such as host codes that reserve all GPU memory for their own pool or arena
   at start-up (a further allocation would fail or break their budget) and
   time-critical loops that must not take the device-wide synchronisation that
   cudaMalloc and cudaFree may cause.
     coeffs  device pointer, FP64, layout [var][mode][ny][nx] (nv*nmodes*ny*nx
             doubles), read only; mode 0 of each variable must be the element
             average, as in every canonical array of this library
     nv      variables (1..4), nmodes modes per variable, nx*ny elements of
             size dx*dy
     out     device pointer to nv doubles, written
     stream  cudaStream_t the two kernels are launched on (NULL: legacy default)
   Its scratch space is a fixed array of 4096 x 4 doubles (128 KiB) inside
   libdg.so; it limits nx*ny to DG_STATIC_MAX_ELEMENTS, and larger inputs return
   DG_ERR_ARG without launching anything.  When CUDA loads modules lazily
   (CUDA_MODULE_LOADING=LAZY, the default of recent CUDA releases), the array
   is committed in a device's memory by the first call made with that device
   current -- that call looks up its device address (cudaGetSymbolAddress),
   which loads this part of the library -- and the GPU then holds it until the
   process exits.  So a caller that reserves all GPU memory for its own pool
   must make one call on each device before it reserves the pool, and that
   first call must also come before any stream capture; later calls allocate
   nothing.  Both pointers are checked before any launch: host memory (pageable
   or page-locked), memory of another device or an address the runtime does not
   know returns DG_ERR_ARG.  All calls share the one array and each call
   overwrites every slot it later reads, so nothing needs clearing between
   calls, but calls whose kernels overlap on the GPU (on different streams or
   from different host threads) race on it and return wrong sums: serialise
   them.  Asynchronous: returns once the kernels are enqueued.  Errors:
   DG_ERR_ARG for a null or non-device pointer, a bad size or no current
   device, DG_ERR_CUDA if the address lookup or a launch fails; the reason is
   in dg_last_error(NULL). */
int dg_conserved_static(const double *coeffs, int nv, int nmodes, int nx, int ny, double dx,
                        double dy, double *out, void *stream);

/* dg_selftest_wait -- a check of the library's bounded device-side waits.  The
   paper has no counterpart.  Every wait of a libdg kernel on something another
   agent completes (a bulk copy landing on an mbarrier, tensor-core MMAs
   committing to one, CTAs of the same persistent launch advancing a counter)
   gives up after a limit, records DG_ERR_TIMEOUT in the handle's status word
   and lets the kernel exit, so a defect cannot hang the GPU.  This call makes
   such a wait run out on purpose: one CTA waits, with the product kernels'
   own wait helper, on something nothing will complete, and reports how it
   ended.
     kind  0: an mbarrier that no copy and no thread arrives on (the stage
              kernel's wait on its damping-offset copy, about 0.3 s);
           1: the same while the CTA holds tensor memory (the tensor-core
              inference kernel's waits), which the CTA frees before it exits;
           2: a counter in global memory that one CTA of a two-CTA cooperative
              launch never advances (the persistent batched kernel's waits
              between stages, 0.5 s).
     freed receives 1 if the CTA freed its tensor memory (kind 1), else 0
           (may be NULL).
   Returns DG_ERR_TIMEOUT when the wait gave up as designed (the expected
   result), DG_OK if it did not, DG_ERR_ARG for another kind and DG_ERR_CUDA
   if a CUDA call failed.  Uses the legacy default stream and synchronises the
   device. */
int dg_selftest_wait(int kind, int *freed);

/* ---- Troubled cells and limiters (FP64 form; DG_ERR_UNSUPPORTED otherwise) --
   The TVB-modified minmod test of Cockburn & Shu, the limited-P1 reduction of
   troubled elements and the positivity limiter of Sec. 2.4 (Zhang & Shu), as
   dg_disc.limiter / tvb_m / positivity describe them.  Flags are one byte per
   element, 1 = troubled, layout [j][i] (nx*ny bytes, caller-owned host
   buffers).  All four synchronise. */

/* Flags of the TVB test with constant M on the current state (state unchanged). */
int dg_indicator(dg_handle *h, double M, unsigned char *flags);

/* The step's limiter (TVB limiting if dg_disc.limiter > 0, then positivity if
   set) applied once to the current state. */
int dg_limit(dg_handle *h);

/* Limited-P1 reduction of the elements flagged in `flags` (from any
   indicator), then positivity if set, on the current state. */
int dg_limit_flags(dg_handle *h, const unsigned char *flags);

/* TVB flags computed by the last limiter pass, i.e. of the last stage value
   before it was limited (the labels of the learned indicator). */
int dg_last_flags(dg_handle *h, unsigned char *flags);

/* ---- Learned troubled-cell indicator ----------------------------------------
   No counterpart in the paper (its only limiter is the positivity limiter of
   Sec. 2.4): a multilayer perceptron nin -> 64 (GELU) -> 64 (GELU) -> 1 logit
   that stands in for the TVB test as the limiter's flagging step
   (dg_disc.limiter = 2), trained on the TVB test's own flags (dg_last_flags).
   BF16 weights (round to nearest even of an FP32 master copy), FP32
   accumulation.  Parameters, flat FP32: W1 [64][nin], b1 [64], W2 [64][64],
   b2 [64], w3 [64], b3.  Loss: mean over the batch of
   w_y (softplus(z) - y z), w_1 = pos_weight, w_0 = 1; Adam (0.9, 0.999, 1e-8).
   Features of an element (nin = 5 nv m^2 FP32): for the stencil element, left,
   right, below and above neighbours (boundary rule for outside elements) and
   each variable v, the modes times 1/S_v, S_v the largest |mode| of v over the
   stencil (1 if all vanish), reciprocal and product in FP64, the product
   rounded once; index (s nv + v) m^2 + k.
   x, y, z and grad pointers marked _dev are device pointers; host pointers are
   caller-owned; `stream` is a cudaStream_t (NULL: legacy default).  The
   network calls synchronise their stream before returning.  A _dev pointer
   that is not device (or managed) memory of the current device is refused
   with DG_ERR_ARG before any launch; the sizes of the buffers behind them
   (B rows of nin, B labels, B logits; n indices, n rows of features) are
   the caller's to guarantee. */
typedef struct dg_mlp dg_mlp;

/* Weights uniform in +-1/sqrt(fan_in) (counter-based SplitMix64 of seed), biases 0. */
int dg_mlp_create(dg_mlp **net, int nin, unsigned long long seed);
int dg_mlp_destroy(dg_mlp *net);
int dg_mlp_nparams(const dg_mlp *net, int *n);
int dg_mlp_get_params(const dg_mlp *net, float *host);
/* Replace the master parameters (and reset Adam). */
int dg_mlp_set_params(dg_mlp *net, const float *host);
/* Logits z_dev[B] of features x_dev[B][nin]. */
int dg_mlp_forward(dg_mlp *net, const float *x_dev, int B, float *z_dev, void *stream);
/* Gradient of the loss w.r.t. the parameters (to grad_host, may be NULL) and the loss. */
int dg_mlp_grad(dg_mlp *net, const float *x_dev, const float *y_dev, int B, float pos_weight,
                float *grad_host, double *loss, void *stream);
/* One Adam step on a batch (labels y_dev[B] in {0, 1}); loss before the step. */
int dg_mlp_train_step(dg_mlp *net, const float *x_dev, const float *y_dev, int B, float pos_weight,
                      float lr, double *loss, void *stream);
/* Features out_dev[n][5 nv m^2] of the elements elems_dev[n] (index j*nx + i)
   of the current state (FP64 form).  Synchronises. */
int dg_features(dg_handle *h, const int *elems_dev, int n, float *out_dev);
/* Hand a copy of the network (BF16) to the handle for limiter 2; flags where
   the logit exceeds threshold.  net = NULL removes it (the TVB test again).
   The handle's inference runs on the tensor cores: activations split into
   BF16 hi + lo against the BF16 weights, FP32 accumulation (logits within
   ~1e-6 of an FP32 evaluation); dg_mlp_forward stays FP32 on the CUDA
   cores.  The weights are packed once here (own device allocation, with
   scratch of 8 nv bytes per element). */
int dg_set_indicator(dg_handle *h, const dg_mlp *net, float threshold);
/* Logits and/or flags ([j][i], host buffers) of the learned indicator on the
   current state.  Synchronises. */
int dg_indicator_logits(dg_handle *h, float *logits, unsigned char *flags);

/* Release the handle and the device memory it allocated. */
int dg_destroy(dg_handle *h);

/* Static description of the last error of h (or of the last failed dg_init
   or dg_batch_* call of this thread for NULL). */
const char *dg_last_error(dg_handle *h);

/* ---- Batched precision form ------------------------------------------------
   Many independent discs (the Sec. 5.1 problem with its own mesh size, degree,
   planet mass and seed each) advanced together on one GPU.  The paper runs one
   disc over many GPUs (Sec. 3.1); it has no batched form.  Two kinds of
   schedule, chosen by dg_batch_config or the autotuner:
   - per-stage launches: each RK stage of every instance is one launch over the
     32-element tiles of all instances (mixed degrees), with persistent CTAs
     that take (instance, tile) work items from a device counter in a tuned
     order (or one CTA per tile); the torque of every instance and its
     end-of-step work (torque sum, time advance, CFL step) are one launch each;
   - the flow schedule: one persistent cooperative launch per step.  Its CTAs
     take work items (runs of up to tiles_per_item tiles of one row) from one
     queue holding every instance's first-stage items, then the second, the
     last, then the torque; an item waits only until the rows it reads (its own
     and the two neighbouring rows) are finished by the stage before, and the
     CTA that finishes an instance's last torque tile does that instance's
     end-of-step work.  Every wait is bounded (one second); one that gives up
     voids the step of its instance, which keeps its state and reports
     DG_ERR_TIMEOUT.
   One step is captured as a CUDA graph and replayed.  Every instance keeps its
   own CFL step, time, torque series and error status, and gives the same
   results as dg_step on its own handle under every schedule (same per-tile
   code, same arithmetic, same order of every sum); after batched steps the
   handles are used as usual (dg_fetch, dg_torque...).

   Requirements: 1 <= n <= DG_BATCH_MAX handles, each created with
   disc.prec = 1 and disc.rk = 3 (locally isothermal), all on the same stream
   and device, each in at most one batch.  The batch keeps pointers to the
   handles, which must outlive it; it owns a CUDA stream, two events, its
   work tables and counters.  Batched work is ordered after everything
   queued on the handles' stream before the call and before everything queued
   there after it.  Errors: DG_ERR_ARG (bad argument), DG_ERR_UNSUPPORTED
   (a handle not in the precision form or not SSP(3,3)), DG_ERR_CUDA,
   DG_ERR_NOMEM; device-side errors of an instance surface on that handle
   (and in dg_batch_sync) as for dg_step. */
#define DG_BATCH_MAX 64
typedef struct dg_batch dg_batch;

int dg_batch_create(dg_batch **b, dg_handle *const *handles, int n);

/* Schedule of the batched steps:
     policy          work order: 0 instances as given, 1 costliest tiles first
                     (highest degree, then largest instance), 2 one tile row of
                     each instance in turn
     dynamic         0: one CTA per tile in each stage launch; 1: persistent
                     CTAs (ctas_per_sm per SM) take items from a counter in
                     each stage launch; 2: the flow schedule (one persistent
                     launch per step), items from a queue counter; 3: the
                     flow schedule with CTA c taking queue positions c,
                     c + G, c + 2G, ... (G CTAs, no counter)
     ctas_per_sm     resident CTAs per SM of the persistent grid (0 or above the
                     occupancy limit: the limit)
     tiles_per_item  1, 2 or 4: tiles (32 elements each) of one row per work
                     item of the flow schedule (ignored by the others)
   Default: policy 1, dynamic 1, the occupancy limit, 1 tile per item. */
int dg_batch_config(dg_batch *b, int policy, int dynamic, int ctas_per_sm, int tiles_per_item);
int dg_batch_get_config(const dg_batch *b, int *policy, int *dynamic, int *ctas_per_sm,
                        int *tiles_per_item);

/* Autotuner: times `steps` batched steps under each schedule (3 work orders x
   {persistent per-stage launches at the occupancy limit and one CTA below it,
   one CTA per tile, the flow schedule with 1, 2 and 4 tiles per item from the
   queue counter and with 1 and 2 in round-robin}), keeps
   the fastest and returns it (any output pointer may be NULL; best_ms is the
   time of one batched step).  The instances are restored afterwards (state,
   time, step count), so tuning does not advance them.  Synchronous. */
int dg_batch_tune(dg_batch *b, int steps, int *policy, int *dynamic, int *ctas_per_sm,
                  int *tiles_per_item, double *best_ms);

/* nsteps SSP(3,3) steps of every instance, each with its own CFL step.
   Asynchronous. */
int dg_batch_step(dg_batch *b, int nsteps);

/* Wait for the batch; DG_OK or the first instance's error code. */
int dg_batch_sync(dg_batch *b);

/* Release the batch (not the handles). */
int dg_batch_destroy(dg_batch *b);

#ifdef __cplusplus
}
#endif
#endif
