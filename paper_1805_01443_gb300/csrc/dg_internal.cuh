// dg_internal.cuh -- declarations shared by the CUDA translation units of libdg.
//
// Device data layout ("element-blocked SoA"): elements are grouped in tiles of
// 32 consecutive elements along x (one warp lane per element).  Tile (it, j)
// holds element i = 32*it + lane of row j; inside a tile the layout is
// [var][mode][lane], so the 32 lanes of a warp read one (var, mode) row of 32
// elements as one coalesced 256-byte (FP64) transaction.  A state buffer is
// [j][it][var][mode][32] doubles; lanes past nx in the last tile are padding.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dg.h"

namespace dg {

constexpr int TILE = 32;
constexpr int MAXP = 4;
constexpr int MAXM = MAXP + 1;
constexpr int SERIES_CAP = 65536;

// Device-resident time state of one handle (no host round trip per step).
struct DevState {
  double t;                    // current time t^n
  double dt;                   // CFL step of the current state (next step's dt)
  double torque;               // Gamma_z of the last completed step
  long long step;              // completed steps
  int status;                  // 0 or a DG_ERR_* code; set => every kernel is a no-op
  int pending;                 // error bits of a stage kernel (1 numeric, 2 timeout), promoted by finish
  unsigned long long dt_bits;  // atomicMin slot for the next CFL step (bits of a double > 0)
  long long series_count;      // torque values written to the ring so far
  // precision form: planet position at t^n + c dt for c = 0, 1/2, 1, each
  // coordinate as an unevaluated pair of floats (x hi, x lo, y hi, y lo),
  // the planet at t^{n+1} in FP64, and the step in use rounded to FP32;
  // written once per step so that no stage CTA evaluates FP64 sin/cos
  float plf[3][4];
  double pl1[2];
  float dtf;
};

// Physical parameters shared by all kernels of a handle.
struct Phys {
  int kind;          // EOS kind (dg_eos.kind)
  double gamma;
  double h;          // aspect ratio or constant sound speed
  int star;          // star potential on
  double rs;         // star softening radius
  int planet;        // planet potential on
  double q, eps2;    // planet mass ratio, smoothing^2
  double r_p, omega_p, phi0;
  double rd_in, rd_out;   // damping radii (<= 0: off)
  double damp_ratio;      // 1.15^(3/2)
  int ic;
  double slope, sig_floor, amp, vx0, vy0;
  double cfl;
  double cfl_fac;    // factor of C in the CFL step (1/(2p+1), or the positivity bound)
  int limiter;       // 0 none, 1 TVB test, 2 given flags (learned indicator)
  double tvb_m;
  int positivity;
  double ring_r, ring_p;  // ic 3
};

struct Mesh {
  int nx, ny, ntx, bc;
  double x0, y0, dx, dy, x1, y1;
};

// Arguments of one RK stage launch.
struct StageArgs {
  const double* U;    // u^(s): the state L is evaluated on (tiled)
  const double* Un;   // u^n for the Shu-Osher combination (tiled)
  double* Out;        // output (tiled)
  const double* GL;   // ghosts (bc 1): left/right columns [j][var][mode]
  const double* GR;
  const double* GB;   // bottom/top rows, tiled [it][var][mode][32]
  const double* GT;
  DevState* ts;
  double* part;       // per-CTA torque partials (gx, gy), last stage only
  Mesh mesh;
  Phys phys;
  double alpha, beta; // Out = alpha u^n + beta (u^(s) + dt L(u^(s)))
  double cstage;      // stage time t^n + cstage dt
  double fixed_dt;    // > 0: use instead of ts->dt
  int mode;           // 0: Out = L(U); 1: RK stage; 2: last RK stage (+ damping, torque, CFL)
  // static fields of the locally isothermal disc with the star (null
  // otherwise): at the nodes [tile][3][M][32] c_s^2 and the star's gradient
  // (x, y); at the x-face points [ny][m][nx+1][2] and the y-face points
  // [ny+1][nx][m][2] c_s^2 and c_s
  const double* SN;
  const double* SXF;
  const double* SYF;
};

// Parameters of the precision form (FP32 operator on delta = u - u_b).
struct Prec32 {
  float rs, irs3, h2;      // star softening radius, 1/r_s^3, aspect ratio^2
  float sqk_out, om_in;    // sqrt(1 + (s-1) h^2), sqrt((1 + (s+2) h^2) / r_s^3)
  float slope, sig_floor;
  int slope_half;          // slope == -1/2: Sigma_b = r^-1/2 by rsqrt
  int star, planet;
  float q, eps2;
  float x0p[2], y0p[2], dxp[2], dyp[2];  // x0, y0, dx, dy as (hi, lo) float pairs
  float eps2p[2];          // planet smoothing^2 as a float pair (torque)
  float rd_in, rd_out, damp_ratio;
  float cfl_fac;           // C / (2p + 1)
  // mesh geometry in FP32 (coefficients only; offsets from the planet are
  // formed per CTA in float-float arithmetic from the pairs above)
  float x0, y0, dx, dy, hdx, hdy, s2x, s2y, idx, idy, area;
};

// Arguments of one precision-form stage launch (tiled FP32 arrays).
struct StageArgs32 {
  const float* D;      // delta^(s)
  const float* Dn;     // delta^n
  float* Out;
  const float* Rb;     // R_b = L(u_b), evaluated in FP64, stored FP32 at the nodes [slot][var][node][32]
  const int* RbIdx;    // tile -> its slot in Rb, or -1 (R_b dropped: below 1e-10 of its maximum)
  const float* Db;     // Q0 - Q_b at the nodes for (Sigma, vx, vy) [tile][3][node][32] (damping)
  const float* Bm0;    // element averages of u_b [tile][3][32] (CFL)
  const float* Bmodes; // u_b at the nodes in FP32 [tile][var][node][32] (exact-background tiles)
  const int* TileFlag; // 1: the tile uses the exact projected background
  const int* TileOrder;  // last stage: CTA -> tile (tiles that touch a damping zone first), or null
  DevState* ts;
  double* part;
  Mesh mesh;
  Prec32 pc;
  int pidx;            // stage time t^n + c dt: DevState::plf row (c = 0, 1/2, 1 -> 0, 1, 2)
  float alpha, beta;
  int mode;
};

// Constant tables of the m-point Gauss-Legendre rule for degree p.
struct Tables {
  double phi[MAXM][MAXM];   // [q][a] = sqrt(2a+1) P_a(xi_q)
  double dphi[MAXM][MAXM];  // [q][a] = d/dxi of the above
  double wh[MAXM];          // w_q / 2 (weights normalised to sum 1 on [-1,1])
  double pp[MAXM];          // sqrt(2a+1) P_a(+1)
  double pm[MAXM];          // sqrt(2a+1) P_a(-1)
  double xi[MAXM];          // nodes
};

// per-order entry points (dg_stage_p{1..4}.cu)
#define DG_DECLARE_ORDER(P)                                                        \
  cudaError_t launch_stage_p##P(const StageArgs& a, cudaStream_t s);              \
  cudaError_t upload_tables_p##P(const Tables& t);                                 \
  size_t stage_smem_p##P(int kind);                                                \
  cudaError_t launch_stage32_p##P(const StageArgs32& a, cudaStream_t s);          \
  cudaError_t launch_torque32_p##P(const float* D, const float* SigbN, const DevState* ts, double* part, \
                                   const Mesh& ms, const Prec32& pc, cudaStream_t s);               \
  cudaError_t upload_tables32_p##P(const Tables& t);                               \
  cudaError_t launch_static_p##P(const Mesh& ms, const Phys& ph, double* SN, double* SXF, double* SYF, \
                                 cudaStream_t s);
DG_DECLARE_ORDER(1)
DG_DECLARE_ORDER(2)
DG_DECLARE_ORDER(3)
DG_DECLARE_ORDER(4)
#undef DG_DECLARE_ORDER

// auxiliary kernels (dg_aux.cu)
struct InitArgs {
  double* out;       // target buffer
  int target;        // 0 interior (tiled), 1 left ghosts, 2 right, 3 bottom (tiled), 4 top (tiled)
  int p, nv;
  Mesh mesh;
  Phys phys;
  unsigned long long seed;
  double noise_amp;
  double xq[MAXM + 1], wq[MAXM + 1];   // (m+1)-point GL rule
  double phq[MAXM + 1][MAXM];          // basis at those nodes
};

cudaError_t launch_init(const InitArgs& a, int count, cudaStream_t s);
// CFL step from the element averages of U, or of U + D (D: the precision
// form's FP32 delta at the nodes, averaged with the weights wn[q*m + r] =
// (w_q/2)(w_r/2); may be null)
cudaError_t launch_cfl(const double* U, const float* D, const double* wn, DevState* ts, const Mesh& mesh,
                       const Phys& phys, int p, int nv, cudaStream_t s);
cudaError_t launch_finish(DevState* ts, const double* part, int nparts, double* series,
                          double fixed_dt, int advance, int planet32, double r_p, double omega_p,
                          double phi0, cudaStream_t s);
// canonical modes -> tiled FP64 state; canon may be mapped page-locked host memory
cudaError_t launch_ingest(const double* canon, double* tiled, const Mesh& mesh, int nv, int M, cudaStream_t s);
cudaError_t launch_to_canon(const double* tiled, double* canon, const Mesh& mesh, int nv, int M,
                            cudaStream_t s);
// precision form (locally isothermal, 3 variables): canonical FP32 delta
// (values at the nodes) -> tiled delta d, with the CFL minimum of U + d (U:
// tiled FP64 u_b; wn: the node weights) folded into *dt_bits (atomic minimum
// of the bits of a double > 0) and a non-finite or non-positive state into
// *pending (bit 0) in the same pass, as launch_cfl would
cudaError_t launch_ingest_delta_cfl(const float* canon, float* d, const double* U, const double* wn,
                                   unsigned long long* dt_bits, int* pending, const Mesh& mesh, const Phys& phys,
                                   int M, cudaStream_t s);
// The CFL slot of an upload converted on its own stream, apart from the time
// state that steps still in flight read and write.
struct UpSlot {
  unsigned long long dt_bits;  // +inf bits when empty
  int pending;                 // 0 when empty
  int pad;
};
// Make the converted upload the handle's state: the time state as
// launch_reset_state(t, step) leaves it, then the step's dt (or the error
// status) from the slot, which is emptied for the upload after next.
cudaError_t launch_adopt_upload(DevState* ts, UpSlot* up, double t, long long step, cudaStream_t s);
cudaError_t launch_to_canon_f32(const float* tiled, float* canon, const Mesh& mesh, int nv, int M,
                                cudaStream_t s);
cudaError_t launch_conserved(const double* U, double* part, double* out, const Mesh& mesh, int nv,
                             int M, cudaStream_t s);
cudaError_t launch_reset_state(DevState* ts, double t, long long step, cudaStream_t s);
// out = u0 + dt sum_{j<nk} c_j k_j + cx X over n doubles (nk <= 5, X may be null)
cudaError_t launch_combine(double* out, const double* u0, const double* const* k, const double* c, int nk,
                           const double* X, double cx, size_t n, const DevState* ts, double fixed_dt,
                           cudaStream_t s);
// planet positions and FP32 step of the precision form for the current t and
// step (fixed_dt > 0 replaces the CFL step)
cudaError_t launch_planet32(DevState* ts, double fixed_dt, double r_p, double omega_p, double phi0,
                            cudaStream_t s);

// troubled-cell indicator and limiters of the FP64 form, in place (dg_limit.cu):
// tvb runs the TVB test (flags to tvb_out if given), `given` replaces its flags
// for the limiting, apply = 0 only writes the flags
cudaError_t launch_limit(double* U, const double* GL, const double* GR, const double* GB, const double* GT,
                         const unsigned char* given, unsigned char* tvb_out, const DevState* ts,
                         const Mesh& ms, const Phys& ph, const Tables& tab, int p, int nv, int tvb,
                         int apply, int positivity, cudaStream_t s);

// ---- learned troubled-cell indicator (dg_mlp.cu) ----------------------------
constexpr int MLP_HIDDEN = 64;

// device buffers of one network and its training scratch (batch <= cap)
struct MlpBufs {
  int nin;
  float* p;   // FP32 master parameters (flat)
  float* m;   // Adam moments
  float* v;
  void* pb;   // BF16 copy of p
  float* g;   // gradient
  int cap;
  float *a1, *h1, *a2, *h2, *z, *dz, *d2, *d1;  // [cap][64] (z, dz: [cap])
  double* lossb;  // [cap]
};
int mlp_nparams(int nin);
cudaError_t mlp_sync_bf16(MlpBufs& b, cudaStream_t s);
cudaError_t mlp_forward(MlpBufs& b, const float* x, int B, float* zout, cudaStream_t s);
cudaError_t mlp_backward(MlpBufs& b, const float* x, const float* y, int B, float pos_weight, double* loss_sum,
                         cudaStream_t s);
cudaError_t mlp_adam(MlpBufs& b, int t, float lr, cudaStream_t s);
// features (FP32 [n][5 nv M]) of the listed elements j*nx+i of a tiled FP64 state
cudaError_t launch_features(const double* U, const double* GL, const double* GR, const double* GB,
                            const double* GT, const Mesh& ms, int p, int nv, const int* elems, int n, float* out,
                            cudaStream_t s);
// flags (logit > threshold) and optionally logits of every element, on the
// tensor cores; wpack holds the weights in the layout mlp_pack writes, work
// is scratch of mlp_work_bytes (per-element maxima of |c| and the
// coefficients as BF16 pairs, the stencil scales)
cudaError_t launch_mlp_flags(const double* U, const double* GL, const double* GR, const double* GB,
                             const double* GT, const Mesh& ms, int p, int nv, const void* wpack, void* work,
                             float threshold, DevState* ts, unsigned char* flags, float* logits, cudaStream_t s);
size_t mlp_work_bytes(const Mesh& ms, int nv, int M);
// host: the flat FP32 parameters as the inference kernel's operands (W1 in
// 64-input chunks and W2 as BF16 tensor-core tiles, then b1, b2, w3, b3 as the
// FP32 values of their BF16 roundings)
size_t mlp_pack_bytes(int nv, int M);
void mlp_pack(const float* prm, int nv, int M, unsigned char* out);

// precision-form setup and conversions (dg_prec.cu)
// tiled (or, with canon, canonical) FP64 modes minus sub (tiled FP64, may be
// null) -> tiled FP32 values at the Gauss-Legendre nodes, the transform in
// FP64 (fp64 set) or FP32
cudaError_t launch_to_nodal32(const double* src, int canon, const double* sub, float* dst, const Mesh& mesh,
                              const Tables& tab, int p, int nv, int fp64, cudaStream_t s);
// tiled FP32 nodal values -> tiled FP64 modes (+ add, tiled FP64 modes, may be null)
cudaError_t launch_to_modal64(const float* src, const double* add, double* dst, const Mesh& mesh,
                              const Tables& tab, int p, int nv, cudaStream_t s);
cudaError_t launch_bg_nodes(const double* bg, float* sigbn, float* db, float* bm0, float* disc,
                            const Mesh& mesh, const Phys& phys, const Tables& tab, int p,
                            cudaStream_t s);
cudaError_t launch_tile_flags(const float* disc, int* flags, const Mesh& mesh, float threshold,
                              cudaStream_t s);

// ---- batched precision form (dg_batch.cu) ----------------------------------
// Many independent discs advanced together: every launch covers the tiles of
// all instances (mixed degrees), and the ping-pong state of each instance is
// chosen on the device from the parity of its step counter, so the launch
// arguments do not change from step to step and one captured step replays.
constexpr int BATCH_MAX = 64;

struct BatchInst32 {
  StageArgs32 a;        // per-instance arguments (D, Dn, Out, alpha, beta, pidx, mode unused)
  float* buf[2];        // delta^n / delta^{n+1} by step parity
  float* DZ;            // stage scratch
  const float* SigbN;   // Sigma_b node pairs (torque)
  double* series;       // torque ring of the instance
  double r_p, omega_p, phi0;
  long long step0;      // step count at which buf[cur0] held the state
  int cur0, p, nparts;
};

// One persistent launch per step (the flow schedule): CTAs take work items
// from one queue -- every stage-1 item, then every stage-2 item, every
// stage-3 item, then the torque groups -- and an item waits, with a bounded
// spin, only for the tile rows it reads to be finished by the stage before.
// The counters live in one int array that is cleared before every step.
struct BatchFlow32 {
  int* ctr;             // [0] queue, [1] abort flag, [2] CTAs done, [FLOW_TQ + k] torque
                        // tiles done of instance k, [FLOW_ROWS + 3 r + s] tiles of global row
                        // r finished by stage s
  const int2* items;    // stage work items {(instance << 25) | first tile, tiles}, stages 1-2 order
  const int2* last;     // the same for the last stage
  const int* tq;        // torque groups: (instance << 25) | first tile (3 tiles, one per warp)
  int nq;               // stage work items of stages 1 and 2
  int nql;              // stage work items of the last stage
  int ntq;              // torque groups
  unsigned long long limit_ns;  // bound of one wait
  int rr;               // 1: CTA c takes positions c, c + G, c + 2G, ... (no queue counter)
  int rowbase[BATCH_MAX + 1];   // first global row of each instance
};
constexpr int FLOW_TQ = 4;
constexpr int FLOW_ROWS = FLOW_TQ + BATCH_MAX;

struct BatchLaunch32 {
  int n;                // instances
  int nitems;           // tiles over all instances
  int stage;            // SSP(3,3) stage 0, 1, 2
  int dynamic;          // 1: persistent CTAs take items from *counter; 0: one item per CTA
  int* counter;         // work counter of this stage (reset every step)
  const int* items;     // work order: (instance << 25) | tile
  int tile0[BATCH_MAX + 1];  // prefix sums of the instances' tile counts
  BatchFlow32 flow;
  BatchInst32 inst[BATCH_MAX];
};

// tables of every degree used by the batch (tabs[p], p = 1..4, or null)
cudaError_t batch_upload_tables32(const Tables* const* tabs);
size_t batch_stage32_smem();
int batch_stage32_ctas_per_sm();
cudaError_t launch_batch_stage32(const BatchLaunch32& L, int grid, cudaStream_t s);
cudaError_t launch_batch_torque32(const BatchLaunch32& L, cudaStream_t s);
cudaError_t launch_batch_finish(const BatchLaunch32& L, cudaStream_t s);
cudaError_t launch_batch_planet32(const BatchLaunch32& L, cudaStream_t s);
// the flow schedule: one cooperative launch of `grid` CTAs per step
int batch_flow_ctas_per_sm();
cudaError_t launch_batch_flow32(const BatchLaunch32& L, int grid, cudaStream_t s);

// Record msg as this thread's last error (dg_last_error(NULL)); returns code.
int set_thread_error(int code, const char* msg);

}  // namespace dg
