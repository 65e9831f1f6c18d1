// dg_stage32.cuh -- precision form of the fused RK-stage kernel: FP32
// operator on the perturbation delta = u - u_b of the locally isothermal disc
// about its projected rotational equilibrium u_b (the Keplerian background).
//
// L(u) = R_b + [L(u_b + delta) - L(u_b)], where R_b = L(u_b) is evaluated once
// in FP64 (the FP64 stage kernel) and stored; the bracket is evaluated here in
// FP32 from flux, source and Riemann-flux DIFFERENCES written so that the
// background only enters as a multiplicative coefficient of delta terms:
//   m v - m_b v_b   = dm v + m_b dv,   dv = (dm - v_b dSigma) / Sigma
//   p - p_b         = c_s^2 dSigma
//   S - S_b         = -dSigma grad Phi_* - Sigma grad Phi_p
//   h(uL,uR) - h_b  = (df_L + df_R)/2 - [alpha (dR - dL) + (alpha - alpha_b)(uR_b - uL_b)]/2
// The background coefficients come from the analytic equilibrium at the point,
// except in tiles flagged at set-up (the singular centre Sigma ~ r^-1/2 and the
// solid-body-core edge, where the analytic and projected backgrounds differ;
// the box edge under periodic or copied-element boundaries, where the
// neighbour's background is its own projection), where the projected one is
// interpolated from its FP32 values at the nodes.
//
// Nodal form.  delta, R_b and the projected background are held as the
// values of their polynomials at the m x m Gauss-Legendre nodes of each
// element, not as Legendre modes.  With the m-point rule the two are the
// same discrete operator (Eq. 2 with the quadrature of the modal scheme): the
// modal basis is orthonormal on the rule, so the map from modes to node values
// is inverted by its transpose times the weights, and the operator's modal
// result mapped to the nodes is the DG weak form in the Lagrange basis of
// the nodes -- volume terms by the weak derivative dw along each node line,
// source terms at the node itself, face traces and the lift by the Lagrange
// values at the element ends.  So no stage contracts modes to nodes, the
// volume sums cost m FMAs per node and direction instead of 2m per mode,
// and damping acts on the node values directly.  The modes appear only where
// the state crosses the library boundary (dg_prec.cu).
//
// Work decomposition: one CTA per 32-element tile of one mesh row, three warps;
// thread (v, e) owns variable v of element e.  Its node values and
// volume/lift accumulators stay in registers; shared memory only exchanges
// the node values, face traces, pointwise fluxes and face fluxes between the
// three variable threads of an element.  Pointwise and face work is dealt
// round-robin over the three threads.  Independent evaluations that share
// their operation sequence (two quadrature nodes, the two sides of a face, two
// node lines of a sum) run as the lanes of packed FP32x2 instructions, each
// lane in its scalar order.  The last stage adds damping in delta form (tiles
// that touch a zone, scheduled first so that an SM holds CTAs on one code
// path) and the CFL minimum; the torque of the new state is a separate
// one-variable pass (k_torque32 below).
#pragma once
#include "dg_async.cuh"
#include "dg_internal.cuh"


namespace dg {

// FP32 tables of degree P for the nodal form (the m-point Gauss-Legendre
// rule and the Lagrange basis l_q of its nodes), one slice per degree so that
// one translation unit can hold kernels of several degrees.  The state of the
// precision form is the polynomial's values at the m x m nodes; with the
// mean-orthonormal modal basis phi_a and weights w_q/2 the two forms are
// related by sum_a phi_a(xi_q) phi_a(xi) = l_q(xi) / (w_q/2), so that
//   weak derivative  dw[q][q'] = (w_q'/2) l_q'(xi_q') / (w_q/2)
//                              = (w_q'/2) sum_a phi_a(xi_q) phi'_a(xi_q'),
//   lift at an end   lp[q] = l_q(+1) / (w_q/2) = sum_a phi_a(xi_q) phi_a(+1)
//   (lm at -1), and traces at an end  bp[q] = l_q(+1), bm[q] = l_q(-1).
struct Tab32 {
  float xi[MAXM], wh[MAXM];
  float bp[MAXM], bm[MAXM];  // l_q(+1), l_q(-1)
  float2 bpm2[MAXM];         // (bp, bm): the two traces of a node line as the lanes of packed FMAs
  float dw[MAXM][MAXM];      // weak derivative [q][q']
  float lp[MAXM], lm[MAXM];  // lift at +1 (its negative enters) and at -1
  float eye[MAXM][MAXM];     // unit vectors: point values of exact-background tiles at a node line
  // operand pairs of the packed volume/lift sums over node pairs (2k, 2k+1);
  // the pair past an odd m has zero coefficients
  float2 dwp[(MAXM + 1) / 2][MAXM];  // (dw[2k][q'], dw[2k+1][q'])
  float2 lmp[(MAXM + 1) / 2], lpn[(MAXM + 1) / 2];  // (lm[2k], lm[2k+1]), (-lp[2k], -lp[2k+1])
  float2 dw2[MAXM][MAXM], lm2[MAXM], lpn2[MAXM];     // (dw, dw), (lm, lm), (-lp, -lp): one entry, both lanes
  // low parts of the FP64 tables as float pairs (float-float torque)
  float xil[MAXM];
  float w2h[MAXM * MAXM], w2l[MAXM * MAXM];  // [q*m + r] (w_q/2)(w_r/2)
};
static __constant__ Tab32 c32t[MAXP + 1];

// Analytic background of the disc and the isothermal sound speed at (x, y).
struct Bg32 {
  float sig, vx, vy, mx, my, c2;
};

// The background enters only as coefficients of perturbation terms, so the
// hardware approximations (a few ulp) of reciprocal and square root serve; the
// correctly rounded library forms run partly on this part's narrow FP64 unit.
// Products that may meet a sum are written as explicitly rounded products, so
// that no code generator fuses them into an FMA in one kernel and not in
// another (the single-disc and batched kernels round alike).
__device__ __forceinline__ float sqrt_fast(float x) { return __fmul_rn(x, rsqrtf(x)); }

__device__ __forceinline__ Bg32 bg32_at(const Prec32& pc, float x, float y) {
  Bg32 b;
  const float r2 = fmaxf(fmaf(x, x, __fmul_rn(y, y)), 1e-24f);  // r >= 1e-12: a node at the origin
  const float ir = rsqrtf(r2);
  const float r = __fmul_rn(r2, ir);
  const float sir = sqrt_fast(ir);  // r^-1/2
  float sig = pc.slope_half ? sir : exp2f(__fmul_rn(pc.slope, __log2f(r)));
  sig = fmaxf(sig, pc.sig_floor);
  float om, vk2;
  if (r >= pc.rs) {
    om = __fmul_rn(__fmul_rn(pc.sqk_out, ir), sir);  // v_phi / r = sqrt((1 + (s-1) h^2) / r) / r
    vk2 = ir;
  } else {
    om = pc.om_in;                     // solid-body core
    vk2 = __fmul_rn(r2, pc.irs3);
  }
  b.sig = sig;
  b.vx = __fmul_rn(-om, y);
  b.vy = __fmul_rn(om, x);
  b.mx = __fmul_rn(sig, b.vx);
  b.my = __fmul_rn(sig, b.vy);
  b.c2 = __fmul_rn(pc.h2, vk2);
  return b;
}

// ---- two evaluations at once: the lanes of packed FP32x2 instructions ------
__device__ __forceinline__ float2 m2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 a2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 d2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 n2(float2 a) { return make_float2(-a.x, -a.y); }

struct Bg32x2 {
  float2 sig, vx, vy, mx, my, c2;
};
__device__ __forceinline__ Bg32x2 bg32_at2(const Prec32& pc, float2 x, float2 y, float2& r2, float2& ir) {
  Bg32x2 b;
  r2 = f2(x, x, m2(y, y));
  r2 = make_float2(fmaxf(r2.x, 1e-24f), fmaxf(r2.y, 1e-24f));  // r >= 1e-12: a node at the origin
  ir = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
  const float2 r = m2(r2, ir);
  const float2 sir = m2(ir, make_float2(rsqrtf(ir.x), rsqrtf(ir.y)));  // r^-1/2
  float2 sig = sir;
  if (!pc.slope_half)
    sig = make_float2(exp2f(pc.slope * __log2f(r.x)), exp2f(pc.slope * __log2f(r.y)));
  sig = make_float2(fmaxf(sig.x, pc.sig_floor), fmaxf(sig.y, pc.sig_floor));
  const float2 omA = m2(m2(d2(pc.sqk_out), ir), sir), vkB = m2(r2, d2(pc.irs3));
  const float2 om = make_float2(r.x >= pc.rs ? omA.x : pc.om_in, r.y >= pc.rs ? omA.y : pc.om_in);
  const float2 vk2 = make_float2(r.x >= pc.rs ? ir.x : vkB.x, r.y >= pc.rs ? ir.y : vkB.y);
  b.sig = sig;
  b.vx = m2(n2(om), y);
  b.vy = m2(om, x);
  b.mx = m2(sig, b.vx);
  b.my = m2(sig, b.vy);
  b.c2 = m2(d2(pc.h2), vk2);
  return b;
}
// flux differences f(u_b + d) - f(u_b) (isothermal, 3 variables) at two points
__device__ __forceinline__ void dflux32x2(const Bg32x2& b, const float2* d, float2* fx, float2* fy, float2& vx,
                                          float2& vy) {
  const float2 sg = a2(b.sig, d[0]);
  const float2 is = make_float2(__fdividef(1.0f, sg.x), __fdividef(1.0f, sg.y));
  const float2 dvx = m2(f2(n2(b.vx), d[0], d[1]), is);
  const float2 dvy = m2(f2(n2(b.vy), d[0], d[2]), is);
  vx = a2(b.vx, dvx);
  vy = a2(b.vy, dvy);
  const float2 dp = m2(b.c2, d[0]);
  fx[0] = d[1];
  fx[1] = f2(d[1], vx, f2(b.mx, dvx, dp));
  fx[2] = f2(d[2], vx, m2(b.my, dvx));
  fy[0] = d[2];
  fy[1] = f2(d[1], vy, m2(b.mx, dvy));
  fy[2] = f2(d[2], vy, f2(b.my, dvy, dp));
}

// LLF flux difference through a face with normal +DIR, with background traces
// bL, bR on the two sides (equal for the analytic background); the flux
// differences of the two sides are the lanes of one packed pass.
template <int DIR>
__device__ __forceinline__ void dllf32(const Bg32& bL, const Bg32& bR, const float* dL,
                                       const float* dR, float* h) {
  Bg32x2 b;
  b.sig = make_float2(bL.sig, bR.sig);
  b.vx = make_float2(bL.vx, bR.vx);
  b.vy = make_float2(bL.vy, bR.vy);
  b.mx = make_float2(bL.mx, bR.mx);
  b.my = make_float2(bL.my, bR.my);
  b.c2 = make_float2(bL.c2, bR.c2);
  const float2 d[3] = {make_float2(dL[0], dR[0]), make_float2(dL[1], dR[1]), make_float2(dL[2], dR[2])};
  float2 fx[3], fy[3], vx, vy;
  dflux32x2(b, d, fx, fy, vx, vy);
  const float2* fn = DIR == 0 ? fx : fy;
  const float2 vn = DIR == 0 ? vx : vy;
  const float c = sqrt_fast(bL.c2);
  const float al = fmaxf(fabsf(vn.x), fabsf(vn.y)) + c;
  const float alb = fmaxf(fabsf(DIR == 0 ? bL.vx : bL.vy), fabsf(DIR == 0 ? bR.vx : bR.vy)) + c;
  const float jb[3] = {bR.sig - bL.sig, bR.mx - bL.mx, bR.my - bL.my};
#pragma unroll
  for (int v = 0; v < 3; v++)
    h[v] = fmaf(0.5f, __fadd_rn(fn[v].x, fn[v].y), __fmul_rn(-0.5f, fmaf(al, dR[v] - dL[v], __fmul_rn(al - alb, jb[v]))));
}

// Exact projected background at a point of one element from its FP32 values
// at the nodes (stride 32 between nodes): u_b = sum_qr b(q, r) fa[q] gb[r],
// with fa, gb the Lagrange weights of the point along each node line (a unit
// vector at a node, bp or bm at an element end); c2 from the analytic sound
// speed of the point.
template <int P>
__device__ __noinline__ Bg32 bg32_poly(const float* bm, const float* fa, const float* gb, float c2) {
  constexpr int m = P + 1, M = m * m;
  float u[3];
#pragma unroll
  for (int v = 0; v < 3; v++) {
    float acc = 0.0f;
#pragma unroll
    for (int aa = 0; aa < m; aa++) {
      float t = 0.0f;
#pragma unroll
      for (int b = 0; b < m; b++) t = fmaf(bm[(v * M + aa * m + b) * 32], gb[b], t);
      acc = fmaf(fa[aa], t, acc);
    }
    u[v] = acc;
  }
  Bg32 r;
  r.sig = u[0];
  r.mx = u[1];
  r.my = u[2];
  r.vx = u[1] / u[0];
  r.vy = u[2] / u[0];
  r.c2 = c2;
  return r;
}

// Shared-memory plan (floats) of the precision-form stage kernel.  The face
// fluxes are formed before the pointwise terms, so the traces that are dead
// once the fluxes exist (own y traces, left x traces) sit in the planes of
// the pointwise terms that are written after them: 32.0 KB at P4, seven CTAs
// per SM.
template <int P>
struct Smem32 {
  static constexpr int m = P + 1, M = m * m;
  // nodal values [3][M][32]; the pointwise terms of the momentum rows fx1,
  // fx2 (times 2/dx), fy1, fy2 (times 2/dy) and the sources src1, src2,
  // [6][M][32], overwrite them in place (planes 0-2 alias U: each node's
  // values are read and replaced by the one thread that owns the node).  The
  // density's fluxes are the momentum perturbations themselves, which its
  // thread reads from the state in global memory, so they need no plane.
  static constexpr int U = 0;
  static constexpr int F = 0;
  static constexpr int PFX = 0;                    // planes of fx_v, fy_v, src_v for v = 1, 2: PFX + v - 1, ...
  static constexpr int PFY = 2;
  static constexpr int PSRC = 4;
  static constexpr int YT = F + 3 * M * 32;        // own y traces [2][3][m][32]: 0 top, 1 bottom (in planes 3..)
  static constexpr int XL = YT + 2 * 3 * m * 32;   // left x traces [3][m][33], slot e (in planes 3..)
  static constexpr int XR0 = F + 6 * M * 32;
  static constexpr int XR = XL + 3 * m * 33 > XR0 ? XL + 3 * m * 33 : XR0;  // right x traces [3][m][33], slot e+1
  static constexpr int YN = XR + 3 * m * 33;       // neighbour traces [2][3][m][32]: 0 below's top, 1 above's bottom
  // face fluxes (times 1/dx, 1/dy) overwrite the traces they are formed from
  // (each face point's traces are read and replaced by the one thread that
  // owns the point):
  static constexpr int FX = XR;                    // x-face flux differences [3][m][33]
  static constexpr int FY = YN;                    // y-face flux differences [2][3][m][32]
  static constexpr int B0 = YN + 2 * 3 * m * 32;   // element averages of the new state [3][32]
  static constexpr int FLAGS = B0 + 3 * 32;        // 32 ints
  static constexpr int TOTAL = FLAGS + 32;
  static constexpr int ND = 8;                     // 8-byte words: offsets, dt, mbarrier
  static constexpr size_t BYTES = (size_t)ND * sizeof(double) + (size_t)TOTAL * sizeof(float);
  static_assert(F + 6 * M * 32 <= XR, "damping offsets (planes 3-5) overlap the x traces");
};

// exact int -> float for 0 <= x < 2^23 on the integer and FP32 pipes (this
// part executes conversion instructions on its narrow FP64 unit)
__device__ __forceinline__ float i2f(int x) { return __int_as_float(0x4B000000 | x) - 8388608.0f; }

// ---- float-float ("double-float") arithmetic on the FP32 pipe --------------
// The _rn intrinsics are never contracted into FMAs, which the error-free
// transformations below rely on.

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// an unevaluated pair h + l with |l| <= ulp(h)/2 (~2^-46 relative)
struct F2 {
  float h, l;
};
__device__ __forceinline__ F2 f2_norm(float s, float e) {  // |e| small against s
  F2 r;
  r.h = __fadd_rn(s, e);
  r.l = __fsub_rn(e, __fsub_rn(r.h, s));
  return r;
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return f2_norm(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {  // exact product of the heads by an FMA
  const float p = __fmul_rn(a.h, b.h);
  const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)));
  return f2_norm(p, e);
}
__device__ __forceinline__ F2 f2_mulf(F2 a, float b) {
  const float p = __fmul_rn(a.h, b);
  const float e = fmaf(a.l, b, fmaf(a.h, b, -p));
  return f2_norm(p, e);
}
// 1/sqrt(d), d > 0: one Newton step y (1 + r/2), r = 1 - d y^2 formed in
// float-float, from the hardware estimate (error ~ (3/2) eps0^2 ~ 2^-44)
__device__ __forceinline__ F2 f2_rsqrt(F2 d) {
  const float y = rsqrtf(d.h);
  F2 y2;
  y2.h = __fmul_rn(y, y);
  y2.l = fmaf(y, y, -y2.h);
  const F2 t = f2_mul(d, y2);
  const float r = __fsub_rn(__fsub_rn(1.0f, t.h), t.l);  // 1 - t.h exact: t.h within [1/2, 2]
  return f2_norm(y, __fmul_rn(__fmul_rn(0.5f, y), r));
}

// Unnormalised forms for the torque sums: the result h + l has |l| within a
// few ulp(h) but is not re-split into head and tail.  Every consumer accepts
// that: a product reads a tail only through FMAs, and a sum splits the heads
// exactly and adds the tails.  Each saves the three-instruction
// renormalisation.
__device__ __forceinline__ F2 f2_mul_u(F2 a, F2 b) {
  const float p = __fmul_rn(a.h, b.h);
  return F2{p, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)))};
}
__device__ __forceinline__ F2 f2_add_u(F2 a, F2 b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return F2{s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}
// d^{-3/2}, d > 0: from the hardware estimate y of d^{-1/2}, r = 1 - d y^2 is
// formed in float-float and d^{-3/2} = y^3 (1 - r)^{-3/2}
// = y^3 (1 + 3r/2 + 15r^2/8 + O(r^3)) by the binomial series.  With |r| ~
// 2^-22 the truncation is ~2^-63 and the rounding of the correction ~2^-45 of
// the result; y^3 is formed as an exact-head pair.
__device__ __forceinline__ F2 f2_rsqrt3_u(F2 d) {
  const float y = rsqrtf(d.h);
  const float y2h = __fmul_rn(y, y);
  const float y2l = fmaf(y, y, -y2h);
  const F2 t = f2_mul_u(d, F2{y2h, y2l});
  const float r = __fsub_rn(__fsub_rn(1.0f, t.h), t.l);  // 1 - t.h exact: t.h within [1/2, 2]
  const float c = __fmul_rn(r, fmaf(1.875f, r, 1.5f));
  const float p = __fmul_rn(y2h, y);
  const float e = fmaf(y2l, y, fmaf(y2h, y, -p));
  return F2{p, fmaf(p, c, e)};
}

// x0 + k dx - p as a normalised (hi, lo) float pair, from the float pairs of
// x0, dx and p (float-float arithmetic on the FP32 pipe, ~2^-46 relative)
__device__ __forceinline__ void ff_offset(float k, const float* x0p, const float* dxp, float ph,
                                          float pl, float& hi, float& lo) {
  const F2 kd = f2_mulf(F2{dxp[0], dxp[1]}, k);
  F2 r = f2_add(F2{x0p[0], x0p[1]}, kd);
  r = f2_add(r, F2{-ph, -pl});
  hi = r.h;
  lo = r.l;
}

// minimum resident CTAs per SM asked of the register allocator (80
// registers and 25.6 KB of shared memory at P4 fit eight)
#ifndef DG_STAGE32_MIN_CTAS
#define DG_STAGE32_MIN_CTAS 8
#endif


// LAST = false: modes 0 (operator only) and 1 (RK stage); LAST = true: mode 2
// (last RK stage with damping, torque and CFL), compiled apart so that the
// first two stages do not carry the epilogue's code
template <int P, bool LAST>
__device__ __forceinline__ void stage32_tile(const StageArgs32& a, const float* Dcur, const float* Dn0,
                                             float* Outp, float alpha, float beta, int pidx, int mode,
                                             int bx, int j, double* smd) {
  constexpr int m = P + 1, M = m * m, NV = 3;
  constexpr int NVM = NV * M;
  using S = Smem32<P>;
  // smd[0..4]: floats sF[0..8] (tile offsets from the planet (hi, lo), dt);
  // smd[7]: the mbarrier of the last stage's TMA copy
  float* sF = reinterpret_cast<float*>(smd);
  float* sm = reinterpret_cast<float*>(smd + S::ND);
  float* sU = sm + S::U;
  float* sFl = sm + S::F;
  float* sXR = sm + S::XR;
  float* sXL = sm + S::XL;
  float* sYT = sm + S::YT;
  float* sYN = sm + S::YN;
  float* sFX = sm + S::FX;
  float* sFY = sm + S::FY;
  float* sB0 = sm + S::B0;
  int* sFlag = reinterpret_cast<int*>(sm + S::FLAGS);

  const Mesh& ms = a.mesh;
  const Prec32& pc = a.pc;
  if (a.ts->status != 0) return;

  const int tid = threadIdx.x, lane = tid & 31, v = tid >> 5;
  const int i0 = bx * 32;
  const int nvalid = min(32, ms.nx - i0);
  const bool valid = lane < nvalid;
  const int lc = valid ? lane : nvalid - 1;

  if (tid == 0) {
    // centre of the tile's first element relative to the planet at the stage
    // time and (last stage) at t^{n+1}, kept as (hi, lo) float pairs: a single
    // rounding here would shift every element of the tile row by the same
    // amount, a correlated error the torque sum does not average out
    const DevState* ts = a.ts;
    sF[8] = ts->dtf;
    const float kx = i2f(i0) + 0.5f, ky = i2f(j) + 0.5f;
    const float* pl = ts->plf[pidx];
    ff_offset(kx, pc.x0p, pc.dxp, pl[0], pl[1], sF[0], sF[4]);
    ff_offset(ky, pc.y0p, pc.dyp, pl[2], pl[3], sF[1], sF[5]);
    if (LAST) mbar_init(smd + 7, 1);
  }
  if (tid < 32) sFlag[tid] = 0;

  // element pointers of this thread's variable (stride 32 between modes);
  // bc 0 periodic wrap, bc 1 ghosts carry the background (delta = 0),
  // bc 2 transmissive (exterior trace = interior trace)
  const size_t tile = (size_t)j * ms.ntx + bx;
  const size_t voff = (size_t)v * M * 32;
  const float* own = Dcur + tile * NVM * 32 + voff + lc;
  const float* pB = nullptr;
  const float* pT = nullptr;
  bool zB = false, zT = false;
  if (j > 0) pB = Dcur + ((size_t)(j - 1) * ms.ntx + bx) * NVM * 32 + voff + lc;
  else if (ms.bc == 0) pB = Dcur + ((size_t)(ms.ny - 1) * ms.ntx + bx) * NVM * 32 + voff + lc;
  else if (ms.bc == 1) zB = true;
  else if (ms.bc == 3) pB = own;  // zero-gradient ghost: a copy of this row
  if (j + 1 < ms.ny) pT = Dcur + ((size_t)(j + 1) * ms.ntx + bx) * NVM * 32 + voff + lc;
  else if (ms.bc == 0) pT = Dcur + (size_t)bx * NVM * 32 + voff + lc;
  else if (ms.bc == 1) zT = true;
  else if (ms.bc == 3) pT = own;
  const bool trB = !pB && !zB, trT = !pT && !zT;
  const int il = i0 - 1, ir = i0 + nvalid;
  const float* pL = nullptr;
  const float* pR = nullptr;
  bool zL = false, zR = false;
  if (il >= 0) pL = Dcur + ((size_t)j * ms.ntx + (il >> 5)) * NVM * 32 + voff + (il & 31);
  else if (ms.bc == 0) { const int iw = ms.nx - 1; pL = Dcur + ((size_t)j * ms.ntx + (iw >> 5)) * NVM * 32 + voff + (iw & 31); }
  else if (ms.bc == 1) zL = true;
  else if (ms.bc == 3) pL = Dcur + (size_t)j * ms.ntx * NVM * 32 + voff;
  if (ir < ms.nx) pR = Dcur + ((size_t)j * ms.ntx + (ir >> 5)) * NVM * 32 + voff + (ir & 31);
  else if (ms.bc == 0) pR = Dcur + (size_t)j * ms.ntx * NVM * 32 + voff;
  else if (ms.bc == 1) zR = true;
  else if (ms.bc == 3) { const int ie = ms.nx - 1; pR = Dcur + ((size_t)j * ms.ntx + (ie >> 5)) * NVM * 32 + voff + (ie & 31); }
  const bool trL = !pL && !zL, trR = !pR && !zR;
  // does any node of the tile lie in a damping zone (last stage; a
  // conservative test on the tile's box, the per-node test decides)
  bool zones = false;
  if (LAST) {
    const float xlo = fmaf(i2f(i0), pc.dx, pc.x0), xhi = fmaf(i2f(nvalid), pc.dx, xlo);
    const float ylo = fmaf(i2f(j), pc.dy, pc.y0), yhi = ylo + pc.dy;
    const float cx = fminf(fmaxf(0.0f, xlo), xhi), cy = fminf(fmaxf(0.0f, ylo), yhi);
    const float rmin2 = fmaf(cx, cx, cy * cy);
    const float rmax2 = fmaxf(xlo * xlo, xhi * xhi) + fmaxf(ylo * ylo, yhi * yhi);
    zones = (pc.rd_in > 0.0f && rmin2 < 1.001f * pc.rd_in * pc.rd_in) ||
            (pc.rd_out > 0.0f && rmax2 > 0.999f * pc.rd_out * pc.rd_out);
  }
  // the tile rows the update reads at the end (u^n, R_b, the damping offsets)
  // are asked of the L2 now, one bulk request each, so that their DRAM
  // latency passes while the tile computes
  const int rbs = a.RbIdx[tile];
  if (tid == 32) {
    const unsigned tbytes = NVM * 32 * sizeof(float);
    if (mode != 0 && alpha != 0.0f) bulk_prefetch_l2(Dn0 + tile * NVM * 32, tbytes);
    if (rbs >= 0) bulk_prefetch_l2(a.Rb + (size_t)rbs * NVM * 32, tbytes);
    if (LAST && zones) bulk_prefetch_l2(a.Db + tile * (size_t)(3 * M * 32), 3 * M * 32 * sizeof(float));
  }
  // tiles near the singular centre use the exact projected background (FP32
  // modes of u_b, same tiled layout as delta, all three variables)
  const int exact = a.TileFlag[tile];
  const float* bgOwn = exact ? a.Bmodes + tile * NVM * 32 + lc : nullptr;
  const float* bgB = (exact && pB) ? a.Bmodes + (pB - Dcur) - voff : nullptr;
  const float* bgT = (exact && pT) ? a.Bmodes + (pT - Dcur) - voff : nullptr;
  const float* bgL = (exact && pL) ? a.Bmodes + (pL - Dcur) - voff : nullptr;
  const float* bgR = (exact && pR) ? a.Bmodes + (pR - Dcur) - voff : nullptr;
  // FP32 geometry of this thread's element
  const float lanef = i2f(lane);
  const float xcf = fmaf(i2f(i0 + lane) + 0.5f, pc.dx, pc.x0);
  const float ycf = fmaf(i2f(j) + 0.5f, pc.dy, pc.y0);
  const float yBf = fmaf(i2f(j), pc.dy, pc.y0), yTf = fmaf(i2f(j + 1), pc.dy, pc.y0);

  // ---- P1: nodal values and face traces of this thread's variable ------------
  // The state is the values at the m x m nodes (k = q*m + r): they go to
  // shared memory as they are, and each face trace is one sum along a node
  // line with the Lagrange weights of the element end.
  // the element below is loaded with the own element and the element above
  // before the traces below are summed, so that each load's latency passes
  // under the sums before it (a missing neighbour reads the own element,
  // unused)
  float cb[M];
  {
    float c[M];
#pragma unroll
    for (int k = 0; k < M; k++) c[k] = own[k * 32];
    {
      const float* qB = pB ? pB : own;
#pragma unroll
      for (int k = 0; k < M; k++) cb[k] = qB[k * 32];
    }
#pragma unroll
    for (int k = 0; k < M; k++) sU[voff + k * 32 + lane] = c[k];
    // x traces at the m y-nodes r: right (xi = +1) and left (xi = -1) as the
    // lanes of one packed sum over q; right trace of element e at slot e+1,
    // left trace at slot e
    float* xr = sXR + v * m * 33;
    float* xl = sXL + v * m * 33;
#pragma unroll
    for (int r = 0; r < m; r++) {
      float2 t = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int q = 0; q < m; q++) t = f2(c32t[P].bpm2[q], d2(c[q * m + r]), t);
      xr[r * 33 + lane + 1] = t.x;
      if (valid) xl[r * 33 + lane] = t.y;
      if (lane == 0 && trL) xr[r * 33] = t.y;  // mirror: exterior = interior
      if (lane == nvalid - 1 && trR) xl[r * 33 + nvalid] = t.x;
    }
    // y traces at the m x-nodes q: top (eta = +1, plane 0) and bottom (plane 1)
#pragma unroll
    for (int q = 0; q < m; q++) {
      float2 t = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int r = 0; r < m; r++) t = f2(c32t[P].bpm2[r], d2(c[q * m + r]), t);
      sYT[((0 * 3 + v) * m + q) * 32 + lane] = t.x;
      sYT[((1 * 3 + v) * m + q) * 32 + lane] = t.y;
      if (trB) sYN[((0 * 3 + v) * m + q) * 32 + lane] = t.y;
      if (trT) sYN[((1 * 3 + v) * m + q) * 32 + lane] = t.x;
    }
  }
  {
    // neighbour rows: the top trace of the element below and the bottom trace
    // of the element above, each summed in the order of its owner's own trace
    // (both CTAs of a face see the same values)
    float c[M];
    {
      const float* qT = pT ? pT : own;
#pragma unroll
      for (int k = 0; k < M; k++) c[k] = qT[k * 32];
    }
    if (pB) {
#pragma unroll
      for (int q = 0; q < m; q++) {
        float acc = 0.0f;
#pragma unroll
        for (int r = 0; r < m; r++) acc = fmaf(c32t[P].bp[r], cb[q * m + r], acc);
        sYN[((0 * 3 + v) * m + q) * 32 + lane] = acc;
      }
    } else if (zB) {
#pragma unroll
      for (int q = 0; q < m; q++) sYN[((0 * 3 + v) * m + q) * 32 + lane] = 0.0f;
    }
    if (pT) {
#pragma unroll
      for (int q = 0; q < m; q++) {
        float acc = 0.0f;
#pragma unroll
        for (int r = 0; r < m; r++) acc = fmaf(c32t[P].bm[r], c[q * m + r], acc);
        sYN[((1 * 3 + v) * m + q) * 32 + lane] = acc;
      }
    } else if (zT) {
#pragma unroll
      for (int q = 0; q < m; q++) sYN[((1 * 3 + v) * m + q) * 32 + lane] = 0.0f;
    }
    // the two x-halo elements: right trace of the left halo, left trace of the
    // right halo, one y-node per lane (lanes 0..m-1 left, 16..16+m-1 right),
    // each summed in the order of the owner tile's own trace
    {
      const bool right = lane >= 16;
      const int r = lane & 15;
      const float* ph = right ? pR : pL;
      if (r < m && (ph || (right ? zR : zL))) {
        float acc = 0.0f;
        if (ph) {
#pragma unroll
          for (int q = 0; q < m; q++) acc = fmaf(right ? c32t[P].bm[q] : c32t[P].bp[q], ph[(q * m + r) * 32], acc);
        }
        if (right) sXL[(v * m + r) * 33 + nvalid] = acc;
        else sXR[(v * m + r) * 33] = acc;
      }
    }
  }
  __syncthreads();
  const float dt = sF[8];
  // ---- P2: face fluxes, then the pointwise flux differences and sources at
  // the nodes (both dealt round-robin over the three threads of an element);
  // the pointwise terms overwrite the traces the face fluxes were formed from
  {
    // y faces of the element: bottom (below | own) and top (own | above)
    for (int kk = v; kk < 2 * m; kk += 3) {
      const int side = kk >= m, q = kk - side * m;
      const float xq = fmaf(pc.hdx, c32t[P].xi[q], xcf);
      float dL[3], dR[3], hf[3];
#pragma unroll
      for (int w3 = 0; w3 < 3; w3++) {
        const int o = ((w3)*m + q) * 32 + lane;
        dL[w3] = side ? sYT[0 * 3 * m * 32 + o] : sYN[0 * 3 * m * 32 + o];
        dR[w3] = side ? sYN[1 * 3 * m * 32 + o] : sYT[1 * 3 * m * 32 + o];
      }
      Bg32 bO = bg32_at(pc, xq, side ? yTf : yBf), bN = bO;
      if (exact) {
        const float c2 = bO.c2;
        bO = bg32_poly<P>(bgOwn, c32t[P].eye[q], side ? c32t[P].bp : c32t[P].bm, c2);
        const float* nb = side ? bgT : bgB;
        if (nb) bN = bg32_poly<P>(nb, c32t[P].eye[q], side ? c32t[P].bm : c32t[P].bp, c2);
        else if (side ? trT : trB) bN = bO;
      }
      dllf32<1>(side ? bO : bN, side ? bN : bO, dL, dR, hf);
#pragma unroll
      for (int w3 = 0; w3 < 3; w3++) sFY[((side * 3 + w3) * m + q) * 32 + lane] = hf[w3] * pc.idy;
    }
    // x faces f = 0..nvalid of the tile row (face f between elements f-1 and f)
    for (int idx = tid; idx < m * 33; idx += 96) {
      const int r = idx / 33, f = idx - 33 * r;
      if (f <= nvalid) {
        float dL[3], dR[3], hf[3];
#pragma unroll
        for (int w3 = 0; w3 < 3; w3++) {
          dL[w3] = sXR[(w3 * m + r) * 33 + f];
          dR[w3] = sXL[(w3 * m + r) * 33 + f];
        }
        const float y = fmaf(pc.hdy, c32t[P].xi[r], ycf);
        Bg32 bL = bg32_at(pc, fmaf(i2f(i0 + f), pc.dx, pc.x0), y), bR = bL;
        if (exact) {
          const float* eL = (f > 0) ? bgOwn - lc + (f - 1) : bgL;
          const float* eR = (f < nvalid) ? bgOwn - lc + f : bgR;
          const float c2 = bL.c2;
          if (eL) bL = bg32_poly<P>(eL, c32t[P].bp, c32t[P].eye[r], c2);
          if (eR) bR = bg32_poly<P>(eR, c32t[P].bm, c32t[P].eye[r], c2);
          if (!eL && trL && f == 0) bL = bR;
          if (!eR && trR && f == nvalid) bR = bL;
        }
        dllf32<0>(bL, bR, dL, dR, hf);
#pragma unroll
        for (int w3 = 0; w3 < 3; w3++) sFX[(w3 * m + r) * 33 + f] = hf[w3] * pc.idx;
      }
    }
  }
  __syncthreads();
  {
    const float pdx0 = fmaf(lanef, pc.dx, sF[0]);
    // two nodes per iteration, n0 = v + 3 kk and n1 = n0 + 3 (an odd last node
    // pairs with itself and its second lane is not stored)
    constexpr int KN = (M + 2) / 3;
#pragma unroll 1
    for (int kk = 0; kk < KN; kk += 2) {
      const int n0 = v + 3 * kk;
      if (n0 >= M) break;  // warp-uniform
      const bool two = n0 + 3 < M;
      const int n1 = two ? n0 + 3 : n0;
      const int q0 = n0 / m, r0 = n0 - q0 * m, q1 = n1 / m, r1 = n1 - q1 * m;
      float2 d[3];
#pragma unroll
      for (int w3 = 0; w3 < 3; w3++) d[w3] = make_float2(sU[(w3 * M + n0) * 32 + lane], sU[(w3 * M + n1) * 32 + lane]);
      const float2 xiq = make_float2(c32t[P].xi[q0], c32t[P].xi[q1]), xir = make_float2(c32t[P].xi[r0], c32t[P].xi[r1]);
      const float2 xq = f2(d2(pc.hdx), xiq, d2(xcf));
      const float2 y = f2(d2(pc.hdy), xir, d2(ycf));
      float2 r2, ir;
      Bg32x2 bgn = bg32_at2(pc, xq, y, r2, ir);
      if (exact) {
        const Bg32 b0 = bg32_poly<P>(bgOwn, c32t[P].eye[q0], c32t[P].eye[r0], bgn.c2.x);
        const Bg32 b1 = bg32_poly<P>(bgOwn, c32t[P].eye[q1], c32t[P].eye[r1], bgn.c2.y);
        bgn.sig = make_float2(b0.sig, b1.sig);
        bgn.vx = make_float2(b0.vx, b1.vx);
        bgn.vy = make_float2(b0.vy, b1.vy);
        bgn.mx = make_float2(b0.mx, b1.mx);
        bgn.my = make_float2(b0.my, b1.my);
      }
      float2 fx[3], fy[3], vxn, vyn;
      dflux32x2(bgn, d, fx, fy, vxn, vyn);
      // star: -dSigma grad Phi_*; planet: -Sigma grad Phi_p
      float2 src1 = d2(0.0f), src2 = d2(0.0f);
      if (pc.star) {
        const float rs2 = pc.rs * pc.rs;
        const float2 ir3 = m2(m2(ir, ir), ir);
        const float2 inv = make_float2(r2.x >= rs2 ? ir3.x : pc.irs3, r2.y >= rs2 ? ir3.y : pc.irs3);
        src1 = m2(m2(n2(d[0]), xq), inv);
        src2 = m2(m2(n2(d[0]), y), inv);
      }
      if (pc.planet) {
        const float2 pdx = a2(d2(pdx0), f2(d2(pc.hdx), xiq, d2(sF[4])));
        const float2 pdy = a2(d2(sF[1]), f2(d2(pc.hdy), xir, d2(sF[5])));
        const float2 dd = f2(pdx, pdx, f2(pdy, pdy, d2(pc.eps2)));
        const float2 id = make_float2(rsqrtf(dd.x), rsqrtf(dd.y));
        const float2 f = m2(m2(m2(m2(d2(pc.q), id), id), id), a2(bgn.sig, d[0]));
        src1 = f2(n2(f), pdx, src1);
        src2 = f2(n2(f), pdy, src2);
      }
      // the momentum rows' terms in planes 0-5 (fx1, fx2, fy1, fy2, src1, src2)
      const float2 s2x = d2(pc.s2x), s2y = d2(pc.s2y);
      const float2 o2[6] = {m2(fx[1], s2x), m2(fx[2], s2x), m2(fy[1], s2y), m2(fy[2], s2y), src1, src2};
      float* o0 = sFl + n0 * 32 + lane;
#pragma unroll
      for (int t = 0; t < 6; t++) o0[t * M * 32] = o2[t].x;
      if (two) {
        float* o1 = sFl + n1 * 32 + lane;
#pragma unroll
        for (int t = 0; t < 6; t++) o1[t * M * 32] = o2[t].y;
      }
    }
  }
  __syncthreads();
  // ---- P3: volume integral and surface lift of this thread's variable -------
  // At node (q, r): L = sum_q' dw[q][q'] fx(q', r) + sum_r' dw[r][r'] fy(q, r')
  //                   + src(q, r) + lm[q] hL(r) - lp[q] hR(r) + lm[r] hB(q) - lp[r] hT(q)
  // (fx, fy carry 2/dx, 2/dy and the face fluxes 1/dx, 1/dy).  Node pairs
  // (2k, 2k+1) along x are the lanes of packed FMAs: the x sums take the
  // pair's two table rows against one value, the y sums one table entry
  // against the pair's two values; each lane keeps its scalar order.
  // The density row's fluxes are the momentum perturbations (times 2/dx,
  // 2/dy), read from the state in global memory (the tile loaded in P1, at
  // hand in the caches); the momentum rows read their terms from planes 0-5.
  constexpr int MP = (m + 1) / 2;  // node pairs along x (the pair past an odd m has a dead lane)
  float2 LP[MP][m];                // LP[k][r] = (L(2k, r), L(2k+1, r))
  {
    const int pfx = S::PFX + v - 1, pfy = S::PFY + v - 1, psrc = S::PSRC + v - 1;
    const float* gmx = Dcur + tile * NVM * 32 + 1 * M * 32 + lc;  // delta m_x, delta m_y of this element
    const float* gmy = gmx + M * 32;
#pragma unroll
    for (int k = 0; k < MP; k++)
#pragma unroll
      for (int r = 0; r < m; r++) {
        const int q0 = 2 * k, q1 = 2 * k + 1;
        LP[k][r] = make_float2(v > 0 ? sFl[(psrc * M + q0 * m + r) * 32 + lane] : 0.0f,
                               (v > 0 && q1 < m) ? sFl[(psrc * M + q1 * m + r) * 32 + lane] : 0.0f);
      }
    // x: one node row r at a time, its m fluxes and its two face fluxes
#pragma unroll
    for (int r = 0; r < m; r++) {
      float X[m];
      if (v > 0) {
#pragma unroll
        for (int q2 = 0; q2 < m; q2++) X[q2] = sFl[(pfx * M + q2 * m + r) * 32 + lane];
      } else {
#pragma unroll
        for (int q2 = 0; q2 < m; q2++) X[q2] = __fmul_rn(pc.s2x, gmx[(q2 * m + r) * 32]);
      }
      const float hl = sFX[(v * m + r) * 33 + lane], hr = sFX[(v * m + r) * 33 + lane + 1];
#pragma unroll
      for (int k = 0; k < MP; k++) {
        float2 acc = LP[k][r];
#pragma unroll
        for (int q2 = 0; q2 < m; q2++) acc = f2(c32t[P].dwp[k][q2], d2(X[q2]), acc);
        acc = f2(c32t[P].lmp[k], d2(hl), acc);
        LP[k][r] = f2(c32t[P].lpn[k], d2(hr), acc);
      }
    }
    // y: one node pair (2k, 2k+1) at a time, its two node columns and their
    // bottom and top face fluxes
#pragma unroll
    for (int k = 0; k < MP; k++) {
      const int q0 = 2 * k, q1 = 2 * k + 1;
      float2 Y[m];
      if (v > 0) {
#pragma unroll
        for (int r2 = 0; r2 < m; r2++)
          Y[r2] = make_float2(sFl[(pfy * M + q0 * m + r2) * 32 + lane],
                              q1 < m ? sFl[(pfy * M + q1 * m + r2) * 32 + lane] : 0.0f);
      } else {
#pragma unroll
        for (int r2 = 0; r2 < m; r2++)
          Y[r2] = make_float2(__fmul_rn(pc.s2y, gmy[(q0 * m + r2) * 32]),
                              q1 < m ? __fmul_rn(pc.s2y, gmy[(q1 * m + r2) * 32]) : 0.0f);
      }
      const float2 hb = make_float2(sFY[((0 * 3 + v) * m + q0) * 32 + lane],
                                    q1 < m ? sFY[((0 * 3 + v) * m + q1) * 32 + lane] : 0.0f);
      const float2 ht = make_float2(sFY[((1 * 3 + v) * m + q0) * 32 + lane],
                                    q1 < m ? sFY[((1 * 3 + v) * m + q1) * 32 + lane] : 0.0f);
#pragma unroll
      for (int r = 0; r < m; r++) {
        float2 acc = LP[k][r];
#pragma unroll
        for (int r2 = 0; r2 < m; r2++) acc = f2(c32t[P].dw2[r][r2], Y[r2], acc);
        acc = f2(c32t[P].lm2[r], hb, acc);
        LP[k][r] = f2(c32t[P].lpn2[r], ht, acc);
      }
    }
  }
  float L[M];
#pragma unroll
  for (int q = 0; q < m; q++)
#pragma unroll
    for (int r = 0; r < m; r++) L[q * m + r] = (q & 1) ? LP[q >> 1][r].y : LP[q >> 1][r].x;
  // background residual R_b (only in the tiles that keep it), then the
  // Shu-Osher combination
  const size_t gbase = tile * NVM * 32 + voff;
  if (rbs >= 0) {
    const float* rb = a.Rb + (size_t)rbs * NVM * 32 + voff + lc;
#pragma unroll
    for (int k = 0; k < M; k++) L[k] += rb[k * 32];
  }
  if (mode == 0) {
    if (valid) {
#pragma unroll
      for (int k = 0; k < M; k++) Outp[gbase + k * 32 + lane] = L[k];
    }
    return;
  }
  float un[M];
#pragma unroll
  for (int k = 0; k < M; k++) {
    const float dn = (alpha != 0.0f) ? Dn0[gbase + k * 32 + lc] : 0.0f;
    un[k] = fmaf(alpha, dn, beta * fmaf(dt, L[k], own[k * 32]));
  }
  if (!LAST) {
    if (valid) {
#pragma unroll
      for (int k = 0; k < M; k++) Outp[gbase + k * 32 + lane] = un[k];
    }
    return;
  }
  // ---- P4 (last stage): damping in delta form, CFL ---------------------------
  if (zones) {
    // the damping targets Q0 - Q_b at the nodes are copied by the TMA unit
    // into planes 3-5 of the pointwise terms, dead from here on, while the
    // nodal values of the new state are stored in planes 0-2
    float* sDb = sm + S::F + 3 * M * 32;
    static_assert(S::F + 6 * M * 32 <= S::XR, "damping offsets exceed the dead pointwise planes 3-5");
    fence_proxy_async_smem();
    __syncthreads();  // every read of the pointwise terms and face fluxes by P3 is done
    if (tid == 0) {
      const unsigned bytes = 3 * M * 32 * sizeof(float);
      mbar_expect_tx(smd + 7, bytes);
      bulk_g2s(sDb, a.Db + tile * (size_t)(3 * M * 32), bytes, smd + 7);
    }
#pragma unroll
    for (int k = 0; k < M; k++) sU[voff + k * 32 + lane] = un[k];
    if (__syncthreads_or(!mbar_wait(smd + 7, 0))) {
      // the copy did not land in time: flag the step (it is discarded) and
      // give the copy a last bounded chance to drain before the CTA exits
      if (tid == 0) atomicOr(&a.ts->pending, 2);
      mbar_wait(smd + 7, 0);
      return;
    }
    int damped = 0;
#pragma unroll 1
    for (int kk = 0; kk < (M + 2) / 3; kk++) {
      const int n = v + 3 * kk;
      if (n >= M) break;  // warp-uniform
      const int q = n / m, r = n - q * m;
      const float xq = fmaf(pc.hdx, c32t[P].xi[q], xcf);
      const float y = fmaf(pc.hdy, c32t[P].xi[r], ycf);
      const float rr = sqrt_fast(fmaxf(fmaf(xq, xq, __fmul_rn(y, y)), 1e-24f));
      float R = 0.0f, rd = 0.0f;
      if (pc.rd_in > 0.0f && rr < pc.rd_in) {
        rd = pc.rd_in;
        const float x = __fdividef(__fsub_rn(rr, rd), __fsub_rn(__fdividef(rd, pc.damp_ratio), rd));
        R = fminf(__fmul_rn(x, x), 1.0f);
      } else if (pc.rd_out > 0.0f && rr > pc.rd_out) {
        rd = pc.rd_out;
        const float x = __fdividef(__fsub_rn(rr, rd), fmaf(rd, pc.damp_ratio, -rd));
        R = fminf(__fmul_rn(x, x), 1.0f);
      }
      if (R > 0.0f) {
        damped = 1;
        // Q_new = Q0 + kappa (Q - Q0), kappa = tau / (tau + dt), written for
        // delta Q = Q - Q_b: dQ_new = kappa dQ + (1 - kappa) (Q0 - Q_b)
        const float tau = __fdividef(__fmul_rn(6.2831853071795864769f, sqrt_fast(__fmul_rn(__fmul_rn(rd, rd), rd))), R);
        const float itd = __fdividef(1.0f, __fadd_rn(tau, dt));
        const float kap = __fmul_rn(tau, itd), omk = __fmul_rn(dt, itd);
        Bg32 bgn = bg32_at(pc, xq, y);
        if (exact) bgn = bg32_poly<P>(bgOwn, c32t[P].eye[q], c32t[P].eye[r], bgn.c2);
        const float d0 = sU[(0 * M + n) * 32 + lane];
        const float d1 = sU[(1 * M + n) * 32 + lane], d2 = sU[(2 * M + n) * 32 + lane];
        const float sg = __fadd_rn(bgn.sig, d0);
        const float isg = __fdividef(1.0f, sg);
        const float dvx = __fmul_rn(fmaf(-bgn.vx, d0, d1), isg);
        const float dvy = __fmul_rn(fmaf(-bgn.vy, d0, d2), isg);
        const float ds2 = fmaf(kap, d0, __fmul_rn(omk, sDb[(0 * M + n) * 32 + lc]));
        const float dvx2 = fmaf(kap, dvx, __fmul_rn(omk, sDb[(1 * M + n) * 32 + lc]));
        const float dvy2 = fmaf(kap, dvy, __fmul_rn(omk, sDb[(2 * M + n) * 32 + lc]));
        const float sg2 = __fadd_rn(bgn.sig, ds2);
        sU[(0 * M + n) * 32 + lane] = ds2;
        sU[(1 * M + n) * 32 + lane] = fmaf(ds2, bgn.vx, __fmul_rn(sg2, dvx2));
        sU[(2 * M + n) * 32 + lane] = fmaf(ds2, bgn.vy, __fmul_rn(sg2, dvy2));
      }
    }
    if (damped) sFlag[lane] = 1;
    if (__syncthreads_or(damped)) {
      // the damped values at the nodes are the new state (the state is its
      // nodal values: no projection back)
      if (sFlag[lane]) {
#pragma unroll
        for (int k = 0; k < M; k++) un[k] = sU[voff + k * 32 + lane];
      }
    }
  }
  if (valid) {
#pragma unroll
    for (int k = 0; k < M; k++) Outp[gbase + k * 32 + lane] = un[k];
  }
  {
    // element average of this variable: the m x m Gauss-Legendre rule
    float avg = 0.0f;
#pragma unroll
    for (int k = 0; k < M; k++) avg = fmaf(c32t[P].w2h[k], un[k], avg);
    sB0[v * 32 + lane] = avg;
  }
  __syncthreads();
  if (v == 0) {
    // CFL minimum of the new state from the element averages of u_b + delta
    float dtf = __int_as_float(0x7f800000);
    int bad = 0;
    if (valid) {
      const float* b0 = a.Bm0 + tile * (size_t)(3 * 32);
      const float rho = b0[0 * 32 + lane] + sB0[0 * 32 + lane];
      const float irho = 1.0f / rho;
      const float vx = (b0[1 * 32 + lane] + sB0[1 * 32 + lane]) * irho;
      const float vy = (b0[2 * 32 + lane] + sB0[2 * 32 + lane]) * irho;
      const float c = sqrtf(bg32_at(pc, xcf, ycf).c2);
      dtf = pc.cfl_fac / ((fabsf(vx) + c) / pc.dx + (fabsf(vy) + c) / pc.dy);
      bad = !(rho > 0.0f) || !(dtf > 0.0f);  // +inf (no wave speed) is no constraint; NaN fails
      if (bad) dtf = __int_as_float(0x7f800000);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dtf = fminf(dtf, __shfl_xor_sync(0xffffffffu, dtf, o));
      bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
      if (bad) atomicOr(&a.ts->pending, 1);
      atomicMin(&a.ts->dt_bits, (unsigned long long)__double_as_longlong((double)dtf));
    }
  }
}

// one tile per CTA: grid (tiles per row, rows)
template <int P, bool LAST>
__global__ void __launch_bounds__(96, DG_STAGE32_MIN_CTAS) k_stage32(const StageArgs32 a) {
  extern __shared__ double smd[];
  pdl_wait();
  pdl_trigger();
  int bx = blockIdx.x, j = blockIdx.y;
  if (LAST && a.TileOrder) {
    // CTAs in an order that keeps the tiles running the damping branch together
    const int t = a.TileOrder[blockIdx.y * gridDim.x + blockIdx.x];
    j = t / a.mesh.ntx;
    bx = t - j * a.mesh.ntx;
  }
  stage32_tile<P, LAST>(a, a.D, a.Dn, a.Out, a.alpha, a.beta, a.pidx, a.mode, bx, j, smd);
}

// Torque on the planet at t^{n+1} from the new state (Sec. 5.2 torque with the
// quadrature-node masses).  One warp per tile, lane e owns element e.  The
// terms w_n m_n (r_n - r_p) / (|r_n - r_p|^2 + eps^2)^{3/2} are large and
// cancel to a few 1e-5 of their absolute sum, and their absolute sum is
// spread evenly over the decades of distance from the planet, so every term
// is evaluated, and summed over the element's nodes, in float-float
// arithmetic (~2^-44 relative); the sums over elements are FP64: node
// mass Sigma_b (a float pair from the FP64 background) + delta Sigma (the
// state's own FP32 value at the node), offsets from the planet as float pairs
// from the FP64 position, the inverse cube by one float-float Newton
// correction.  The x offset depends on the node row q only and the y offset
// on the node column r only, so the force sums as sum_q dx_q (sum_r f_qr)
// and sum_r dy_r (sum_q f_qr).  Each element's pair is rounded to a double
// and the warp sums its elements in FP64; the finish kernel sums the tiles in
// FP64.
template <int P>
__device__ __forceinline__ void torque32_tile(const float* D, const float* SigbN, const DevState* ts,
                                              double* part, const Mesh& ms, const Prec32& pc, int tile) {
  constexpr int m = P + 1, M = m * m, NVM = 3 * M;
  if (ts->status != 0) return;
  const int lane = threadIdx.x & 31;
  const int j = tile / ms.ntx, bx = tile - j * ms.ntx;
  const int i = bx * 32 + lane;
  const bool valid = i < ms.nx;
  const int lc = valid ? lane : 0;
  const float* sD = D + (size_t)tile * NVM * 32 + lc;  // variable 0 at the nodes
  const float* sbh = SigbN + (size_t)tile * 2 * M * 32 + lc;
  const float* sbl = sbh + M * 32;
  const float* p1 = ts->plf[2];
  F2 ox, oy;
  ff_offset(i2f(i) + 0.5f, pc.x0p, pc.dxp, p1[0], p1[1], ox.h, ox.l);
  ff_offset(i2f(j) + 0.5f, pc.y0p, pc.dyp, p1[2], p1[3], oy.h, oy.l);
  const F2 hdx{0.5f * pc.dxp[0], 0.5f * pc.dxp[1]}, hdy{0.5f * pc.dyp[0], 0.5f * pc.dyp[1]};
  const F2 eps2{pc.eps2p[0], pc.eps2p[1]};
  // offsets of the node columns from the planet and their squares plus eps^2
  F2 py[m], pye[m];
#pragma unroll
  for (int r = 0; r < m; r++) {
    py[r] = f2_add(oy, f2_mul(hdy, F2{c32t[P].xi[r], c32t[P].xil[r]}));
    pye[r] = f2_add(f2_mul(py[r], py[r]), eps2);
  }
  F2 gx{0.0f, 0.0f}, gy{0.0f, 0.0f};
  if (valid) {
    F2 C[m];  // column sums sum_q f_qr
#pragma unroll
    for (int r = 0; r < m; r++) C[r] = F2{0.0f, 0.0f};
    // one node row q per iteration (rolled: the float-float body is long);
    // the next row's values are loaded while this row computes
    float nh[m], nl[m], nd[m];
#pragma unroll
    for (int r = 0; r < m; r++) {
      nh[r] = sbh[r * 32];
      nl[r] = sbl[r * 32];
      nd[r] = sD[r * 32];
    }
#pragma unroll 1
    for (int q = 0; q < m; q++) {
      float sh[m], sl[m], dd[m];
#pragma unroll
      for (int r = 0; r < m; r++) {
        sh[r] = nh[r];
        sl[r] = nl[r];
        dd[r] = nd[r];
      }
      if (q + 1 < m) {
#pragma unroll
        for (int r = 0; r < m; r++) {
          nh[r] = sbh[((q + 1) * m + r) * 32];
          nl[r] = sbl[((q + 1) * m + r) * 32];
          nd[r] = sD[((q + 1) * m + r) * 32];
        }
      }
      const F2 px = f2_add(ox, f2_mul(hdx, F2{c32t[P].xi[q], c32t[P].xil[q]}));
      const F2 px2 = f2_mul_u(px, px);
      F2 S{0.0f, 0.0f};  // row sum sum_r f_qr
#pragma unroll
      for (int r = 0; r < m; r++) {
        const int n = q * m + r;
        const F2 ds{dd[r], 0.0f};
        // w_n (Sigma_b + delta Sigma) / (d^2 + eps^2)^{3/2}
        const F2 mass = f2_mul_u(f2_add_u(F2{sh[r], sl[r]}, ds), F2{c32t[P].w2h[n], c32t[P].w2l[n]});
        const F2 f = f2_mul_u(mass, f2_rsqrt3_u(f2_add_u(px2, pye[r])));
        S = r ? f2_add_u(S, f) : f;
        C[r] = f2_add_u(C[r], f);
      }
      gx = f2_add_u(gx, f2_mul_u(S, px));
    }
#pragma unroll
    for (int r = 0; r < m; r++) gy = f2_add_u(gy, f2_mul_u(C[r], py[r]));
  }
  // the element's sums to FP64, then the warp's sum over its elements in FP64
  double ex = (double)gx.h + (double)gx.l, ey = (double)gy.h + (double)gy.l;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ex += __shfl_xor_sync(0xffffffffu, ex, o);
    ey += __shfl_xor_sync(0xffffffffu, ey, o);
  }
  if (lane == 0) {
    const double area = ms.dx * ms.dy;
    part[2 * tile] = ex * area;
    part[2 * tile + 1] = ey * area;
  }
}

// four tiles (warps) per CTA
template <int P>
__global__ void __launch_bounds__(128, 6) k_torque32(const float* D, const float* SigbN, const DevState* ts,
                                                   double* part, const Mesh ms, const Prec32 pc) {
  pdl_wait();
  pdl_trigger();
  const int w = threadIdx.x >> 5;
  const int tile = blockIdx.x * 4 + w;
  if (tile < ms.ntx * ms.ny) torque32_tile<P>(D, SigbN, ts, part, ms, pc, tile);  // warp-uniform
}

template <int P, bool LAST>
static cudaError_t launch_stage32_kind(const StageArgs32& a, cudaStream_t s) {
  static bool configured = false;
  const size_t bytes = Smem32<P>::BYTES;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_stage32<P, LAST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    // the whole unified L1 as shared memory: the occupancy the kernel is
    // built for, not the carveout the driver would pick for it
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_stage32<P, LAST>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  return launch_pdl(k_stage32<P, LAST>, dim3(a.mesh.ntx, a.mesh.ny), dim3(96), bytes, s, a);
}

template <int P>
static cudaError_t launch_stage32_impl(const StageArgs32& a, cudaStream_t s) {
  return a.mode == 2 ? launch_stage32_kind<P, true>(a, s) : launch_stage32_kind<P, false>(a, s);
}

template <int P>
static cudaError_t launch_torque32_impl(const float* D, const float* SigbN, const DevState* ts, double* part,
                                 const Mesh& ms, const Prec32& pc, cudaStream_t s) {
  const int ntiles = ms.ntx * ms.ny;
  return launch_pdl(k_torque32<P>, dim3((ntiles + 3) / 4), dim3(128), 0, s, D, SigbN, ts, part, ms, pc);
}

template <int P>
static Tab32 make_tab32(const Tables& t) {
  constexpr int m = P + 1;
  Tab32 c{};
  double dw[MAXM][MAXM] = {}, lp[MAXM] = {}, lm[MAXM] = {};
  for (int q = 0; q < m; q++) {
    for (int a = 0; a < m; a++) {
      lp[q] += t.phi[q][a] * t.pp[a];
      lm[q] += t.phi[q][a] * t.pm[a];
    }
    for (int q2 = 0; q2 < m; q2++) {
      double s = 0.0;
      for (int a = 0; a < m; a++) s += t.phi[q][a] * t.dphi[q2][a];
      dw[q][q2] = t.wh[q2] * s;
    }
  }
  for (int q = 0; q < m; q++) {
    c.xi[q] = (float)t.xi[q];
    c.xil[q] = (float)(t.xi[q] - (double)c.xi[q]);
    c.wh[q] = (float)t.wh[q];
    c.bp[q] = (float)(t.wh[q] * lp[q]);
    c.bm[q] = (float)(t.wh[q] * lm[q]);
    c.bpm2[q] = make_float2(c.bp[q], c.bm[q]);
    c.lp[q] = (float)lp[q];
    c.lm[q] = (float)lm[q];
    c.eye[q][q] = 1.0f;
    for (int q2 = 0; q2 < m; q2++) {
      c.dw[q][q2] = (float)dw[q][q2];
      c.dw2[q][q2] = make_float2(c.dw[q][q2], c.dw[q][q2]);
    }
    c.lm2[q] = make_float2(c.lm[q], c.lm[q]);
    c.lpn2[q] = make_float2(-c.lp[q], -c.lp[q]);
    for (int r = 0; r < m; r++) {
      const double w2 = t.wh[q] * t.wh[r];
      c.w2h[q * m + r] = (float)w2;
      c.w2l[q * m + r] = (float)(w2 - (double)c.w2h[q * m + r]);
    }
  }
  for (int k = 0; 2 * k < m; k++) {
    const int q0 = 2 * k, q1 = 2 * k + 1;
    const bool two = q1 < m;
    for (int q2 = 0; q2 < m; q2++) c.dwp[k][q2] = make_float2(c.dw[q0][q2], two ? c.dw[q1][q2] : 0.0f);
    c.lmp[k] = make_float2(c.lm[q0], two ? c.lm[q1] : 0.0f);
    c.lpn[k] = make_float2(-c.lp[q0], two ? -c.lp[q1] : 0.0f);
  }
  return c;
}

// this translation unit's slice P of the tables (internal linkage: every
// translation unit that includes this header has its own copy of the tables,
// and a merged instantiation would fill another unit's copy)
template <int P>
static cudaError_t upload_tables32_impl(const Tables& t) {
  const Tab32 c = make_tab32<P>(t);
  return cudaMemcpyToSymbol(c32t, &c, sizeof(Tab32), P * sizeof(Tab32));
}

}  // namespace dg
