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
// solid-body-core edge), where the analytic and projected backgrounds differ
// and the projected one is contracted from its FP32 modes.  Same CTA structure
// as dg_stage.cuh (one 32-element tile, m warps).  The last stage adds damping
// in delta form, the torque (FP64 terms within a radius of the planet, FP32
// terms beyond, FP64 reduction) and the CFL minimum.  All mesh geometry is
// passed as FP32 scalars; offsets from the planet are formed once per CTA in
// FP64 and rounded, so the FP64 pipe is left to the near-planet torque.
#pragma once
#include "dg_internal.cuh"

#ifndef DG_P
#error "define DG_P before including dg_stage32.cuh"
#endif

namespace dg {

static __constant__ float c32_phi[MAXM][MAXM];    // [q][a] sqrt(2a+1) P_a(xi_q)
static __constant__ float c32_wphi[MAXM][MAXM];   // w_q/2 phi_a(xi_q)
static __constant__ float c32_wdphi[MAXM][MAXM];  // w_q/2 phi'_a(xi_q)
static __constant__ float c32_pp[MAXM], c32_pm[MAXM], c32_xi[MAXM], c32_wh[MAXM];
static __constant__ double c32_phi64[MAXM][MAXM], c32_xi64[MAXM], c32_wh64[MAXM];

// Analytic background of the disc and the isothermal sound speed at (x, y).
struct Bg32 {
  float sig, vx, vy, mx, my, c2;
};

__device__ __forceinline__ Bg32 bg32_at(const Prec32& pc, float x, float y) {
  Bg32 b;
  const float r2 = fmaf(x, x, y * y);
  const float ir = rsqrtf(r2);
  const float r = r2 * ir;
  float sig = pc.slope_half ? sqrtf(ir) : exp2f(pc.slope * __log2f(r));
  sig = fmaxf(sig, pc.sig_floor);
  float om, vk2;
  if (r >= pc.rs) {
    om = pc.sqk_out * ir * sqrtf(ir);  // v_phi / r = sqrt((1 + (s-1) h^2) / r) / r
    vk2 = ir;
  } else {
    om = pc.om_in;                     // solid-body core
    vk2 = r2 * pc.irs3;
  }
  b.sig = sig;
  b.vx = -om * y;
  b.vy = om * x;
  b.mx = sig * b.vx;
  b.my = sig * b.vy;
  b.c2 = pc.h2 * vk2;
  return b;
}

// flux differences f(u_b + d) - f(u_b) (isothermal, 3 variables)
__device__ __forceinline__ void dflux32(const Bg32& b, const float* d, float* fx, float* fy,
                                        float& vx, float& vy) {
  const float sg = b.sig + d[0];
  const float is = __frcp_rn(sg);
  const float dvx = (d[1] - b.vx * d[0]) * is;
  const float dvy = (d[2] - b.vy * d[0]) * is;
  vx = b.vx + dvx;
  vy = b.vy + dvy;
  const float dp = b.c2 * d[0];
  fx[0] = d[1];
  fx[1] = fmaf(d[1], vx, fmaf(b.mx, dvx, dp));
  fx[2] = fmaf(d[2], vx, b.my * dvx);
  fy[0] = d[2];
  fy[1] = fmaf(d[1], vy, b.mx * dvy);
  fy[2] = fmaf(d[2], vy, fmaf(b.my, dvy, dp));
}

// LLF flux difference through a face with normal +DIR, with background traces
// bL, bR on the two sides (equal for the analytic background).
template <int DIR>
__device__ __forceinline__ void dllf32(const Bg32& bL, const Bg32& bR, const float* dL,
                                       const float* dR, float* h) {
  float fxL[3], fyL[3], fxR[3], fyR[3], vxL, vyL, vxR, vyR;
  dflux32(bL, dL, fxL, fyL, vxL, vyL);
  dflux32(bR, dR, fxR, fyR, vxR, vyR);
  const float* fL = DIR == 0 ? fxL : fyL;
  const float* fR = DIR == 0 ? fxR : fyR;
  const float c = sqrtf(bL.c2);
  const float al = fmaxf(fabsf(DIR == 0 ? vxL : vyL), fabsf(DIR == 0 ? vxR : vyR)) + c;
  const float alb = fmaxf(fabsf(DIR == 0 ? bL.vx : bL.vy), fabsf(DIR == 0 ? bR.vx : bR.vy)) + c;
  const float jb[3] = {bR.sig - bL.sig, bR.mx - bL.mx, bR.my - bL.my};
#pragma unroll
  for (int v = 0; v < 3; v++)
    h[v] = 0.5f * (fL[v] + fR[v]) - 0.5f * fmaf(al, dR[v] - dL[v], (al - alb) * jb[v]);
}

// Exact projected background at a point of one element from its FP32 modes
// (stride 32 between modes): u_b = sum_ab b_ab fa[a] gb[b]; c2 from the
// analytic sound speed of the point.
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

// FP64 torque terms of the m nodes (xi_q, eta_r) of one element near the
// planet: node mass from the FP64 background modes plus the FP32 perturbation.
template <int P>
__device__ __noinline__ void torque_near64(const double* bg, const float* dsig, int q, double xcd,
                                           double ycd, double xp, double yp, double hdx,
                                           double hdy, double area, double eps2, double& gx,
                                           double& gy) {
  constexpr int m = P + 1;
  double t[m][m];  // t[a][r] = sum_b u_b,ab phi_b(eta_r)
#pragma unroll
  for (int aa = 0; aa < m; aa++)
#pragma unroll
    for (int r = 0; r < m; r++) {
      double acc = 0.0;
#pragma unroll
      for (int b = 0; b < m; b++) acc = fma(bg[(aa * m + b) * 32], c32_phi64[r][b], acc);
      t[aa][r] = acc;
    }
  const double ddx = xcd + hdx * c32_xi64[q] - xp;
#pragma unroll
  for (int r = 0; r < m; r++) {
    double sb = 0.0;
#pragma unroll
    for (int aa = 0; aa < m; aa++) sb = fma(c32_phi64[q][aa], t[aa][r], sb);
    const double mass = (sb + (double)dsig[r]) * c32_wh64[q] * c32_wh64[r] * area;
    const double ddy = ycd + hdy * c32_xi64[r] - yp;
    const double d2 = fma(ddx, ddx, fma(ddy, ddy, eps2));
    const double id = rsqrt(d2);
    const double f = mass * id * id * id;
    gx = fma(f, ddx, gx);
    gy = fma(f, ddy, gy);
  }
}

template <int P>
struct Smem32 {
  static constexpr int m = P + 1, M = m * m, NV = 3;
  static constexpr int C = 0;                      // delta^(s) of the tile [NV][M][32]
  static constexpr int T = C + NV * M * 32;        // T_a(r) / A_b(q)   [NV][m][m][32]
  static constexpr int B = T + NV * m * m * 32;    // B_b(q)            [NV][m][m][32]
  static constexpr int R = B + NV * m * m * 32;    // R+-, neighbours [4][NV][m][32]; x fluxes [NV][m][33]
  static constexpr int XR = R + 4 * NV * m * 32;   // right x traces [NV][m][33]; then HL
  static constexpr int XL = XR + NV * m * 33;      // left x traces  [NV][m][33]; then HR
  static constexpr int FYB = XL + NV * m * 33;
  static constexpr int FYT = FYB + NV * m * 32;
  static constexpr int H = FYT + NV * m * 32;      // x-halo coefficients [2][NV*M]
  static constexpr int FLAGS = H + 2 * NV * M;     // 32 ints
  static constexpr int TOTAL = FLAGS + 32;         // floats
  static constexpr int ND = 16 + 2 * m * 32;       // doubles: planet data, torque partials
  static constexpr size_t BYTES = (size_t)TOTAL * sizeof(float) + ND * sizeof(double);
};

// minimum resident CTAs per SM asked of the register allocator
#ifndef DG_STAGE32_MIN_CTAS
#define DG_STAGE32_MIN_CTAS 3
#endif

template <int P>
__global__ void __launch_bounds__(32 * (P + 1), DG_STAGE32_MIN_CTAS) k_stage32(const StageArgs32 a) {
  constexpr int m = P + 1, M = m * m, NV = 3, NT = 32 * m;
  constexpr int NVM = NV * M;
  using S = Smem32<P>;
  extern __shared__ double smd[];
  double* sD = smd;                       // [0..3] planet (stage, end); [16..] torque partials
  float* sF = reinterpret_cast<float*>(smd + 4);  // [0..3] tile offsets from the planets
  float* sm = reinterpret_cast<float*>(smd + S::ND);
  float* sC = sm + S::C;
  float* sT = sm + S::T;
  float* sB = sm + S::B;
  float* sR = sm + S::R;
  float* sFX = sm + S::R;
  float* sXR = sm + S::XR;
  float* sXL = sm + S::XL;
  float* sHL = sm + S::XR;
  float* sHR = sm + S::XL;
  float* sFYB = sm + S::FYB;
  float* sFYT = sm + S::FYT;
  float* sH = sm + S::H;
  int* sFlag = reinterpret_cast<int*>(sm + S::FLAGS);

  const Mesh& ms = a.mesh;
  const Prec32& pc = a.pc;
  if (a.ts->status != 0) return;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int bx = blockIdx.x, j = blockIdx.y;
  const int i0 = bx * 32;
  const int nvalid = min(32, ms.nx - i0);
  const bool valid = lane < nvalid;
  const int lc = valid ? lane : nvalid - 1;
  const double dtd = (a.fixed_dt > 0.0) ? a.fixed_dt : a.ts->dt;
  const float dt = (float)dtd;

  if (tid == 0) {
    // planet at the stage time and at t^{n+1}; centre of the tile's first
    // element relative to each, formed in FP64 and kept as a pair of floats
    // (hi, lo): a single rounding here would shift every element of the tile
    // row by the same amount, a correlated error the torque sum does not
    // average out
    const double tn = a.ts->t;
    const double xc0 = ms.x0 + (i0 + 0.5) * ms.dx, yc0 = ms.y0 + (j + 0.5) * ms.dy;
    double sn, cs;
    sincos(pc.omega_p * (tn + a.cstage * dtd) + pc.phi0, &sn, &cs);
    double ox = xc0 - pc.r_p * cs, oy = yc0 - pc.r_p * sn;
    sF[0] = (float)ox;
    sF[1] = (float)oy;
    sF[4] = (float)(ox - (double)sF[0]);
    sF[5] = (float)(oy - (double)sF[1]);
    sincos(pc.omega_p * (tn + dtd) + pc.phi0, &sn, &cs);
    sD[0] = pc.r_p * cs;
    sD[1] = pc.r_p * sn;
    ox = xc0 - sD[0];
    oy = yc0 - sD[1];
    sF[2] = (float)ox;
    sF[3] = (float)oy;
    sF[6] = (float)(ox - (double)sF[2]);
    sF[7] = (float)(oy - (double)sF[3]);
  }
  if (tid < 32) sFlag[tid] = 0;

  // ---- loads -----------------------------------------------------------------
  const size_t tile = (size_t)j * ms.ntx + bx;
  const float* Ut = a.D + tile * NVM * 32;
  for (int idx = tid; idx < NVM * 32; idx += NT) {
    const int l = idx & 31;
    sC[idx] = Ut[(l < nvalid) ? idx : idx - l + nvalid - 1];
  }
  // x neighbours: periodic wrap; bc 1 ghosts carry the background (delta = 0);
  // bc 2 transmissive mirrors the interior trace
  const int il = i0 - 1, ir = i0 + nvalid;
  const float* pL = nullptr;
  const float* pR = nullptr;
  bool zL = false, zR = false;
  if (il >= 0) pL = a.D + ((size_t)j * ms.ntx + (il >> 5)) * NVM * 32 + (il & 31);
  else if (ms.bc == 0) { const int iw = ms.nx - 1; pL = a.D + ((size_t)j * ms.ntx + (iw >> 5)) * NVM * 32 + (iw & 31); }
  else if (ms.bc == 1) zL = true;
  if (ir < ms.nx) pR = a.D + ((size_t)j * ms.ntx + (ir >> 5)) * NVM * 32 + (ir & 31);
  else if (ms.bc == 0) pR = a.D + (size_t)j * ms.ntx * NVM * 32;
  else if (ms.bc == 1) zR = true;
  const bool trL = (pL == nullptr) && !zL, trR = (pR == nullptr) && !zR;
  for (int idx = tid; idx < 2 * NVM; idx += NT) {
    const int side = idx >= NVM;
    const int vk = idx - side * NVM;
    const float* p = side ? pR : pL;
    sH[idx] = p ? p[(size_t)vk * 32] : 0.0f;
  }
  const float* pB = nullptr;
  const float* pT = nullptr;
  bool zB = false, zT = false;
  if (j > 0) pB = a.D + ((size_t)(j - 1) * ms.ntx + bx) * NVM * 32;
  else if (ms.bc == 0) pB = a.D + ((size_t)(ms.ny - 1) * ms.ntx + bx) * NVM * 32;
  else if (ms.bc == 1) zB = true;
  if (j + 1 < ms.ny) pT = a.D + ((size_t)(j + 1) * ms.ntx + bx) * NVM * 32;
  else if (ms.bc == 0) pT = a.D + (size_t)bx * NVM * 32;
  else if (ms.bc == 1) zT = true;
  const bool trB = (pB == nullptr) && !zB, trT = (pT == nullptr) && !zT;
  // tiles near the singular centre use the exact projected background (FP32
  // modes of u_b, same tiled layout as delta); all others the analytic one
  const int exact = a.TileFlag[tile];
  const float* bOwn = exact ? a.Bmodes + tile * NVM * 32 + lc : nullptr;
  const float* pLm = (exact && pL) ? a.Bmodes + (pL - a.D) : nullptr;
  const float* pRm = (exact && pR) ? a.Bmodes + (pR - a.D) : nullptr;
  const float* pBm = (exact && pB) ? a.Bmodes + (pB - a.D) : nullptr;
  const float* pTm = (exact && pT) ? a.Bmodes + (pT - a.D) : nullptr;
  // FP32 geometry of this thread's element
  const float xcf = pc.x0 + ((float)(i0 + lane) + 0.5f) * pc.dx;
  const float ycf = pc.y0 + ((float)j + 0.5f) * pc.dy;
  const float yBf = pc.y0 + (float)j * pc.dy, yTf = yBf + pc.dy;
  const float xt0 = pc.x0 + (float)i0 * pc.dx;
  __syncthreads();

  // ---- P1 ---------------------------------------------------------------------
  {
    const int aa = w;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      float c[m];
#pragma unroll
      for (int b = 0; b < m; b++) c[b] = sC[(v * M + aa * m + b) * 32 + lane];
#pragma unroll
      for (int r = 0; r < m; r++) {
        float acc = 0.0f;
#pragma unroll
        for (int b = 0; b < m; b++) acc = fmaf(c[b], c32_phi[r][b], acc);
        sT[((v * m + aa) * m + r) * 32 + lane] = acc;
      }
      float rp = 0.0f, rm = 0.0f;
#pragma unroll
      for (int b = 0; b < m; b++) {
        rp = fmaf(c[b], c32_pp[b], rp);
        rm = fmaf(c[b], c32_pm[b], rm);
      }
      sR[((0 * NV + v) * m + aa) * 32 + lane] = rp;
      sR[((1 * NV + v) * m + aa) * 32 + lane] = rm;
      float acc = 0.0f;
      if (pB) {
#pragma unroll
        for (int b = 0; b < m; b++) acc = fmaf(pB[(v * M + aa * m + b) * 32 + lc], c32_pp[b], acc);
      }
      sR[((2 * NV + v) * m + aa) * 32 + lane] = acc;
      acc = 0.0f;
      if (pT) {
#pragma unroll
        for (int b = 0; b < m; b++) acc = fmaf(pT[(v * M + aa * m + b) * 32 + lc], c32_pm[b], acc);
      }
      sR[((3 * NV + v) * m + aa) * 32 + lane] = acc;
    }
  }
  if (lane < 2) {
    const int r = w, side = lane;
    if ((side == 0 && !trL) || (side == 1 && !trR)) {
      const float* hc = sH + side * NVM;
#pragma unroll
      for (int v = 0; v < NV; v++) {
        float acc = 0.0f;
#pragma unroll
        for (int aa = 0; aa < m; aa++) {
          float t = 0.0f;
#pragma unroll
          for (int b = 0; b < m; b++) t = fmaf(hc[v * M + aa * m + b], c32_phi[r][b], t);
          acc = fmaf(side == 0 ? c32_pp[aa] : c32_pm[aa], t, acc);
        }
        if (side == 0) sXR[(v * m + r) * 33 + 0] = acc;
        else sXL[(v * m + r) * 33 + nvalid] = acc;
      }
    }
  }
  __syncthreads();

  // ---- P2 ---------------------------------------------------------------------
  float A[NV][m], Bv[NV][m];
  {
    const int q = w;
    float u[NV][m];
#pragma unroll
    for (int v = 0; v < NV; v++)
#pragma unroll
      for (int r = 0; r < m; r++) {
        float acc = 0.0f;
#pragma unroll
        for (int aa = 0; aa < m; aa++) acc = fmaf(c32_phi[q][aa], sT[((v * m + aa) * m + r) * 32 + lane], acc);
        u[v][r] = acc;
      }
#pragma unroll
    for (int v = 0; v < NV; v++) {
      float xr = 0.0f, xl = 0.0f;
#pragma unroll
      for (int aa = 0; aa < m; aa++) {
        const float t = sT[((v * m + aa) * m + w) * 32 + lane];
        xr = fmaf(c32_pp[aa], t, xr);
        xl = fmaf(c32_pm[aa], t, xl);
      }
      sXR[(v * m + w) * 33 + lane + 1] = xr;
      if (valid) sXL[(v * m + w) * 33 + lane] = xl;
      if (trL && lane == 0) sXR[(v * m + w) * 33 + 0] = xl;
      if (trR && lane == nvalid - 1) sXL[(v * m + w) * 33 + nvalid] = xr;
      if (zL && lane == 0) sXR[(v * m + w) * 33 + 0] = 0.0f;
      if (zR && lane == nvalid - 1) sXL[(v * m + w) * 33 + nvalid] = 0.0f;
    }
    const float xq = fmaf(pc.hdx, c32_xi[q], xcf);
    {
      float yt[NV], yb[NV], nb[NV], na[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) {
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
        for (int aa = 0; aa < m; aa++) {
          const float f = c32_phi[q][aa];
          s0 = fmaf(f, sR[((0 * NV + v) * m + aa) * 32 + lane], s0);
          s1 = fmaf(f, sR[((1 * NV + v) * m + aa) * 32 + lane], s1);
          s2 = fmaf(f, sR[((2 * NV + v) * m + aa) * 32 + lane], s2);
          s3 = fmaf(f, sR[((3 * NV + v) * m + aa) * 32 + lane], s3);
        }
        yt[v] = s0;
        yb[v] = s1;
        nb[v] = trB ? s1 : s2;  // zB: s2 = 0 (background ghost)
        na[v] = trT ? s0 : s3;
      }
      float hf[NV];
      {
        Bg32 bO = bg32_at(pc, xq, yBf), bN = bO;
        if (exact) {
          bO = bg32_poly<P>(bOwn, c32_phi[q], c32_pm, bO.c2);
          if (pBm) bN = bg32_poly<P>(pBm + lc, c32_phi[q], c32_pp, bO.c2);
          else if (trB) bN = bO;
        }
        dllf32<1>(bN, bO, nb, yb, hf);
      }
#pragma unroll
      for (int v = 0; v < NV; v++) sFYB[(v * m + q) * 32 + lane] = hf[v];
      {
        Bg32 bO = bg32_at(pc, xq, yTf), bN = bO;
        if (exact) {
          bO = bg32_poly<P>(bOwn, c32_phi[q], c32_pp, bO.c2);
          if (pTm) bN = bg32_poly<P>(pTm + lc, c32_phi[q], c32_pm, bO.c2);
          else if (trT) bN = bO;
        }
        dllf32<1>(bO, bN, yt, na, hf);
      }
#pragma unroll
      for (int v = 0; v < NV; v++) sFYT[(v * m + q) * 32 + lane] = hf[v];
    }
#pragma unroll
    for (int v = 0; v < NV; v++)
#pragma unroll
      for (int b = 0; b < m; b++) {
        A[v][b] = 0.0f;
        Bv[v][b] = 0.0f;
      }
    // node offsets from the planet at the stage time
    const float pdx = fmaf((float)lane, pc.dx, sF[0]) + fmaf(pc.hdx, c32_xi[q], sF[4]);
#pragma unroll
    for (int r = 0; r < m; r++) {
      const float y = fmaf(pc.hdy, c32_xi[r], ycf);
      Bg32 bgn = bg32_at(pc, xq, y);
      if (exact) bgn = bg32_poly<P>(bOwn, c32_phi[q], c32_phi[r], bgn.c2);
      float d[NV], fx[NV], fy[NV], vx, vy;
#pragma unroll
      for (int v = 0; v < NV; v++) d[v] = u[v][r];
      dflux32(bgn, d, fx, fy, vx, vy);
      // star: -dSigma grad Phi_*; planet: -Sigma grad Phi_p
      float src1 = 0.0f, src2 = 0.0f;
      if (pc.star) {
        const float r2 = fmaf(xq, xq, y * y);
        float inv;
        if (r2 >= pc.rs * pc.rs) {
          const float irr = rsqrtf(r2);
          inv = irr * irr * irr;
        } else {
          inv = pc.irs3;
        }
        src1 = -d[0] * xq * inv;
        src2 = -d[0] * y * inv;
      }
      if (pc.planet) {
        const float pdy = sF[1] + fmaf(pc.hdy, c32_xi[r], sF[5]);
        const float d2 = fmaf(pdx, pdx, fmaf(pdy, pdy, pc.eps2));
        const float id = rsqrtf(d2);
        const float f = pc.q * id * id * id * (bgn.sig + d[0]);
        src1 = fmaf(-f, pdx, src1);
        src2 = fmaf(-f, pdy, src2);
      }
#pragma unroll
      for (int v = 0; v < NV; v++) {
        const float fyy = fy[v] * pc.s2y;
#pragma unroll
        for (int b = 0; b < m; b++) {
          A[v][b] = fmaf(c32_wphi[r][b], fx[v], A[v][b]);
          Bv[v][b] = fmaf(c32_wdphi[r][b], fyy, Bv[v][b]);
        }
      }
#pragma unroll
      for (int b = 0; b < m; b++) {
        Bv[1][b] = fmaf(c32_wphi[r][b], src1, Bv[1][b]);
        Bv[2][b] = fmaf(c32_wphi[r][b], src2, Bv[2][b]);
      }
    }
  }
  __syncthreads();

  // ---- P2b: publish A, B; x-face fluxes ----------------------------------------
#pragma unroll
  for (int v = 0; v < NV; v++)
#pragma unroll
    for (int b = 0; b < m; b++) {
      sT[((v * m + b) * m + w) * 32 + lane] = A[v][b];
      sB[((v * m + b) * m + w) * 32 + lane] = Bv[v][b];
    }
  {
    const int r = w;
    const float y = fmaf(pc.hdy, c32_xi[r], ycf);
    for (int f = lane; f <= nvalid; f += 32) {
      float uL[NV], uR[NV], hf[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) {
        uL[v] = sXR[(v * m + r) * 33 + f];
        uR[v] = sXL[(v * m + r) * 33 + f];
      }
      Bg32 bL = bg32_at(pc, fmaf((float)f, pc.dx, xt0), y), bR = bL;
      if (exact) {
        // left element: lane f-1 or the left halo; right: lane f or the right halo
        const float* eL = (f > 0) ? bOwn - lc + (f - 1) : pLm;
        const float* eR = (f < nvalid) ? bOwn - lc + f : pRm;
        const float c2 = bL.c2;
        if (eL) bL = bg32_poly<P>(eL, c32_pp, c32_phi[r], c2);
        if (eR) bR = bg32_poly<P>(eR, c32_pm, c32_phi[r], c2);
        if (!eL && trL && f == 0) bL = bR;
        if (!eR && trR && f == nvalid) bR = bL;
      }
      dllf32<0>(bL, bR, uL, uR, hf);
#pragma unroll
      for (int v = 0; v < NV; v++) sFX[(v * m + r) * 33 + f] = hf[v];
    }
  }
  __syncthreads();

  // ---- P3 ---------------------------------------------------------------------
  const int aa = w;
  float L[NV][m];
  {
    const int b = w;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      float hl = 0.0f, hr = 0.0f;
#pragma unroll
      for (int r = 0; r < m; r++) {
        hl = fmaf(c32_wphi[r][b], sFX[(v * m + r) * 33 + lane], hl);
        hr = fmaf(c32_wphi[r][b], sFX[(v * m + r) * 33 + lane + 1], hr);
      }
      sHL[(v * m + b) * 32 + lane] = hl;
      sHR[(v * m + b) * 32 + lane] = hr;
    }
#pragma unroll
    for (int v = 0; v < NV; v++) {
      float ht = 0.0f, hb = 0.0f;
#pragma unroll
      for (int q = 0; q < m; q++) {
        ht = fmaf(c32_wphi[q][aa], sFYT[(v * m + q) * 32 + lane], ht);
        hb = fmaf(c32_wphi[q][aa], sFYB[(v * m + q) * 32 + lane], hb);
      }
#pragma unroll
      for (int bb = 0; bb < m; bb++) {
        float va = 0.0f, vb = 0.0f;
#pragma unroll
        for (int q = 0; q < m; q++) {
          va = fmaf(c32_wdphi[q][aa], sT[((v * m + bb) * m + q) * 32 + lane], va);
          vb = fmaf(c32_wphi[q][aa], sB[((v * m + bb) * m + q) * 32 + lane], vb);
        }
        L[v][bb] = fmaf(pc.s2x, va, vb) + pc.idy * (c32_pm[bb] * hb - c32_pp[bb] * ht);
      }
    }
  }
  // the background residual and u^n of this thread's modes, issued before the sync
  const size_t obase = tile * NVM * 32;
  float rb[NV][m], dn[NV][m];
#pragma unroll
  for (int v = 0; v < NV; v++)
#pragma unroll
    for (int bb = 0; bb < m; bb++) {
      const size_t idx = obase + (v * M + aa * m + bb) * 32 + lc;
      rb[v][bb] = a.Rb[idx];
      dn[v][bb] = (a.mode != 0 && a.alpha != 0.0f) ? a.Dn[idx] : 0.0f;
    }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; v++)
#pragma unroll
    for (int bb = 0; bb < m; bb++) {
      L[v][bb] += pc.idx * (c32_pm[aa] * sHL[(v * m + bb) * 32 + lane] - c32_pp[aa] * sHR[(v * m + bb) * 32 + lane]);
      L[v][bb] += rb[v][bb];
    }
  if (a.mode == 0) {
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; v++)
#pragma unroll
        for (int bb = 0; bb < m; bb++) a.Out[obase + (v * M + aa * m + bb) * 32 + lane] = L[v][bb];
    }
    return;
  }
  float un[NV][m];
#pragma unroll
  for (int v = 0; v < NV; v++)
#pragma unroll
    for (int bb = 0; bb < m; bb++) {
      const int idx = (v * M + aa * m + bb) * 32 + lane;
      un[v][bb] = fmaf(a.alpha, dn[v][bb], a.beta * fmaf(dt, L[v][bb], sC[idx]));
    }
  if (a.mode == 1) {
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; v++)
#pragma unroll
        for (int bb = 0; bb < m; bb++) a.Out[obase + (v * M + aa * m + bb) * 32 + lane] = un[v][bb];
    }
    return;
  }

  // ---- P4 (last stage): damping in delta form, torque, CFL ---------------------
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; v++)
#pragma unroll
    for (int bb = 0; bb < m; bb++) sC[(v * M + aa * m + bb) * 32 + lane] = un[v][bb];
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; v++) {
    float c[m];
#pragma unroll
    for (int b = 0; b < m; b++) c[b] = sC[(v * M + aa * m + b) * 32 + lane];
#pragma unroll
    for (int r = 0; r < m; r++) {
      float acc = 0.0f;
#pragma unroll
      for (int b = 0; b < m; b++) acc = fmaf(c[b], c32_phi[r][b], acc);
      sT[((v * m + aa) * m + r) * 32 + lane] = acc;
    }
  }
  __syncthreads();
  int damped = 0;
  {
    const int q = w;
    float u[NV][m];
#pragma unroll
    for (int v = 0; v < NV; v++)
#pragma unroll
      for (int r = 0; r < m; r++) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < m; k++) acc = fmaf(c32_phi[q][k], sT[((v * m + k) * m + r) * 32 + lane], acc);
        u[v][r] = acc;
      }
    const float xq = fmaf(pc.hdx, c32_xi[q], xcf);
    const bool zones = (pc.rd_in > 0.0f) || (pc.rd_out > 0.0f);
    const float* db = a.Db + tile * (size_t)(3 * M * 32);
#pragma unroll
    for (int r = 0; r < m; r++) {
      const float y = fmaf(pc.hdy, c32_xi[r], ycf);
      if (zones) {
        const float rr = sqrtf(fmaf(xq, xq, y * y));
        float R = 0.0f, rd = 0.0f;
        if (pc.rd_in > 0.0f && rr < pc.rd_in) {
          rd = pc.rd_in;
          const float x = (rr - rd) / (rd / pc.damp_ratio - rd);
          R = fminf(x * x, 1.0f);
        } else if (pc.rd_out > 0.0f && rr > pc.rd_out) {
          rd = pc.rd_out;
          const float x = (rr - rd) / (rd * pc.damp_ratio - rd);
          R = fminf(x * x, 1.0f);
        }
        if (R > 0.0f) {
          damped = 1;
          // Q_new = Q0 + kappa (Q - Q0), kappa = tau / (tau + dt), written for
          // delta Q = Q - Q_b: dQ_new = kappa dQ + (1 - kappa) (Q0 - Q_b)
          const float tau = 6.2831853071795864769f * sqrtf(rd * rd * rd) / R;
          const float kap = tau / (tau + dt), omk = dt / (tau + dt);
          Bg32 bgn = bg32_at(pc, xq, y);
          if (exact) bgn = bg32_poly<P>(bOwn, c32_phi[q], c32_phi[r], bgn.c2);
          const int nn = q * m + r;
          const float sg = bgn.sig + u[0][r];
          const float dvx = (u[1][r] - bgn.vx * u[0][r]) / sg;
          const float dvy = (u[2][r] - bgn.vy * u[0][r]) / sg;
          const float ds2 = fmaf(kap, u[0][r], omk * db[(0 * M + nn) * 32 + lc]);
          const float dvx2 = fmaf(kap, dvx, omk * db[(1 * M + nn) * 32 + lc]);
          const float dvy2 = fmaf(kap, dvy, omk * db[(2 * M + nn) * 32 + lc]);
          const float sg2 = bgn.sig + ds2;
          u[0][r] = ds2;
          u[1][r] = fmaf(ds2, bgn.vx, sg2 * dvx2);
          u[2][r] = fmaf(ds2, bgn.vy, sg2 * dvy2);
        }
      }
    }
    // torque on the planet at t^{n+1}.  Elements within sqrt(near2) of the
    // planet: FP64 terms from the FP64 background modes.  Beyond: unweighted
    // FP32 terms Sigma(node) (r_n - r_p) / (d^2 + eps^2)^(3/2) with a correctly
    // rounded rsqrt, summed over the 32 lanes per node class (q, r); the
    // quadrature weights w_q w_r |K| / 4 are applied to the class sums in FP64
    // once per CTA, so no rounding is shared by every element.
    double gxd = 0.0, gyd = 0.0;
    float fx[m], fy[m];
#pragma unroll
    for (int r = 0; r < m; r++) fx[r] = fy[r] = 0.0f;
    if (valid) {
      const float cdx = fmaf((float)lane, pc.dx, sF[2]), cdy = sF[3];
      if (fmaf(cdx, cdx, cdy * cdy) < pc.near2) {
        const double xcd = ms.x0 + (i0 + lane + 0.5) * ms.dx, ycd = ms.y0 + (j + 0.5) * ms.dy;
        torque_near64<P>(a.BG64 + tile * NVM * 32 + lane, u[0], q, xcd, ycd, sD[0], sD[1],
                         0.5 * ms.dx, 0.5 * ms.dy, ms.dx * ms.dy, pc.eps2_d, gxd, gyd);
      } else {
        const float* sbn = a.SigbN + tile * (size_t)(M * 32);
        const float pdx = cdx + fmaf(pc.hdx, c32_xi[q], sF[6]);
#pragma unroll
        for (int r = 0; r < m; r++) {
          const float sig = sbn[(q * m + r) * 32 + lane] + u[0][r];
          const float pdy = cdy + fmaf(pc.hdy, c32_xi[r], sF[7]);
          const float d2 = fmaf(pdx, pdx, fmaf(pdy, pdy, pc.eps2));
          const float id = __frsqrt_rn(d2);
          const float f = sig * (id * id * id);
          fx[r] = f * pdx;
          fy[r] = f * pdy;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < m; r++)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        fx[r] += __shfl_xor_sync(0xffffffffu, fx[r], o);
        fy[r] += __shfl_xor_sync(0xffffffffu, fy[r], o);
      }
    if (lane == 0) {
      // this warp's node classes (q, r), weighted in FP64
      const double wq = c32_wh64[q] * ms.dx * ms.dy;
#pragma unroll
      for (int r = 0; r < m; r++) {
        gxd += wq * c32_wh64[r] * (double)fx[r];
        gyd += wq * c32_wh64[r] * (double)fy[r];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gxd += __shfl_xor_sync(0xffffffffu, gxd, o);
      gyd += __shfl_xor_sync(0xffffffffu, gyd, o);
    }
    if (lane == 0) {
      sD[16 + w] = gxd;
      sD[16 + m + w] = gyd;
    }
    if (damped) sFlag[lane] = 1;
    if (__syncthreads_or(damped)) {
#pragma unroll
      for (int v = 0; v < NV; v++)
#pragma unroll
        for (int b = 0; b < m; b++) {
          float acc = 0.0f;
#pragma unroll
          for (int r = 0; r < m; r++) acc = fmaf(c32_wphi[r][b], u[v][r], acc);
          sB[((v * m + b) * m + q) * 32 + lane] = acc;
        }
      __syncthreads();
      if (sFlag[lane]) {
#pragma unroll
        for (int v = 0; v < NV; v++)
#pragma unroll
          for (int bb = 0; bb < m; bb++) {
            float acc = 0.0f;
#pragma unroll
            for (int qq = 0; qq < m; qq++) acc = fmaf(c32_wphi[qq][aa], sB[((v * m + bb) * m + qq) * 32 + lane], acc);
            un[v][bb] = acc;
          }
      }
    }
  }
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; v++)
#pragma unroll
      for (int bb = 0; bb < m; bb++) a.Out[obase + (v * M + aa * m + bb) * 32 + lane] = un[v][bb];
  }
  if (w == 0) {
    // CFL minimum of the new state (mode 0 of the full state), then the torque
    // partial of the CTA in a fixed order
    double dtk = __longlong_as_double(0x7ff0000000000000LL);
    int bad = 0;
    if (valid) {
      const float* b0 = a.Bm0 + tile * (size_t)(3 * 32);
      const float rho = b0[0 * 32 + lane] + un[0][0];
      const float irho = 1.0f / rho;
      const float vx = (b0[1 * 32 + lane] + un[1][0]) * irho, vy = (b0[2 * 32 + lane] + un[2][0]) * irho;
      const float c = sqrtf(bg32_at(pc, xcf, ycf).c2);
      const float dtf = pc.cfl_fac / ((fabsf(vx) + c) / pc.dx + (fabsf(vy) + c) / pc.dy);
      dtk = (double)dtf;
      bad = !(rho > 0.0f) || !(dtf > 0.0f) || !isfinite(dtf);
      if (bad) dtk = __longlong_as_double(0x7ff0000000000000LL);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dtk = fmin(dtk, __shfl_xor_sync(0xffffffffu, dtk, o));
      bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
      if (bad) atomicOr(&a.ts->pending, 1);
      atomicMin(&a.ts->dt_bits, (unsigned long long)__double_as_longlong(dtk));
    }
  }
  __syncthreads();
  if (tid == 0) {
    double gx = 0.0, gy = 0.0;
#pragma unroll
    for (int k = 0; k < m; k++) {
      gx += sD[16 + k];
      gy += sD[16 + m + k];
    }
    a.part[2 * tile] = gx;
    a.part[2 * tile + 1] = gy;
  }
}

template <int P>
cudaError_t launch_stage32_impl(const StageArgs32& a, cudaStream_t s) {
  static bool configured = false;
  const size_t bytes = Smem32<P>::BYTES;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_stage32<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid(a.mesh.ntx, a.mesh.ny);
  k_stage32<P><<<grid, 32 * (P + 1), bytes, s>>>(a);
  return cudaGetLastError();
}

template <int P>
cudaError_t upload_tables32_impl(const Tables& t) {
  float phi[MAXM][MAXM] = {}, wphi[MAXM][MAXM] = {}, wdphi[MAXM][MAXM] = {};
  float pp[MAXM] = {}, pm[MAXM] = {}, xi[MAXM] = {}, wh[MAXM] = {};
  for (int q = 0; q <= P; q++) {
    xi[q] = (float)t.xi[q];
    wh[q] = (float)t.wh[q];
    pp[q] = (float)t.pp[q];
    pm[q] = (float)t.pm[q];
    for (int a = 0; a <= P; a++) {
      phi[q][a] = (float)t.phi[q][a];
      wphi[q][a] = (float)(t.wh[q] * t.phi[q][a]);
      wdphi[q][a] = (float)(t.wh[q] * t.dphi[q][a]);
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c32_phi, phi, sizeof(phi));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c32_wphi, wphi, sizeof(wphi));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c32_wdphi, wdphi, sizeof(wdphi));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c32_pp, pp, sizeof(pp));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c32_pm, pm, sizeof(pm));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c32_xi, xi, sizeof(xi));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c32_wh, wh, sizeof(wh));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c32_phi64, t.phi, sizeof(t.phi));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c32_xi64, t.xi, sizeof(t.xi));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c32_wh64, t.wh, sizeof(t.wh));
  return e;
}

}  // namespace dg
