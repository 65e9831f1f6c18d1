// dg_stage.cuh -- fused RK-stage kernel of the DG operator (Eq. 2 of
// arXiv:1805.01443), included once per polynomial degree by dg_stage_p{P}.cu
// with DG_P defined.
//
// One CTA = one tile of 32 elements of one mesh row, m = p+1 warps.  Thread
// (warp w, lane e) owns element e of the tile and, depending on the phase, the
// x-mode a = w, the x-node q = w or the y-node r = w of that element.  The
// modal <-> nodal contractions are sum-factorised (two passes of m^3 per
// variable, Sec. 2.2 tensor-product basis), intermediate results move between
// phases through shared memory, and every face flux is computed once per CTA:
//
//   S0  load u^(s) of the tile (coalesced 256 B rows), the two x-neighbour
//       elements, and collapse the y-neighbours to their face polynomials
//   P1  T_a(eta_r) = sum_b u_ab phi_b(eta_r); R^+-_a = sum_b u_ab phi_b(+-1)
//   P2  nodal values u(xi_q, eta_r), x traces, y traces and the two y-face
//       LLF fluxes; f_x, f_y, S at the nodes folded into the first pass of the
//       volume integral (A_b(q), B_b(q))
//   P3  x-face LLF fluxes; second pass of the volume integral; surface lift;
//       Shu-Osher combination u_new = alpha u^n + beta (u^(s) + dt L)
//   P4  (last stage) damping zones at the nodes (Sec. 5.1), per-CTA torque
//       partial on the new state (Sec. 5.2), per-CTA CFL minimum (Sec. 2.3)
#pragma once
#include "dg_internal.cuh"
#include "dg_physics.cuh"

#ifndef DG_P
#error "define DG_P before including dg_stage.cuh"
#endif

namespace dg {

// Per-translation-unit copy of the quadrature/basis tables of degree DG_P.
static __constant__ Tables c_tab;
// w_q/2 * phi_a(xi_q) and w_q/2 * phi'_a(xi_q), [q][a]
static __constant__ double c_wphi[MAXM][MAXM];
static __constant__ double c_wdphi[MAXM][MAXM];

template <int KIND>
struct NVar {
  static constexpr int value = (KIND == 1) ? 4 : 3;
};

// Isothermal sound speed squared at (x, y): kind 2 constant h^2, kind 0
// h^2 v_K^2 with v_K^2 = r dPhi_s/dr of the softened star (1/r outside r_s,
// r^2/r_s^3 inside).
template <int KIND>
__device__ __forceinline__ double cs2_at(const Phys& ph, double x, double y) {
  if (KIND == 2) return ph.h * ph.h;
  if (KIND == 1) return 0.0;
  double r2 = x * x + y * y;
  double r = sqrt(r2);
  double vk2 = (r >= ph.rs) ? 1.0 / r : r2 / (ph.rs * ph.rs * ph.rs);
  return ph.h * ph.h * vk2;
}

// Physical fluxes f_x, f_y of Eq. 1.
template <int KIND>
__device__ __forceinline__ void phys_flux(const double* u, double cs2, double gam, double* fx,
                                          double* fy) {
  const double rho = u[0], mx = u[1], my = u[2];
  const double ir = 1.0 / rho;
  const double vx = mx * ir, vy = my * ir;
  double p;
  if (KIND == 1)
    p = (gam - 1.0) * (u[3] - 0.5 * (mx * vx + my * vy));
  else
    p = cs2 * rho;
  fx[0] = mx;
  fx[1] = fma(mx, vx, p);
  fx[2] = my * vx;
  fy[0] = my;
  fy[1] = mx * vy;
  fy[2] = fma(my, vy, p);
  if (KIND == 1) {
    fx[3] = (u[3] + p) * vx;
    fy[3] = (u[3] + p) * vy;
  }
}

// Local Lax-Friedrichs flux through a face with normal +DIR (0: x, 1: y):
// h = (f(uL) + f(uR))/2 - alpha (uR - uL)/2, alpha = max(|v_n| + c) of the two sides.
template <int KIND, int DIR>
__device__ __forceinline__ void llf(const double* uL, const double* uR, double cs2, double cs, double gam,
                                    double* h) {
  constexpr int NV = NVar<KIND>::value;
  double f[2][NV], s[2];
  const double* us[2] = {uL, uR};
#pragma unroll
  for (int side = 0; side < 2; side++) {
    const double* u = us[side];
    const double rho = u[0], mx = u[1], my = u[2];
    const double ir = 1.0 / rho;
    const double vx = mx * ir, vy = my * ir;
    double p, c2;
    if (KIND == 1) {
      p = (gam - 1.0) * (u[3] - 0.5 * (mx * vx + my * vy));
      c2 = gam * p * ir;
    } else {
      p = cs2 * rho;
      c2 = cs2;
    }
    const double vn = DIR == 0 ? vx : vy;
    f[side][0] = DIR == 0 ? mx : my;
    f[side][1] = DIR == 0 ? fma(mx, vx, p) : mx * vy;
    f[side][2] = DIR == 0 ? my * vx : fma(my, vy, p);
    if (KIND == 1) f[side][3] = (u[3] + p) * vn;
    s[side] = fabs(vn) + (KIND == 1 ? sqrt(c2) : cs);
  }
  const double al = fmax(s[0], s[1]);
#pragma unroll
  for (int v = 0; v < NV; v++) h[v] = 0.5 * (f[0][v] + f[1][v]) - 0.5 * al * (uR[v] - uL[v]);
}

// grad(Phi_* + Phi_p) at (x, y): softened star (solid-body core inside r_s)
// plus Plummer planet at (px, py).
__device__ __forceinline__ void grad_star(const Phys& ph, double x, double y, double& gx, double& gy) {
  gx = 0.0;
  gy = 0.0;
  if (ph.star) {
    double r2 = x * x + y * y;
    double inv;
    if (r2 >= ph.rs * ph.rs) {
      double ir = rsqrt(r2);
      inv = ir * ir * ir;
    } else {
      inv = 1.0 / (ph.rs * ph.rs * ph.rs);
    }
    gx = x * inv;
    gy = y * inv;
  }
}
__device__ __forceinline__ void grad_planet(const Phys& ph, double x, double y, double px, double py,
                                            double& gx, double& gy) {
  if (ph.planet) {
    double ddx = x - px, ddy = y - py;
    double d2 = fma(ddx, ddx, fma(ddy, ddy, ph.eps2));
    double id = rsqrt(d2);
    double f = ph.q * id * id * id;
    gx = fma(f, ddx, gx);
    gy = fma(f, ddy, gy);
  }
}

// Shared-memory plan (doubles) of the stage kernel.
template <int P, int KIND>
struct Smem {
  static constexpr int m = P + 1, M = m * m, NV = NVar<KIND>::value;
  static constexpr int C = 0;                      // u^(s) of the tile [NV][M][32]
  static constexpr int T = C + NV * M * 32;        // T_a(r) / A_b(q)   [NV][m][m][32]
  static constexpr int B = T + NV * m * m * 32;    // B_b(q)            [NV][m][m][32]
  static constexpr int R = B + NV * m * m * 32;    // R+-, neighbours   [4][NV][m][32]; then x fluxes [NV][m][33]
  static constexpr int XR = R + 4 * NV * m * 32;   // right x traces    [NV][m][33]; then HL [NV][m][32]
  static constexpr int XL = XR + NV * m * 33;      // left x traces     [NV][m][33]; then HR [NV][m][32]
  static constexpr int FYB = XL + NV * m * 33;     // bottom y fluxes   [NV][m][32]
  static constexpr int FYT = FYB + NV * m * 32;    // top y fluxes      [NV][m][32]
  static constexpr int H = FYT + NV * m * 32;      // x-halo coefficients [2][NV*M]
  static constexpr int MISC = H + 2 * NV * M;      // planet positions, warp partials (16)
  static constexpr int FLAGS = MISC + 16;          // 32 ints
  static constexpr int TOTAL = FLAGS + 16;
  static constexpr size_t BYTES = (size_t)TOTAL * sizeof(double);
};

template <int P, int KIND>
__global__ void __launch_bounds__(32 * (P + 1)) k_stage(const StageArgs a) {
  constexpr int m = P + 1, M = m * m, NV = NVar<KIND>::value, NT = 32 * m;
  constexpr int NVM = NV * M;
  using S = Smem<P, KIND>;
  extern __shared__ double sm[];
  double* sC = sm + S::C;
  double* sT = sm + S::T;
  double* sB = sm + S::B;
  double* sR = sm + S::R;
  double* sFX = sm + S::R;
  double* sXR = sm + S::XR;
  double* sXL = sm + S::XL;
  double* sHL = sm + S::XR;
  double* sHR = sm + S::XL;
  double* sFYB = sm + S::FYB;
  double* sFYT = sm + S::FYT;
  double* sH = sm + S::H;
  double* sMisc = sm + S::MISC;
  int* sFlag = reinterpret_cast<int*>(sm + S::FLAGS);

  const Mesh& ms = a.mesh;
  const Phys& ph = a.phys;
  if (a.ts->status != 0) return;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int bx = blockIdx.x, j = blockIdx.y;
  const int i0 = bx * 32;
  const int nvalid = min(32, ms.nx - i0);
  const bool valid = lane < nvalid;
  const int lc = valid ? lane : nvalid - 1;
  const double dt = (a.fixed_dt > 0.0) ? a.fixed_dt : a.ts->dt;
  const double tn = a.ts->t;

  if (tid == 0) {
    double sn, cs;
    sincos(ph.omega_p * (tn + a.cstage * dt) + ph.phi0, &sn, &cs);
    sMisc[0] = ph.r_p * cs;
    sMisc[1] = ph.r_p * sn;
    sincos(ph.omega_p * (tn + dt) + ph.phi0, &sn, &cs);
    sMisc[2] = ph.r_p * cs;
    sMisc[3] = ph.r_p * sn;
  }
  if (tid < 32) sFlag[tid] = 0;

  // ---- S0: loads -----------------------------------------------------------
  const size_t tile = (size_t)j * ms.ntx + bx;
  const double* Ut = a.U + tile * NVM * 32;
  for (int idx = tid; idx < NVM * 32; idx += NT) {
    const int l = idx & 31;
    sC[idx] = Ut[(l < nvalid) ? idx : idx - l + nvalid - 1];
  }
  // x neighbours of the tile (periodic wrap, ghost column, transmissive, or
  // the zero-gradient copy of the boundary element)
  const int il = i0 - 1, ir = i0 + nvalid;
  const double* pL = nullptr;
  const double* pR = nullptr;
  int stL = 32, stR = 32;
  if (il >= 0) {
    pL = a.U + ((size_t)j * ms.ntx + (il >> 5)) * NVM * 32 + (il & 31);
  } else if (ms.bc == 0) {
    const int iw = ms.nx - 1;
    pL = a.U + ((size_t)j * ms.ntx + (iw >> 5)) * NVM * 32 + (iw & 31);
  } else if (ms.bc == 1) {
    pL = a.GL + (size_t)j * NVM;
    stL = 1;
  } else if (ms.bc == 3) {  // zero-gradient ghost: a copy of the boundary element
    pL = a.U + (size_t)j * ms.ntx * NVM * 32;
  }
  if (ir < ms.nx) {
    pR = a.U + ((size_t)j * ms.ntx + (ir >> 5)) * NVM * 32 + (ir & 31);
  } else if (ms.bc == 0) {
    pR = a.U + (size_t)j * ms.ntx * NVM * 32;
  } else if (ms.bc == 1) {
    pR = a.GR + (size_t)j * NVM;
    stR = 1;
  } else if (ms.bc == 3) {
    const int ie = ms.nx - 1;
    pR = a.U + ((size_t)j * ms.ntx + (ie >> 5)) * NVM * 32 + (ie & 31);
  }
  const bool trL = (pL == nullptr), trR = (pR == nullptr);
  for (int idx = tid; idx < 2 * NVM; idx += NT) {
    const int side = idx >= NVM;
    const int vk = idx - side * NVM;
    const double* p = side ? pR : pL;
    if (p) sH[idx] = p[(size_t)vk * (side ? stR : stL)];
  }
  // y neighbours: rows j-1 and j+1 of the same tile column (tiled, stride 32)
  const double* pB = nullptr;
  const double* pT = nullptr;
  if (j > 0)
    pB = a.U + ((size_t)(j - 1) * ms.ntx + bx) * NVM * 32;
  else if (ms.bc == 0)
    pB = a.U + ((size_t)(ms.ny - 1) * ms.ntx + bx) * NVM * 32;
  else if (ms.bc == 1)
    pB = a.GB + (size_t)bx * NVM * 32;
  else if (ms.bc == 3)
    pB = Ut;
  if (j + 1 < ms.ny)
    pT = a.U + ((size_t)(j + 1) * ms.ntx + bx) * NVM * 32;
  else if (ms.bc == 0)
    pT = a.U + (size_t)bx * NVM * 32;
  else if (ms.bc == 1)
    pT = a.GT + (size_t)bx * NVM * 32;
  else if (ms.bc == 3)
    pT = Ut;
  const bool trB = (pB == nullptr), trT = (pT == nullptr);
  __syncthreads();

  // ---- P1: first modal->nodal pass, face collapses ----------------------------
  {
    const int aa = w;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      double c[m];
#pragma unroll
      for (int b = 0; b < m; b++) c[b] = sC[(v * M + aa * m + b) * 32 + lane];
#pragma unroll
      for (int r = 0; r < m; r++) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < m; b++) acc = fma(c[b], c_tab.phi[r][b], acc);
        sT[((v * m + aa) * m + r) * 32 + lane] = acc;
      }
      double rp = 0.0, rm = 0.0;
#pragma unroll
      for (int b = 0; b < m; b++) {
        rp = fma(c[b], c_tab.pp[b], rp);
        rm = fma(c[b], c_tab.pm[b], rm);
      }
      sR[((0 * NV + v) * m + aa) * 32 + lane] = rp;
      sR[((1 * NV + v) * m + aa) * 32 + lane] = rm;
      if (!trB) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < m; b++) acc = fma(pB[(v * M + aa * m + b) * 32 + lc], c_tab.pp[b], acc);
        sR[((2 * NV + v) * m + aa) * 32 + lane] = acc;
      }
      if (!trT) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < m; b++) acc = fma(pT[(v * M + aa * m + b) * 32 + lc], c_tab.pm[b], acc);
        sR[((3 * NV + v) * m + aa) * 32 + lane] = acc;
      }
    }
  }
  // traces of the x-halo elements at y-node r = w: lane 0 the left halo's
  // right trace, lane 1 the right halo's left trace
  if (lane < 2) {
    const int r = w, side = lane;
    if ((side == 0 && !trL) || (side == 1 && !trR)) {
      const double* hc = sH + side * NVM;
#pragma unroll
      for (int v = 0; v < NV; v++) {
        double acc = 0.0;
#pragma unroll
        for (int aa = 0; aa < m; aa++) {
          double t = 0.0;
#pragma unroll
          for (int b = 0; b < m; b++) t = fma(hc[v * M + aa * m + b], c_tab.phi[r][b], t);
          acc = fma(side == 0 ? c_tab.pp[aa] : c_tab.pm[aa], t, acc);
        }
        if (side == 0)
          sXR[(v * m + r) * 33 + 0] = acc;
        else
          sXL[(v * m + r) * 33 + nvalid] = acc;
      }
    }
  }
  __syncthreads();

  // ---- P2: nodal values, traces, y fluxes, pointwise flux and source -------------
  double A[NV][m], Bv[NV][m];
  {
    const int q = w;
    double u[NV][m];
#pragma unroll
    for (int v = 0; v < NV; v++)
#pragma unroll
      for (int r = 0; r < m; r++) {
        double acc = 0.0;
#pragma unroll
        for (int aa = 0; aa < m; aa++) acc = fma(c_tab.phi[q][aa], sT[((v * m + aa) * m + r) * 32 + lane], acc);
        u[v][r] = acc;
      }
    // x traces at y-node r = w
#pragma unroll
    for (int v = 0; v < NV; v++) {
      double xr = 0.0, xl = 0.0;
#pragma unroll
      for (int aa = 0; aa < m; aa++) {
        const double t = sT[((v * m + aa) * m + w) * 32 + lane];
        xr = fma(c_tab.pp[aa], t, xr);
        xl = fma(c_tab.pm[aa], t, xl);
      }
      sXR[(v * m + w) * 33 + lane + 1] = xr;
      if (valid) sXL[(v * m + w) * 33 + lane] = xl;
      if (trL && lane == 0) sXR[(v * m + w) * 33 + 0] = xl;
      if (trR && lane == nvalid - 1) sXL[(v * m + w) * 33 + nvalid] = xr;
    }
    // y traces at x-node q and the bottom/top y-face fluxes
    const double xq = ms.x0 + (i0 + lane + 0.5) * ms.dx + 0.5 * ms.dx * c_tab.xi[q];
    {
      double yt[NV], yb[NV], nb[NV], na[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
        for (int aa = 0; aa < m; aa++) {
          const double f = c_tab.phi[q][aa];
          s0 = fma(f, sR[((0 * NV + v) * m + aa) * 32 + lane], s0);
          s1 = fma(f, sR[((1 * NV + v) * m + aa) * 32 + lane], s1);
          if (!trB) s2 = fma(f, sR[((2 * NV + v) * m + aa) * 32 + lane], s2);
          if (!trT) s3 = fma(f, sR[((3 * NV + v) * m + aa) * 32 + lane], s3);
        }
        yt[v] = s0;
        yb[v] = s1;
        nb[v] = trB ? s1 : s2;
        na[v] = trT ? s0 : s3;
      }
      double hf[NV];
      double c2b, cb, c2t, ct;
      if (KIND == 0 && a.SYF) {
        const size_t o = ((size_t)j * ms.nx + i0 + lc) * m + q;
        const size_t stride = (size_t)ms.nx * m;
        c2b = a.SYF[2 * o];
        cb = a.SYF[2 * o + 1];
        c2t = a.SYF[2 * (o + stride)];
        ct = a.SYF[2 * (o + stride) + 1];
      } else {
        c2b = cs2_at<KIND>(ph, xq, ms.y0 + j * ms.dy);
        cb = sqrt(c2b);
        c2t = cs2_at<KIND>(ph, xq, ms.y0 + (j + 1) * ms.dy);
        ct = sqrt(c2t);
      }
      llf<KIND, 1>(nb, yb, c2b, cb, ph.gamma, hf);
#pragma unroll
      for (int v = 0; v < NV; v++) sFYB[(v * m + q) * 32 + lane] = hf[v];
      llf<KIND, 1>(yt, na, c2t, ct, ph.gamma, hf);
#pragma unroll
      for (int v = 0; v < NV; v++) sFYT[(v * m + q) * 32 + lane] = hf[v];
    }
    // volume: f_x, f_y and S at the nodes (xi_q, eta_r), first contraction over r
#pragma unroll
    for (int v = 0; v < NV; v++)
#pragma unroll
      for (int b = 0; b < m; b++) {
        A[v][b] = 0.0;
        Bv[v][b] = 0.0;
      }
    const double yc = ms.y0 + (j + 0.5) * ms.dy;
    const double px = sMisc[0], py = sMisc[1];
    const double s2y = 2.0 / ms.dy;
#pragma unroll
    for (int r = 0; r < m; r++) {
      const double y = yc + 0.5 * ms.dy * c_tab.xi[r];
      double uu[NV], fx[NV], fy[NV], src[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) uu[v] = u[v][r];
      double gx, gy, c2n;
      if (KIND == 0 && a.SN) {
        const double* sn = a.SN + tile * 3 * M * 32 + (size_t)(q * m + r) * 32 + lane;
        c2n = sn[0];
        gx = sn[M * 32];
        gy = sn[2 * M * 32];
      } else {
        c2n = cs2_at<KIND>(ph, xq, y);
        grad_star(ph, xq, y, gx, gy);
      }
      phys_flux<KIND>(uu, c2n, ph.gamma, fx, fy);
      grad_planet(ph, xq, y, px, py, gx, gy);
      src[0] = 0.0;
      src[1] = -uu[0] * gx;
      src[2] = -uu[0] * gy;
      if (NV == 4) src[NV - 1] = -(uu[1] * gx + uu[2] * gy);
#pragma unroll
      for (int v = 0; v < NV; v++) {
        const double fyy = fy[v] * s2y;
#pragma unroll
        for (int b = 0; b < m; b++) {
          A[v][b] = fma(c_wphi[r][b], fx[v], A[v][b]);
          Bv[v][b] = fma(c_wdphi[r][b], fyy, Bv[v][b]);
          if (v > 0) Bv[v][b] = fma(c_wphi[r][b], src[v], Bv[v][b]);
        }
      }
    }
  }
  __syncthreads();

  // ---- P2b: publish A, B; x-face fluxes -----------------------------------------
#pragma unroll
  for (int v = 0; v < NV; v++)
#pragma unroll
    for (int b = 0; b < m; b++) {
      sT[((v * m + b) * m + w) * 32 + lane] = A[v][b];
      sB[((v * m + b) * m + w) * 32 + lane] = Bv[v][b];
    }
  {
    const int r = w;
    const double y = ms.y0 + (j + 0.5) * ms.dy + 0.5 * ms.dy * c_tab.xi[r];
    for (int f = lane; f <= nvalid; f += 32) {
      double uL[NV], uR[NV], hf[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) {
        uL[v] = sXR[(v * m + r) * 33 + f];
        uR[v] = sXL[(v * m + r) * 33 + f];
      }
      double c2f, cf;
      if (KIND == 0 && a.SXF) {
        const size_t o = ((size_t)j * m + r) * (ms.nx + 1) + i0 + f;
        c2f = a.SXF[2 * o];
        cf = a.SXF[2 * o + 1];
      } else {
        c2f = cs2_at<KIND>(ph, ms.x0 + (i0 + f) * ms.dx, y);
        cf = sqrt(c2f);
      }
      llf<KIND, 0>(uL, uR, c2f, cf, ph.gamma, hf);
#pragma unroll
      for (int v = 0; v < NV; v++) sFX[(v * m + r) * 33 + f] = hf[v];
    }
  }
  __syncthreads();

  // ---- P3: second volume pass, lift ------------------------------------------
  const int aa = w;
  double L[NV][m];
  {
    const int b = w;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      double hl = 0.0, hr = 0.0;
#pragma unroll
      for (int r = 0; r < m; r++) {
        hl = fma(c_wphi[r][b], sFX[(v * m + r) * 33 + lane], hl);
        hr = fma(c_wphi[r][b], sFX[(v * m + r) * 33 + lane + 1], hr);
      }
      sHL[(v * m + b) * 32 + lane] = hl;
      sHR[(v * m + b) * 32 + lane] = hr;
    }
    const double s2x = 2.0 / ms.dx, idy = 1.0 / ms.dy;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      double ht = 0.0, hb = 0.0;
#pragma unroll
      for (int q = 0; q < m; q++) {
        ht = fma(c_wphi[q][aa], sFYT[(v * m + q) * 32 + lane], ht);
        hb = fma(c_wphi[q][aa], sFYB[(v * m + q) * 32 + lane], hb);
      }
#pragma unroll
      for (int bb = 0; bb < m; bb++) {
        double va = 0.0, vb = 0.0;
#pragma unroll
        for (int q = 0; q < m; q++) {
          va = fma(c_wdphi[q][aa], sT[((v * m + bb) * m + q) * 32 + lane], va);
          vb = fma(c_wphi[q][aa], sB[((v * m + bb) * m + q) * 32 + lane], vb);
        }
        L[v][bb] = fma(s2x, va, vb) + idy * (c_tab.pm[bb] * hb - c_tab.pp[bb] * ht);
      }
    }
  }
  __syncthreads();
  {
    const double idx_ = 1.0 / ms.dx;
#pragma unroll
    for (int v = 0; v < NV; v++)
#pragma unroll
      for (int bb = 0; bb < m; bb++)
        L[v][bb] += idx_ * (c_tab.pm[aa] * sHL[(v * m + bb) * 32 + lane] -
                            c_tab.pp[aa] * sHR[(v * m + bb) * 32 + lane]);
  }

  const size_t obase = tile * NVM * 32;
  if (a.mode == 0) {
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; v++)
#pragma unroll
        for (int bb = 0; bb < m; bb++) a.Out[obase + (v * M + aa * m + bb) * 32 + lane] = L[v][bb];
    }
    return;
  }

  // Shu-Osher combination
  double un[NV][m];
#pragma unroll
  for (int v = 0; v < NV; v++)
#pragma unroll
    for (int bb = 0; bb < m; bb++) {
      const int idx = (v * M + aa * m + bb) * 32 + lane;
      const double us = fma(dt, L[v][bb], sC[idx]);
      double r = a.beta * us;
      if (a.alpha != 0.0 && valid) r = fma(a.alpha, a.Un[obase + idx], r);
      un[v][bb] = r;
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

  // ---- P4 (last stage): damping, torque partial, CFL ---------------------------
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; v++)
#pragma unroll
    for (int bb = 0; bb < m; bb++) sC[(v * M + aa * m + bb) * 32 + lane] = un[v][bb];
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; v++) {
    double c[m];
#pragma unroll
    for (int b = 0; b < m; b++) c[b] = sC[(v * M + aa * m + b) * 32 + lane];
#pragma unroll
    for (int r = 0; r < m; r++) {
      double acc = 0.0;
#pragma unroll
      for (int b = 0; b < m; b++) acc = fma(c[b], c_tab.phi[r][b], acc);
      sT[((v * m + aa) * m + r) * 32 + lane] = acc;
    }
  }
  __syncthreads();
  int damped = 0;
  double gxs = 0.0, gys = 0.0;
  {
    const int q = w;
    double u[NV][m];
#pragma unroll
    for (int v = 0; v < NV; v++)
#pragma unroll
      for (int r = 0; r < m; r++) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < m; k++) acc = fma(c_tab.phi[q][k], sT[((v * m + k) * m + r) * 32 + lane], acc);
        u[v][r] = acc;
      }
    const double xq = ms.x0 + (i0 + lane + 0.5) * ms.dx + 0.5 * ms.dx * c_tab.xi[q];
    const double yc = ms.y0 + (j + 0.5) * ms.dy;
    const bool zones = (ph.rd_in > 0.0) || (ph.rd_out > 0.0);
#pragma unroll
    for (int r = 0; r < m; r++) {
      const double y = yc + 0.5 * ms.dy * c_tab.xi[r];
      if (zones) {
        const double rr = sqrt(xq * xq + y * y);
        double R = 0.0, rd = 0.0;
        if (ph.rd_in > 0.0 && rr < ph.rd_in) {
          rd = ph.rd_in;
          const double rb = rd / ph.damp_ratio, x = (rr - rd) / (rb - rd);
          R = fmin(x * x, 1.0);
        } else if (ph.rd_out > 0.0 && rr > ph.rd_out) {
          rd = ph.rd_out;
          const double rb = rd * ph.damp_ratio, x = (rr - rd) / (rb - rd);
          R = fmin(x * x, 1.0);
        }
        if (R > 0.0) {
          damped = 1;
          const double tau = 6.283185307179586476925286766559 * sqrt(rd * rd * rd) / R;
          double w0[4];
          ic_prim(ph, ms, xq, y, w0);
          const double rho = u[0][r];
          double Q[4] = {rho, u[1][r] / rho, u[2][r] / rho, 0.0};
          double Q0[4] = {w0[0], w0[1], w0[2], 0.0};
          if (NV == 4) {
            const double p = (ph.gamma - 1.0) * (u[NV - 1][r] - 0.5 * (u[1][r] * Q[1] + u[2][r] * Q[2]));
            Q[3] = p / rho;
            Q0[3] = w0[3] / w0[0];
          }
#pragma unroll
          for (int v = 0; v < NV; v++) Q[v] = (dt * Q0[v] + tau * Q[v]) / (tau + dt);
          u[0][r] = Q[0];
          u[1][r] = Q[0] * Q[1];
          u[2][r] = Q[0] * Q[2];
          if (NV == 4)
            u[NV - 1][r] = Q[3] * Q[0] / (ph.gamma - 1.0) + 0.5 * Q[0] * (Q[1] * Q[1] + Q[2] * Q[2]);
        }
      }
      if (valid) {
        // torque on the planet at t^{n+1} from the node masses
        const double mass = u[0][r] * c_tab.wh[q] * c_tab.wh[r] * ms.dx * ms.dy;
        const double ddx = xq - sMisc[2], ddy = y - sMisc[3];
        const double d2 = fma(ddx, ddx, fma(ddy, ddy, ph.eps2));
        const double id = rsqrt(d2);
        const double f = mass * id * id * id;
        gxs = fma(f, ddx, gxs);
        gys = fma(f, ddy, gys);
      }
    }
    if (damped) sFlag[lane] = 1;
    if (__syncthreads_or(damped)) {
#pragma unroll
      for (int v = 0; v < NV; v++)
#pragma unroll
        for (int b = 0; b < m; b++) {
          double acc = 0.0;
#pragma unroll
          for (int r = 0; r < m; r++) acc = fma(c_wphi[r][b], u[v][r], acc);
          sB[((v * m + b) * m + q) * 32 + lane] = acc;
        }
      __syncthreads();
      if (sFlag[lane]) {
#pragma unroll
        for (int v = 0; v < NV; v++)
#pragma unroll
          for (int bb = 0; bb < m; bb++) {
            double acc = 0.0;
#pragma unroll
            for (int qq = 0; qq < m; qq++) acc = fma(c_wphi[qq][aa], sB[((v * m + bb) * m + qq) * 32 + lane], acc);
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
  // CFL minimum of the new state from the element averages (warp 0 holds mode 0)
  if (w == 0) {
    double dtk = __longlong_as_double(0x7ff0000000000000LL);
    int bad = 0;
    if (valid) {
      const double rho = un[0][0], vx = un[1][0] / rho, vy = un[2][0] / rho;
      double c;
      if (KIND == 1) {
        const double p = (ph.gamma - 1.0) * (un[NV - 1][0] - 0.5 * (un[1][0] * vx + un[2][0] * vy));
        c = sqrt(ph.gamma * p / rho);
      } else {
        const double xc = ms.x0 + (i0 + lane + 0.5) * ms.dx, yc = ms.y0 + (j + 0.5) * ms.dy;
        c = sqrt(cs2_at<KIND>(ph, xc, yc));
      }
      dtk = ph.cfl * ph.cfl_fac / ((fabs(vx) + c) / ms.dx + (fabs(vy) + c) / ms.dy);
      bad = !(rho > 0.0) || !(dtk > 0.0);  // +inf (no wave speed) is no constraint; NaN fails
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
  // torque partial of the CTA, fixed reduction order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gxs += __shfl_xor_sync(0xffffffffu, gxs, o);
    gys += __shfl_xor_sync(0xffffffffu, gys, o);
  }
  if (lane == 0) {
    sMisc[4 + 2 * w] = gxs;
    sMisc[5 + 2 * w] = gys;
  }
  __syncthreads();
  if (tid == 0) {
    double gx = 0.0, gy = 0.0;
#pragma unroll
    for (int k = 0; k < m; k++) {
      gx += sMisc[4 + 2 * k];
      gy += sMisc[5 + 2 * k];
    }
    a.part[2 * tile] = gx;
    a.part[2 * tile + 1] = gy;
  }
}

// Static fields of the locally isothermal disc with the star, evaluated
// once with the expressions (and the operand order) the stage kernel uses
// without them, so a kernel that reads them computes the same values: at the
// nodes c_s^2 and the star's gradient, at the face points c_s^2 and c_s.
template <int P>
__global__ void k_static_fields(const Mesh ms, const Phys ph, double* SN, double* SXF, double* SYF) {
  constexpr int m = P + 1, M = m * m;
  const long long nn = (long long)ms.ny * ms.ntx * M * 32;
  const long long nxf = (long long)ms.ny * m * (ms.nx + 1);
  const long long nyf = (long long)(ms.ny + 1) * ms.nx * m;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nn + nxf + nyf;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < nn) {
      // [tile][field][q m + r][lane]
      const int lane = (int)(t & 31);
      const int n = (int)((t >> 5) % M);
      const long long tile = (t >> 5) / M;
      const int j = (int)(tile / ms.ntx), i0 = (int)(tile % ms.ntx) * 32;
      const int q = n / m, r = n - q * m;
      const double xq = ms.x0 + (i0 + lane + 0.5) * ms.dx + 0.5 * ms.dx * c_tab.xi[q];
      const double yc = ms.y0 + (j + 0.5) * ms.dy;
      const double y = yc + 0.5 * ms.dy * c_tab.xi[r];
      double gx, gy;
      grad_star(ph, xq, y, gx, gy);
      double* o = SN + tile * 3 * M * 32 + (size_t)n * 32 + lane;
      o[0] = cs2_at<0>(ph, xq, y);
      o[M * 32] = gx;
      o[2 * M * 32] = gy;
    } else if (t < nn + nxf) {
      // [j][r][f]: face f of row j at y-node r
      const long long u = t - nn;
      const int f = (int)(u % (ms.nx + 1));
      const int r = (int)((u / (ms.nx + 1)) % m);
      const int j = (int)(u / ((long long)(ms.nx + 1) * m));
      const int i0 = (f / 32) * 32, ff = f - i0;
      const double y = ms.y0 + (j + 0.5) * ms.dy + 0.5 * ms.dy * c_tab.xi[r];
      const double c2 = cs2_at<0>(ph, ms.x0 + (i0 + ff) * ms.dx, y);
      SXF[2 * u] = c2;
      SXF[2 * u + 1] = sqrt(c2);
    } else {
      // [j'][i][q]: the face y = y0 + j' dy at x-node q of element i
      const long long u = t - nn - nxf;
      const int q = (int)(u % m);
      const int i = (int)((u / m) % ms.nx);
      const int jf = (int)(u / ((long long)m * ms.nx));
      const int i0 = (i / 32) * 32, lane = i - i0;
      const double xq = ms.x0 + (i0 + lane + 0.5) * ms.dx + 0.5 * ms.dx * c_tab.xi[q];
      const double c2 = cs2_at<0>(ph, xq, ms.y0 + jf * ms.dy);
      SYF[2 * u] = c2;
      SYF[2 * u + 1] = sqrt(c2);
    }
  }
}

template <int P>
static cudaError_t launch_static_impl(const Mesh& ms, const Phys& ph, double* SN, double* SXF, double* SYF,
                                      cudaStream_t s) {
  k_static_fields<P><<<1216, 256, 0, s>>>(ms, ph, SN, SXF, SYF);
  return cudaGetLastError();
}

template <int P>
static size_t stage_smem_impl(int kind) {
  return kind == 1 ? Smem<P, 1>::BYTES : Smem<P, 0>::BYTES;
}

template <int P, int KIND>
static cudaError_t launch_kind(const StageArgs& a, cudaStream_t s) {
  static bool configured = false;
  const size_t bytes = Smem<P, KIND>::BYTES;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_stage<P, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid(a.mesh.ntx, a.mesh.ny);
  k_stage<P, KIND><<<grid, 32 * (P + 1), bytes, s>>>(a);
  return cudaGetLastError();
}

template <int P>
static cudaError_t launch_stage_impl(const StageArgs& a, cudaStream_t s) {
  switch (a.phys.kind) {
    case 0: return launch_kind<P, 0>(a, s);
    case 1: return launch_kind<P, 1>(a, s);
    case 2: return launch_kind<P, 2>(a, s);
  }
  return cudaErrorInvalidValue;
}

template <int P>
static cudaError_t upload_tables_impl(const Tables& t) {
  double wphi[MAXM][MAXM] = {}, wdphi[MAXM][MAXM] = {};
  for (int q = 0; q <= P; q++)
    for (int a = 0; a <= P; a++) {
      wphi[q][a] = t.wh[q] * t.phi[q][a];
      wdphi[q][a] = t.wh[q] * t.dphi[q][a];
    }
  cudaError_t e = cudaMemcpyToSymbol(c_tab, &t, sizeof(Tables));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_wphi, wphi, sizeof(wphi));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_wdphi, wdphi, sizeof(wdphi));
  return e;
}

}  // namespace dg
