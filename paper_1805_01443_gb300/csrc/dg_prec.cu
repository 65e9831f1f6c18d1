// dg_prec.cu -- setup and conversions of the precision form: delta = u - u_b
// in FP32 about the FP64 projected background u_b, held as its values at the
// Gauss-Legendre nodes, and the static background fields the FP32 stage
// kernel reads (nodal Sigma_b for the torque, damping offsets Q0 - Q_b,
// element averages of u_b for the CFL step).
#include "dg_internal.cuh"
#include "dg_physics.cuh"

namespace dg {

namespace {

// Modal <-> nodal transforms of the precision form's tiled arrays (its state,
// R_b and the exact background are values at the m x m Gauss-Legendre nodes
// of each element).  One thread per (element, variable): a block of (32, nv)
// threads per tile, grid (tiles per row, rows); lanes past nx write zeros.
//   to nodes:  u(q, r) = sum_ab c_ab phi_a(xi_q) phi_b(eta_r), with c the
//              source modes minus `sub` (both FP64, the difference rounded to
//              T), summed over b then a in T
//   to modes:  c_ab = sum_qr (w_q/2)(w_r/2) phi_a(xi_q) phi_b(eta_r) u(q, r) in
//              FP64 (the discrete orthonormality of the basis on the m-point
//              rule), plus `add` (FP64 modes) when given
// The source of k_to_nodal32 is a tiled array or, with canon set, the
// canonical array [var][a*m+b][j][i].
template <int P, typename T>
__global__ void k_to_nodal32(const double* __restrict__ src, int canon, const double* __restrict__ sub,
                             float* __restrict__ dst, const Mesh ms, const Tables tab, int nv) {
  constexpr int m = P + 1, M = m * m;
  const int lane = threadIdx.x, v = threadIdx.y;
  const int i = blockIdx.x * TILE + lane, j = blockIdx.y;
  const size_t tile = (size_t)j * ms.ntx + blockIdx.x;
  float* out = dst + (tile * nv + v) * M * TILE + lane;
  if (i >= ms.nx) {
    for (int k = 0; k < M; k++) out[k * TILE] = 0.0f;
    return;
  }
  const size_t to = (tile * nv + v) * M * TILE + lane;
  T c[M];
  for (int k = 0; k < M; k++) {
    const double x = canon ? src[((size_t)(v * M + k) * ms.ny + j) * ms.nx + i] : src[to + (size_t)k * TILE];
    c[k] = (T)(sub ? x - sub[to + (size_t)k * TILE] : x);
  }
  T Tm[m][m];
  for (int a = 0; a < m; a++)
    for (int r = 0; r < m; r++) {
      T acc = 0;
      for (int b = 0; b < m; b++) acc += c[a * m + b] * (T)tab.phi[r][b];
      Tm[a][r] = acc;
    }
  for (int q = 0; q < m; q++)
    for (int r = 0; r < m; r++) {
      T acc = 0;
      for (int a = 0; a < m; a++) acc += (T)tab.phi[q][a] * Tm[a][r];
      out[(q * m + r) * TILE] = (float)acc;
    }
}

template <int P>
__global__ void k_to_modal64(const float* __restrict__ src, const double* __restrict__ add,
                             double* __restrict__ dst, const Mesh ms, const Tables tab, int nv) {
  constexpr int m = P + 1, M = m * m;
  const int lane = threadIdx.x, v = threadIdx.y;
  const int i = blockIdx.x * TILE + lane, j = blockIdx.y;
  const size_t to = (((size_t)j * ms.ntx + blockIdx.x) * nv + v) * M * TILE + lane;
  if (i >= ms.nx) {
    for (int k = 0; k < M; k++) dst[to + (size_t)k * TILE] = 0.0;
    return;
  }
  double u[M];
  for (int k = 0; k < M; k++) u[k] = (double)src[to + (size_t)k * TILE];
  double Pq[m][m];  // [b][q] = sum_r (w_r/2) phi_b(eta_r) u(q, r)
  for (int b = 0; b < m; b++)
    for (int q = 0; q < m; q++) {
      double acc = 0.0;
      for (int r = 0; r < m; r++) acc += tab.wh[r] * tab.phi[r][b] * u[q * m + r];
      Pq[b][q] = acc;
    }
  for (int a = 0; a < m; a++)
    for (int b = 0; b < m; b++) {
      double acc = 0.0;
      for (int q = 0; q < m; q++) acc += tab.wh[q] * tab.phi[q][a] * Pq[b][q];
      dst[to + (size_t)(a * m + b) * TILE] = add ? add[to + (size_t)(a * m + b) * TILE] + acc : acc;
    }
}

// One thread per element: FP64 nodal values of the projected background u_b
// at the m x m Gauss-Legendre nodes (dense contraction), giving
//   Sigma_b(node) as a (hi, lo) float pair -> sigbn [tile][2][node][32] (torque node masses)
//   Q0 - Q_b for Q = (Sigma, vx, vy)      -> db    (damping target offsets)
//   element averages (mode 0) of u_b      -> bm0   (CFL step)
__global__ void k_bg_nodes(const double* __restrict__ bg, float* __restrict__ sigbn,
                           float* __restrict__ db, float* __restrict__ bm0,
                           float* __restrict__ disc, const Mesh ms, const Phys ph,
                           const Tables tab, int p) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ms.nx * ms.ny) return;
  const int i = e % ms.nx, j = e / ms.nx;
  const int m = p + 1, M = m * m, NV = 3;
  const size_t tile = (size_t)j * ms.ntx + (i >> 5);
  const int lane = i & 31;
  const double* c = bg + tile * NV * M * TILE + lane;
  const double xc = ms.x0 + (i + 0.5) * ms.dx, yc = ms.y0 + (j + 0.5) * ms.dy;
  for (int v = 0; v < NV; v++) bm0[(tile * 3 + v) * TILE + lane] = (float)c[(size_t)v * M * TILE];
  // largest relative difference between the projected and the analytic
  // background over the volume nodes and the face points of the element
  auto rel = [](const double* up, const double* w0) {
    const double vs = fmax(sqrt(w0[1] * w0[1] + w0[2] * w0[2]), 1e-6);
    const double ds = fabs(up[0] - w0[0]) / fabs(w0[0]);
    const double dv = fmax(fabs(up[1] / up[0] - w0[1]), fabs(up[2] / up[0] - w0[2])) / vs;
    return fmax(ds, dv);
  };
  double dmax = 0.0;
  for (int face = 0; face < 4; face++)
    for (int k = 0; k < m; k++) {
      double fa[MAXM], gb[MAXM];
      for (int t = 0; t < m; t++) {
        fa[t] = face < 2 ? (face == 0 ? tab.pm[t] : tab.pp[t]) : tab.phi[k][t];
        gb[t] = face < 2 ? tab.phi[k][t] : (face == 2 ? tab.pm[t] : tab.pp[t]);
      }
      double up[3];
      for (int v = 0; v < NV; v++) {
        double acc = 0.0;
        for (int a = 0; a < m; a++)
          for (int b = 0; b < m; b++) acc += c[((size_t)v * M + a * m + b) * TILE] * fa[a] * gb[b];
        up[v] = acc;
      }
      const double x = face < 2 ? xc + (face == 0 ? -0.5 : 0.5) * ms.dx : xc + 0.5 * ms.dx * tab.xi[k];
      const double y = face < 2 ? yc + 0.5 * ms.dy * tab.xi[k] : yc + (face == 2 ? -0.5 : 0.5) * ms.dy;
      double w0[4];
      ic_prim(ph, ms, x, y, w0);
      dmax = fmax(dmax, rel(up, w0));
    }
  for (int q = 0; q < m; q++)
    for (int r = 0; r < m; r++) {
      double u[3];
      for (int v = 0; v < NV; v++) {
        double acc = 0.0;
        for (int a = 0; a < m; a++)
          for (int b = 0; b < m; b++)
            acc += c[((size_t)v * M + a * m + b) * TILE] * tab.phi[q][a] * tab.phi[r][b];
        u[v] = acc;
      }
      const int n = q * m + r;
      const double x = xc + 0.5 * ms.dx * tab.xi[q], y = yc + 0.5 * ms.dy * tab.xi[r];
      double w0[4];
      ic_prim(ph, ms, x, y, w0);
      const float shi = (float)u[0];
      sigbn[((tile * 2 + 0) * M + n) * TILE + lane] = shi;
      sigbn[((tile * 2 + 1) * M + n) * TILE + lane] = (float)(u[0] - (double)shi);
      db[((tile * 3 + 0) * M + n) * TILE + lane] = (float)(w0[0] - u[0]);
      db[((tile * 3 + 1) * M + n) * TILE + lane] = (float)(w0[1] - u[1] / u[0]);
      db[((tile * 3 + 2) * M + n) * TILE + lane] = (float)(w0[2] - u[2] / u[0]);
      dmax = fmax(dmax, rel(u, w0));
    }
  disc[tile * TILE + lane] = (float)dmax;
}

// A tile takes the exact background when it, or one of its four neighbour
// tiles, holds an element whose projected background departs from the
// analytic one by more than `thr` (relative).  Under periodic (bc 0) and
// copied-element (bc 3) boundaries the tiles along the box edge take it too:
// the neighbour across the edge is an element elsewhere (or the edge element
// itself, extended outward), whose background at the shared face is its own
// projection, not the analytic background at the face point.
__global__ void k_tile_flags(const float* __restrict__ disc, int* __restrict__ flags, const Mesh ms,
                             float thr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ms.ntx * ms.ny) return;
  const int bx = t % ms.ntx, j = t / ms.ntx;
  int f = 0;
  const int nb[5][2] = {{0, 0}, {-1, 0}, {1, 0}, {0, -1}, {0, 1}};
  for (int k = 0; k < 5; k++) {
    const int tx = bx + nb[k][0], ty = j + nb[k][1];
    if (tx < 0 || tx >= ms.ntx || ty < 0 || ty >= ms.ny) continue;
    const int nval = min(TILE, ms.nx - tx * TILE);
    for (int l = 0; l < nval; l++) f |= disc[((size_t)ty * ms.ntx + tx) * TILE + l] > thr;
  }
  if ((ms.bc == 0 || ms.bc == 3) && (bx == 0 || bx + 1 == ms.ntx || j == 0 || j + 1 == ms.ny)) f = 1;
  flags[t] = f;
}

}  // namespace

template <typename T>
static cudaError_t to_nodal32(const double* src, int canon, const double* sub, float* dst, const Mesh& ms,
                              const Tables& tab, int p, int nv, cudaStream_t s) {
  const dim3 grid(ms.ntx, ms.ny), block(TILE, nv);
  switch (p) {
    case 1: k_to_nodal32<1, T><<<grid, block, 0, s>>>(src, canon, sub, dst, ms, tab, nv); break;
    case 2: k_to_nodal32<2, T><<<grid, block, 0, s>>>(src, canon, sub, dst, ms, tab, nv); break;
    case 3: k_to_nodal32<3, T><<<grid, block, 0, s>>>(src, canon, sub, dst, ms, tab, nv); break;
    default: k_to_nodal32<4, T><<<grid, block, 0, s>>>(src, canon, sub, dst, ms, tab, nv); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_to_nodal32(const double* src, int canon, const double* sub, float* dst, const Mesh& mesh,
                              const Tables& tab, int p, int nv, int fp64, cudaStream_t s) {
  return fp64 ? to_nodal32<double>(src, canon, sub, dst, mesh, tab, p, nv, s)
              : to_nodal32<float>(src, canon, sub, dst, mesh, tab, p, nv, s);
}

cudaError_t launch_to_modal64(const float* src, const double* add, double* dst, const Mesh& ms,
                              const Tables& tab, int p, int nv, cudaStream_t s) {
  const dim3 grid(ms.ntx, ms.ny), block(TILE, nv);
  switch (p) {
    case 1: k_to_modal64<1><<<grid, block, 0, s>>>(src, add, dst, ms, tab, nv); break;
    case 2: k_to_modal64<2><<<grid, block, 0, s>>>(src, add, dst, ms, tab, nv); break;
    case 3: k_to_modal64<3><<<grid, block, 0, s>>>(src, add, dst, ms, tab, nv); break;
    default: k_to_modal64<4><<<grid, block, 0, s>>>(src, add, dst, ms, tab, nv); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_bg_nodes(const double* bg, float* sigbn, float* db, float* bm0, float* disc,
                            const Mesh& mesh, const Phys& phys, const Tables& tab, int p,
                            cudaStream_t s) {
  const int n = mesh.nx * mesh.ny;
  k_bg_nodes<<<(n + 127) / 128, 128, 0, s>>>(bg, sigbn, db, bm0, disc, mesh, phys, tab, p);
  return cudaGetLastError();
}

cudaError_t launch_tile_flags(const float* disc, int* flags, const Mesh& mesh, float threshold,
                              cudaStream_t s) {
  const int n = mesh.ntx * mesh.ny;
  k_tile_flags<<<(n + 127) / 128, 128, 0, s>>>(disc, flags, mesh, threshold);
  return cudaGetLastError();
}

}  // namespace dg
