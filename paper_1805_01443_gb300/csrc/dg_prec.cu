// dg_prec.cu -- setup and conversions of the precision form: delta = u - u_b
// in FP32 about the FP64 projected background u_b, and the static background
// fields the FP32 stage kernel reads (nodal Sigma_b for the torque, damping
// offsets Q0 - Q_b, element averages of u_b for the CFL step).
#include "dg_internal.cuh"
#include "dg_physics.cuh"

namespace dg {

namespace {

__global__ void k_delta_from_full(const double* __restrict__ full, const double* __restrict__ bg,
                                  float* __restrict__ d, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    d[e] = (float)(full[e] - bg[e]);
}

__global__ void k_full_from_delta(const double* __restrict__ bg, const float* __restrict__ d,
                                  double* __restrict__ full, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    full[e] = bg[e] + (double)d[e];
}

__global__ void k_f64_to_f32(const double* __restrict__ x, float* __restrict__ y, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = (float)x[e];
}

__global__ void k_f32_to_f64(const float* __restrict__ x, double* __restrict__ y, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = (double)x[e];
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

cudaError_t launch_delta_from_full(const double* full, const double* bg, float* d, size_t n,
                                   cudaStream_t s) {
  k_delta_from_full<<<1216, 256, 0, s>>>(full, bg, d, n);
  return cudaGetLastError();
}

cudaError_t launch_full_from_delta(const double* bg, const float* d, double* full, size_t n,
                                   cudaStream_t s) {
  k_full_from_delta<<<1216, 256, 0, s>>>(bg, d, full, n);
  return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(const double* x, float* y, size_t n, cudaStream_t s) {
  k_f64_to_f32<<<1216, 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float* x, double* y, size_t n, cudaStream_t s) {
  k_f32_to_f64<<<1216, 256, 0, s>>>(x, y, n);
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
