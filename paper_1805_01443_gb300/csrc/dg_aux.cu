// dg_aux.cu -- initial-condition projection, CFL reduction, per-step finish,
// layout transforms and conserved sums.
#include <math.h>

#include "dg_async.cuh"
#include "dg_finish.cuh"
#include "dg_internal.cuh"
#include "dg_physics.cuh"

namespace dg {

namespace {

constexpr unsigned long long INF_BITS = DT_INF_BITS;

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator:
// value(c) = mix(seed + (c + 1) * 0x9E3779B97F4A7C15), top 53 bits -> [0, 1).
__device__ __forceinline__ double splitmix_uniform(unsigned long long seed, unsigned long long c) {
  unsigned long long z = seed + (c + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

// L2 projection of the initial data onto the modes (Eq. 2, first line) with
// the (m+1)-point Gauss-Legendre rule; one thread per element.
__global__ void k_init(const InitArgs a, int count) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const Mesh& ms = a.mesh;
  int i, j;
  switch (a.target) {
    case 0: i = e % ms.nx; j = e / ms.nx; break;
    case 1: i = -1; j = e; break;
    case 2: i = ms.nx; j = e; break;
    case 3: i = e; j = -1; break;
    default: i = e; j = ms.ny; break;
  }
  const int m = a.p + 1, mq = m + 1, M = m * m, nv = a.nv;
  double c[4][MAXM * MAXM];
  for (int v = 0; v < 4; v++)
    for (int k = 0; k < M; k++) c[v][k] = 0.0;
  const double xc = ms.x0 + (i + 0.5) * ms.dx, yc = ms.y0 + (j + 0.5) * ms.dy;
  for (int q = 0; q < mq; q++)
    for (int r = 0; r < mq; r++) {
      const double x = xc + 0.5 * ms.dx * a.xq[q], y = yc + 0.5 * ms.dy * a.xq[r];
      double w[4], u[4];
      ic_prim(a.phys, ms, x, y, w);
      if (a.target == 0 && (a.phys.ic == 0 || a.phys.ic == 3) && a.noise_amp > 0.0) {
        const unsigned long long ctr =
            ((unsigned long long)j * ms.nx + i) * (unsigned long long)(mq * mq) + q * mq + r;
        w[0] += a.noise_amp * (2.0 * splitmix_uniform(a.seed, ctr) - 1.0);
      }
      u[0] = w[0];
      u[1] = w[0] * w[1];
      u[2] = w[0] * w[2];
      u[3] = w[3] / (a.phys.gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2]);
      const double wt = 0.25 * a.wq[q] * a.wq[r];
      for (int aa = 0; aa < m; aa++)
        for (int b = 0; b < m; b++) {
          const double f = wt * a.phq[q][aa] * a.phq[r][b];
          for (int v = 0; v < nv; v++) c[v][aa * m + b] += f * u[v];
        }
    }
  const size_t NVM = (size_t)nv * M;
  for (int v = 0; v < nv; v++)
    for (int k = 0; k < M; k++) {
      const double val = c[v][k];
      size_t o;
      if (a.target == 0)
        o = (((size_t)j * ms.ntx + (i >> 5)) * NVM + v * M + k) * TILE + (i & 31);
      else if (a.target <= 2)
        o = (size_t)j * NVM + v * M + k;
      else
        o = (((size_t)(i >> 5)) * NVM + v * M + k) * TILE + (i & 31);
      a.out[o] = val;
    }
}

// CFL time step of Sec. 2.3 from the element averages; block minimum folded
// into the device slot with an atomic minimum on the (positive) bit pattern.
// CFL minimum of the element averages of U (tiled FP64), or of U + D when D
// (tiled FP32, the precision form's delta about U = u_b, values at the nodes)
// is given: the average of D is sum_n w_n D_n with the weights w_n = (w_q/2)
// (w_r/2) as float pairs (wh, wl), each product and the sum formed in
// float-float arithmetic (~2^-44 relative to sum |w_n D_n|), then added to
// U's FP64 average
struct NodeW {
  float wh[MAXM * MAXM], wl[MAXM * MAXM];
};

// one term w_n d of the float-float sum (sh, sl), in node order
__device__ __forceinline__ void ff_acc(const NodeW& w, int n, float d, float& sh, float& sl) {
  const float p = __fmul_rn(w.wh[n], d);
  const float e = fmaf(w.wl[n], d, fmaf(w.wh[n], d, -p));  // w d - p, to ~2^-48 of w d
  const float t = __fadd_rn(sh, p);                          // two-sum of sh and p
  const float bb = __fsub_rn(t, sh);
  sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(p, bb)), e));
  sh = t;
}

// the CFL bound of element (i, j) from its averages (E: adiabatic only);
// +inf (no wave speed) is no constraint, and bad is set for a NaN or
// non-positive bound or density
__device__ __forceinline__ double cfl_bound(double rho, double mx, double my, double E, int i, int j,
                                            const Mesh& ms, const Phys& ph, double idx, double idy, int& bad) {
  const double irho = 1.0 / rho;
  const double vx = mx * irho, vy = my * irho;
  double c;
  if (ph.kind == 1) {
    const double pr = (ph.gamma - 1.0) * (E - 0.5 * (mx * vx + my * vy));
    c = sqrt(ph.gamma * pr * irho);
  } else if (ph.kind == 2) {
    c = ph.h;
  } else {
    const double xc = ms.x0 + (i + 0.5) * ms.dx, yc = ms.y0 + (j + 0.5) * ms.dy;
    const double r = sqrt(xc * xc + yc * yc);
    // h v_K: h / sqrt(r) outside the softened core, h r / r_s^(3/2) inside
    c = ph.h * (r >= ph.rs ? rsqrt(r) : sqrt(vk2_of(ph, r)));
  }
  double dtk = ph.cfl * ph.cfl_fac / ((fabs(vx) + c) * idx + (fabs(vy) + c) * idy);
  bad = !(rho > 0.0) || !(dtk > 0.0);
  if (bad) dtk = __longlong_as_double((long long)INF_BITS);
  return dtk;
}

__global__ void k_cfl(const double* U, const float* D, const NodeW w, DevState* ts, const Mesh ms, const Phys ph,
                      int p, int nv, double idx, double idy) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int M = (p + 1) * (p + 1);
  double dtk = __longlong_as_double((long long)INF_BITS);
  int bad = 0;
  if (e < ms.nx * ms.ny) {
    const int i = e % ms.nx, j = e / ms.nx;
    const size_t base = (((size_t)j * ms.ntx + (i >> 5)) * nv * M) * TILE + (i & 31);
    auto avg = [&](int v) {
      const size_t o = base + (size_t)v * M * TILE;
      if (!D) return U[o];
      float sh = 0.0f, sl = 0.0f;
      for (int n = 0; n < M; n++) ff_acc(w, n, D[o + (size_t)n * TILE], sh, sl);
      return U[o] + ((double)sh + (double)sl);
    };
    dtk = cfl_bound(avg(0), avg(1), avg(2), ph.kind == 1 ? avg(3) : 0.0, i, j, ms, ph, idx, idy, bad);
  }
  for (int o = 16; o > 0; o >>= 1) {
    dtk = fmin(dtk, __shfl_xor_sync(0xffffffffu, dtk, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(&ts->pending, 1);
    atomicMin(&ts->dt_bits, (unsigned long long)__double_as_longlong(dtk));
  }
}

// the three stage-time positions, one per thread (FP64 sincos each)
__global__ void k_planet32(DevState* ts, double fixed_dt, double r_p, double omega_p, double phi0) {
  const int k = threadIdx.x;
  const double dt = fixed_dt > 0.0 ? fixed_dt : ts->dt;
  if (k < 3) store_planet32_k(ts, k, ts->t, dt, r_p, omega_p, phi0);
  if (k == 0) ts->dtf = (float)dt;
}

__global__ void k_finish(DevState* ts, const double* part, int nparts, double* series,
                         double fixed_dt, int advance, int planet32, double r_p, double omega_p,
                         double phi0) {
  pdl_wait();
  pdl_trigger();
  finish_step(ts, part, nparts, series, fixed_dt, advance, planet32, r_p, omega_p, phi0);
}

__global__ void k_reset(DevState* ts, double t, long long step) {
  ts->t = t;
  ts->dt = 0.0;
  ts->torque = 0.0;
  ts->step = step;
  ts->status = 0;
  ts->pending = 0;
  ts->dt_bits = INF_BITS;
  ts->series_count = 0;
}

// canonical <-> tiled layout kernels: a block of 8 warps per (tile bx, row
// j), thread x = lane, warp y taking var-modes vk = y, y + 8, ...; each warp
// moves one row of 32 elements of one (var, mode) per iteration on both sides.
// k_ingest: canonical modes (device memory, or mapped page-locked host memory
// read in place) -> tiled FP64 state
__global__ void k_ingest(const double* __restrict__ canon, double* __restrict__ tiled, const Mesh ms, int nvm) {
  const int i = blockIdx.x * TILE + threadIdx.x, j = blockIdx.y;
  if (i >= ms.nx) return;
  for (int vk = threadIdx.y; vk < nvm; vk += blockDim.y)
    tiled[(((size_t)j * ms.ntx + blockIdx.x) * nvm + vk) * TILE + threadIdx.x] =
        canon[((size_t)vk * ms.ny + j) * ms.nx + i];
}

// canonical FP32 delta (values at the nodes) -> tiled delta, with the CFL
// step of u_b + delta (the precision form's upload): a block of (32, 3)
// threads per tile, thread (lane, v) moving variable v of one element in node
// order and summing its average as k_cfl does, warp 0 forming the bounds; the
// M loads of a thread are issued before any is used
template <int M>
__global__ void k_ingest_delta_cfl(const float* __restrict__ canon, float* __restrict__ d,
                                   const double* __restrict__ U, const NodeW w, unsigned long long* dt_bits,
                                   int* pending, const Mesh ms, const Phys ph, double idx, double idy) {
  __shared__ float s_sum[3][2][TILE];
  const int lane = threadIdx.x, v = threadIdx.y;
  const int i = blockIdx.x * TILE + lane, j = blockIdx.y;
  const size_t base = ((size_t)j * ms.ntx + blockIdx.x) * 3 * M * TILE + lane;
  float sh = 0.0f, sl = 0.0f;
  if (i < ms.nx) {
    float x[M];
#pragma unroll
    for (int n = 0; n < M; n++) x[n] = __ldg(canon + ((size_t)(v * M + n) * ms.ny + j) * ms.nx + i);
#pragma unroll
    for (int n = 0; n < M; n++) {
      d[base + (size_t)(v * M + n) * TILE] = x[n];
      ff_acc(w, n, x[n], sh, sl);
    }
  }
  s_sum[v][0][lane] = sh;
  s_sum[v][1][lane] = sl;
  __syncthreads();
  if (v != 0) return;
  double dtk = __longlong_as_double((long long)INF_BITS);
  int bad = 0;
  if (i < ms.nx) {
    double a[3];
    for (int k = 0; k < 3; k++)
      a[k] = U[base + (size_t)k * M * TILE] + ((double)s_sum[k][0][lane] + (double)s_sum[k][1][lane]);
    dtk = cfl_bound(a[0], a[1], a[2], 0.0, i, j, ms, ph, idx, idy, bad);
  }
  for (int o = 16; o > 0; o >>= 1) {
    dtk = fmin(dtk, __shfl_xor_sync(0xffffffffu, dtk, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (lane == 0) {
    if (bad) atomicOr(pending, 1);
    atomicMin(dt_bits, (unsigned long long)__double_as_longlong(dtk));
  }
}

// what k_reset, the CFL pass into ts and k_finish without advance leave in the
// time state, from a CFL slot filled apart from it
__global__ void k_adopt_upload(DevState* ts, UpSlot* up, double t, long long step) {
  const unsigned long long bits = up->dt_bits;
  const int pend = up->pending;
  up->dt_bits = INF_BITS;
  up->pending = 0;
  ts->t = t;
  ts->dt = 0.0;
  ts->torque = 0.0;
  ts->step = step;
  ts->series_count = 0;
  ts->pending = pend;
  ts->status = 0;
  if (pend) {
    ts->status = (pend & 2) ? DG_ERR_TIMEOUT : DG_ERR_NUMERIC;
    ts->dt_bits = bits;
    return;
  }
  const double dtn = __longlong_as_double((long long)bits);
  if (!(dtn > 0.0) || !isfinite(dtn)) ts->status = DG_ERR_NUMERIC;
  else ts->dt = dtn;
  ts->dt_bits = INF_BITS;
}

__global__ void k_to_canon_f32(const float* tiled, float* canon, const Mesh ms, int nvm) {
  const int i = blockIdx.x * TILE + threadIdx.x, j = blockIdx.y;
  if (i >= ms.nx) return;
  for (int vk = threadIdx.y; vk < nvm; vk += blockDim.y)
    canon[((size_t)vk * ms.ny + j) * ms.nx + i] = tiled[(((size_t)j * ms.ntx + blockIdx.x) * nvm + vk) * TILE + threadIdx.x];
}

__global__ void k_to_canon(const double* tiled, double* canon, const Mesh ms, int nvm) {
  const int i = blockIdx.x * TILE + threadIdx.x, j = blockIdx.y;
  if (i >= ms.nx) return;
  for (int vk = threadIdx.y; vk < nvm; vk += blockDim.y)
    canon[((size_t)vk * ms.ny + j) * ms.nx + i] = tiled[(((size_t)j * ms.ntx + blockIdx.x) * nvm + vk) * TILE + threadIdx.x];
}

// FP64 sums of element average x |K| per variable: per-block partials in a
// fixed order, then one block sums the partials in a fixed order.
__global__ void k_conserved_part(const double* U, double* part, const Mesh ms, int nv, int M) {
  __shared__ double s[4][256];
  const int tid = threadIdx.x;
  const int e = blockIdx.x * 256 + tid;
  for (int v = 0; v < 4; v++) s[v][tid] = 0.0;
  if (e < ms.nx * ms.ny) {
    const int i = e % ms.nx, j = e / ms.nx;
    const size_t base = (((size_t)j * ms.ntx + (i >> 5)) * nv * M) * TILE + (i & 31);
    for (int v = 0; v < nv; v++) s[v][tid] = U[base + (size_t)v * M * TILE] * ms.dx * ms.dy;
  }
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (tid < st)
      for (int v = 0; v < 4; v++) s[v][tid] += s[v][tid + st];
    __syncthreads();
  }
  if (tid == 0)
    for (int v = 0; v < nv; v++) part[(size_t)blockIdx.x * 4 + v] = s[v][0];
}

__global__ void k_conserved_final(const double* part, int nblk, double* out, int nv) {
  __shared__ double s[4][256];
  const int tid = threadIdx.x;
  for (int v = 0; v < 4; v++) {
    double acc = 0.0;
    for (int b = tid; b < nblk; b += 256) acc += part[(size_t)b * 4 + v];
    s[v][tid] = acc;
  }
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (tid < st)
      for (int v = 0; v < 4; v++) s[v][tid] += s[v][tid + st];
    __syncthreads();
  }
  if (tid == 0)
    for (int v = 0; v < nv; v++) out[v] = s[v][0];
}

}  // namespace

cudaError_t launch_init(const InitArgs& a, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_init<<<(count + 127) / 128, 128, 0, s>>>(a, count);
  return cudaGetLastError();
}

cudaError_t launch_cfl(const double* U, const float* D, const double* wn, DevState* ts, const Mesh& mesh,
                       const Phys& phys, int p, int nv, cudaStream_t s) {
  const int n = mesh.nx * mesh.ny;
  NodeW w{};
  if (D)
    for (int k = 0; k < (p + 1) * (p + 1); k++) {
      w.wh[k] = (float)wn[k];
      w.wl[k] = (float)(wn[k] - (double)w.wh[k]);
    }
  k_cfl<<<(n + 255) / 256, 256, 0, s>>>(U, D, w, ts, mesh, phys, p, nv, 1.0 / mesh.dx, 1.0 / mesh.dy);
  return cudaGetLastError();
}

cudaError_t launch_finish(DevState* ts, const double* part, int nparts, double* series,
                          double fixed_dt, int advance, int planet32, double r_p, double omega_p,
                          double phi0, cudaStream_t s) {
  return launch_pdl(k_finish, dim3(1), dim3(256), 0, s, ts, part, nparts, series, fixed_dt, advance, planet32,
                    r_p, omega_p, phi0);
}

// out = u0 + dt sum_{j<nk} c_j k_j + cx X (dt the step in use)
__global__ void k_combine(double* __restrict__ out, const double* __restrict__ u0, const double* k0,
                          const double* k1, const double* k2, const double* k3, const double* k4, double c0,
                          double c1, double c2, double c3, double c4, int nk, const double* X, double cx,
                          size_t n, const DevState* ts, double fixed_dt) {
  if (ts->status != 0) return;
  const double dt = fixed_dt > 0.0 ? fixed_dt : ts->dt;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (nk > 0) acc += c0 * k0[e];
    if (nk > 1) acc += c1 * k1[e];
    if (nk > 2) acc += c2 * k2[e];
    if (nk > 3) acc += c3 * k3[e];
    if (nk > 4) acc += c4 * k4[e];
    double r = u0[e] + dt * acc;
    if (X) r += cx * X[e];
    out[e] = r;
  }
}

cudaError_t launch_combine(double* out, const double* u0, const double* const* k, const double* c, int nk,
                           const double* X, double cx, size_t n, const DevState* ts, double fixed_dt,
                           cudaStream_t s) {
  const double* kk[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double cc[5] = {0, 0, 0, 0, 0};
  for (int j = 0; j < nk && j < 5; j++) {
    kk[j] = k[j];
    cc[j] = c[j];
  }
  k_combine<<<1216, 256, 0, s>>>(out, u0, kk[0], kk[1], kk[2], kk[3], kk[4], cc[0], cc[1], cc[2], cc[3], cc[4], nk,
                                  X, cx, n, ts, fixed_dt);
  return cudaGetLastError();
}

cudaError_t launch_planet32(DevState* ts, double fixed_dt, double r_p, double omega_p, double phi0,
                            cudaStream_t s) {
  k_planet32<<<1, 32, 0, s>>>(ts, fixed_dt, r_p, omega_p, phi0);
  return cudaGetLastError();
}

cudaError_t launch_adopt_upload(DevState* ts, UpSlot* up, double t, long long step, cudaStream_t s) {
  k_adopt_upload<<<1, 1, 0, s>>>(ts, up, t, step);
  return cudaGetLastError();
}

cudaError_t launch_reset_state(DevState* ts, double t, long long step, cudaStream_t s) {
  k_reset<<<1, 1, 0, s>>>(ts, t, step);
  return cudaGetLastError();
}

cudaError_t launch_ingest(const double* canon, double* tiled, const Mesh& mesh, int nv, int M, cudaStream_t s) {
  k_ingest<<<dim3(mesh.ntx, mesh.ny), dim3(TILE, 8), 0, s>>>(canon, tiled, mesh, nv * M);
  return cudaGetLastError();
}

cudaError_t launch_ingest_delta_cfl(const float* canon, float* d, const double* U, const double* wn,
                                   unsigned long long* dt_bits, int* pending, const Mesh& mesh, const Phys& phys,
                                   int M, cudaStream_t s) {
  NodeW w{};
  for (int k = 0; k < M; k++) {
    w.wh[k] = (float)wn[k];
    w.wl[k] = (float)(wn[k] - (double)w.wh[k]);
  }
  const dim3 g(mesh.ntx, mesh.ny), b(TILE, 3);
  const double idx = 1.0 / mesh.dx, idy = 1.0 / mesh.dy;
  switch (M) {
    case 4: k_ingest_delta_cfl<4><<<g, b, 0, s>>>(canon, d, U, w, dt_bits, pending, mesh, phys, idx, idy); break;
    case 9: k_ingest_delta_cfl<9><<<g, b, 0, s>>>(canon, d, U, w, dt_bits, pending, mesh, phys, idx, idy); break;
    case 16: k_ingest_delta_cfl<16><<<g, b, 0, s>>>(canon, d, U, w, dt_bits, pending, mesh, phys, idx, idy); break;
    case 25: k_ingest_delta_cfl<25><<<g, b, 0, s>>>(canon, d, U, w, dt_bits, pending, mesh, phys, idx, idy); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_to_canon_f32(const float* tiled, float* canon, const Mesh& mesh, int nv, int M,
                                cudaStream_t s) {
  k_to_canon_f32<<<dim3(mesh.ntx, mesh.ny), dim3(TILE, 8), 0, s>>>(tiled, canon, mesh, nv * M);
  return cudaGetLastError();
}

cudaError_t launch_to_canon(const double* tiled, double* canon, const Mesh& mesh, int nv, int M,
                            cudaStream_t s) {
  k_to_canon<<<dim3(mesh.ntx, mesh.ny), dim3(TILE, 8), 0, s>>>(tiled, canon, mesh, nv * M);
  return cudaGetLastError();
}

cudaError_t launch_conserved(const double* U, double* part, double* out, const Mesh& mesh, int nv,
                             int M, cudaStream_t s) {
  const int n = mesh.nx * mesh.ny, nblk = (n + 255) / 256;
  k_conserved_part<<<nblk, 256, 0, s>>>(U, part, mesh, nv, M);
  k_conserved_final<<<1, 256, 0, s>>>(part, nblk, out, nv);
  return cudaGetLastError();
}

}  // namespace dg
