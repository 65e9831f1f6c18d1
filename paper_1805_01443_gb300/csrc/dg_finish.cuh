// dg_finish.cuh -- end-of-step work shared by the single-handle and the
// batched drivers: fixed-order torque sum, time advance, next CFL step and
// the planet positions of the precision form.
#pragma once
#include "dg_internal.cuh"

namespace dg {

constexpr unsigned long long DT_INF_BITS = 0x7ff0000000000000ULL;  // +inf, the empty CFL slot

// planet position k (times t, t + dt/2, t + dt) of the precision form for the
// step starting at t with step dt (see DevState::plf)
__device__ __forceinline__ void store_planet32_k(DevState* ts, int k, double t, double dt, double r_p,
                                                 double omega_p, double phi0) {
  const double c = k == 0 ? 0.0 : k == 1 ? 0.5 : 1.0;
  double sn, cs;
  sincos(omega_p * (t + c * dt) + phi0, &sn, &cs);
  const double x = r_p * cs, y = r_p * sn;
  const float xh = (float)x, yh = (float)y;
  ts->plf[k][0] = xh;
  ts->plf[k][1] = (float)(x - (double)xh);
  ts->plf[k][2] = yh;
  ts->plf[k][3] = (float)(y - (double)yh);
  if (k == 2) {
    ts->pl1[0] = x;
    ts->pl1[1] = y;
  }
}

// all three positions by one thread
__device__ __forceinline__ void store_planet32(DevState* ts, double dt, double r_p, double omega_p,
                                               double phi0) {
  for (int k = 0; k < 3; k++) store_planet32_k(ts, k, ts->t, dt, r_p, omega_p, phi0);
  ts->dtf = (float)dt;
}

// End of a step, by one CTA of NT threads: fixed-order sum of the per-tile
// torque partials, torque on the planet at t^{n+1} (Sec. 5.2), time advance,
// the next CFL step and (planet32) the next step's planet positions, one per
// thread.  With advance = 0 only the CFL slot is turned into ts->dt.  With
// planet32 the position at t^{n+1} is the one stored for this step (pl1, the
// same expression), so no trigonometry runs before the torque.  The sum is
// the same for every NT: 256 virtual lanes (lane v adds partials v, v + 256,
// ... in order, then a pairwise tree over the lanes), the real threads taking
// lanes tid, tid + NT, ...; sx and sy are 256 doubles of shared scratch each.
template <int NT>
__device__ __forceinline__ void finish_step_nt(double* sx, double* sy, DevState* ts, const double* part,
                                               int nparts, double* series, double fixed_dt, int advance,
                                               int planet32, double r_p, double omega_p, double phi0) {
  __shared__ double s_t, s_dt;
  __shared__ int s_go;
  constexpr int NL = 256;
  const int tid = threadIdx.x;
  if (ts->status != 0) return;
  if (advance) {
    const double2* p2 = reinterpret_cast<const double2*>(part);
    for (int v = tid; v < NL; v += NT) {
      double gx = 0.0, gy = 0.0;
      // unrolled so that 16 loads are in flight; the additions keep their order
#pragma unroll 16
      for (int k = v; k < nparts; k += NL) {
        const double2 g = p2[k];
        gx += g.x;
        gy += g.y;
      }
      sx[v] = gx;
      sy[v] = gy;
    }
    __syncthreads();
    for (int s = NL / 2; s > 0; s >>= 1) {
      for (int v = tid; v < s; v += NT) {
        sx[v] += sx[v + s];
        sy[v] += sy[v + s];
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    s_go = 0;
    if (ts->pending) {
      // bit 0: non-finite or non-positive state; bit 1: a bounded wait gave up
      ts->status = (ts->pending & 2) ? DG_ERR_TIMEOUT : DG_ERR_NUMERIC;
    } else {
      if (advance) {
        const double dt = fixed_dt > 0.0 ? fixed_dt : ts->dt;
        const double tn1 = ts->t + dt;
        double xp, yp;
        if (planet32) {
          xp = ts->pl1[0];
          yp = ts->pl1[1];
        } else {
          double sn, cs;
          sincos(omega_p * tn1 + phi0, &sn, &cs);
          xp = r_p * cs;
          yp = r_p * sn;
        }
        const double gz = xp * sy[0] - yp * sx[0];
        series[ts->series_count % SERIES_CAP] = gz;
        ts->series_count += 1;
        ts->torque = gz;
        ts->t = tn1;
        ts->step += 1;
      }
      const double dtn = __longlong_as_double((long long)ts->dt_bits);
      if (!(dtn > 0.0) || !isfinite(dtn)) {
        if (fixed_dt <= 0.0) ts->status = DG_ERR_NUMERIC;
      } else {
        ts->dt = dtn;
      }
      ts->dt_bits = DT_INF_BITS;
      if (planet32 && ts->status == 0) {
        s_go = 1;
        s_t = ts->t;
        s_dt = fixed_dt > 0.0 ? fixed_dt : ts->dt;
        ts->dtf = (float)s_dt;
      }
    }
  }
  __syncthreads();
  if (s_go && tid < 3) store_planet32_k(ts, tid, s_t, s_dt, r_p, omega_p, phi0);
}

// the same by one CTA of 256 threads with its own scratch
__device__ __forceinline__ void finish_step(DevState* ts, const double* part, int nparts, double* series,
                                            double fixed_dt, int advance, int planet32, double r_p,
                                            double omega_p, double phi0) {
  __shared__ double sx[256], sy[256];
  finish_step_nt<256>(sx, sy, ts, part, nparts, series, fixed_dt, advance, planet32, r_p, omega_p, phi0);
}

}  // namespace dg
