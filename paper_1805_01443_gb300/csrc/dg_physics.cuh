// dg_physics.cuh -- device definitions of the initial/background state shared
// by the initial projection, the FP64 damping target and the precision-form
// setup (one definition, so the three agree to the last bit).
#pragma once
#include "dg_internal.cuh"

namespace dg {

// r dPhi_*/dr of the softened star: 1/r outside r_s, r^2/r_s^3 in the
// solid-body core (Sec. 5.1).
__device__ __forceinline__ double vk2_of(const Phys& ph, double r) {
  return (r >= ph.rs) ? 1.0 / r : r * r / (ph.rs * ph.rs * ph.rs);
}

// Primitive state (rho, vx, vy, p) of the initial condition without noise:
// ic 0 the rotational-equilibrium disc Sigma = max(r^s, floor),
// v_phi^2 = (1 + (s-1) h^2)/r outside r_s and (1 + (s+2) h^2) r^2/r_s^3
// inside, p = h^2 v_K^2 Sigma; ic 3 the same with p x ring_p inside r < ring_r;
// ic 1 the density wave; ic 2 a uniform state; ic 4 and 5 the vortices of
// Sec. 4; ic 6 the paper's own disc of Sec. 5.1.
__device__ __forceinline__ void ic_prim(const Phys& ph, const Mesh& ms, double x, double y,
                                        double* w) {
  if (ph.ic == 0 || ph.ic == 3) {
    double r = fmax(sqrt(x * x + y * y), 1e-12);
    double h2 = ph.h * ph.h, rs3 = ph.rs * ph.rs * ph.rs;
    double sig = fmax(pow(r, ph.slope), ph.sig_floor);
    double vphi2 = (r >= ph.rs) ? (1.0 + (ph.slope - 1.0) * h2) / r
                                : (1.0 + (ph.slope + 2.0) * h2) * r * r / rs3;
    double vphi = sqrt(fmax(vphi2, 0.0));
    w[0] = sig;
    w[1] = -vphi * y / r;
    w[2] = vphi * x / r;
    w[3] = h2 * vk2_of(ph, r) * sig;
    if (ph.ic == 3 && r < ph.ring_r) w[3] *= ph.ring_p;  // the imposed shock ring
  } else if (ph.ic == 4) {
    // isentropic vortex (Sec. 4.1) of strength amp in the free stream (vx0, vy0)
    const double g = ph.gamma, beta = ph.amp, pi = 3.141592653589793238462643383279503;
    const double xc = 0.5 * (ms.x0 + ms.x1), yc = 0.5 * (ms.y0 + ms.y1);
    const double dx = x - xc, dy = y - yc, r2 = dx * dx + dy * dy;
    const double T = 1.0 - (g - 1.0) * beta * beta / (8.0 * g * pi * pi) * exp(1.0 - r2);
    const double du = beta / (2.0 * pi) * exp(0.5 * (1.0 - r2));
    w[0] = pow(T, 1.0 / (g - 1.0));
    w[1] = ph.vx0 - du * dy;
    w[2] = ph.vy0 + du * dx;
    w[3] = pow(w[0], g);
  } else if (ph.ic == 5) {
    // Gresho vortex (Sec. 4.2) about the box centre
    const double xc = 0.5 * (ms.x0 + ms.x1), yc = 0.5 * (ms.y0 + ms.y1);
    const double dx = x - xc, dy = y - yc, r = sqrt(dx * dx + dy * dy);
    double vphi, p;
    if (r < 0.2) {
      vphi = 5.0 * r;
      p = 5.0 + 12.5 * r * r;
    } else if (r < 0.4) {
      vphi = 2.0 - 5.0 * r;
      p = 9.0 - 4.0 * log(0.2) + 12.5 * r * r - 20.0 * r + 4.0 * log(r);
    } else {
      vphi = 0.0;
      p = 3.0 + 4.0 * log(2.0);
    }
    w[0] = 1.0;
    w[1] = r > 0.0 ? -vphi * dy / r : 0.0;
    w[2] = r > 0.0 ? vphi * dx / r : 0.0;
    w[3] = p;
  } else if (ph.ic == 6) {
    // the paper's own disc (Sec. 5.1): Sigma = max(1/(1+f), floor),
    // p = h^2 Sigma, f = exp((r - r_ex)/h), v_phi^2 = r^2 Omega^2 - r h f/(1+f)
    // with the softened star's r^2 Omega^2 (no pressure term where the floor
    // holds); r_ex = the outer damping radius x 1.15^(3/2)
    const double r = fmax(sqrt(x * x + y * y), 1e-12);
    const double rex = ph.rd_out * ph.damp_ratio;
    const double f = exp((r - rex) / ph.h);
    double sig = 1.0 / (1.0 + f), g = f / (1.0 + f);
    if (sig < ph.sig_floor) {
      sig = ph.sig_floor;
      g = 0.0;
    }
    const double vphi = sqrt(fmax(vk2_of(ph, r) - r * ph.h * g, 0.0));
    w[0] = sig;
    w[1] = -vphi * y / r;
    w[2] = vphi * x / r;
    w[3] = ph.h * ph.h * sig;
  } else if (ph.ic == 1) {
    double lx = ms.x1 - ms.x0, ly = ms.y1 - ms.y0;
    w[0] = 1.0 + ph.amp * sin(6.283185307179586476925286766559 * ((x - ms.x0) / lx + (y - ms.y0) / ly));
    w[1] = ph.vx0;
    w[2] = ph.vy0;
    w[3] = 1.0;
  } else {
    w[0] = 1.0;
    w[1] = ph.vx0;
    w[2] = ph.vy0;
    w[3] = 1.0;
  }
}

}  // namespace dg
