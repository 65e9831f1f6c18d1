// dg_limit.cu -- troubled-cell indicator and limiters of the FP64 form, applied
// in place to a stage value (tiled layout [j][tile][var][mode][32]).
//
// One thread per element.  (1) The TVB-modified minmod test (Cockburn & Shu):
// per variable and direction, the face increment of the linear mode,
// sqrt(3) u_(1,0) in x and sqrt(3) u_(0,1) in y, against the forward and
// backward differences of the element means; |increment| <= M h^2 is never
// limited.  The element is troubled when any increment would change.  (2) A
// troubled element (by the test, or by given flags from the learned
// indicator) keeps its mean and the limited linear modes, every other mode
// zero.  (3) The positivity limiter of Sec. 2.4 (Zhang & Shu): density, then
// pressure (adiabatic), >= 1e-13 at the m x m volume nodes and the 4m face
// points, by scaling the non-mean modes towards the mean.  Limiting never
// writes mode 0, so reading the neighbours' means while they are limited in
// place is safe.
#include "dg_internal.cuh"

namespace dg {

namespace {

constexpr double SQRT3 = 1.7320508075688772935274463415059;  // phi_1(+1) / phi_0
constexpr double POS_EPS = 1e-13;

__device__ __forceinline__ double minmod3(double a, double b, double c) {
  if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
  if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
  return 0.0;
}

__device__ __forceinline__ double tvb_minmod(double a1, double a2, double a3, double mh2) {
  if (fabs(a1) <= mh2) return a1;
  return minmod3(a1, a2, a3);
}

struct LimitArgs {
  double* U;                  // tiled state, limited in place
  const double* GL;           // bc 1 ghosts: left/right columns [j][var][mode]
  const double* GR;
  const double* GB;           // bottom/top rows, tiled [it][var][mode][32]
  const double* GT;
  const unsigned char* given; // flags of another indicator [j][i], or null
  unsigned char* tvb_out;     // the TVB flags of the input state [j][i], or null
  const DevState* ts;
  Mesh ms;
  double tvb_m;
  int tvb;                    // run the TVB test (and its limiting when apply)
  int apply;                  // 0: flags only, the state is left alone
  int positivity;
  double gamma;
  Tables tab;
};

// mean of variable v of the element at (i, j) (maybe outside), boundary rule
template <int NV, int M>
__device__ __forceinline__ double mean_of(const LimitArgs& a, int i, int j, int v, double own) {
  const Mesh& ms = a.ms;
  if (i < 0 || i >= ms.nx || j < 0 || j >= ms.ny) {
    if (ms.bc == 0) {
      i = (i + ms.nx) % ms.nx;
      j = (j + ms.ny) % ms.ny;
    } else if (ms.bc == 1) {
      if (i < 0) return a.GL[((size_t)j * NV + v) * M];
      if (i >= ms.nx) return a.GR[((size_t)j * NV + v) * M];
      const double* g = j < 0 ? a.GB : a.GT;
      return g[(((size_t)(i >> 5) * NV + v) * M) * 32 + (i & 31)];
    } else {
      return own;  // transmissive: the element's own mean
    }
  }
  const size_t tile = (size_t)j * ms.ntx + (i >> 5);
  return a.U[((tile * NV + v) * M) * 32 + (i & 31)];
}

template <int NV>
__device__ __forceinline__ double pressure_of(const double* U, double gamma) {
  return (gamma - 1.0) * (U[NV - 1] - 0.5 * (U[1] * U[1] + U[2] * U[2]) / U[0]);
}

// values of all variables at check point n (volume node (q, r) = n / m, n % m
// for n < M; then the m points of the faces x = +1, x = -1, y = +1, y = -1)
template <int P, int NV>
__device__ __forceinline__ void eval_point(const double (&c)[NV][(P + 1) * (P + 1)], const Tables& t, int n,
                                           double* U) {
  constexpr int m = P + 1, M = m * m;
#pragma unroll
  for (int v = 0; v < NV; v++) {
    double acc = 0.0;
#pragma unroll
    for (int aa = 0; aa < m; aa++)
#pragma unroll
      for (int b = 0; b < m; b++) {
        double phi;
        if (n < M) phi = t.phi[n / m][aa] * t.phi[n % m][b];
        else {
          const int f = (n - M) / m, r = (n - M) % m;
          phi = f == 0 ? t.pp[aa] * t.phi[r][b]
              : f == 1 ? t.pm[aa] * t.phi[r][b]
              : f == 2 ? t.phi[r][aa] * t.pp[b]
                       : t.phi[r][aa] * t.pm[b];
        }
        acc += c[v][aa * m + b] * phi;
      }
    U[v] = acc;
  }
}

template <int P, int NV>
__global__ void __launch_bounds__(128) k_limit(const LimitArgs a) {
  constexpr int m = P + 1, M = m * m;
  if (a.ts->status != 0) return;
  const Mesh& ms = a.ms;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = (int)(gid & 31);
  const long long tile = gid >> 5;
  if (tile >= (long long)ms.ntx * ms.ny) return;
  const int j = (int)(tile / ms.ntx), bx = (int)(tile - (long long)j * ms.ntx);
  const int i = bx * 32 + lane;
  if (i >= ms.nx) return;
  double* base = a.U + ((size_t)tile * NV * M) * 32 + lane;
  double c[NV][M];
#pragma unroll
  for (int v = 0; v < NV; v++)
#pragma unroll
    for (int k = 0; k < M; k++) c[v][k] = base[(v * M + k) * 32];
  bool changed = false;

  if (a.tvb) {
    double sx[NV], sy[NV];
    const double mhx = a.tvb_m * ms.dx * ms.dx, mhy = a.tvb_m * ms.dy * ms.dy;
    int troubled = 0;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const double mean = c[v][0];
      const double mL = mean_of<NV, M>(a, i - 1, j, v, mean), mR = mean_of<NV, M>(a, i + 1, j, v, mean);
      const double mB = mean_of<NV, M>(a, i, j - 1, v, mean), mT = mean_of<NV, M>(a, i, j + 1, v, mean);
      const double ax = SQRT3 * c[v][m], ay = SQRT3 * c[v][1];
      sx[v] = tvb_minmod(ax, mR - mean, mean - mL, mhx);
      sy[v] = tvb_minmod(ay, mT - mean, mean - mB, mhy);
      if (sx[v] != ax || sy[v] != ay) troubled = 1;
    }
    const size_t e = (size_t)j * ms.nx + i;
    if (a.tvb_out) a.tvb_out[e] = (unsigned char)troubled;
    const int use = a.given ? a.given[e] : troubled;
    if (use && a.apply) {
#pragma unroll
      for (int v = 0; v < NV; v++) {
#pragma unroll
        for (int k = 1; k < M; k++) c[v][k] = 0.0;
        c[v][m] = sx[v] / SQRT3;
        c[v][1] = sy[v] / SQRT3;
      }
      changed = true;
    }
  }

  if (a.positivity && a.apply) {
    // conservative bound first: |U_v(x) - mean_v| <= sum_{k>0} |c_vk| max|phi_k|
    // with max|phi_ab| = sqrt(2a+1) sqrt(2b+1); elements provably positive at
    // every point skip the point checks (their limiter factor would be 1)
    double B[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      double s = 0.0;
#pragma unroll
      for (int k = 1; k < M; k++) s += fabs(c[v][k]) * sqrt((2.0 * (k / m) + 1.0) * (2.0 * (k % m) + 1.0));
      B[v] = s;
    }
    bool check = c[0][0] - B[0] < POS_EPS;
    if (NV == 4 && !check) {
      const double rl = c[0][0] - B[0];
      const double mxa = fabs(c[1][0]) + B[1], mya = fabs(c[2][0]) + B[2];
      const double pl = (a.gamma - 1.0) * (c[NV - 1][0] - B[NV - 1] - 0.5 * (mxa * mxa + mya * mya) / rl);
      check = !(pl >= POS_EPS);
    }
    if (check) {
      constexpr int NP = M + 4 * m;
      double U[NV];
      double rmin = INFINITY;
      for (int n = 0; n < NP; n++) {
        eval_point<P, NV>(c, a.tab, n, U);
        rmin = fmin(rmin, U[0]);
      }
      const double rbar = c[0][0];
      if (rmin < POS_EPS && rbar > POS_EPS) {
        const double th = fmax((rbar - POS_EPS) / (rbar - rmin), 0.0);
#pragma unroll
        for (int k = 1; k < M; k++) c[0][k] *= th;
        changed = true;
      }
      if (NV == 4) {
        double Ub[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) Ub[v] = c[v][0];
        const double pbar = pressure_of<NV>(Ub, a.gamma);
        if (pbar > POS_EPS) {
          double th = 1.0;
          for (int n = 0; n < NP; n++) {
            eval_point<P, NV>(c, a.tab, n, U);
            const double p = pressure_of<NV>(U, a.gamma);
            if (p < POS_EPS) th = fmin(th, (pbar - POS_EPS) / (pbar - p));
          }
          if (th < 1.0) {
            th = fmax(th, 0.0);
#pragma unroll
            for (int v = 0; v < NV; v++)
#pragma unroll
              for (int k = 1; k < M; k++) c[v][k] *= th;
            changed = true;
          }
        }
      }
    }
  }

  if (changed) {
#pragma unroll
    for (int v = 0; v < NV; v++)
#pragma unroll
      for (int k = 1; k < M; k++) base[(v * M + k) * 32] = c[v][k];
  }
}

template <int P, int NV>
cudaError_t launch_p(const LimitArgs& a, cudaStream_t s) {
  const long long threads = (long long)a.ms.ntx * a.ms.ny * 32;
  k_limit<P, NV><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_limit(double* U, const double* GL, const double* GR, const double* GB, const double* GT,
                         const unsigned char* given, unsigned char* tvb_out, const DevState* ts,
                         const Mesh& ms, const Phys& ph, const Tables& tab, int p, int nv, int tvb,
                         int apply, int positivity, cudaStream_t s) {
  LimitArgs a;
  a.U = U;
  a.GL = GL;
  a.GR = GR;
  a.GB = GB;
  a.GT = GT;
  a.given = given;
  a.tvb_out = tvb_out;
  a.ts = ts;
  a.ms = ms;
  a.tvb_m = ph.tvb_m;
  a.tvb = tvb;
  a.apply = apply;
  a.positivity = positivity;
  a.gamma = ph.gamma;
  a.tab = tab;
  if (nv == 4) {
    switch (p) {
      case 1: return launch_p<1, 4>(a, s);
      case 2: return launch_p<2, 4>(a, s);
      case 3: return launch_p<3, 4>(a, s);
      case 4: return launch_p<4, 4>(a, s);
    }
  } else {
    switch (p) {
      case 1: return launch_p<1, 3>(a, s);
      case 2: return launch_p<2, 3>(a, s);
      case 3: return launch_p<3, 3>(a, s);
      case 4: return launch_p<4, 3>(a, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace dg
