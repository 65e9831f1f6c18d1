// dg_mlp.cu -- the learned troubled-cell indicator: a multilayer perceptron
// nin -> 64 (GELU) -> 64 (GELU) -> 1 logit on the modal coefficients of an
// element and its four neighbours, with BF16 weights and FP32 accumulation.
//
// Features of element e (FP32): for the stencil s = 0 the element, 1 left,
// 2 right, 3 below, 4 above (outside elements by the boundary rule), variable
// v and mode k, x[(s * nv + v) * M + k] = c_s[v][k] * (1 / S_v) with S_v the
// largest |c_s[v][k]| over the stencil and the modes (1 when all vanish): the
// reciprocal and the product in FP64, the product rounded once to FP32
// (dg_features, the training inputs).  The inference kernel on the tensor
// cores applies the scale after the first layer's sums instead: the
// coefficients, truncated to FP32 and held as BF16 pairs hi + lo (2^-17
// relative), enter the products unscaled, and the sums of each variable are
// multiplied by 1 / S_v rounded to FP32 -- no FP64 instruction per input.
//
// Parameters (FP32 master copy, flat): W1 [64][nin], b1 [64], W2 [64][64],
// b2 [64], w3 [64], b3.  The products use the weights rounded to BF16
// (round to nearest even); gradients are taken through that rounding as the
// identity.  Loss: mean over the batch of the weighted binary cross entropy
// w_y (softplus(z) - y z), w_1 = pos_weight, w_0 = 1.  Optimiser: Adam
// (beta 0.9, 0.999, eps 1e-8) on the master copy.
//
// Training (forward, backward, Adam) runs on the CUDA cores in FP32; the
// inference inside the limiter (k_mlp_tc) runs its two dense layers on the
// tensor cores, the activations split into BF16 hi + lo against the BF16
// weights with FP32 accumulators in tensor memory.
#include <cuda_bf16.h>

#include <string.h>

#include <new>
#include <vector>

#include "dg_internal.cuh"
#include "dg_tc.cuh"

namespace dg {

namespace {

constexpr int H = MLP_HIDDEN;

__device__ __forceinline__ float gelu(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float a) {
  return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) + a * 0.39894228040143268f * expf(-0.5f * a * a);
}

struct Offs {
  int W1, b1, W2, b2, w3, b3, n;
};
__host__ __device__ inline Offs offs(int nin) {
  Offs o;
  o.W1 = 0;
  o.b1 = H * nin;
  o.W2 = o.b1 + H;
  o.b2 = o.W2 + H * H;
  o.w3 = o.b2 + H;
  o.b3 = o.w3 + H;
  o.n = o.b3 + 1;
  return o;
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ q, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = __float2bfloat16_rn(p[i]);
}

// out[b][o] = act(sum_i in[b][i] W[o][i] + bias[o]); pre-activation kept
__global__ void k_dense(const float* __restrict__ in, const __nv_bfloat16* __restrict__ W,
                        const __nv_bfloat16* __restrict__ bias, float* __restrict__ pre,
                        float* __restrict__ out, int B, int nin, int nout, int act) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * nout) return;
  const int b = (int)(t / nout), o = (int)(t - (long long)b * nout);
  const float* x = in + (size_t)b * nin;
  const __nv_bfloat16* w = W + (size_t)o * nin;
  float acc = __bfloat162float(bias[o]);
  for (int i = 0; i < nin; i++) acc = fmaf(x[i], __bfloat162float(w[i]), acc);
  if (pre) pre[t] = acc;
  out[t] = act ? gelu(acc) : acc;
}

// dz[b] = w_y (sigmoid(z) - y) / B and the per-example loss w_y (softplus(z) - y z)
__global__ void k_out_grad(const float* __restrict__ z, const float* __restrict__ y, float* __restrict__ dz,
                           double* __restrict__ loss, int B, float pos_weight) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float zz = z[b], yy = y[b];
  const float w = yy > 0.5f ? pos_weight : 1.0f;
  const float sig = 1.0f / (1.0f + expf(-zz));
  dz[b] = w * (sig - yy) / (float)B;
  const float sp = zz > 0.0f ? zz + log1pf(expf(-zz)) : log1pf(expf(zz));
  loss[b] = (double)(w * (sp - yy * zz));
}

// G[o][i] = sum_b A[b][o] X[b][i] (weight gradient) and, for i == nin, the
// bias gradient sum_b A[b][o]
__global__ void k_wgrad(const float* __restrict__ A, const float* __restrict__ X, float* __restrict__ Gw,
                        float* __restrict__ Gb, int B, int nout, int nin) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nout * (nin + 1)) return;
  const int o = (int)(t / (nin + 1)), i = (int)(t - (long long)o * (nin + 1));
  float acc = 0.0f;
  if (i < nin) {
    for (int b = 0; b < B; b++) acc = fmaf(A[(size_t)b * nout + o], X[(size_t)b * nin + i], acc);
    Gw[(size_t)o * nin + i] = acc;
  } else {
    for (int b = 0; b < B; b++) acc += A[(size_t)b * nout + o];
    Gb[o] = acc;
  }
}

// D[b][i] = act'(pre[b][i]) sum_o A[b][o] W[o][i]  (gradient at the pre-activation below)
__global__ void k_igrad(const float* __restrict__ A, const __nv_bfloat16* __restrict__ W,
                        const float* __restrict__ pre, float* __restrict__ D, int B, int nout, int nin) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * nin) return;
  const int b = (int)(t / nin), i = (int)(t - (long long)b * nin);
  float acc = 0.0f;
  for (int o = 0; o < nout; o++) acc = fmaf(A[(size_t)b * nout + o], __bfloat162float(W[(size_t)o * nin + i]), acc);
  D[t] = acc * gelu_d(pre[t]);
}

__global__ void k_sum(const double* __restrict__ x, int n, double* __restrict__ out) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += x[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int n, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---- features of the FP64 tiled state -----------------------------------------

namespace {

struct FeatArgs {
  const double* U;
  const double *GL, *GR, *GB, *GT;
  Mesh ms;
};

// coefficient k of variable v of the stencil element (i, j) (maybe outside)
template <int NV, int M>
__device__ __forceinline__ double coef(const FeatArgs& a, int i, int j, int ci, int cj, int v, int k) {
  const Mesh& ms = a.ms;
  if (i < 0 || i >= ms.nx || j < 0 || j >= ms.ny) {
    if (ms.bc == 0) {
      i = (i + ms.nx) % ms.nx;
      j = (j + ms.ny) % ms.ny;
    } else if (ms.bc == 1) {
      if (i < 0) return a.GL[((size_t)j * NV + v) * M + k];
      if (i >= ms.nx) return a.GR[((size_t)j * NV + v) * M + k];
      const double* g = j < 0 ? a.GB : a.GT;
      return g[(((size_t)(i >> 5) * NV + v) * M + k) * 32 + (i & 31)];
    } else {
      i = ci;
      j = cj;
    }
  }
  const size_t tile = (size_t)j * ms.ntx + (i >> 5);
  return a.U[((tile * NV + v) * M + k) * 32 + (i & 31)];
}

// R[v] = 1 / S_v.  The largest |c| is found on the bit patterns (sign bit
// cleared, compared as integers: the order of non-negative doubles), which
// keeps the scan off the narrow FP64 unit; one FP64 reciprocal per variable.
template <int NV, int M>
__device__ __forceinline__ void stencil_scales(const FeatArgs& a, int i, int j, double* R) {
  const int di[5] = {0, -1, 1, 0, 0}, dj[5] = {0, 0, 0, -1, 1};
  unsigned long long mx[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) mx[v] = 0ull;
  for (int s = 0; s < 5; s++)
#pragma unroll
    for (int v = 0; v < NV; v++)
      for (int k = 0; k < M; k++) {
        const unsigned long long b =
            (unsigned long long)__double_as_longlong(coef<NV, M>(a, i + di[s], j + dj[s], i, j, v, k)) &
            0x7fffffffffffffffull;
        mx[v] = b > mx[v] ? b : mx[v];
      }
#pragma unroll
  for (int v = 0; v < NV; v++) R[v] = mx[v] ? 1.0 / __longlong_as_double((long long)mx[v]) : 1.0;
}

template <int NV, int M>
__global__ void k_features(const FeatArgs a, const int* __restrict__ elems, int n, float* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int e = elems[t];
  if (e < 0 || e >= a.ms.nx * a.ms.ny) return;
  const int i = e % a.ms.nx, j = e / a.ms.nx;
  const int di[5] = {0, -1, 1, 0, 0}, dj[5] = {0, 0, 0, -1, 1};
  double S[NV];
  stencil_scales<NV, M>(a, i, j, S);
  float* o = out + (size_t)t * 5 * NV * M;
  for (int s = 0; s < 5; s++)
#pragma unroll
    for (int v = 0; v < NV; v++)
      for (int k = 0; k < M; k++)
        o[(s * NV + v) * M + k] = (float)(coef<NV, M>(a, i + di[s], j + dj[s], i, j, v, k) * S[v]);
}

// ---- fused inference on the tensor cores ----------------------------------
// One CTA of 256 threads per 128 elements (4 mesh tiles); element row r is
// the MMA row r.  The scale 1/S_v of a feature depends only on the element's
// stencil and the variable, so layer 1 is sum_v (1/S_v) (W1_v c_v): the
// unscaled coefficients enter the MMAs and four accumulators in tensor memory
// (one per variable, 64 columns each) are scaled and summed in the epilogue.
// Each element's coefficients are then converted once, not once per stencil
// they enter: a pre-pass (k_elem_prep) writes every coefficient as a BF16
// pair hi + lo of its FP32 truncation (x = hi + lo to 2^-16 relative; the
// weights are BF16 already, so the two MMAs reproduce the FP32 products) and
// every element's max |c| per variable.  Layer 1 runs over the inputs in
// chunks of 64, ordered by variable (each variable's stencil groups of 8
// modes, padded to an even count so that an MMA's K = 16 never spans two
// variables): the 256 threads gather the chunk's pairs (two threads per row,
// 32 inputs each) into the hi and lo operands, and one thread issues the
// chunk's MMAs (M 128, N 64, K 16) into the accumulator of their variable.
// The A operand is double-buffered: the next chunk's pairs are loaded while
// this one is stored and its MMAs run.  The W1 chunks arrive by bulk copies
// into a four-stage ring, two chunks ahead.  1/S_v of every element's stencil
// comes from its own pass (k_stencil_scale).  The epilogue reads the four
// accumulators back (warp w: lanes 32 (w mod 4).., columns 32 (w / 4)..),
// forms sum_v (1/S_v) D1_v + b1, applies GELU and splits the hidden units into
// BF16 hi + lo, the A operand of layer 2 (64 -> 64, same scheme, its
// accumulator in the first variable's columns); the last epilogue forms the
// logit.
constexpr int TC_ROWS = 128, TC_KC = 64, TC_THREADS = 256, TC_WST = 4;
constexpr int TC_A = 0;                          // [2 buffers][hi, lo][128 x 64] BF16, 16 KB each
constexpr int TC_B = TC_A + 4 * 16384;           // W1 chunks [TC_WST stages][64 x 64] BF16
constexpr int TC_W2 = TC_B + TC_WST * 8192;      // W2 [64 x 64] BF16
constexpr int TC_PAR = TC_W2 + 8192;             // b1, b2, w3 [64] and b3, FP32 (1 KB)
constexpr int TC_PZ = TC_PAR + 1024;             // partial logits [128] FP32
constexpr int TC_BAR = TC_PZ + 512;              // mbarriers: A buffer [2], W1 stage [4], W2, layer 2
constexpr int TC_TM = TC_BAR + 64;               // tensor-memory base address
constexpr int TC_SMEM = TC_TM + 16;              // 105.6 KB: two CTAs per SM, 2 x 256 tensor-memory columns

// byte offset of (row, k) in a K-major no-swizzle operand of `rows` rows
__host__ __device__ inline int tc_off(int rows, int row, int k) {
  return (k >> 3) * (rows * 16) + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ unsigned pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a in the low half
  return *reinterpret_cast<const unsigned*>(&h);
}

// x = hi + lo exactly in FP32 terms: lo is the BF16 rounding of x - hi
__device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo) {
  unsigned h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
    h[e] = *reinterpret_cast<const unsigned*>(&hh);
    l[e] = pack_bf16(x[2 * e] - __low2float(hh), x[2 * e + 1] - __high2float(hh));
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// double -> float, round to nearest even, on the integer pipe (this part
// runs the conversion instruction on its narrow FP64 unit); finite |x| < 2^128
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int e = (int)((hi >> 20) & 0x7ffu);
  unsigned f;
  if (e >= 897) {  // normal result: keep 23 fraction bits, round on the 29 dropped
    const unsigned rest = lo & 0x1FFFFFFFu;
    f = ((unsigned)(e - 896) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    f += (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ? 1u : 0u;
  } else if (e >= 872) {  // subnormal result: the significand shifted right by 926 - e
    const unsigned long long sig = (1ull << 52) | (b & 0xFFFFFFFFFFFFFull);
    const int sh = 926 - e;
    const unsigned long long q = sig >> sh, r = sig & ((1ull << sh) - 1), h = 1ull << (sh - 1);
    f = (unsigned)q + ((r > h || (r == h && (q & 1ull))) ? 1u : 0u);
  } else {
    f = 0u;
  }
  return __uint_as_float(f | (hi & 0x80000000u));
}

// double -> float by truncation of the 29 dropped fraction bits, branch-free on
// the integer pipe: |x| in [2^-126, 2^128) keeps its exponent and top 23
// fraction bits (within one FP32 unit, toward zero), smaller |x| gives zero
__device__ __forceinline__ float d2f_rz(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ah = hi & 0x7FFFFFFFu;
  const unsigned f = ah >= (897u << 20) ? (((ah - (896u << 20)) << 3) | (lo >> 29)) : 0u;
  return __uint_as_float(f | (hi & 0x80000000u));
}

// GELU a Phi(a) of a pair, for the inference epilogues, in packed FP32x2
// arithmetic.  Phi(a) = (1 + erf(a / sqrt 2)) / 2 with erf from Abramowitz &
// Stegun 7.1.26 (Hastings' rational form, |error| <= 1.5e-7): for x >= 0,
// erf x = 1 - q, q = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),
// t = 1 / (1 + p x).  With x = |a| / sqrt 2 and h = a q / 2, a Phi(a) is
// a - h for a >= 0 and h for a < 0.  exp(-a^2 / 2) = 2^(-a^2 log2(e) / 2) by
// the hardware base-2 exponential (zero for |a| > 13).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float2 gelu_pair(float2 a) {
  const float2 x = make_float2(fabsf(a.x) * 0.70710678118654752f, fabsf(a.y) * 0.70710678118654752f);
  const float2 d = __ffma2_rn(x, make_float2(0.3275911f, 0.3275911f), make_float2(1.0f, 1.0f));
  const float2 t = make_float2(__fdividef(1.0f, d.x), __fdividef(1.0f, d.y));
  float2 q = __ffma2_rn(t, make_float2(1.061405429f, 1.061405429f), make_float2(-1.453152027f, -1.453152027f));
  q = __ffma2_rn(q, t, make_float2(1.421413741f, 1.421413741f));
  q = __ffma2_rn(q, t, make_float2(-0.284496736f, -0.284496736f));
  q = __ffma2_rn(q, t, make_float2(0.254829592f, 0.254829592f));
  q = __fmul2_rn(q, t);
  const float2 g = __fmul2_rn(__fmul2_rn(a, a), make_float2(-0.72134752044448170f, -0.72134752044448170f));
  q = __fmul2_rn(q, make_float2(ex2_approx(g.x), ex2_approx(g.y)));
  const float2 h = __fmul2_rn(__fmul2_rn(a, make_float2(0.5f, 0.5f)), q);
  return make_float2(a.x >= 0.0f ? a.x - h.x : h.x, a.y >= 0.0f ? a.y - h.y : h.y);
}

// the mesh element standing for stencil element (ii, jj) of element (ci, cj):
// false for a fixed ghost element (bc 1)
__device__ __forceinline__ bool mesh_elem(const Mesh& ms, int ii, int jj, int ci, int cj, long long& tile,
                                          int& lane) {
  if (ii < 0 || ii >= ms.nx || jj < 0 || jj >= ms.ny) {
    if (ms.bc == 0) {
      ii = (ii + ms.nx) % ms.nx;
      jj = (jj + ms.ny) % ms.ny;
    } else if (ms.bc == 1) {
      return false;
    } else {
      ii = ci;
      jj = cj;
    }
  }
  tile = (long long)jj * ms.ntx + (ii >> 5);
  lane = ii & 31;
  return true;
}

// an FP64 coefficient as the BF16 pair of its FP32 truncation: hi in the low
// half, lo = the BF16 rounding of x - hi in the high half
__device__ __forceinline__ unsigned bf16_pair(double c) {
  const float x = d2f_rz(c);
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  return (unsigned)__bfloat16_as_ushort(h) | ((unsigned)__bfloat16_as_ushort(l) << 16);
}

// input groups of 8 modes of one (variable, stencil element): per variable
// 5 * GPB groups padded to an even count GPV (an MMA's K = 16 is two groups),
// group G = v * GPV + s * GPB + g holding modes 8 g .. 8 g + 7 of variable v
// of stencil element s (zero past M)
__host__ __device__ constexpr int tc_gpb(int M) { return (M + 7) / 8; }
__host__ __device__ constexpr int tc_gpv(int M) { return (5 * tc_gpb(M) + 1) / 2 * 2; }

// The BF16 pairs of an element's variable as GPB groups of 8 words (zero past
// mode M), so that a thread loads a group with two 16-byte loads:
//   mesh elements   [tile][v][g][lane][8]   (32 elements of a tile row side by side)
//   bc 1 ghosts     GL, GR: [j][v][g][8];  GB, GT: [x tile][v][g][lane][8]
// Per element and variable the prep pass also writes the bits of max |c| over
// the modes, [tile][v][32] (the order of non-negative doubles as integers).
template <int M>
__device__ __forceinline__ void put_groups(const double* __restrict__ src, int stride, unsigned* __restrict__ dst,
                                           int gstride, unsigned long long* mx) {
  constexpr int GPB = tc_gpb(M);
  unsigned long long m = 0ull;
#pragma unroll
  for (int g = 0; g < GPB; g++) {
    unsigned w[8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
      const int k = g * 8 + e;
      double x = 0.0;
      if (k < M) x = src[k * stride];
      const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
      m = b > m ? b : m;
      w[e] = bf16_pair(x);
    }
    uint4* q = reinterpret_cast<uint4*>(dst + (size_t)g * gstride);
    q[0] = make_uint4(w[0], w[1], w[2], w[3]);
    q[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
  if (mx) *mx = m;
}

// one thread per (tile, variable, lane) of the state: t = (tile * NV + v) * 32 + lane
template <int NV, int M>
__global__ void k_elem_prep(const double* __restrict__ U, unsigned long long* __restrict__ mx,
                            unsigned* __restrict__ img, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  put_groups<M>(U + (size_t)(t >> 5) * (M * 32) + (t & 31), 32,
                img + ((size_t)(t >> 5) * tc_gpb(M) * 32 + (t & 31)) * 8, 256, mx + t);
}

// the fixed ghost elements (bc 1): GL, GR ([j][v][k], ny * NV rows each), then
// GB, GT ([x tile][v][k][32], ntx * NV * 32 columns each)
template <int NV, int M>
__global__ void k_ghost_prep(const double* __restrict__ GL, const double* __restrict__ GR,
                             const double* __restrict__ GB, const double* __restrict__ GT, unsigned* __restrict__ gl,
                             unsigned* __restrict__ gr, unsigned* __restrict__ gb, unsigned* __restrict__ gt, int ny,
                             int ntx) {
  constexpr int GPB = tc_gpb(M);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nside = (long long)ny * NV, ntop = (long long)ntx * NV * 32;
  if (t < 2 * nside) {
    const bool r = t >= nside;
    const long long q = t - (r ? nside : 0);  // j * NV + v
    put_groups<M>((r ? GR : GL) + (size_t)q * M, 1, (r ? gr : gl) + (size_t)q * GPB * 8, 8, nullptr);
  } else if (t < 2 * nside + 2 * ntop) {
    const long long u = t - 2 * nside;
    const bool top = u >= ntop;
    const long long q = u - (top ? ntop : 0);  // (x tile * NV + v) * 32 + lane
    put_groups<M>((top ? GT : GB) + (size_t)(q >> 5) * (M * 32) + (q & 31), 32,
                  (top ? gt : gb) + ((size_t)(q >> 5) * GPB * 32 + (q & 31)) * 8, 256, nullptr);
  }
}

// 1 / S_v of every element's stencil, FP32, [tile][lane] as 4 floats (the
// fourth unused for 3 variables): S_v from the per-element maxima (the fixed
// ghost elements of bc 1 scanned here) rounded to FP32, its FP32 reciprocal,
// 1 where S_v vanishes or is below the FP32 normal range (its coefficients
// truncate to zero)
template <int NV, int M>
__global__ void k_stencil_scale(const FeatArgs a, const unsigned long long* __restrict__ emax,
                                float4* __restrict__ rs, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int tile = (int)(t >> 5);  // ntiles < 2^31
  const int j = tile / a.ms.ntx, i = (tile - j * a.ms.ntx) * 32 + (int)(t & 31);
  float R[4] = {1.0f, 1.0f, 1.0f, 1.0f};
  if (i < a.ms.nx) {
    unsigned long long mx[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) mx[v] = 0ull;
#pragma unroll
    for (int s = 0; s < 5; s++) {
      const int ii = i + (s == 1 ? -1 : s == 2 ? 1 : 0), jj = j + (s == 3 ? -1 : s == 4 ? 1 : 0);
      long long te;
      int le;
      if (mesh_elem(a.ms, ii, jj, i, j, te, le)) {
#pragma unroll
        for (int v = 0; v < NV; v++) {
          const unsigned long long b = emax[((size_t)te * NV + v) * 32 + le];
          mx[v] = b > mx[v] ? b : mx[v];
        }
      } else {
#pragma unroll
        for (int v = 0; v < NV; v++)
          for (int k = 0; k < M; k++) {
            const unsigned long long b =
                (unsigned long long)__double_as_longlong(coef<NV, M>(a, ii, jj, i, j, v, k)) & 0x7fffffffffffffffull;
            mx[v] = b > mx[v] ? b : mx[v];
          }
      }
    }
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const float m = d2f_rn(__longlong_as_double((long long)mx[v]));
      R[v] = m >= 1.17549435e-38f ? __frcp_rn(m) : 1.0f;
    }
  }
  rs[t] = make_float4(R[0], R[1], R[2], R[3]);
}

// the inference's scratch: per-element maxima, the BF16 pair images of
// the state and of the four ghost arrays, the stencil scales (byte offsets,
// 256-byte aligned)
struct WorkPlan {
  size_t img, gl, gr, gb, gt, rs, total;
};
inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }
inline WorkPlan work_plan(const Mesh& ms, int nv, int M) {
  const size_t nt = (size_t)ms.ntx * ms.ny, grp = (size_t)nv * tc_gpb(M) * 8 * sizeof(unsigned);
  WorkPlan w;
  w.img = al256(nt * nv * 32 * sizeof(unsigned long long));
  w.gl = w.img + al256(nt * 32 * grp);
  w.gr = w.gl + al256((size_t)ms.ny * grp);
  w.gb = w.gr + al256((size_t)ms.ny * grp);
  w.gt = w.gb + al256((size_t)ms.ntx * 32 * grp);
  w.rs = w.gt + al256((size_t)ms.ntx * 32 * grp);
  w.total = w.rs + al256(nt * 32 * sizeof(float4));
  return w;
}

struct ImgArgs {
  const float4* rs;
  const unsigned *img, *gl, *gr, *gb, *gt;
};

// words of a group of 8 modes of stencil element s of this row (zeros for an
// invalid row, a padding group or one past the last)
template <int NV, int M>
__device__ __forceinline__ void tc_load_group(const unsigned* const* sp, const int* sst, bool valid, int G,
                                              uint4& w0, uint4& w1) {
  constexpr int GPB = tc_gpb(M), GPV = tc_gpv(M);
  const int v = G / GPV, r = G - v * GPV, s = r / GPB, g = r - s * GPB;
  w0 = w1 = make_uint4(0u, 0u, 0u, 0u);
  if (valid && v < NV && s < 5) {
    const uint4* q = reinterpret_cast<const uint4*>(sp[s] + (v * GPB + g) * sst[s]);
    w0 = __ldg(q);
    w1 = __ldg(q + 1);
  }
}

// a group's 8 pairs as the hi and lo operand rows (low halves, high halves)
__device__ __forceinline__ void tc_unpair(const uint4& w0, const uint4& w1, uint4& hi, uint4& lo) {
  hi = make_uint4(__byte_perm(w0.x, w0.y, 0x5410), __byte_perm(w0.z, w0.w, 0x5410), __byte_perm(w1.x, w1.y, 0x5410),
                  __byte_perm(w1.z, w1.w, 0x5410));
  lo = make_uint4(__byte_perm(w0.x, w0.y, 0x7632), __byte_perm(w0.z, w0.w, 0x7632), __byte_perm(w1.x, w1.y, 0x7632),
                  __byte_perm(w1.z, w1.w, 0x7632));
}

template <int NV, int M>
__global__ void __launch_bounds__(TC_THREADS, 2)
    k_mlp_tc(const FeatArgs a, const ImgArgs im, const unsigned char* __restrict__ wp, float threshold,
             DevState* ts, unsigned char* __restrict__ flags, float* __restrict__ logits, long long ntiles,
             int ahead) {
  constexpr int GPB = tc_gpb(M), GPV = tc_gpv(M), NGT = NV * GPV, NC = (NGT + 7) / 8, H2 = MLP_HIDDEN;
  static_assert(MLP_HIDDEN == 64 && NV <= 4, "tile plan: NV accumulators of 64 columns in 256");
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TC_BAR);
  unsigned* s_taddr = reinterpret_cast<unsigned*>(sm + TC_TM);
  // this row's element and where its stencil's pairs are are found first,
  // so that the first chunk's loads are in flight during the set-up; the
  // status is read here too and decides only whether the CTA writes (a set
  // status leaves every output as it was), so that no CTA waits for it
  const int status = *(volatile const int*)&ts->status;
  const int tid = threadIdx.x, warp = tid >> 5, row = tid & (TC_ROWS - 1), half = tid >> 7;
  const unsigned idesc = tc_idesc_bf16(TC_ROWS, H2);

  // this row's element and its stencil (s = 0 own, 1 left, 2 right, 3 below, 4 above)
  const int tile = (int)blockIdx.x * 4 + (row >> 5);  // ntiles < 2^31
  int i = 0, j = 0;
  bool valid = false;
  if (tile < ntiles) {
    j = tile / a.ms.ntx;
    i = (tile - j * a.ms.ntx) * 32 + (row & 31);
    valid = i < a.ms.nx;
  }
  // each stencil element's pairs: the first word of its group 0 of variable
  // 0 and the words from one group to the next
  const unsigned* sp[5];
  int sst[5];
#pragma unroll
  for (int s = 0; s < 5; s++) {
    const int ii = i + (s == 1 ? -1 : s == 2 ? 1 : 0), jj = j + (s == 3 ? -1 : s == 4 ? 1 : 0);
    long long te;
    int le;
    sp[s] = im.img;
    sst[s] = 0;
    if (!valid) continue;
    if (mesh_elem(a.ms, ii, jj, i, j, te, le)) {
      sp[s] = im.img + ((size_t)te * NV * GPB * 32 + le) * 8;
      sst[s] = 256;
    } else if (ii < 0 || ii >= a.ms.nx) {  // [j][v][g][8]
      sp[s] = (ii < 0 ? im.gl : im.gr) + (size_t)j * NV * GPB * 8;
      sst[s] = 8;
    } else {  // [x tile][v][g][lane][8]
      sp[s] = (jj < 0 ? im.gb : im.gt) + ((size_t)(i >> 5) * NV * GPB * 32 + (i & 31)) * 8;
      sst[s] = 256;
    }
  }

  // ---- layer 1 over the input chunks ----
  // this thread's four groups of chunk c, at K positions 8 kg(g): with an even
  // GPB the groups c * 8 + 2 g + half (a group pair shares its variable and
  // stencil element, so one code serves both halves); else c * 8 + 4 half + g,
  // the branch on the warp-uniform half making every group index a constant
  auto kg = [&](int g) { return GPB % 2 == 0 ? 2 * g + half : 4 * half + g; };
  auto load4 = [&](int c, uint4* w) {
    if constexpr (GPB % 2 == 0) {
#pragma unroll
      for (int g = 0; g < 4; g++) {
        const int G0 = c * 8 + 2 * g, v = G0 / GPV, r = G0 - v * GPV, s = r / GPB, gg = r - s * GPB + half;
        w[2 * g] = w[2 * g + 1] = make_uint4(0u, 0u, 0u, 0u);
        if (valid && v < NV) {
          const uint4* q = reinterpret_cast<const uint4*>(sp[s] + (v * GPB + gg) * sst[s]);
          w[2 * g] = __ldg(q);
          w[2 * g + 1] = __ldg(q + 1);
        }
      }
    } else if (half == 0) {
#pragma unroll
      for (int g = 0; g < 4; g++) tc_load_group<NV, M>(sp, sst, valid, c * 8 + g, w[2 * g], w[2 * g + 1]);
    } else {
#pragma unroll
      for (int g = 0; g < 4; g++) tc_load_group<NV, M>(sp, sst, valid, c * 8 + 4 + g, w[2 * g], w[2 * g + 1]);
    }
  };
  uint4 cur[8];
  load4(0, cur);
  // 1 / S_v of this row's stencil (used by the first epilogue)
  const float4 r4 = valid ? im.rs[(size_t)tile * 32 + (row & 31)] : make_float4(1.0f, 1.0f, 1.0f, 1.0f);
  const float R[4] = {r4.x, r4.y, r4.z, r4.w};
  if (warp == 0) tmem_alloc(s_taddr, 256);  // variable v's layer-1 sums: columns 64 v ..; layer 2: 0..63
  if (tid == 64) {
    // the CTA `ahead` places on (one wave later) first touches the pairs of
    // the tile row above its own and its scales: ask the L2 for them now
    const long long nb = (long long)blockIdx.x + ahead, t0 = nb * 4 + a.ms.ntx;
    const long long t1 = t0 + 4 < ntiles ? t0 + 4 : ntiles;
    if (t0 < t1) bulk_prefetch_l2(im.img + (size_t)t0 * NV * GPB * 256, (unsigned)(t1 - t0) * NV * GPB * 1024);
    if (nb * 4 < ntiles)
      bulk_prefetch_l2(im.rs + nb * 128, (unsigned)((ntiles - nb * 4 < 4 ? ntiles - nb * 4 : 4) * 32 * sizeof(float4)));
  }
  if (tid == 32) {  // warp 1, while warp 0 allocates
#pragma unroll
    for (int b = 0; b < 8; b++) mbar_init(&bar[b], 1);
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[6], 8192 + 1024);
    bulk_g2s(sm + TC_W2, wp + (size_t)NC * 8192, 8192, &bar[6]);
    bulk_g2s(sm + TC_PAR, wp + (size_t)NC * 8192 + 8192, 1024, &bar[6]);
#pragma unroll
    for (int c = 0; c < (NC < TC_WST ? NC : TC_WST); c++) {
      mbar_expect_tx(&bar[2 + c], 8192);
      bulk_g2s(sm + TC_B + c * 8192, wp + (size_t)c * 8192, 8192, &bar[2 + c]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned taddr = *s_taddr;
  bool ok = true;

#pragma unroll
  for (int c = 0; c < NC; c++) {
    // the next chunk's pairs are in flight while this one is stored and multiplied
    uint4 nxt[8];
    if (c + 1 < NC) load4(c + 1, nxt);
    unsigned char* Ahi = sm + TC_A + (c & 1) * 32768;
    unsigned char* Alo = Ahi + 16384;
    if (c >= 2) {
      // the MMAs of chunk c - 2, the last readers of this A buffer and of W1
      // stage (c + 2) mod 4, are done
      ok &= mbar_wait(&bar[c & 1], ((c - 2) >> 1) & 1);
      if (tid == 0 && c + 2 < NC) {
        const int st = (c + 2) & 3;
        mbar_expect_tx(&bar[2 + st], 8192);
        bulk_g2s(sm + TC_B + st * 8192, wp + (size_t)(c + 2) * 8192, 8192, &bar[2 + st]);
      }
    }
#pragma unroll
    for (int g = 0; g < 4; g++) {
      uint4 hi, lo;
      tc_unpair(cur[2 * g], cur[2 * g + 1], hi, lo);
      const int off = tc_off(TC_ROWS, row, kg(g) * 8);
      *reinterpret_cast<uint4*>(Ahi + off) = hi;
      *reinterpret_cast<uint4*>(Alo + off) = lo;
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      ok &= mbar_wait(&bar[2 + (c & 3)], (c >> 2) & 1);
      tc_fence_after();
      const unsigned aH = smem_addr(Ahi), aL = smem_addr(Alo), bB = smem_addr(sm + TC_B + (c & 3) * 8192);
#pragma unroll
      for (int ks = 0; ks < TC_KC / 16; ks++) {
        // K step ks: groups c * 8 + 2 ks and + 1, both of variable v; its
        // first K step of a variable starts that variable's sums
        const int G0 = c * 8 + 2 * ks, v = G0 / GPV;
        if (G0 < NGT) {
          const unsigned d = taddr + 64 * v;
          const uint64_t db = tc_sdesc(bB + ks * 2048, 1024, 128);
          tc_mma(d, tc_sdesc(aH + ks * 4096, 2048, 128), db, idesc, G0 > v * GPV ? 1 : 0);
          tc_mma(d, tc_sdesc(aL + ks * 4096, 2048, 128), db, idesc, 1);
        }
      }
      tc_commit(&bar[c & 1]);
    }
    if (c + 1 < NC) {
#pragma unroll
      for (int q = 0; q < 8; q++) cur[q] = nxt[q];
    }
  }
  // the commits of the last two chunks (each covers every earlier MMA)
  ok &= mbar_wait(&bar[(NC - 1) & 1], ((NC - 1) >> 1) & 1);
  if (NC >= 2) ok &= mbar_wait(&bar[NC & 1], ((NC - 2) >> 1) & 1);
  ok &= mbar_wait(&bar[6], 0);
  tc_fence_after();
  const float* par = reinterpret_cast<const float*>(sm + TC_PAR);  // b1, b2, w3, b3
  const int quarter = warp & 3, ch = warp >> 2;
  const unsigned tl = taddr + ((unsigned)(quarter * 32) << 16);
  // ---- epilogue 1: h1 = GELU(sum_v (1 / S_v) D1_v + b1) as the layer-2 A operand ----
  // (8 hidden units at a time: the loop is not unrolled, to keep the code small)
#pragma unroll 1
  for (int g = 0; g < 4; g++) {
    const int col = ch * 32 + g * 8;
    float d[32], x[8];
    tmem_ld8x4(tl + col, tl + 64 + col, tl + (NV > 2 ? 128 : 0) + col, tl + (NV > 3 ? 192 : 0) + col, d);
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      float2 h = make_float2(par[col + e], par[col + e + 1]);
#pragma unroll
      for (int v = 0; v < NV; v++) h = __ffma2_rn(make_float2(R[v], R[v]), make_float2(d[8 * v + e], d[8 * v + e + 1]), h);
      h = gelu_pair(h);
      x[e] = h.x;
      x[e + 1] = h.y;
    }
    uint4 hi, lo;
    split8(x, hi, lo);
    const int off = tc_off(TC_ROWS, row, col);
    *reinterpret_cast<uint4*>(sm + TC_A + off) = hi;
    *reinterpret_cast<uint4*>(sm + TC_A + 16384 + off) = lo;
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    tc_fence_after();
    const unsigned aH = smem_addr(sm + TC_A), aL = aH + 16384, bW = smem_addr(sm + TC_W2);
#pragma unroll
    for (int ks = 0; ks < H2 / 16; ks++) {
      const uint64_t db = tc_sdesc(bW + ks * 2048, 1024, 128);
      tc_mma(taddr, tc_sdesc(aH + ks * 4096, 2048, 128), db, idesc, ks > 0 ? 1 : 0);
      tc_mma(taddr, tc_sdesc(aL + ks * 4096, 2048, 128), db, idesc, 1);
    }
    tc_commit(&bar[7]);
  }
  ok &= mbar_wait(&bar[7], 0);
  tc_fence_after();
  // ---- epilogue 2: z = w3 . GELU(D2 + b2) + b3 ----
  float2 zp2 = make_float2(0.0f, 0.0f);
#pragma unroll 1
  for (int g = 0; g < 4; g++) {
    const int col = ch * 32 + g * 8;
    float d[8];
    tmem_ld8(tl + col, d);
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const float2 h = gelu_pair(__fadd2_rn(make_float2(d[e], d[e + 1]), make_float2(par[H2 + col + e], par[H2 + col + e + 1])));
      zp2 = __ffma2_rn(h, make_float2(par[2 * H2 + col + e], par[2 * H2 + col + e + 1]), zp2);
    }
  }
  const float zp = zp2.x + zp2.y;
  float* szp = reinterpret_cast<float*>(sm + TC_PZ);
  if (ch == 1) szp[row] = zp;
  tc_fence_before();
  __syncthreads();
  if (ch == 0 && valid && status == 0) {
    const float z = zp + szp[row] + par[3 * H2];
    const size_t e = (size_t)j * a.ms.nx + i;
    flags[e] = (unsigned char)(z > threshold);
    if (logits) logits[e] = z;
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, 256);
  }
  if (!ok && status == 0) atomicOr(&ts->pending, 2);
}

template <int NV, int M>
cudaError_t launch_flags_t(const FeatArgs& fa, const void* wpack, void* work, float threshold, DevState* ts,
                           unsigned char* flags, float* logits, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<NV, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const Mesh& ms = fa.ms;
  const WorkPlan wl = work_plan(ms, NV, M);
  unsigned char* w = static_cast<unsigned char*>(work);
  unsigned long long* emax = reinterpret_cast<unsigned long long*>(w);
  unsigned* img = reinterpret_cast<unsigned*>(w + wl.img);
  unsigned *gl = reinterpret_cast<unsigned*>(w + wl.gl), *gr = reinterpret_cast<unsigned*>(w + wl.gr);
  unsigned *gb = reinterpret_cast<unsigned*>(w + wl.gb), *gt = reinterpret_cast<unsigned*>(w + wl.gt);
  const long long ntiles = (long long)ms.ntx * ms.ny;
  if (ntiles >= (1ll << 29)) return cudaErrorInvalidValue;  // tile indices in int, CTA indices * 4 too
  const long long n = ntiles * NV * 32;
  k_elem_prep<NV, M><<<blocks(n, 128), 128, 0, s>>>(fa.U, emax, img, n);
  if (ms.bc == 1) {
    const long long ng = 2LL * ms.ny * NV + 2LL * ms.ntx * NV * 32;
    k_ghost_prep<NV, M><<<blocks(ng, 128), 128, 0, s>>>(fa.GL, fa.GR, fa.GB, fa.GT, gl, gr, gb, gt, ms.ny, ms.ntx);
  }
  float4* rs = reinterpret_cast<float4*>(w + wl.rs);
  const long long ne = ntiles * 32;
  k_stencil_scale<NV, M><<<blocks(ne, 128), 128, 0, s>>>(fa, emax, rs, ne);
  const ImgArgs im = {rs, img, gl, gr, gb, gt};
  static int resident = 0;  // CTAs in one wave: two per SM
  if (!resident) {
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    resident = 2 * nsm;
  }
  const long long nblk = (ntiles + 3) / 4;
  k_mlp_tc<NV, M><<<(unsigned)nblk, TC_THREADS, TC_SMEM, s>>>(fa, im, static_cast<const unsigned char*>(wpack),
                                                              threshold, ts, flags, logits, ntiles, resident);
  return cudaGetLastError();
}

template <int NV, int M>
cudaError_t launch_feat_t(const FeatArgs& fa, const int* elems, int n, float* out, cudaStream_t s) {
  k_features<NV, M><<<blocks(n, 128), 128, 0, s>>>(fa, elems, n, out);
  return cudaGetLastError();
}

FeatArgs feat_args(const double* U, const double* GL, const double* GR, const double* GB, const double* GT,
                   const Mesh& ms) {
  FeatArgs fa;
  fa.U = U;
  fa.GL = GL;
  fa.GR = GR;
  fa.GB = GB;
  fa.GT = GT;
  fa.ms = ms;
  return fa;
}

}  // namespace

#define DG_MLP_DISPATCH(NVv, p, CALL)                         \
  do {                                                        \
    if (NVv == 4) {                                           \
      switch (p) {                                            \
        case 1: return CALL(4, 4);                            \
        case 2: return CALL(4, 9);                            \
        case 3: return CALL(4, 16);                           \
        case 4: return CALL(4, 25);                           \
      }                                                       \
    } else {                                                  \
      switch (p) {                                            \
        case 1: return CALL(3, 4);                            \
        case 2: return CALL(3, 9);                            \
        case 3: return CALL(3, 16);                           \
        case 4: return CALL(3, 25);                           \
      }                                                       \
    }                                                         \
    return cudaErrorInvalidValue;                             \
  } while (0)

cudaError_t launch_features(const double* U, const double* GL, const double* GR, const double* GB,
                            const double* GT, const Mesh& ms, int p, int nv, const int* elems, int n, float* out,
                            cudaStream_t s) {
  const FeatArgs fa = feat_args(U, GL, GR, GB, GT, ms);
#define CALL(a, b) launch_feat_t<a, b>(fa, elems, n, out, s)
  DG_MLP_DISPATCH(nv, p, CALL);
#undef CALL
}

cudaError_t launch_mlp_flags(const double* U, const double* GL, const double* GR, const double* GB,
                             const double* GT, const Mesh& ms, int p, int nv, const void* wpack, void* work,
                             float threshold, DevState* ts, unsigned char* flags, float* logits, cudaStream_t s) {
  const FeatArgs fa = feat_args(U, GL, GR, GB, GT, ms);
#define CALL(a, b) launch_flags_t<a, b>(fa, wpack, work, threshold, ts, flags, logits, s)
  DG_MLP_DISPATCH(nv, p, CALL);
#undef CALL
}

size_t mlp_pack_bytes(int nv, int M) { return (size_t)((nv * tc_gpv(M) + 7) / 8) * 8192 + 8192 + 1024; }
size_t mlp_work_bytes(const Mesh& ms, int nv, int M) { return work_plan(ms, nv, M).total; }

namespace {
unsigned short bf16_bits(float f) {  // round to nearest even, as __float2bfloat16_rn
  unsigned u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x7fffffu)) return (unsigned short)((u >> 16) | 0x40);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (unsigned short)(u >> 16);
}
float bf16_value(float f) {
  const unsigned u = (unsigned)bf16_bits(f) << 16;
  float r;
  memcpy(&r, &u, 4);
  return r;
}
void put_bf16(unsigned char* base, int off, float f) {
  const unsigned short b = bf16_bits(f);
  memcpy(base + off, &b, 2);
}
}  // namespace

void mlp_pack(const float* prm, int nv, int M, unsigned char* out) {
  const int nin = 5 * nv * M, gpb = tc_gpb(M), gpv = tc_gpv(M), ng = nv * gpv, nc = (ng + 7) / 8;
  const Offs o = offs(nin);
  memset(out, 0, mlp_pack_bytes(nv, M));
  // input k' = G * 8 + e of group G = v * gpv + s * gpb + g is input
  // (s * nv + v) * M + 8 g + e of the network (zero for the padding group
  // s = 5 and the padding modes 8 g + e >= M)
  for (int c = 0; c < nc; c++)
    for (int kc = 0; kc < TC_KC; kc++) {
      const int kp = c * TC_KC + kc, G = kp / 8;
      if (G >= ng) continue;
      const int v = G / gpv, r = G - v * gpv, s = r / gpb, kk = (r - s * gpb) * 8 + kp % 8;
      if (s >= 5 || kk >= M) continue;
      const int in = (s * nv + v) * M + kk;
      for (int n = 0; n < H; n++) put_bf16(out + (size_t)c * 8192, tc_off(H, n, kc), prm[o.W1 + (size_t)n * nin + in]);
    }
  unsigned char* w2 = out + (size_t)nc * 8192;
  for (int u = 0; u < H; u++)
    for (int q = 0; q < H; q++) put_bf16(w2, tc_off(H, u, q), prm[o.W2 + u * H + q]);
  float pf[3 * H + 1];
  for (int u = 0; u < H; u++) {
    pf[u] = bf16_value(prm[o.b1 + u]);
    pf[H + u] = bf16_value(prm[o.b2 + u]);
    pf[2 * H + u] = bf16_value(prm[o.w3 + u]);
  }
  pf[3 * H] = bf16_value(prm[o.b3]);
  memcpy(w2 + 8192, pf, sizeof(pf));
}

// ---- training ------------------------------------------------------------

cudaError_t mlp_sync_bf16(MlpBufs& b, cudaStream_t s) {
  const int n = offs(b.nin).n;
  k_to_bf16<<<blocks(n, 256), 256, 0, s>>>(b.p, reinterpret_cast<__nv_bfloat16*>(b.pb), n);
  return cudaGetLastError();
}

cudaError_t mlp_forward(MlpBufs& b, const float* x, int B, float* zout, cudaStream_t s) {
  const Offs o = offs(b.nin);
  const __nv_bfloat16* pb = reinterpret_cast<const __nv_bfloat16*>(b.pb);
  k_dense<<<blocks((long long)B * H, 128), 128, 0, s>>>(x, pb + o.W1, pb + o.b1, b.a1, b.h1, B, b.nin, H, 1);
  k_dense<<<blocks((long long)B * H, 128), 128, 0, s>>>(b.h1, pb + o.W2, pb + o.b2, b.a2, b.h2, B, H, H, 1);
  k_dense<<<blocks(B, 128), 128, 0, s>>>(b.h2, pb + o.w3, pb + o.b3, nullptr, zout, B, H, 1, 0);
  return cudaGetLastError();
}

cudaError_t mlp_backward(MlpBufs& b, const float* x, const float* y, int B, float pos_weight, double* loss_sum,
                         cudaStream_t s) {
  const Offs o = offs(b.nin);
  const __nv_bfloat16* pb = reinterpret_cast<const __nv_bfloat16*>(b.pb);
  cudaError_t e = mlp_forward(b, x, B, b.z, s);
  if (e != cudaSuccess) return e;
  k_out_grad<<<blocks(B, 256), 256, 0, s>>>(b.z, y, b.dz, b.lossb, B, pos_weight);
  k_sum<<<1, 256, 0, s>>>(b.lossb, B, loss_sum);
  k_wgrad<<<blocks(H + 1, 128), 128, 0, s>>>(b.dz, b.h2, b.g + o.w3, b.g + o.b3, B, 1, H);
  k_igrad<<<blocks((long long)B * H, 128), 128, 0, s>>>(b.dz, pb + o.w3, b.a2, b.d2, B, 1, H);
  k_wgrad<<<blocks((long long)H * (H + 1), 128), 128, 0, s>>>(b.d2, b.h1, b.g + o.W2, b.g + o.b2, B, H, H);
  k_igrad<<<blocks((long long)B * H, 128), 128, 0, s>>>(b.d2, pb + o.W2, b.a1, b.d1, B, H, H);
  k_wgrad<<<blocks((long long)H * (b.nin + 1), 128), 128, 0, s>>>(b.d1, x, b.g + o.W1, b.g + o.b1, B, H, b.nin);
  return cudaGetLastError();
}

cudaError_t mlp_adam(MlpBufs& b, int t, float lr, cudaStream_t s) {
  const int n = offs(b.nin).n;
  const float c1 = 1.0f - powf(0.9f, (float)t), c2 = 1.0f - powf(0.999f, (float)t);
  k_adam<<<blocks(n, 256), 256, 0, s>>>(b.p, b.m, b.v, b.g, n, lr, c1, c2);
  return cudaGetLastError();
}

int mlp_nparams(int nin) { return offs(nin).n; }

}  // namespace dg
