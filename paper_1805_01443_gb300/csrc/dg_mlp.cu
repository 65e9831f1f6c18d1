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
// cores forms the same inputs in FP32 -- the coefficient truncated and the
// reciprocal rounded to FP32, then their FP32 product -- within 2^-22
// relative of those and without an FP64 instruction per input.
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
// the MMA row r.  Layer 1 runs over the inputs in chunks of 64: the 256
// threads form the chunk's features (two threads per row, 32 inputs each),
// split each into BF16 hi + lo (x = hi + lo to 2^-16 relative; the weights are
// BF16 already, so the two MMAs reproduce the FP32 products), and one thread
// issues the chunk's MMAs (M 128, N 64, K 16) into tensor memory.  The next
// chunk's coefficients are loaded and scaled while those MMAs run; its
// features are stored once they are done (one A buffer: the MMAs take a
// small fraction of the feature time, and the smaller footprint lets three
// CTAs share an SM).  The W1 chunks arrive by bulk copies into a two-stage
// ring.  The epilogue reads the accumulators back (warp w: lanes 32 (w mod 4)..,
// columns 32 (w / 4)..), adds the bias, applies GELU and splits the hidden
// units into BF16 hi + lo, the A operand of layer 2 (64 -> 64, same scheme);
// the last epilogue forms the logit.
constexpr int TC_ROWS = 128, TC_KC = 64, TC_THREADS = 256;
constexpr int TC_A = 0;                          // [hi, lo][128 x 64] BF16, 16 KB each
constexpr int TC_B = TC_A + 2 * 16384;           // W1 chunks [2 stages][64 x 64] BF16
constexpr int TC_W2 = TC_B + 2 * 8192;           // W2 [64 x 64] BF16
constexpr int TC_PAR = TC_W2 + 8192;             // b1, b2, w3 [64] and b3, FP32 (1 KB); then partial logits
constexpr int TC_BAR = TC_PAR + 1024;            // mbarriers: MMA done, (unused), W1 chunk [2], W2, layer 2
constexpr int TC_TM = TC_BAR + 64;               // tensor-memory base address
constexpr int TC_SMEM = TC_TM + 16;
constexpr int TC_PZ = TC_A + 8192;               // partial logits [128] (A is dead by then)

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

// bits of max |c| over the modes of variable v of every element, [tile][v][32]
template <int NV, int M>
__global__ void k_elem_max(const double* __restrict__ U, unsigned long long* __restrict__ mx, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double* p = U + (t >> 5) * (M * 32) + (t & 31);
  unsigned long long m = 0ull;
#pragma unroll
  for (int k = 0; k < M; k++) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(p[k * 32]) & 0x7fffffffffffffffull;
    m = b > m ? b : m;
  }
  mx[t] = m;
}

#ifdef DG_TC_SWAP_LBO
#define TC_DESC(addr, lbo, sbo) tc_sdesc(addr, sbo, lbo)
#else
#define TC_DESC(addr, lbo, sbo) tc_sdesc(addr, lbo, sbo)
#endif

template <int NV, int M>
__global__ void __launch_bounds__(TC_THREADS, 3)
    k_mlp_tc(const FeatArgs a, const unsigned char* __restrict__ wp, const unsigned long long* __restrict__ emax,
             float threshold, DevState* ts, unsigned char* __restrict__ flags, float* __restrict__ logits,
             long long ntiles) {
  // inputs in groups of 8 modes of one (stencil element, variable), the modes
  // of a variable padded to a multiple of 8 (zero weights): a group has one
  // base address, one stride and one scale
  constexpr int GPB = (M + 7) / 8, NG = 5 * NV * GPB, NC = (NG + 7) / 8, H2 = MLP_HIDDEN;
  static_assert(MLP_HIDDEN == 64 && NV <= 4, "tile plan");
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TC_BAR);
  unsigned* s_taddr = reinterpret_cast<unsigned*>(sm + TC_TM);
  if (ts->status != 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, row = tid & (TC_ROWS - 1), half = tid >> 7;
  const unsigned idesc = tc_idesc_bf16(TC_ROWS, H2);

  if (warp == 0) tmem_alloc(s_taddr, 128);  // D1: columns 0..63, D2: 64..127
  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < 6; b++) mbar_init(&bar[b], 1);
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[4], 8192 + 1024);
    bulk_g2s(sm + TC_W2, wp + (size_t)NC * 8192, 8192, &bar[4]);
    bulk_g2s(sm + TC_PAR, wp + (size_t)NC * 8192 + 8192, 1024, &bar[4]);
#pragma unroll
    for (int c = 0; c < (NC < 2 ? NC : 2); c++) {
      mbar_expect_tx(&bar[2 + c], 8192);
      bulk_g2s(sm + TC_B + c * 8192, wp + (size_t)c * 8192, 8192, &bar[2 + c]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned taddr = *s_taddr;
  bool ok = true;

  // this row's element and its stencil (s = 0 own, 1 left, 2 right, 3 below, 4 above)
  const long long tile = (long long)blockIdx.x * 4 + (row >> 5);
  int i = 0, j = 0;
  bool valid = false;
  if (tile < ntiles) {
    j = (int)(tile / a.ms.ntx);
    i = (int)(tile - (long long)j * a.ms.ntx) * 32 + (row & 31);
    valid = i < a.ms.nx;
  }
  // 1 / S_v over the stencil, from the per-element maxima (fixed ghost elements
  // scanned here), rounded to FP32
  float R[NV];
  {
    unsigned long long mx[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) mx[v] = 0ull;
    if (valid) {
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
    }
#pragma unroll
    for (int v = 0; v < NV; v++) R[v] = mx[v] ? d2f_rn(1.0 / __longlong_as_double((long long)mx[v])) : 1.0f;
  }

  // base address and stride (elements) of each stencil element's coefficients
  const double* sp[5];
  int sst[5];
#pragma unroll
  for (int s = 0; s < 5; s++) {
    const int ii = i + (s == 1 ? -1 : s == 2 ? 1 : 0), jj = j + (s == 3 ? -1 : s == 4 ? 1 : 0);
    long long te;
    int le;
    sp[s] = a.U;
    sst[s] = 0;
    if (!valid) continue;
    if (mesh_elem(a.ms, ii, jj, i, j, te, le)) {
      sp[s] = a.U + (size_t)te * NV * M * 32 + le;
      sst[s] = 32;
    } else if (ii < 0 || ii >= a.ms.nx) {  // fixed ghost elements [j][v][k]
      sp[s] = (ii < 0 ? a.GL : a.GR) + (size_t)j * NV * M;
      sst[s] = 1;
    } else {  // [tile][v][k][32]
      sp[s] = (jj < 0 ? a.GB : a.GT) + (size_t)(i >> 5) * NV * M * 32 + (i & 31);
      sst[s] = 32;
    }
  }

  // ---- layer 1 over the input chunks ----
  unsigned char* Ahi = sm + TC_A;
  unsigned char* Alo = Ahi + 16384;
  for (int c = 0; c < NC; c++) {
    const int st = c & 1;
    if (c >= 2 && tid == 0) {
      // the MMAs of chunk c - 2, the last readers of this W1 stage, are done:
      // every thread saw their commit before it wrote chunk c - 1
      mbar_expect_tx(&bar[2 + st], 8192);
      bulk_g2s(sm + TC_B + st * 8192, wp + (size_t)c * 8192, 8192, &bar[2 + st]);
    }
#pragma unroll 1
    for (int g = 0; g < 4; g += 2) {
      // the two groups' 16 coefficients are loaded first (all in flight at
      // once), then scaled and rounded
      double cv[16];
      float rv2[2];
#pragma unroll
      for (int h8 = 0; h8 < 2; h8++) {
        const int G = c * 8 + half * 4 + g + h8;
        const int sv = G / GPB, kk0 = (G - sv * GPB) * 8, s = sv / NV, v = sv - s * NV;
        const double* q = sp[0];
        int qs = sst[0];
#pragma unroll
        for (int w = 1; w < 5; w++)
          if (s == w) {
            q = sp[w];
            qs = sst[w];
          }
        float rv = R[0];
#pragma unroll
        for (int w = 1; w < NV; w++) rv = (v == w) ? R[w] : rv;
        rv2[h8] = rv;
        const bool on = valid && G < NG;
        q += (size_t)(v * M + kk0) * qs;
#pragma unroll
        for (int e = 0; e < 8; e++) cv[h8 * 8 + e] = (on && kk0 + e < M) ? q[e * qs] : 0.0;
      }
      // each coefficient truncated to FP32 on the integer pipe, then scaled
      // in FP32: within 2^-22 of the features of the FP64 product
      // (dg_features), and no FP64 instruction per input
      float x[16];
#pragma unroll
      for (int t = 0; t < 16; t++) x[t] = d2f_rz(cv[t]) * rv2[t >> 3];
      // the previous chunk's MMAs have read the A buffer
      if (c > 0 && g == 0) ok &= mbar_wait(&bar[0], (c - 1) & 1);
#pragma unroll
      for (int h8 = 0; h8 < 2; h8++) {
        uint4 hi, lo;
        split8(x + 8 * h8, hi, lo);
        const int off = tc_off(TC_ROWS, row, half * 32 + (g + h8) * 8);
        *reinterpret_cast<uint4*>(Ahi + off) = hi;
        *reinterpret_cast<uint4*>(Alo + off) = lo;
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      ok &= mbar_wait(&bar[2 + st], (c >> 1) & 1);
      tc_fence_after();
      const unsigned aH = smem_addr(Ahi), aL = smem_addr(Alo), bB = smem_addr(sm + TC_B + st * 8192);
#pragma unroll
      for (int ks = 0; ks < TC_KC / 16; ks++) {
        const uint64_t db = TC_DESC(bB + ks * 2048, 1024, 128);
        tc_mma(taddr, TC_DESC(aH + ks * 4096, 2048, 128), db, idesc, (c > 0 || ks > 0) ? 1 : 0);
        tc_mma(taddr, TC_DESC(aL + ks * 4096, 2048, 128), db, idesc, 1);
      }
      tc_commit(&bar[0]);
    }
  }
  // the last commit covers every earlier MMA
  ok &= mbar_wait(&bar[0], (NC - 1) & 1);
  ok &= mbar_wait(&bar[4], 0);
  tc_fence_after();
  const float* par = reinterpret_cast<const float*>(sm + TC_PAR);  // b1, b2, w3, b3
  const int quarter = warp & 3, ch = warp >> 2;
  const unsigned tl = taddr + ((unsigned)(quarter * 32) << 16);
  float acc[32];
  // ---- epilogue 1: h1 = GELU(D1 + b1) as the layer-2 A operand (the A buffer) ----
  tmem_ld32(tl + ch * 32, acc);
  {
    unsigned char* Hhi = sm + TC_A;
    unsigned char* Hlo = Hhi + 16384;
#pragma unroll
    for (int g = 0; g < 4; g++) {
      float x[8];
#pragma unroll
      for (int e = 0; e < 8; e++) x[e] = gelu(acc[g * 8 + e] + par[ch * 32 + g * 8 + e]);
      uint4 hi, lo;
      split8(x, hi, lo);
      const int off = tc_off(TC_ROWS, row, ch * 32 + g * 8);
      *reinterpret_cast<uint4*>(Hhi + off) = hi;
      *reinterpret_cast<uint4*>(Hlo + off) = lo;
    }
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    tc_fence_after();
    const unsigned aH = smem_addr(sm + TC_A), aL = aH + 16384, bW = smem_addr(sm + TC_W2);
#pragma unroll
    for (int ks = 0; ks < H2 / 16; ks++) {
      const uint64_t db = TC_DESC(bW + ks * 2048, 1024, 128);
      tc_mma(taddr + H2, TC_DESC(aH + ks * 4096, 2048, 128), db, idesc, ks > 0 ? 1 : 0);
      tc_mma(taddr + H2, TC_DESC(aL + ks * 4096, 2048, 128), db, idesc, 1);
    }
    tc_commit(&bar[5]);
  }
  ok &= mbar_wait(&bar[5], 0);
  tc_fence_after();
  // ---- epilogue 2: z = w3 . GELU(D2 + b2) + b3 ----
  tmem_ld32(tl + H2 + ch * 32, acc);
  float zp = 0.0f;
#pragma unroll
  for (int e = 0; e < 32; e++) zp = fmaf(gelu(acc[e] + par[H2 + ch * 32 + e]), par[2 * H2 + ch * 32 + e], zp);
  float* szp = reinterpret_cast<float*>(sm + TC_PZ);
  if (ch == 1) szp[row] = zp;
  tc_fence_before();
  __syncthreads();
  if (ch == 0 && valid) {
    const float z = zp + szp[row] + par[3 * H2];
    const size_t e = (size_t)j * a.ms.nx + i;
    flags[e] = (unsigned char)(z > threshold);
    if (logits) logits[e] = z;
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, 128);
  }
  if (!ok) atomicOr(&ts->pending, 2);
}

template <int NV, int M>
cudaError_t launch_flags_t(const FeatArgs& fa, const void* wpack, unsigned long long* emax, float threshold,
                           DevState* ts, unsigned char* flags, float* logits, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<NV, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const long long ntiles = (long long)fa.ms.ntx * fa.ms.ny;
  const long long nmax = ntiles * NV * 32;
  k_elem_max<NV, M><<<blocks(nmax, 256), 256, 0, s>>>(fa.U, emax, nmax);
  const long long nblk = (ntiles + 3) / 4;
  k_mlp_tc<NV, M><<<(unsigned)nblk, TC_THREADS, TC_SMEM, s>>>(
      fa, static_cast<const unsigned char*>(wpack), emax, threshold, ts, flags, logits, ntiles);
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
  unsigned long long* emax = static_cast<unsigned long long*>(work);
#define CALL(a, b) launch_flags_t<a, b>(fa, wpack, emax, threshold, ts, flags, logits, s)
  DG_MLP_DISPATCH(nv, p, CALL);
#undef CALL
}

size_t mlp_pack_bytes(int nv, int M) {
  const int ng = 5 * nv * ((M + 7) / 8);
  return (size_t)((ng + 7) / 8) * 8192 + 8192 + 1024;
}
size_t mlp_work_bytes(const Mesh& ms, int nv) { return (size_t)ms.ntx * ms.ny * nv * 32 * sizeof(unsigned long long); }

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
  const int nin = 5 * nv * M, gpb = (M + 7) / 8, ng = 5 * nv * gpb, nc = (ng + 7) / 8;
  const Offs o = offs(nin);
  memset(out, 0, mlp_pack_bytes(nv, M));
  // input k' = (sv * gpb + kk / 8) * 8 + kk % 8 of group sv = s * nv + v is
  // input (s * nv + v) * M + kk of the network (zero for the padding kk >= M)
  for (int c = 0; c < nc; c++)
    for (int kc = 0; kc < TC_KC; kc++) {
      const int kp = c * TC_KC + kc, G = kp / 8;
      if (G >= ng) continue;
      const int sv = G / gpb, kk = (G - sv * gpb) * 8 + kp % 8;
      if (kk >= M) continue;
      const int in = sv * M + kk;
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
