// dg_mlp.cu -- the learned troubled-cell indicator: a multilayer perceptron
// nin -> 64 (GELU) -> 64 (GELU) -> 1 logit on the modal coefficients of an
// element and its four neighbours, with BF16 weights and FP32 accumulation.
//
// Features of element e (FP32): for the stencil s = 0 the element, 1 left,
// 2 right, 3 below, 4 above (outside elements by the boundary rule), variable
// v and mode k, x[(s * nv + v) * M + k] = c_s[v][k] * (1 / S_v) with S_v the
// largest |c_s[v][k]| over the stencil and the modes (1 when all vanish): the
// reciprocal and the product in FP64, the product rounded once to FP32.
//
// Parameters (FP32 master copy, flat): W1 [64][nin], b1 [64], W2 [64][64],
// b2 [64], w3 [64], b3.  The products use the weights rounded to BF16
// (round to nearest even); gradients are taken through that rounding as the
// identity.  Loss: mean over the batch of the weighted binary cross entropy
// w_y (softplus(z) - y z), w_1 = pos_weight, w_0 = 1.  Optimiser: Adam
// (beta 0.9, 0.999, eps 1e-8) on the master copy.
#include <cuda_bf16.h>

#include <new>
#include <vector>

#include "dg_internal.cuh"

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

// ---- features and fused inference on the FP64 tiled state -------------------

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

// one thread per element: features on the fly, the first layer against the
// BF16 weights staged in shared memory ([input][unit]: every thread reads the
// same row, a broadcast), the second layer and the logit; writes the flag
// (logit > threshold) and, when asked, the logit
template <int NV, int M>
__global__ void __launch_bounds__(256) k_mlp_flags(const FeatArgs a, const __nv_bfloat16* __restrict__ Wt1,
                                                   const __nv_bfloat16* __restrict__ rest, float threshold,
                                                   const DevState* ts, unsigned char* __restrict__ flags,
                                                   float* __restrict__ logits) {
  constexpr int NIN = 5 * NV * M;
  // BF16 weights widened to FP32 once (exact), [NIN][H] then b1, W2 [H][H],
  // b2, w3, b3: the inner loop reads rows of four weights per load
  extern __shared__ float4 sw4[];
  float* sw = reinterpret_cast<float*>(sw4);
  const int nrest = H + H * H + H + H + 1;
  for (int k = threadIdx.x; k < NIN * H; k += blockDim.x) sw[k] = __bfloat162float(Wt1[k]);
  for (int k = threadIdx.x; k < nrest; k += blockDim.x) sw[NIN * H + k] = __bfloat162float(rest[k]);
  __syncthreads();
  if (ts->status != 0) return;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = (int)(gid & 31);
  const long long tile = gid >> 5;
  if (tile >= (long long)a.ms.ntx * a.ms.ny) return;
  const int j = (int)(tile / a.ms.ntx), i = (int)(tile - (long long)j * a.ms.ntx) * 32 + lane;
  if (i >= a.ms.nx) return;
  const int di[5] = {0, -1, 1, 0, 0}, dj[5] = {0, 0, 0, -1, 1};
  double S[NV];
  stencil_scales<NV, M>(a, i, j, S);
  const float* b1 = sw + NIN * H;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* w3 = b2 + H;
  const float* b3 = w3 + H;
  float h[H];
#pragma unroll
  for (int u = 0; u < H; u++) h[u] = b1[u];
  for (int s = 0; s < 5; s++)
    for (int v = 0; v < NV; v++)
      for (int k = 0; k < M; k++) {
        const float x = (float)(coef<NV, M>(a, i + di[s], j + dj[s], i, j, v, k) * S[v]);
        const float4* row = reinterpret_cast<const float4*>(sw + (size_t)((s * NV + v) * M + k) * H);
#pragma unroll
        for (int u4 = 0; u4 < H / 4; u4++) {
          const float4 w = row[u4];
          h[4 * u4 + 0] = fmaf(x, w.x, h[4 * u4 + 0]);
          h[4 * u4 + 1] = fmaf(x, w.y, h[4 * u4 + 1]);
          h[4 * u4 + 2] = fmaf(x, w.z, h[4 * u4 + 2]);
          h[4 * u4 + 3] = fmaf(x, w.w, h[4 * u4 + 3]);
        }
      }
#pragma unroll
  for (int u = 0; u < H; u++) h[u] = gelu(h[u]);
  float z = b3[0];
  for (int u = 0; u < H; u++) {
    float acc = b2[u];
#pragma unroll
    for (int q = 0; q < H; q++) acc = fmaf(h[q], W2[u * H + q], acc);
    z = fmaf(gelu(acc), w3[u], z);
  }
  const size_t e = (size_t)j * a.ms.nx + i;
  flags[e] = (unsigned char)(z > threshold);
  if (logits) logits[e] = z;
}

template <int NV, int M>
cudaError_t launch_flags_t(const FeatArgs& fa, const __nv_bfloat16* Wt1, const __nv_bfloat16* rest,
                           float threshold, const DevState* ts, unsigned char* flags, float* logits,
                           cudaStream_t s) {
  constexpr int NIN = 5 * NV * M;
  const size_t smem = (size_t)(NIN * H + H + H * H + H + H + 1) * sizeof(float);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_flags<NV, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const long long threads = (long long)fa.ms.ntx * fa.ms.ny * 32;
  k_mlp_flags<NV, M><<<blocks(threads, 256), 256, smem, s>>>(fa, Wt1, rest, threshold, ts, flags, logits);
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
                             const double* GT, const Mesh& ms, int p, int nv, const __nv_bfloat16* Wt1,
                             const __nv_bfloat16* rest, float threshold, const DevState* ts,
                             unsigned char* flags, float* logits, cudaStream_t s) {
  const FeatArgs fa = feat_args(U, GL, GR, GB, GT, ms);
#define CALL(a, b) launch_flags_t<a, b>(fa, Wt1, rest, threshold, ts, flags, logits, s)
  DG_MLP_DISPATCH(nv, p, CALL);
#undef CALL
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
