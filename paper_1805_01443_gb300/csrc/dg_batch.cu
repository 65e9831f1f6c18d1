// dg_batch.cu -- batched precision form: the tiles of many discs (of mixed
// size and degree) in one launch per RK stage, with persistent CTAs taking
// (instance, tile) items from a work counter in a tuned order; one launch for
// the torque of every instance and one for their end-of-step work.
#include "dg_finish.cuh"
#include "dg_stage32.cuh"

namespace dg {

namespace {

__device__ __forceinline__ int upper_tile0(const BatchLaunch32& L, int item) {
  int lo = 0, hi = L.n;  // largest k with tile0[k] <= item
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (L.tile0[mid] <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <bool LAST>
__device__ __forceinline__ void batch_item(const BatchLaunch32& L, int code, double* smd) {
  const int k = code >> 25, tile = code & ((1 << 25) - 1);
  const BatchInst32& I = L.inst[k];
  const Mesh& ms = I.a.mesh;
  const int j = tile / ms.ntx, bx = tile - j * ms.ntx;
  // state buffers of this step from the parity of the instance's step counter
  const int cur = I.cur0 ^ (int)((I.a.ts->step - I.step0) & 1);
  const float* un = I.buf[cur];
  float* nx = I.buf[cur ^ 1];
  const float* D = L.stage == 0 ? un : (L.stage == 1 ? nx : I.DZ);
  float* Out = L.stage == 1 ? I.DZ : nx;
  const float alpha = L.stage == 0 ? 0.0f : (L.stage == 1 ? 0.75f : 1.0f / 3.0f);
  const float beta = L.stage == 0 ? 1.0f : (L.stage == 1 ? 0.25f : 2.0f / 3.0f);
  const int pidx = L.stage == 0 ? 0 : (L.stage == 1 ? 2 : 1);
  const int mode = LAST ? 2 : 1;
  switch (I.p) {
    case 1: stage32_tile<1, LAST>(I.a, D, un, Out, alpha, beta, pidx, mode, bx, j, smd); break;
    case 2: stage32_tile<2, LAST>(I.a, D, un, Out, alpha, beta, pidx, mode, bx, j, smd); break;
    case 3: stage32_tile<3, LAST>(I.a, D, un, Out, alpha, beta, pidx, mode, bx, j, smd); break;
    default: stage32_tile<4, LAST>(I.a, D, un, Out, alpha, beta, pidx, mode, bx, j, smd); break;
  }
}

template <bool LAST>
__global__ void __launch_bounds__(96, DG_STAGE32_MIN_CTAS) k_batch_stage32(const __grid_constant__ BatchLaunch32 L) {
  extern __shared__ double smd[];
  __shared__ int s_item;
  if (!L.dynamic) {
    if ((int)blockIdx.x < L.nitems) batch_item<LAST>(L, L.items[blockIdx.x], smd);
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(L.counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();  // every thread holds the item before thread 0 takes the next
    if (item >= L.nitems) break;
    batch_item<LAST>(L, L.items[item], smd);
    __syncthreads();  // the tile's shared memory is free for the next item
  }
}

__global__ void __launch_bounds__(128, 7) k_batch_torque32(const __grid_constant__ BatchLaunch32 L) {
  __shared__ float sD[4][2 * MAXM * MAXM * 32];  // per warp: nodal delta Sigma of its tile
  const int w = threadIdx.x >> 5;
  const int item = blockIdx.x * 4 + w;  // warp-uniform
  if (item >= L.nitems) return;
  float* sd = sD[w] + (threadIdx.x & 31);
  const int k = upper_tile0(L, item), tile = item - L.tile0[k];
  const BatchInst32& I = L.inst[k];
  // the new state: the last stage wrote buf[cur ^ 1]; the step counter
  // advances in the finish launch that follows
  const int cur = I.cur0 ^ (int)((I.a.ts->step - I.step0) & 1);
  const float* nx = I.buf[cur ^ 1];
  switch (I.p) {
    case 1: torque32_tile<1>(nx, I.SigbN, I.a.ts, I.a.part, I.a.mesh, I.a.pc, tile, sd); break;
    case 2: torque32_tile<2>(nx, I.SigbN, I.a.ts, I.a.part, I.a.mesh, I.a.pc, tile, sd); break;
    case 3: torque32_tile<3>(nx, I.SigbN, I.a.ts, I.a.part, I.a.mesh, I.a.pc, tile, sd); break;
    default: torque32_tile<4>(nx, I.SigbN, I.a.ts, I.a.part, I.a.mesh, I.a.pc, tile, sd); break;
  }
}

// one CTA of 256 threads per instance
__global__ void __launch_bounds__(256) k_batch_finish(const __grid_constant__ BatchLaunch32 L) {
  const BatchInst32& I = L.inst[blockIdx.x];
  finish_step(I.a.ts, I.a.part, I.nparts, I.series, 0.0, 1, 1, I.r_p, I.omega_p, I.phi0);
}

__global__ void k_batch_planet32(const __grid_constant__ BatchLaunch32 L) {
  const int k = threadIdx.x;
  if (k >= L.n) return;
  const BatchInst32& I = L.inst[k];
  if (I.a.ts->status == 0) store_planet32(I.a.ts, I.a.ts->dt, I.r_p, I.omega_p, I.phi0);
}

size_t smem_bytes() { return Smem32<4>::BYTES; }

}  // namespace

cudaError_t batch_upload_tables32(const Tables* const* tabs) {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess && tabs[1]) e = upload_tables32_impl<1>(*tabs[1]);
  if (e == cudaSuccess && tabs[2]) e = upload_tables32_impl<2>(*tabs[2]);
  if (e == cudaSuccess && tabs[3]) e = upload_tables32_impl<3>(*tabs[3]);
  if (e == cudaSuccess && tabs[4]) e = upload_tables32_impl<4>(*tabs[4]);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_batch_stage32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_stage32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes());
  return e;
}

size_t batch_stage32_smem() { return smem_bytes(); }

int batch_stage32_ctas_per_sm() {
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch_stage32<false>, 96, smem_bytes()) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_stage32<true>, 96, smem_bytes()) != cudaSuccess)
    return 0;
  return a < b ? a : b;
}

cudaError_t launch_batch_stage32(const BatchLaunch32& L, int grid, cudaStream_t s) {
  if (L.stage == 2) k_batch_stage32<true><<<grid, 96, smem_bytes(), s>>>(L);
  else k_batch_stage32<false><<<grid, 96, smem_bytes(), s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_batch_torque32(const BatchLaunch32& L, cudaStream_t s) {
  k_batch_torque32<<<(L.nitems + 3) / 4, 128, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_batch_finish(const BatchLaunch32& L, cudaStream_t s) {
  k_batch_finish<<<L.n, 256, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_batch_planet32(const BatchLaunch32& L, cudaStream_t s) {
  k_batch_planet32<<<1, BATCH_MAX, 0, s>>>(L);
  return cudaGetLastError();
}

}  // namespace dg
