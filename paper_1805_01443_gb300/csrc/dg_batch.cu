// dg_batch.cu -- batched precision form: the tiles of many discs (of mixed
// size and degree) either in one launch per RK stage, with persistent CTAs
// taking (instance, tile) items from a work counter in a tuned order, one
// launch for the torque of every instance and one for their end-of-step work;
// or in one persistent cooperative launch per step (the flow schedule), whose
// items wait for the tile rows they read instead of for a whole stage.
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

// stage `stage` of tile (bx, j) of instance k
template <bool LAST>
__device__ __forceinline__ void batch_tile(const BatchLaunch32& L, int stage, int k, int bx, int j, double* smd) {
  const BatchInst32& I = L.inst[k];
  // state buffers of this step from the parity of the instance's step counter
  const int cur = I.cur0 ^ (int)((I.a.ts->step - I.step0) & 1);
  const float* un = I.buf[cur];
  float* nx = I.buf[cur ^ 1];
  const float* D = stage == 0 ? un : (stage == 1 ? nx : I.DZ);
  float* Out = stage == 1 ? I.DZ : nx;
  const float alpha = stage == 0 ? 0.0f : (stage == 1 ? 0.75f : 1.0f / 3.0f);
  const float beta = stage == 0 ? 1.0f : (stage == 1 ? 0.25f : 2.0f / 3.0f);
  const int pidx = stage == 0 ? 0 : (stage == 1 ? 2 : 1);
  const int mode = LAST ? 2 : 1;
  switch (I.p) {
    case 1: stage32_tile<1, LAST>(I.a, D, un, Out, alpha, beta, pidx, mode, bx, j, smd); break;
    case 2: stage32_tile<2, LAST>(I.a, D, un, Out, alpha, beta, pidx, mode, bx, j, smd); break;
    case 3: stage32_tile<3, LAST>(I.a, D, un, Out, alpha, beta, pidx, mode, bx, j, smd); break;
    default: stage32_tile<4, LAST>(I.a, D, un, Out, alpha, beta, pidx, mode, bx, j, smd); break;
  }
}

template <bool LAST>
__device__ __forceinline__ void batch_item(const BatchLaunch32& L, int code, double* smd) {
  const int k = code >> 25, tile = code & ((1 << 25) - 1);
  const Mesh& ms = L.inst[k].a.mesh;
  const int j = tile / ms.ntx, bx = tile - j * ms.ntx;
  batch_tile<LAST>(L, L.stage, k, bx, j, smd);
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

// torque of tile `tile` of instance k (one warp)
__device__ __forceinline__ void batch_torque_tile(const BatchLaunch32& L, int k, int tile) {
  const BatchInst32& I = L.inst[k];
  // the new state: the last stage wrote buf[cur ^ 1]; the step counter
  // advances in the end-of-step work that follows
  const int cur = I.cur0 ^ (int)((I.a.ts->step - I.step0) & 1);
  const float* nx = I.buf[cur ^ 1];
  switch (I.p) {
    case 1: torque32_tile<1>(nx, I.SigbN, I.a.ts, I.a.part, I.a.mesh, I.a.pc, tile); break;
    case 2: torque32_tile<2>(nx, I.SigbN, I.a.ts, I.a.part, I.a.mesh, I.a.pc, tile); break;
    case 3: torque32_tile<3>(nx, I.SigbN, I.a.ts, I.a.part, I.a.mesh, I.a.pc, tile); break;
    default: torque32_tile<4>(nx, I.SigbN, I.a.ts, I.a.part, I.a.mesh, I.a.pc, tile); break;
  }
}

__global__ void __launch_bounds__(128, 6) k_batch_torque32(const __grid_constant__ BatchLaunch32 L) {
  const int w = threadIdx.x >> 5;
  const int item = blockIdx.x * 4 + w;  // warp-uniform
  if (item >= L.nitems) return;
  const int k = upper_tile0(L, item), tile = item - L.tile0[k];
  batch_torque_tile(L, k, tile);
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

// ---- the flow schedule: one persistent launch per step ----------------------

// bounded wait of one thread until *ctr >= target: gives up after the
// launch's limit, or soon after another wait of the launch gave up (the abort
// flag), so that nothing waits on work that will not come
__device__ __forceinline__ bool flow_wait(const BatchFlow32& F, const int* ctr, int target) {
  return counter_wait(ctr, target, F.limit_ns, F.ctr + 1);
}

// a wait of instance k gave up: the instance's step is void (its state stays
// at the last good step and its status becomes DG_ERR_TIMEOUT at the end of
// the step), and every other wait of the launch gives up at once
__device__ __forceinline__ void flow_fail(const BatchLaunch32& L, int k) {
  atomicOr(&L.inst[k].a.ts->pending, 2);
  atomicExch(L.flow.ctr + 1, 1);
}

// `len` tiles of one row of instance k at stage `stage`, once the rows they
// read are finished by the stage before (rows j-1, j, j+1, wrapped under the
// periodic boundary).  Those rows are also the only readers, in the stage
// before, of the buffer this stage writes, so the wait orders those reads
// before these writes too.
template <bool LAST>
__device__ __forceinline__ void flow_stage_item(const BatchLaunch32& L, int stage, int2 it, double* smd) {
  const BatchFlow32& F = L.flow;
  const int k = it.x >> 25, t0 = it.x & ((1 << 25) - 1), len = it.y;
  const Mesh& ms = L.inst[k].a.mesh;
  const int j = t0 / ms.ntx, bx0 = t0 - j * ms.ntx;
  int* rows = F.ctr + FLOW_ROWS + 3 * F.rowbase[k];
  bool ok = true;
  if (stage > 0 && threadIdx.x == 0) {
    // the three rows' counters read together (one round trip); the bounded
    // waits only for a row that is not finished yet; then the acquiring fence
    int rr[3];
#pragma unroll
    for (int d = -1; d <= 1; d++) {
      int r = j + d;
      if (r < 0) r = ms.bc == 0 ? ms.ny - 1 : -1;
      else if (r >= ms.ny) r = ms.bc == 0 ? 0 : -1;
      rr[d + 1] = r;
    }
    int cv[3];
#pragma unroll
    for (int d = 0; d < 3; d++) cv[d] = rr[d] >= 0 ? counter_load_relaxed(rows + 3 * rr[d] + (stage - 1)) : ms.ntx;
#pragma unroll 1
    for (int d = 0; d < 3 && ok; d++)
      if (cv[d] < ms.ntx) ok = flow_wait(F, rows + 3 * rr[d] + (stage - 1), ms.ntx);
    __threadfence();
  }
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) flow_fail(L, k);
  } else {
#pragma unroll 1
    for (int u = 0; u < len; u++) {
      batch_tile<LAST>(L, stage, k, bx0 + u, j, smd);
      __syncthreads();  // the tile's shared memory is free for the next one
    }
  }
  // every thread's writes are ordered before thread 0's fence by the barrier
  // (the pattern of a grid barrier); then the rows' counter
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(rows + 3 * j + stage, len);
  }
}

// torque of up to three tiles of instance k (one warp each), each once its
// row is finished by the last stage; the CTA that completes the instance's
// last torque tile does its end-of-step work
__device__ __forceinline__ void flow_torque_item(const BatchLaunch32& L, int code, double* smd) {
  const BatchFlow32& F = L.flow;
  __shared__ int s_last;
  const int k = code >> 25, t0 = code & ((1 << 25) - 1);
  const BatchInst32& I = L.inst[k];
  const Mesh& ms = I.a.mesh;
  const int nt = L.tile0[k + 1] - L.tile0[k];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = t0 + w;
  bool ok = true;
  if (tile < nt) {  // warp-uniform
    if (lane == 0) {
      ok = flow_wait(F, F.ctr + FLOW_ROWS + 3 * (F.rowbase[k] + tile / ms.ntx) + 2, ms.ntx);
      __threadfence();
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) batch_torque_tile(L, k, tile);
  }
  const bool fail = __syncthreads_or(!ok);
  if (threadIdx.x == 0) {
    __threadfence();
    if (fail) flow_fail(L, k);
    const int cnt = min(3, nt - t0);
    s_last = atomicAdd(F.ctr + FLOW_TQ + k, cnt) + cnt == nt;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    finish_step_nt<96>(smd + 8, smd + 8 + 256, I.a.ts, I.a.part, I.nparts, I.series, 0.0, 1, 1, I.r_p,
                       I.omega_p, I.phi0);
  }
}

// CTAs take queue positions from ctr[0] (the next one fetched while the
// current one runs), or, with F.rr, CTA c takes positions c, c + G, c + 2G, ...
// in turn.  Position q: [0, nq) stage 1, [nq, 2 nq) stage 2, [2 nq, 2 nq +
// nql) the last stage, then the torque groups.  An item waits only for items
// earlier in the queue.  Every CTA of the (cooperative) launch is resident
// and takes its positions in increasing order, holding at most one it has
// not started, taken after the one it runs; so the CTA that owns the
// earliest unfinished position is running it, its inputs are finished, and
// it progresses.
__global__ void __launch_bounds__(96, DG_STAGE32_MIN_CTAS) k_batch_flow32(const __grid_constant__ BatchLaunch32 L) {
  extern __shared__ double smd[];
  __shared__ int s_q;
  const BatchFlow32& F = L.flow;
  const int nq = F.nq, nql = F.nql, total = 2 * nq + nql + F.ntq;
  if (threadIdx.x == 0) s_q = F.rr ? (int)blockIdx.x : atomicAdd(F.ctr, 1);
  __syncthreads();
  int q = s_q;
  while (q < total) {
    __syncthreads();  // every thread holds q before thread 0 fetches the next
    if (threadIdx.x == 0) s_q = F.rr ? q + (int)gridDim.x : atomicAdd(F.ctr, 1);
    if (q < nq) flow_stage_item<false>(L, 0, F.items[q], smd);
    else if (q < 2 * nq) flow_stage_item<false>(L, 1, F.items[q - nq], smd);
    else if (q < 2 * nq + nql) flow_stage_item<true>(L, 2, F.last[q - 2 * nq], smd);
    else flow_torque_item(L, F.tq[q - 2 * nq - nql], smd);
    __syncthreads();
    q = s_q;
  }
}

size_t smem_bytes() { return Smem32<4>::BYTES; }
static_assert((8 + 512) * sizeof(double) <= Smem32<4>::BYTES, "end-of-step scratch");
static_assert(sizeof(BatchLaunch32) <= 32000, "kernel parameter size");

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
  // the whole unified L1 as shared memory (the occupancy the kernel is built for)
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_stage32<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_stage32<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
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

int batch_flow_ctas_per_sm() {
  int a = 0;
  if (cudaFuncSetAttribute(k_batch_flow32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes()) !=
      cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch_flow32, 96, smem_bytes()) != cudaSuccess) return 0;
  return a;
}

// cooperative: the launch fails rather than start more CTAs than can be
// resident together
cudaError_t launch_batch_flow32(const BatchLaunch32& L, int grid, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(96);
  cfg.dynamicSmemBytes = smem_bytes();
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch_flow32, L);
}

cudaError_t launch_batch_planet32(const BatchLaunch32& L, cudaStream_t s) {
  k_batch_planet32<<<1, BATCH_MAX, 0, s>>>(L);
  return cudaGetLastError();
}

}  // namespace dg
