// dg_selftest.cu -- dg_selftest_wait: makes the library's bounded device-side
// waits run out on purpose and reports how they ended.
//
// Each kernel here waits, with the same helper the product kernels use, on
// something that nothing will ever complete: an mbarrier with no arrival and
// no copy (the stage kernel's wait on its bulk copy), the same while the CTA
// holds tensor memory (the tensor-core inference kernel's waits on its copies
// and MMA commits), and a counter that one CTA of the launch never advances
// (the persistent batched kernel's waits between stages).  The wait gives up
// after its limit, the kernel records that in a status word and, for the
// tensor-memory case, frees its columns before it exits, as the product
// kernels do.  Nothing faults and nothing hangs: every wait ends.
#include <cuda_runtime.h>

#include <cstdio>

#include "dg_internal.cuh"
#include "dg_tc.cuh"

namespace dg {
namespace {

// out[0]: CTAs whose wait gave up; out[1]: 1 once the tensor memory is freed
__global__ void k_selftest_mbar(int hold_tmem, int* out) {
  __shared__ __align__(8) unsigned long long bar;
  __shared__ unsigned taddr;
  const int warp = threadIdx.x >> 5;
  if (hold_tmem && warp == 0) tmem_alloc(&taddr, 32);
  if (threadIdx.x == 0) mbar_init(&bar, 1);  // one arrival expected, none will come
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const bool ok = mbar_wait(&bar, 0);
  const bool any_timeout = __syncthreads_or(!ok);
  if (hold_tmem && warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, 32);
    if (threadIdx.x == 0) atomicExch(&out[1], 1);
  }
  if (threadIdx.x == 0 && any_timeout) atomicAdd(&out[0], 1);
}

// two CTAs; CTA 1 never signals the counter that CTA 0 waits for (ctr[1] is
// an abort word that stays zero, as in the persistent batched kernel)
__global__ void k_selftest_counter(int* ctr, int* out) {
  if (blockIdx.x == 1) return;
  if (threadIdx.x == 0) {
    __threadfence();
    counter_signal(ctr);
  }
  bool ok = true;
  if (threadIdx.x == 0) ok = counter_wait(ctr, 2, 500000000ull, ctr + 1);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicAdd(&out[0], 1);
}

}  // namespace
}  // namespace dg

extern "C" int dg_selftest_wait(int kind, int* freed) {
  using namespace dg;
  if (kind < 0 || kind > 2) return set_thread_error(DG_ERR_ARG, "dg_selftest_wait: kind is 0, 1 or 2");
  int* d = nullptr;
  cudaError_t e = cudaMalloc((void**)&d, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d, 0, 4 * sizeof(int));
  if (e == cudaSuccess) {
    if (kind < 2) {
      k_selftest_mbar<<<1, 64>>>(kind == 1 ? 1 : 0, d);
      e = cudaGetLastError();
    } else {
      int* ctr = d + 2;
      int* outp = d;
      void* args[] = {(void*)&ctr, (void*)&outp};
      e = cudaLaunchCooperativeKernel((const void*)k_selftest_counter, dim3(2), dim3(32), args, 0, nullptr);
    }
  }
  int h[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof(msg), "dg_selftest_wait: %s", cudaGetErrorString(e));
    return set_thread_error(DG_ERR_CUDA, msg);
  }
  if (freed) *freed = h[1];
  if (h[0] == 1) return set_thread_error(DG_ERR_TIMEOUT, "dg_selftest_wait: the wait gave up, as designed");
  return set_thread_error(DG_OK, "dg_selftest_wait: the wait did not give up");
}
