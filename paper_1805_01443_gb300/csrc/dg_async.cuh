// dg_async.cuh -- asynchronous-copy primitives shared by the kernels: 1D bulk
// copies global -> shared by the TMA unit with completion counted on an
// mbarrier, and bounded mbarrier waits.
#pragma once
#include <cuda_runtime.h>

namespace dg {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(void* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (TMA) writes to it
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(void* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// bytes and both addresses multiples of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, void* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// ask the L2 for `bytes` of global memory (a hint: no completion, no
// register); address and size multiples of 16
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(void* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of the given parity: false after ~2^22 polls
// (a fraction of a second), so that a copy that never lands cannot hang the GPU
__device__ __forceinline__ bool mbar_wait(void* bar, unsigned parity) {
  for (int i = 0; i < (1 << 22); i++) {
    if (mbar_test(bar, parity)) return true;
    if (i >= 8) __nanosleep(64);
  }
  return false;
}

// ---- counters in global memory (waits between CTAs of one launch) ---------
// Only for CTAs that are resident together: a cooperative launch, or CTAs of
// one launch that wait only for work other running CTAs have already taken.

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// add 1 to *ctr with release semantics (this CTA's earlier writes, made
// visible to the GPU by the caller's __threadfence, are ordered before it)
__device__ __forceinline__ void counter_signal(int* ctr) {
  asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(ctr) : "memory");
}
__device__ __forceinline__ int counter_load_relaxed(const int* ctr) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
  return v;
}
__device__ __forceinline__ int counter_load(const int* ctr) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
  return v;
}
// bounded wait until *ctr >= target: false once ~limit_ns have passed on the
// GPU's global timer (or 2^26 polls, whichever comes first), or soon after
// *abort (if given) becomes non-zero, so that a counter nobody advances cannot
// hang the GPU
__device__ __forceinline__ bool counter_wait(const int* ctr, int target, unsigned long long limit_ns,
                                             const int* abort = nullptr) {
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < (1 << 26); i++) {
    if (counter_load(ctr) >= target) return true;
    if (i >= 16) {
      __nanosleep(128);
      if ((i & 63) == 0 && ((abort && counter_load(abort) != 0) || global_ns() - t0 > limit_ns)) return false;
    }
  }
  return false;
}

// ---- programmatic dependent launch (consecutive kernels on one stream) ----
// Wait until the grid this launch depends on has completed and its writes are
// visible (an ordinary launch returns at once); called first in a kernel, so
// nothing of the previous kernel's output is read before it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Let the next launch on the stream start its CTAs (which then wait in
// pdl_wait) once every CTA of this grid has started.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// host: launch `kern` so that it may start while the previous kernel on the
// stream drains (the kernel calls pdl_wait before touching its inputs)
template <typename... Exp, typename... Act>
static cudaError_t launch_pdl(void (*kern)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Act&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Act&&>(args)...);
}

}  // namespace dg
