// dg_static.cu -- dg_conserved_static: the FP64 conserved sums of a canonical
// coefficient array without any device allocation.
//
// Its per-block partial sums live in the file-scope device array below instead
// of memory from cudaMalloc.  The array belongs to this file's module of
// libdg.so (4096 blocks x 4 doubles = 128 KiB).  Under lazy module loading
// (CUDA_MODULE_LOADING=LAZY, the default of recent CUDA releases) the module,
// and with it the array, is loaded into a device's memory at the first call
// made with that device current; from then on that GPU holds it until the
// process exits.  In host code `g_partials` only names a host-side stand-in
// for the symbol, so the kernels are given the device address that
// cudaGetSymbolAddress returns, looked up once per device.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "dg_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;
constexpr int kMaxBlocks = DG_STATIC_MAX_ELEMENTS / kThreads;  // 4096

static __device__ __align__(256) double g_partials[kMaxBlocks * 4];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// block b sums (mode-0 coefficient x |K|) of elements [256 b, 256 b + 256) for
// every variable, in a fixed tree order, into partials[4 b + v]
__global__ void k_static_part(const double* __restrict__ coeffs, int nv, int nmodes, long long nel,
                              double area, double* __restrict__ partials) {
  __shared__ double s[4][kThreads];
  const int tid = threadIdx.x;
  const long long e = (long long)blockIdx.x * kThreads + tid;
  for (int v = 0; v < 4; v++) s[v][tid] = 0.0;
  if (e < nel)
    for (int v = 0; v < nv; v++) s[v][tid] = coeffs[(long long)v * nmodes * nel + e] * area;
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if (tid < st)
      for (int v = 0; v < 4; v++) s[v][tid] += s[v][tid + st];
    __syncthreads();
  }
  if (tid == 0)
    for (int v = 0; v < 4; v++) partials[(long long)blockIdx.x * 4 + v] = s[v][0];
}

// one block: fixed-order sum of the nblk partials written by this call
__global__ void k_static_final(const double* __restrict__ partials, int nblk, int nv,
                               double* __restrict__ out) {
  __shared__ double s[4][kThreads];
  const int tid = threadIdx.x;
  for (int v = 0; v < 4; v++) {
    double acc = 0.0;
    for (int b = tid; b < nblk; b += kThreads) acc += partials[(long long)b * 4 + v];
    s[v][tid] = acc;
  }
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if (tid < st)
      for (int v = 0; v < 4; v++) s[v][tid] += s[v][tid + st];
    __syncthreads();
  }
  if (tid == 0)
    for (int v = 0; v < nv; v++) out[v] = s[v][0];
}

// Device address of g_partials on device `dev` (the current device), looked
// up on the first call made with that device current.  That lookup also loads
// this file's module on the device when modules are loaded lazily.
int scratch_address(int dev, double** out) {
  if (dev >= kMaxDevices) return dg::set_thread_error(DG_ERR_CUDA, "dg_conserved_static: device index");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess || !p) {
      char msg[160];
      snprintf(msg, sizeof(msg), "dg_conserved_static: scratch address: %s", cudaGetErrorString(e));
      return dg::set_thread_error(DG_ERR_CUDA, msg);
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return DG_OK;
}

// DG_OK if p is device (or managed) memory that kernels on device `dev` can
// read and write; anything else -- pageable or page-locked host memory, memory
// of another device, an address the runtime does not know -- is refused before
// a kernel could fault on it.
int check_device_pointer(const void* p, int dev, const char* what) {
  cudaPointerAttributes at;
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // the failed query is this call's own; do not leave it behind
    char msg[160];
    snprintf(msg, sizeof(msg), "dg_conserved_static: %s: pointer attributes unavailable (%s)", what,
             cudaGetErrorString(e));
    return dg::set_thread_error(DG_ERR_ARG, msg);
  }
  const bool device_mem = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  if (!device_mem || (at.type == cudaMemoryTypeDevice && at.device != dev)) {
    char msg[160];
    snprintf(msg, sizeof(msg), "dg_conserved_static: %s is not device memory of the current device %d",
             what, dev);
    return dg::set_thread_error(DG_ERR_ARG, msg);
  }
  return DG_OK;
}

}  // namespace

extern "C" int dg_conserved_static(const double* coeffs, int nv, int nmodes, int nx, int ny,
                                   double dx, double dy, double* out, void* stream) {
  if (!coeffs || !out) return dg::set_thread_error(DG_ERR_ARG, "dg_conserved_static: null pointer");
  if (nv < 1 || nv > 4 || nmodes < 1 || nx < 1 || ny < 1)
    return dg::set_thread_error(DG_ERR_ARG, "dg_conserved_static: bad nv, nmodes, nx or ny");
  if (!(dx > 0.0) || !(dy > 0.0))
    return dg::set_thread_error(DG_ERR_ARG, "dg_conserved_static: dx and dy must be > 0");
  const long long nel = (long long)nx * ny;
  if (nel > (long long)DG_STATIC_MAX_ELEMENTS)
    return dg::set_thread_error(DG_ERR_ARG,
                                "dg_conserved_static: nx * ny above DG_STATIC_MAX_ELEMENTS (1048576)");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    return dg::set_thread_error(DG_ERR_ARG, "dg_conserved_static: no current CUDA device");
  }
  int rc = check_device_pointer(coeffs, dev, "coeffs");
  if (rc == DG_OK) rc = check_device_pointer(out, dev, "out");
  if (rc != DG_OK) return rc;
  const int nblk = (int)((nel + kThreads - 1) / kThreads);
  double* partials = nullptr;
  rc = scratch_address(dev, &partials);
  if (rc != DG_OK) return rc;
  // launched through cudaLaunchKernel so that each launch's own status is
  // returned, not an earlier, unrelated error left in the runtime's record
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double area = dx * dy;
  void* a1[] = {(void*)&coeffs, (void*)&nv, (void*)&nmodes, (void*)&nel, (void*)&area, (void*)&partials};
  cudaError_t e = cudaLaunchKernel((const void*)k_static_part, dim3(nblk), dim3(kThreads), a1, 0, s);
  if (e == cudaSuccess) {
    void* a2[] = {(void*)&partials, (void*)&nblk, (void*)&nv, (void*)&out};
    e = cudaLaunchKernel((const void*)k_static_final, dim3(1), dim3(kThreads), a2, 0, s);
  }
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof(msg), "dg_conserved_static: launch: %s", cudaGetErrorString(e));
    return dg::set_thread_error(DG_ERR_CUDA, msg);
  }
  return DG_OK;
}
