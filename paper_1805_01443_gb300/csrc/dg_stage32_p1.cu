// dg_stage32_p1.cu -- precision-form stage kernel for polynomial degree p = 1.
#define DG_P 1
#include "dg_stage32.cuh"

namespace dg {
cudaError_t launch_stage32_p1(const StageArgs32& a, cudaStream_t s) { return launch_stage32_impl<1>(a, s); }
cudaError_t launch_torque32_p1(const float* D, const float* SigbN, const DevState* ts, double* part,
                                const Mesh& ms, const Prec32& pc, cudaStream_t s) {
  return launch_torque32_impl<1>(D, SigbN, ts, part, ms, pc, s);
}
cudaError_t upload_tables32_p1(const Tables& t) { return upload_tables32_impl<1>(t); }
}  // namespace dg
