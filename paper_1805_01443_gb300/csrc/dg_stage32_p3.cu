// dg_stage32_p3.cu -- precision-form stage kernel for polynomial degree p = 3.
#define DG_P 3
#include "dg_stage32.cuh"

namespace dg {
cudaError_t launch_stage32_p3(const StageArgs32& a, cudaStream_t s) { return launch_stage32_impl<3>(a, s); }
cudaError_t launch_torque32_p3(const float* D, const float* SigbN, const DevState* ts, double* part,
                                const Mesh& ms, const Prec32& pc, cudaStream_t s) {
  return launch_torque32_impl<3>(D, SigbN, ts, part, ms, pc, s);
}
cudaError_t upload_tables32_p3(const Tables& t) { return upload_tables32_impl<3>(t); }
}  // namespace dg
