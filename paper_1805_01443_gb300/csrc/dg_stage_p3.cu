// dg_stage_p3.cu -- stage kernel instantiations for polynomial degree p = 3.
#define DG_P 3
#include "dg_stage.cuh"

namespace dg {
cudaError_t launch_stage_p3(const StageArgs& a, cudaStream_t s) { return launch_stage_impl<3>(a, s); }
cudaError_t upload_tables_p3(const Tables& t) { return upload_tables_impl<3>(t); }
size_t stage_smem_p3(int kind) { return stage_smem_impl<3>(kind); }
cudaError_t launch_static_p3(const Mesh& ms, const Phys& ph, double* SN, double* SXF, double* SYF,
                               cudaStream_t s) {
  return launch_static_impl<3>(ms, ph, SN, SXF, SYF, s);
}
}  // namespace dg
