// dg_stage_p1.cu -- stage kernel instantiations for polynomial degree p = 1.
#define DG_P 1
#include "dg_stage.cuh"

namespace dg {
cudaError_t launch_stage_p1(const StageArgs& a, cudaStream_t s) { return launch_stage_impl<1>(a, s); }
cudaError_t upload_tables_p1(const Tables& t) { return upload_tables_impl<1>(t); }
size_t stage_smem_p1(int kind) { return stage_smem_impl<1>(kind); }
cudaError_t launch_static_p1(const Mesh& ms, const Phys& ph, double* SN, double* SXF, double* SYF,
                               cudaStream_t s) {
  return launch_static_impl<1>(ms, ph, SN, SXF, SYF, s);
}
}  // namespace dg
