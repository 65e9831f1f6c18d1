// dg_stage_p2.cu -- stage kernel instantiations for polynomial degree p = 2.
#define DG_P 2
#include "dg_stage.cuh"

namespace dg {
cudaError_t launch_stage_p2(const StageArgs& a, cudaStream_t s) { return launch_stage_impl<2>(a, s); }
cudaError_t upload_tables_p2(const Tables& t) { return upload_tables_impl<2>(t); }
size_t stage_smem_p2(int kind) { return stage_smem_impl<2>(kind); }
cudaError_t launch_static_p2(const Mesh& ms, const Phys& ph, double* SN, double* SXF, double* SYF,
                               cudaStream_t s) {
  return launch_static_impl<2>(ms, ph, SN, SXF, SYF, s);
}
}  // namespace dg
