// dg_stage_p4.cu -- stage kernel instantiations for polynomial degree p = 4.
#define DG_P 4
#include "dg_stage.cuh"

namespace dg {
cudaError_t launch_stage_p4(const StageArgs& a, cudaStream_t s) { return launch_stage_impl<4>(a, s); }
cudaError_t upload_tables_p4(const Tables& t) { return upload_tables_impl<4>(t); }
size_t stage_smem_p4(int kind) { return stage_smem_impl<4>(kind); }
cudaError_t launch_static_p4(const Mesh& ms, const Phys& ph, double* SN, double* SXF, double* SYF,
                               cudaStream_t s) {
  return launch_static_impl<4>(ms, ph, SN, SXF, SYF, s);
}
}  // namespace dg
