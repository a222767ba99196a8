// Tensor-core M2L: not available in this build yet; build_bc_tree rejects
// the BF16 precision modes with BCFMM_ERR_ARG.
#include "m2l_tc.cuh"

namespace bcfmm {

bool m2l_tc_supported(int) { return false; }
cudaError_t m2l_tc_prepare_tables(int, int, const double*, int, M2LTensorTables*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_m2l_tc(const DevGeom&, const DevTaskLists&, const M2LTensorTables&, int, const float*, float*,
                          cudaStream_t) {
  return cudaErrorNotSupported;
}
void m2l_tc_free_tables(M2LTensorTables*) {}

}  // namespace bcfmm
