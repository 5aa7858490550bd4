// 3D instantiations of the fused stage kernel (5 conserved variables).
#include "fv_stage.cuh"

namespace fvk {
cudaError_t launch_stage_3d(int mode, const CUtensorMap *tmap, const StageArgs &a, int threads, cudaStream_t st) {
  return launch_stage_dim<3, kStage3dMaxThreads>(mode, tmap, a, threads, st);
}
cudaError_t set_stage_attributes_3d(size_t smem) { return set_stage_attributes_dim<3, kStage3dMaxThreads>(smem); }
}  // namespace fvk
