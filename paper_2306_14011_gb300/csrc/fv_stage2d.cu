// 2D instantiations of the fused stage kernel (4 conserved variables), CTAs
// of up to kStage2dMaxThreads threads.
#include "fv_stage.cuh"

namespace fvk {
cudaError_t launch_stage_2d(int mode, const CUtensorMap *tmap, const StageArgs &a, int threads, cudaStream_t st) {
  return launch_stage_dim<2, kStage2dMaxThreads>(mode, tmap, a, threads, st);
}
cudaError_t set_stage_attributes_2d(size_t smem) { return set_stage_attributes_dim<2, kStage2dMaxThreads>(smem); }
}  // namespace fvk
