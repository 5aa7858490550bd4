// 2D instantiations of the fused stage kernel for CTAs of more than
// kStage2dMaxThreads (up to 256) threads, with the smaller register budget.
#include "fv_stage.cuh"

namespace fvk {
cudaError_t launch_stage_2d_wide(int mode, const CUtensorMap *tmap, const StageArgs &a, int threads,
                                 cudaStream_t st) {
  return launch_stage_dim<2, 256>(mode, tmap, a, threads, st);
}
cudaError_t set_stage_attributes_2d_wide(size_t smem) { return set_stage_attributes_dim<2, 256>(smem); }
}  // namespace fvk
