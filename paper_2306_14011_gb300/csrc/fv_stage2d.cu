// 2D instantiations of the fused stage kernel (4 conserved variables).
#include "fv_stage.cuh"

namespace fvk {
cudaError_t launch_stage_2d(int mode, const CUtensorMap *tmap, const StageArgs &a, int threads, cudaStream_t st) {
  return launch_stage_dim<2>(mode, tmap, a, threads, st);
}
cudaError_t set_stage_attributes_2d(size_t smem) { return set_stage_attributes_dim<2>(smem); }
}  // namespace fvk
