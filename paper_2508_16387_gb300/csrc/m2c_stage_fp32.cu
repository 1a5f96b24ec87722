// FP32 (mixed-precision) instantiations of the bulk stage kernel.
#include "m2c_stage.cuh"

namespace m2c {

cudaError_t launch_stage_fp32(const Grid* grids, const long long* tiles, int ngrid, long long ntiles, int mode,
                              const LaunchPlan& lp, cudaStream_t s) {
  if (lp.ty == 4) return launch_stage_pair<float, 4>(grids, tiles, ngrid, ntiles, mode, lp, s);
  if (lp.ty == 16) return launch_stage_pair<float, 16>(grids, tiles, ngrid, ntiles, mode, lp, s);
  return launch_stage_pair<float, 8>(grids, tiles, ngrid, ntiles, mode, lp, s);
}

void setup_stage_fp32() {
  stage_smem_setup_pairs<float, 4>();
  stage_smem_setup_pairs<float, 8>();
  stage_smem_setup_pairs<float, 16>();
}

}  // namespace m2c
