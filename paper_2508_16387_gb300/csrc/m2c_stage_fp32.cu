// FP32 (mixed-precision) instantiations of the bulk stage kernel.
#include "m2c_stage.cuh"

namespace m2c {

cudaError_t launch_stage_fp32(const Grid* grids, const long long* tiles, int ngrid, long long ntiles, int mode,
                              const LaunchPlan& lp, cudaStream_t s) {
  if (lp.ty == 4) return launch_stage_t<float, 4, false>(grids, tiles, ngrid, ntiles, mode, lp, s);
  if (lp.ty == 16) return launch_stage_t<float, 16, false>(grids, tiles, ngrid, ntiles, mode, lp, s);
  return launch_stage_t<float, 8, false>(grids, tiles, ngrid, ntiles, mode, lp, s);
}

void setup_stage_fp32() {
  stage_smem_setup<float, 4, false>();
  stage_smem_setup<float, 8, false>();
  stage_smem_setup<float, 16, false>();
}

}  // namespace m2c
