// FP64 instantiations of the bulk stage kernel (at most 8 rows: registers).
#include "m2c_stage.cuh"

namespace m2c {

cudaError_t launch_stage_fp64(const Grid* grids, const long long* tiles, int ngrid, long long ntiles, int mode,
                              const LaunchPlan& lp, cudaStream_t s) {
  if (lp.ty == 4) return launch_stage_pair<double, 4>(grids, tiles, ngrid, ntiles, mode, lp, s);
  return launch_stage_pair<double, 8>(grids, tiles, ngrid, ntiles, mode, lp, s);
}

void setup_stage_fp64() {
  stage_smem_setup_pairs<double, 4>();
  stage_smem_setup_pairs<double, 8>();
}

}  // namespace m2c
