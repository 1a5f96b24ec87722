// General instantiations of the bulk stage kernel (both precisions, 8-row
// tiles): the scheme options of m2c_set_options are taken at run time.
#include "m2c_stage.cuh"

namespace m2c {

cudaError_t launch_stage_gen(int prec, const Grid* grids, const long long* tiles, int ngrid, long long ntiles,
                             int mode, const LaunchPlan& lp, cudaStream_t s) {
  if (prec == M2C_FP64) return launch_stage_t<double, 8, true>(grids, tiles, ngrid, ntiles, mode, lp, s);
  return launch_stage_t<float, 8, true>(grids, tiles, ngrid, ntiles, mode, lp, s);
}

void setup_stage_gen() {
  stage_smem_setup<double, 8, true>();
  stage_smem_setup<float, 8, true>();
}

}  // namespace m2c
