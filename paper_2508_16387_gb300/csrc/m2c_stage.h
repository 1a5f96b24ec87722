// Host-side entry to the bulk stage kernel, compiled in its own translation
// units (one per precision) so that the library builds in parallel.
#pragma once
#include <cuda_runtime.h>

#include "m2c_kernels.cuh"

namespace m2c {

struct LaunchPlan {
  int ty = 8;            // tile rows (4, 8 or, FP32 only, 16)
  int sched = 0;         // 0: fixed stride over tiles, 1: atomic tile counter
  int blocks_per_sm = 0; // persistent grid of blocks_per_sm x SMs blocks; 0: one block per tile
  unsigned long long* counter = nullptr;
  int mats = -1;         // EOS types of the two materials of every grid, T0 + 4 T1 (SG / MG); -1: mixed or other
};

// Host-side state kept per device (index of the current device, clamped to
// kMaxDevices - 1) and the current device's SM count.
constexpr int kMaxDevices = 64;
int current_device();
int sm_count();

// Launch of k_stage<R, lp.ty> over ntiles tiles of ngrid grids (FP32: 4, 8 or
// 16 rows; FP64: 4 or 8 rows) and the one-time shared-memory opt-in.
cudaError_t launch_stage_fp32(const Grid* grids, const long long* tiles, int ngrid, long long ntiles, int mode,
                              const LaunchPlan& lp, cudaStream_t s);
cudaError_t launch_stage_fp64(const Grid* grids, const long long* tiles, int ngrid, long long ntiles, int mode,
                              const LaunchPlan& lp, cudaStream_t s);
void setup_stage_fp32();
void setup_stage_fp64();
// The general instantiation (k_stage<R, 8, true>) of either precision.
cudaError_t launch_stage_gen(int prec, const Grid* grids, const long long* tiles, int ngrid, long long ntiles,
                             int mode, const LaunchPlan& lp, cudaStream_t s);
void setup_stage_gen();

}  // namespace m2c
